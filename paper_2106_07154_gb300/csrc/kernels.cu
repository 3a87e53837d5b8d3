// kernels.cu -- sm_103a kernels of the LTS3 / SSP-RK3 hot path.
//
// One evaluation of the right-hand side of Eq. (1) restricted to a band
// range, fused with the SSP stage combination (Algorithm 2.1) or with the
// correction accumulation of Steps 3.x.2, is three launches:
//   kind 0 (vertex): q_v = (zeta_v + f_v) / h_v (Appendix B, reading R7) for
//     the vertices the ring pass reads;
//   kind 1 (ring, one thread per cell): reads the cell's counter-clockwise
//     ring once with coalesced slot-major loads and forms F_e = [h]_{i->e} u_e,
//     K_i, H_i = -[div F]_i (compensated sum, then the stage update or the
//     accumulation) and, for every edge e_p of the cell, the cell's share of
//     F^perp_e [q]_{v->e} with the weights w_{e,e'} of Eq. (weights) taken
//     from prefix sums of the kite fractions;
//   kind 2 (edge): U_e = -F^perp_e [q]_{v->e} - [g grad(h+b) + grad K]_e from
//     the two cells' ring results, then the stage update or accumulation.
// Pointwise segments (interface predictions of Steps 3.x.1, snapshots,
// Step 5) ride in these launches.  Every restricted phase is a set of
// contiguous band ranges; the path is a sparse gather stencil, so no tensor
// cores are used.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lts_internal.h"

namespace lts {
namespace {

template <class T>
struct DevSeg {
    int type, begin, end, base, base2, flag, block0, pad;
    T c[6];
    void* p[10];
};

template <class T>
struct DevArgs {
    Tables<T> t;
    DevSeg<T> seg[MAXSEG];
    int nseg;
    const T* in_h;
    const T* in_hl;   // compensation words of the input thickness (COMP only)
    const T* in_u;
    const T* in_ul;   // compensation words of the input velocity (COMP only)
    T* q;
    T* ring_c;        // [maxE*nC] per-slot PV contributions
    T* ring_k;        // [nC] K_i
    T g;
    int* flag;
    int l2;           // 0 no hint, 1 keep in L2 (evict_last), 2 stream (evict_first)
    int smem;         // dynamic shared memory of the launch (fused tiles)
    int L;            // layers per element (multi-layer states; 1 otherwise)
    int lpt;          // multi-layer states: layers per thread (consecutive layers of one element)
    int G;            // multi-layer states: thread groups per element, ceil(L / lpt)
    int v2;           // multi-layer states: 1 when every pair of layers a thread runs is one
                      // aligned two-word access (checked on the host), else 0
    int v4;           // FP32 multi-layer states: 1 when every thread's four layers are one
                      // aligned four-word access (checked on the host), else 0
    // segment-table launches (ensembles): segments in device memory
    const DevSeg<T>* gseg;
    int ngseg;
    int vblocks;      // virtual blocks over all segments
};

// ------------------------------------------------------------- L2 residency
// The fine substeps revisit the fine region's mesh tables (~65 MB on a
// 655k-cell mesh with an 8:1 cap) 3M times per coarse step, and again every
// coarse step, while its state (~25 MB per right-hand side) is rewritten by
// every stage and the coarse-band launches stream the rest of the mesh
// once.  Loads and stores carry an L2 eviction-priority policy per launch
// mode: fine launches (1) keep their tables (evict_last) and let their state
// go first (evict_first); coarse launches (2) stream both (evict_first).
// Measured on GB300, this beats keeping everything of the fine launches
// (the fine working set as a whole is about as large as the L2 holds).
// Hints only: results do not depend on them.
__device__ __forceinline__ uint64_t l2_policy(int mode) {
    uint64_t p;
    if (mode == 1)
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else if (mode == 2)
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Loads of mesh tables (never written by any kernel): free to be scheduled.
#define LTS_LD_STATIC(TY, PTXT, CONS)                                                    \
    __device__ __forceinline__ TY ld_static(const TY* q, uint64_t p) {                   \
        TY x;                                                                            \
        asm("ld.global.nc.L2::cache_hint." PTXT " %0, [%1], %2;" : CONS(x) : "l"(q), "l"(p)); \
        return x;                                                                        \
    }
#define LTS_LD_STATE(TY, PTXT, CONS)                                                     \
    __device__ __forceinline__ TY ld_state(const TY* q, uint64_t p) {                    \
        TY x;                                                                            \
        asm volatile("ld.global.nc.L2::cache_hint." PTXT " %0, [%1], %2;"                \
                     : CONS(x) : "l"(q), "l"(p) : "memory");                             \
        return x;                                                                        \
    }
#define LTS_R(x) "=r"(x)
#define LTS_F(x) "=f"(x)
#define LTS_D(x) "=d"(x)
LTS_LD_STATIC(int, "b32", LTS_R)
LTS_LD_STATIC(uint32_t, "b32", LTS_R)
LTS_LD_STATIC(float, "f32", LTS_F)
LTS_LD_STATIC(double, "f64", LTS_D)
LTS_LD_STATE(float, "f32", LTS_F)
LTS_LD_STATE(double, "f64", LTS_D)
// Two consecutive layers of one element (words x and x + 1) in one access.
// Used only by launches whose host has checked that every such pair starts
// on a multiple of the pair's size (even layer count, even first layer of
// every pair, aligned buffers).
template <class T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};
template <class T>
using vec2_t = typename Vec2<T>::type;
__device__ __forceinline__ float2 ld_state2(const float* q, uint64_t p) {
    float2 x;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(x.x), "=f"(x.y) : "l"(q), "l"(p) : "memory");
    return x;
}
__device__ __forceinline__ double2 ld_state2(const double* q, uint64_t p) {
    double2 x;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(x.x), "=d"(x.y) : "l"(q), "l"(p) : "memory");
    return x;
}
__device__ __forceinline__ int4 ld_static(const int4* q, uint64_t p) {
    int4 x;
    asm("ld.global.nc.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(x.x), "=r"(x.y), "=r"(x.z), "=r"(x.w) : "l"(q), "l"(p));
    return x;
}
__device__ __forceinline__ float4 ld_static(const float4* q, uint64_t p) {
    float4 x;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w) : "l"(q), "l"(p));
    return x;
}
__device__ __forceinline__ float2 ld_static(const float2* q, uint64_t p) {
    float2 x;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(x.x), "=f"(x.y) : "l"(q), "l"(p));
    return x;
}
__device__ __forceinline__ uint8_t ld_static(const uint8_t* q, uint64_t p) {
    uint32_t x;
    asm("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(x) : "l"(q), "l"(p));
    return static_cast<uint8_t>(x);
}
// Stores with an L2 eviction-priority policy: a launch's results carry the
// priority of its state loads (see above).
__device__ __forceinline__ void st_hint(float* q, float v, uint64_t p) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(q), "f"(v), "l"(p) : "memory");
}
__device__ __forceinline__ void st_hint(double* q, double v, uint64_t p) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(q), "d"(v), "l"(p) : "memory");
}
__device__ __forceinline__ void st_hint(float* q, float2 v, uint64_t p) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(q), "f"(v.x), "f"(v.y), "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st_hint(double* q, double2 v, uint64_t p) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(q), "d"(v.x), "d"(v.y), "l"(p)
                 : "memory");
}
// W consecutive layers of one element (W = 2 or 4 words) in one access, for
// launches whose host has checked that every such group is aligned to its
// size.
template <class T, int W>
struct Lanes {
    T v[W];
};
template <int W>
__device__ __forceinline__ Lanes<float, W> ld_lanes(const float* q, uint64_t p) {
    static_assert(W == 2 || W == 4, "two or four FP32 words per access");
    Lanes<float, W> r;
    if constexpr (W == 2) {
        const float2 x = ld_state2(q, p);
        r.v[0] = x.x, r.v[1] = x.y;
    } else {
        asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "l"(q), "l"(p) : "memory");
    }
    return r;
}
template <int W>
__device__ __forceinline__ Lanes<double, W> ld_lanes(const double* q, uint64_t p) {
    static_assert(W == 2, "two FP64 words per access");
    const double2 x = ld_state2(q, p);
    Lanes<double, W> r;
    r.v[0] = x.x, r.v[1] = x.y;
    return r;
}
template <int W>
__device__ __forceinline__ void st_lanes(float* q, const Lanes<float, W>& v, uint64_t p) {
    static_assert(W == 2 || W == 4, "two or four FP32 words per access");
    if constexpr (W == 2) {
        st_hint(q, make_float2(v.v[0], v.v[1]), p);
    } else {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(q), "f"(v.v[0]),
                     "f"(v.v[1]), "f"(v.v[2]), "f"(v.v[3]), "l"(p)
                     : "memory");
    }
}
template <int W>
__device__ __forceinline__ void st_lanes(double* q, const Lanes<double, W>& v, uint64_t p) {
    static_assert(W == 2, "two FP64 words per access");
    st_hint(q, make_double2(v.v[0], v.v[1]), p);
}

// Policy of a launch mode's state accesses (see above): the fine launches'
// state goes first, like the coarse launches' data.
__device__ __forceinline__ int state_mode(int m) { return m == 1 ? 2 : m; }

struct St {
    uint64_t pol;
    __device__ __forceinline__ explicit St(int m) : pol(l2_policy(state_mode(m))) {}
    template <class V>
    __device__ __forceinline__ void operator()(V* q, V v) const { st_hint(q, v, pol); }
    // words q[0], q[1] (two layers) in one aligned access
    template <class V>
    __device__ __forceinline__ void pair(V* q, vec2_t<V> v) const { st_hint(q, v, pol); }
    // words q[0..W-1] (W layers) in one aligned access
    template <int W, class V>
    __device__ __forceinline__ void lanes(V* q, const Lanes<V, W>& v) const { st_lanes<W>(q, v, pol); }
};

// Read-only loads with the launch's L2 policy: `stat` for mesh tables, `operator()`
// for state written by earlier kernels (ordered after griddep_wait).
struct Ld {
    uint64_t pol, spol;   // tables, state
    __device__ __forceinline__ explicit Ld(int m) : pol(l2_policy(m)), spol(l2_policy(state_mode(m))) {}
    template <class V>
    __device__ __forceinline__ V stat(const V* q) const { return ld_static(q, pol); }
    template <class V>
    __device__ __forceinline__ V operator()(const V* q) const { return ld_state(q, spol); }
    // state words q[0], q[1] (two layers) in one aligned access
    template <class V>
    __device__ __forceinline__ vec2_t<V> pair(const V* q) const { return ld_state2(q, spol); }
    // state words q[0..W-1] (W layers) in one aligned access
    template <int W, class V>
    __device__ __forceinline__ Lanes<V, W> lanes(const V* q) const { return ld_lanes<W>(q, spol); }
};

// ------------------------------------------------------------------ layers
// Element index -> array index of the state and the intermediates.  A
// multi-layer state stores the layers of an element next to each other
// ([element * L + layer]); its kernels run one thread per (element, group
// of consecutive layers) with the groups fastest, so the threads of a warp
// share their table loads (one broadcast transaction) and read the state
// contiguously.  Mesh tables are indexed by the element alone.  The
// single-layer map is the identity.
template <bool LAYERED>
struct Lay;
template <>
struct Lay<false> {
    __device__ __forceinline__ int operator()(int x) const { return x; }
};
template <>
struct Lay<true> {
    int L, l;
    __device__ __forceinline__ long long operator()(long long x) const { return x * L + l; }
};

// ---------------------------------------------------------------- arithmetic
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Knuth's TwoSum: s + e == a + b exactly.
template <class T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// Dekker's FastTwoSum (|a| >= |b|).
template <class T>
__device__ __forceinline__ void fast_two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    e = b - (s - a);
}

// SSP stage combination of Algorithm 2.1 in increment form:
//   y = x_s + a (x_old - x_s) + D R
// (stage 1: a = 0, D = dt; stage 2: a = 3/4, D = dt/4; stage 3: a = 1/3,
// D = 2 dt/3), which keeps a constant state exactly constant.  With COMP the
// states are (hi, lo) pairs and the large term x_s is added with TwoSum, so
// the rounding of each stage is carried in lo instead of being lost.
template <class T, bool COMP>
__device__ __forceinline__ void combine(T oh, T ol, T sh, T sl, T a, T D, T R, T& yh, T& yl) {
    if (COMP) {
        T d = (oh - sh) + (ol - sl);
        T inc = fma_rn(D, R, mul_rn(a, d));
        T s, e;
        two_sum(sh, inc, s, e);
        T lo = sl + e;
        fast_two_sum(s, lo, yh, yl);
    } else {
        T inc = fma_rn(D, R, mul_rn(a, oh - sh));
        yh = sh + inc;
        yl = T(0);
    }
}

// Interface-1 prediction of Steps 3.x.1 in increment form,
// x = x_old + c1 (x_1st - x_old) + c2 (x_2nd - x_old); sel != 0 when the
// coefficients select one vector exactly (then the value is copied).
template <class T, bool COMP>
__device__ __forceinline__ void predict(T oh, T ol, T h1, T l1, T h2, T l2, T c1, T c2, int sel,
                                        T& yh, T& yl) {
    if (sel == 1) { yh = oh; yl = ol; return; }
    if (sel == 2) { yh = h1; yl = l1; return; }
    if (sel == 3) { yh = h2; yl = l2; return; }
    T d1 = COMP ? (h1 - oh) + (l1 - ol) : h1 - oh;
    T d2 = COMP ? (h2 - oh) + (l2 - ol) : h2 - oh;
    T inc = fma_rn(c2, d2, mul_rn(c1, d1));
    if (COMP) {
        T s, e;
        two_sum(oh, inc, s, e);
        T lo = ol + e;
        fast_two_sum(s, lo, yh, yl);
    } else {
        yh = oh + inc;
        yl = T(0);
    }
}

__device__ __forceinline__ bool finite_pos(double x) { return x > 0.0 && x < 1e300; }
__device__ __forceinline__ bool finite_pos(float x) { return x > 0.0f && x < 3.0e38f; }
__device__ __forceinline__ bool finite_val(double x) { return fabs(x) < 1e300; }
__device__ __forceinline__ bool finite_val(float x) { return fabsf(x) < 3.0e38f; }

// Programmatic dependent launch: let the next kernel of the stream start
// launching now, and wait until the previous kernel's results are visible.
// Both are no-ops without PDL.  Every kernel loads its static mesh tables
// before griddep_wait, so those loads overlap the previous kernel's tail; no
// state is read or written before the wait.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------- stage-update operands
// The operands of an element's stage update (UPD: old value, input value and
// their compensation words) or accumulation (ACC: the running sum).  The
// edge pass loads them right after the dependency wait, beside its stencil
// gathers, so the update adds no memory round trip after the tendency.
// UPD: oh, ol = old value and its compensation word, xh, xl = input value
// and its word; ACC: oh = the running sum (0 for the first term).
template <class T>
struct EpiOps {
    T oh, ol, xh, xl;
};

enum : int { EPI_NONE = 0, EPI_UPD = 1, EPI_ACC = 2 };

// in_x = null: the caller already holds the input value (it sets xh).
template <class T, bool COMP, bool LY>
__device__ __forceinline__ void epi_load(const Ld& ld, const DevSeg<T>& s, int mode, int i, const T* in_x,
                                         EpiOps<T>& o, const Lay<LY>& y) {
    if (mode == EPI_ACC) {
        o.oh = s.flag ? T(0) : ld((const T*)s.p[0] + y(i - s.base));
    } else if (mode == EPI_UPD) {
        o.oh = ld((const T*)s.p[0] + y(i));
        o.ol = COMP ? ld((const T*)s.p[1] + y(i)) : T(0);
        if (in_x) o.xh = ld(in_x + y(i));
        o.xl = COMP ? ld((const T*)s.p[2] + y(i)) : T(0);
    }
}

// epi_load of W consecutive layers (y.l .. y.l + W - 1) with one access per
// array.
template <class T, bool COMP, int W>
__device__ __forceinline__ void epi_load_group(const Ld& ld, const DevSeg<T>& s, int mode, int i, const T* in_x,
                                               EpiOps<T> (&o)[W], const Lay<true>& y) {
    if (mode == EPI_ACC) {
        if (s.flag) {
#pragma unroll
            for (int k = 0; k < W; ++k) o[k].oh = T(0);
        } else {
            const Lanes<T, W> v = ld.lanes<W>((const T*)s.p[0] + y(i - s.base));
#pragma unroll
            for (int k = 0; k < W; ++k) o[k].oh = v.v[k];
        }
    } else if (mode == EPI_UPD) {
        const Lanes<T, W> oh = ld.lanes<W>((const T*)s.p[0] + y(i));
#pragma unroll
        for (int k = 0; k < W; ++k) o[k].oh = oh.v[k], o[k].ol = T(0), o[k].xl = T(0);
        if (COMP) {
            const Lanes<T, W> ol = ld.lanes<W>((const T*)s.p[1] + y(i));
            const Lanes<T, W> xl = ld.lanes<W>((const T*)s.p[2] + y(i));
#pragma unroll
            for (int k = 0; k < W; ++k) o[k].ol = ol.v[k], o[k].xl = xl.v[k];
        }
        if (in_x) {
            const Lanes<T, W> x = ld.lanes<W>(in_x + y(i));
#pragma unroll
            for (int k = 0; k < W; ++k) o[k].xh = x.v[k];
        }
    }
}

// ------------------------------------------------------------- kind 0: vertex

// q_v = (zeta_v + f_v) / h_v with zeta_v = sum t_{e,v} (d_e/A_v) u_e and
// h_v = sum (A_{i,v}/A_v) h_i.
// The vertex's mesh-table operands (loaded before the dependency wait).
template <class T>
struct VertStat {
    int e0, e1, e2, c0, c1, c2;
    T d0, d1, d2, k0, k1, k2, f;
};

template <class T>
__device__ __forceinline__ void vertex_stat(const Tables<T>& t, const Ld& ld, int v, VertStat<T>& s) {
    // packed rows: {e0, e1, e2, c0}, and in FP32 {d0, d1, d2, f}, {k0, k1, k2, c1}
    const int4 ie = ld.stat(t.vri + v);
    s.e0 = ie.x, s.e1 = ie.y, s.e2 = ie.z, s.c0 = ie.w;
    s.c2 = ld.stat(t.vc2 + v);
    if constexpr (sizeof(T) == 4) {
        const float4 d = ld.stat(t.vrd + v);
        const float4 k = ld.stat(t.vrk + v);
        s.d0 = d.x, s.d1 = d.y, s.d2 = d.z, s.f = d.w;
        s.k0 = k.x, s.k1 = k.y, s.k2 = k.z, s.c1 = __float_as_int(k.w);
    } else {
        s.c1 = ld.stat(t.vc1 + v);
        s.d0 = ld.stat(t.vd0 + v), s.d1 = ld.stat(t.vd1 + v), s.d2 = ld.stat(t.vd2 + v);
        s.k0 = ld.stat(t.vk0 + v), s.k1 = ld.stat(t.vk1 + v), s.k2 = ld.stat(t.vk2 + v);
        s.f = ld.stat(t.f + v);
    }
}

// q_v from the vertex's three edge velocities and cell thicknesses, with the
// roundings spelled out, so every pass that forms q (vertex, fused tiles)
// gets the same bits.
template <class T>
__device__ __forceinline__ T q_value(T d0, T d1, T d2, T u0, T u1, T u2, T k0, T k1, T k2, T h0, T h1, T h2,
                                     T f) {
    const T zeta = fma_rn(d2, u2, fma_rn(d1, u1, mul_rn(d0, u0)));
    const T hv = fma_rn(k2, h2, fma_rn(k1, h1, mul_rn(k0, h0)));
    return (zeta + f) / hv;
}

// Gathers u and h (after the wait) and returns q_v.
template <class T, bool LY>
__device__ __forceinline__ T vertex_q(const DevArgs<T>& a, const Ld& ld, const VertStat<T>& s, const Lay<LY>& y) {
    const T u0 = ld(a.in_u + y(s.e0)), u1 = ld(a.in_u + y(s.e1)), u2 = ld(a.in_u + y(s.e2));
    const T h0 = ld(a.in_h + y(s.c0)), h1 = ld(a.in_h + y(s.c1)), h2 = ld(a.in_h + y(s.c2));
    return q_value(s.d0, s.d1, s.d2, u0, u1, u2, s.k0, s.k1, s.k2, h0, h1, h2, s.f);
}

template <class T, bool LY>
__device__ __forceinline__ void vertex_pv(const DevArgs<T>& a, int v, const Lay<LY>& y) {
    const Ld ld(a.l2);
    VertStat<T> s;
    vertex_stat(a.t, ld, v, s);
    griddep_wait();
    St(a.l2)(a.q + y(v), vertex_q<T, LY>(a, ld, s, y));
}

// --------------------------------------------------------------- kind 1: ring
//
// One thread per cell c, slots j = 0..n-1 (edge e_j, neighbour across it,
// vertex v_j between e_j and e_{j+1}, kite fraction R_j = A_{c,v_j}/A_c):
//   F_j  = (h_c + h_nb)/2 u_j,   G_j = n_{e_j,c} l_j F_j,   qt_j = (q_{v_{j-1}} + q_{v_j})/2
//   K_c  = sum_j l_j d_j u_j^2 / (4 A_c),      H_c = -(1/A_c) sum_j G_j
// and for every slot p the share of the PV flux of edge e_p,
//   C_p = sum_{j != p} (S_{j->p} - 1/2) G_j (qt_p + qt_j),
// where S_{j->p} = sum of R_m over the vertices met going counter-clockwise
// from e_j to e_p (so w_{e_p,e_j} = n_{e_j,c} (-n_{e_p,c}) (S_{j->p} - 1/2),
// t_{e_p,v_{p-1}} = -n_{e_p,c} on a counter-clockwise ring).  With prefix sums
// P_p = R_0 + ... + R_{p-1}, S_{j->p} = P_p - P_j + [j > p] P_n.  Writing
// A = sum_j G_j, A' = sum_j P_j G_j, Asuf_p = sum_{j>p} G_j and B, B', Bsuf
// the same with b_j = G_j qt_j, the sum over j != p regroups into O(n) work:
//   C_p = qt_p (w_p A - A' + P_n Asuf_p) + (w_p B - B' + P_n Bsuf_p) + b_p,
// w_p = P_p - 1/2 (the j = p terms of A and B cancel into the last b_p).

// Arithmetic of the ring core on a value type V: one layer in T (float or
// double), or two layers in float2, where every operation is one packed
// Blackwell FP32x2 instruction whose lanes round exactly as the scalar
// operation (so a two-layer run equals two one-layer runs bit for bit).
template <class V>
struct VA;
template <>
struct VA<float> {
    static __device__ __forceinline__ float cst(float x) { return x; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
};
template <>
struct VA<double> {
    static __device__ __forceinline__ double cst(double x) { return x; }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double neg(double a) { return -a; }
};
template <>
struct VA<float2> {
    static __device__ __forceinline__ float2 cst(float x) { return make_float2(x, x); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
    // a - b is a + (-b) exactly
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, neg(b)); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
};

// The ring arithmetic of one cell from its gathered slot values (slots
// j >= n are ignored), shared by the ring pass and the fused tiles so both
// give the same bits.  V = T for one layer, float2 for two FP32 layers
// (the slot coefficients then hold the same value in both lanes).
// Returns H_c; C[p] for p < n and K_c on output.
template <class V, bool COMP, int NR>
__device__ __forceinline__ V ring_core(int n, V hc, V rA, const V (&uj)[NR], const V (&hn)[NR],
                                       const V (&qv)[NR], const V (&snl)[NR], const V (&Rj)[NR],
                                       const V (&sK)[NR], V (&C)[NR], V& Kc_out) {
    using A = VA<V>;
    const V zero = A::cst(0.0f), half = A::cst(0.5f);
    V G[NR], R[NR];
    V Kc = zero, s = zero, comp = zero;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const bool in = j < n;
        const V F = A::mul(A::mul(half, A::add(hc, hn[j])), uj[j]);
        const V g = in ? A::mul(snl[j], F) : zero;
        G[j] = g;
        R[j] = in ? Rj[j] : zero;
        if (in) {
            Kc = A::fma(A::mul(sK[j], uj[j]), uj[j], Kc);
            if (COMP) {
                // Knuth's TwoSum of (s, g): s + e == s_old + g exactly
                const V ss = A::add(s, g);
                const V bb = A::sub(ss, s);
                const V ee = A::add(A::sub(s, A::sub(ss, bb)), A::sub(g, bb));
                s = ss;
                comp = A::add(comp, ee);
            } else {
                s = A::add(s, g);
            }
        }
    }
    // q at v_{n-1} closes the ring for slot 0
    V qlast = qv[0];
#pragma unroll
    for (int j = 1; j < NR; ++j)
        if (j == n - 1) qlast = qv[j];
    V qt[NR], P[NR], b[NR];
    V Pacc = zero, Asum = zero, Bsum = zero, A1 = zero, B1 = zero;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        qt[j] = A::mul(half, A::add(j == 0 ? qlast : qv[j - 1], qv[j]));
        P[j] = Pacc;
        b[j] = A::mul(G[j], qt[j]);
        if (j < n) {
            Pacc = A::add(Pacc, R[j]);
            Asum = A::add(Asum, G[j]);
            Bsum = A::add(Bsum, b[j]);
            A1 = A::fma(P[j], G[j], A1);
            B1 = A::fma(P[j], b[j], B1);
        }
    }
    const V Pn = Pacc;
    V Asuf = zero, Bsuf = zero;
#pragma unroll
    for (int p = NR - 1; p >= 0; --p) {
        if (p < n) {
            const V w = A::sub(P[p], half);
            const V al = A::fma(Pn, Asuf, A::fma(w, Asum, A::neg(A1)));
            const V be = A::fma(Pn, Bsuf, A::fma(w, Bsum, A::neg(B1)));
            C[p] = A::add(A::fma(qt[p], al, be), b[p]);
            Asuf = A::add(Asuf, G[p]);
            Bsuf = A::add(Bsuf, b[p]);
        }
    }
    Kc_out = Kc;
    return A::mul(A::neg(A::add(s, comp)), rA);
}

// The first UNCOND slots' tables are loaded before the dependency wait
// without waiting for the cell's degree (padding slots are valid copies of
// slot 0), so the table loads and the state gathers of a thread are two
// independent waves.  Seven slots cover the heptagons of variable-resolution
// Voronoi meshes (about one cell in eleven, so nearly every warp has one),
// whose last slot would otherwise cost the warp a further round trip.  Each
// slot is two vector loads in FP32: {edge, neighbour, vertex, n l} and
// {kite fraction, K coefficient}.
constexpr int UNCOND = 7;
static_assert(UNCOND <= kSlotRowsMin, "the slot tables must hold the unconditional slots");

template <class T>
struct RingSlot {
    int e, nb, v;
    T snl, R, sK;
};

template <class T>
__device__ __forceinline__ RingSlot<T> ring_slot(const Tables<T>& t, const Ld& ld, int j, int c) {
    const int N = t.nC;
    const int4 x = ld.stat(t.sidx + j * N + c);
    RingSlot<T> r;
    r.e = x.x;
    r.nb = x.y;
    r.v = x.z;
    if constexpr (sizeof(T) == 4) {
        const float2 z = ld.stat(t.scf + j * N + c);
        r.snl = __int_as_float(x.w);
        r.R = z.x;
        r.sK = z.y;
    } else {
        r.snl = ld.stat(t.snl + j * N + c);
        r.R = ld.stat(t.sR + j * N + c);
        r.sK = ld.stat(t.sK + j * N + c);
    }
    return r;
}

// Gathers the state of NR slots (the warp's largest degree, so the unrolled
// loops run no further than some lane needs) and runs the ring arithmetic.
template <class T, bool COMP, int NR, bool LY>
__device__ __forceinline__ T ring_body(const DevArgs<T>& a, const Ld& ld, int c, int n, T rA,
                                       const RingSlot<T> (&S0)[UNCOND], const Lay<LY>& y) {
    const int N = a.t.nC;
    const T hc = ld(a.in_h + y(c));
    T uj[NR], hn[NR], qv[NR], snl[NR], Rj[NR], sK[NR], C[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const RingSlot<T> r = j < UNCOND ? S0[j % UNCOND] : (j < n ? ring_slot(a.t, ld, j, c) : S0[0]);
        uj[j] = ld(a.in_u + y(r.e));
        hn[j] = ld(a.in_h + y(r.nb));
        qv[j] = ld(a.q + y(r.v));
        snl[j] = r.snl;
        Rj[j] = r.R;
        sK[j] = r.sK;
    }
    T Kc;
    const T H = ring_core<T, COMP, NR>(n, hc, rA, uj, hn, qv, snl, Rj, sK, C, Kc);
    const St st(a.l2);
#pragma unroll
    for (int p = 0; p < NR; ++p)
        if (p < n) st(a.ring_c + y(p * N + c), C[p]);
    st(a.ring_k + y(c), Kc);
    return H;
}

template <class T, bool COMP, int MAXR, bool LY>
__device__ __forceinline__ T ring_pass(const DevArgs<T>& a, int c, const Lay<LY>& y) {
    const Tables<T>& t = a.t;
    const Ld ld(a.l2);
    const int n = ld.stat(t.cn + c);
    RingSlot<T> S0[UNCOND];
#pragma unroll
    for (int j = 0; j < UNCOND; ++j) S0[j] = ring_slot(t, ld, j, c);
    const T rA = ld.stat(t.rA + c);
    griddep_wait();
    // the unrolled width follows the largest degree among the warp's cells
    // (warp-uniform, so the lanes of a warp stay converged)
    const int nmax = __reduce_max_sync(__activemask(), n);
    if (nmax <= 6) return ring_body<T, COMP, 6, LY>(a, ld, c, n, rA, S0, y);
    if (nmax <= 7 || MAXR <= 7) return ring_body<T, COMP, (MAXR < 7 ? MAXR : 7), LY>(a, ld, c, n, rA, S0, y);
    if (nmax <= 8 || MAXR <= 8) return ring_body<T, COMP, (MAXR < 8 ? MAXR : 8), LY>(a, ld, c, n, rA, S0, y);
    return ring_body<T, COMP, MAXR, LY>(a, ld, c, n, rA, S0, y);
}

// Two consecutive layers (y.l and y.l + 1) of an FP32 multi-layer state in
// one ring pass: the slot tables are loaded once, the two layers' state is
// gathered into float2 values (one aligned two-word access each) and the
// ring core runs on both at once.  The
// cells' update operands are loaded with the gathers (the many waves of a
// multi-layer launch leave the registers for them), so the pass has one
// dependent round trip after the wait; o[0].xh, o[1].xh are the input
// thicknesses the ring reads anyway.
template <bool COMP, int NR>
__device__ __forceinline__ float2 ring_body_pair(const DevArgs<float>& a, const Ld& ld, int c, int n, float rA,
                                                 const RingSlot<float> (&S0)[UNCOND], const Lay<true>& y0,
                                                 EpiOps<float> (&o)[2]) {
    const int N = a.t.nC;
    const float2 hc = ld.pair(a.in_h + y0(c));
    o[0].xh = hc.x;
    o[1].xh = hc.y;
    float2 uj[NR], hn[NR], qv[NR], snl[NR], Rj[NR], sK[NR], C[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const RingSlot<float> r = j < UNCOND ? S0[j % UNCOND] : (j < n ? ring_slot(a.t, ld, j, c) : S0[0]);
        uj[j] = ld.pair(a.in_u + y0(r.e));
        hn[j] = ld.pair(a.in_h + y0(r.nb));
        qv[j] = ld.pair(a.q + y0(r.v));
        snl[j] = make_float2(r.snl, r.snl);
        Rj[j] = make_float2(r.R, r.R);
        sK[j] = make_float2(r.sK, r.sK);
    }
    float2 Kc;
    const float2 H = ring_core<float2, COMP, NR>(n, hc, make_float2(rA, rA), uj, hn, qv, snl, Rj, sK, C, Kc);
    const St st(a.l2);
#pragma unroll
    for (int p = 0; p < NR; ++p)
        if (p < n) st.pair(a.ring_c + y0(p * N + c), C[p]);
    st.pair(a.ring_k + y0(c), Kc);
    return H;
}

template <bool COMP, int MAXR>
__device__ __forceinline__ float2 ring_pass_pair(const DevArgs<float>& a, const DevSeg<float>& s, int epi, int c,
                                                 const Lay<true>& y0, EpiOps<float> (&o)[2]) {
    const Tables<float>& t = a.t;
    const Ld ld(a.l2);
    const int n = ld.stat(t.cn + c);
    RingSlot<float> S0[UNCOND];
#pragma unroll
    for (int j = 0; j < UNCOND; ++j) S0[j] = ring_slot(t, ld, j, c);
    const float rA = ld.stat(t.rA + c);
    griddep_wait();
    epi_load_group<float, COMP, 2>(ld, s, epi, c, nullptr, o, y0);
    const int nmax = __reduce_max_sync(__activemask(), n);
    if (nmax <= 6) return ring_body_pair<COMP, 6>(a, ld, c, n, rA, S0, y0, o);
    if (nmax <= 7 || MAXR <= 7)
        return ring_body_pair<COMP, (MAXR < 7 ? MAXR : 7)>(a, ld, c, n, rA, S0, y0, o);
    if (nmax <= 8 || MAXR <= 8)
        return ring_body_pair<COMP, (MAXR < 8 ? MAXR : 8)>(a, ld, c, n, rA, S0, y0, o);
    return ring_body_pair<COMP, MAXR>(a, ld, c, n, rA, S0, y0, o);
}

// --------------------------------------------------------------- kind 2: edge
// U_e = -(1/d_e) [ (C_{c1,p1} - C_{c0,p0})/2 + g((h1 - h0) + (b1 - b0)) + K1 - K0 ]
// (-n_{e,c0} = -1, -n_{e,c1} = +1 carry the signs of the two ring shares).
// The edge's mesh-table operands (loaded before the dependency wait).
template <class T>
struct EdgeStat {
    int c0, c1, p0, p1;
    T rdc, db;
};

template <class T>
__device__ __forceinline__ void edge_stat(const Tables<T>& t, const Ld& ld, int e, EdgeStat<T>& s) {
    // packed row {c0, c1, ep, the bits of 1/d_e in FP32}
    const int4 r = ld.stat(t.erow + e);
    s.c0 = r.x, s.c1 = r.y;
    const uint32_t pp = static_cast<uint32_t>(r.z);
    s.p0 = pp & 0xff, s.p1 = (pp >> 8) & 0xff;
    if constexpr (sizeof(T) == 4) s.rdc = __int_as_float(r.w);
    else s.rdc = ld.stat(t.rdc + e);
    s.db = ld.stat(t.db + e);
}

// U_e from the two ring shares, thicknesses (and compensation words) and
// kinetic energies of the edge's cells, with the roundings spelled out so
// the edge and fused-tile passes get the same bits.  h1 - h0 is
// exact for nearby thicknesses (Sterbenz); with COMP the compensation words
// restore the digits the FP32 thickness dropped.
template <class T, bool COMP>
__device__ __forceinline__ T edge_u(T C0, T C1, T h0, T h1, T hl0, T hl1, T K0, T K1, T db, T rdc, T g) {
    T dh = h1 - h0;
    if (COMP) dh += hl1 - hl0;
    const T grad = fma_rn(g, dh + db, K1 - K0);
    return -rdc * fma_rn(T(0.5), C1 - C0, grad);
}

// Gathers the two cells' ring results and thicknesses (after the wait) and
// returns U_e.
template <class T, bool COMP, bool LY>
__device__ __forceinline__ T edge_value(const DevArgs<T>& a, const Ld& ld, const EdgeStat<T>& s, const Lay<LY>& y) {
    const int N = a.t.nC;
    const T C0 = ld(a.ring_c + y(s.p0 * N + s.c0)), C1 = ld(a.ring_c + y(s.p1 * N + s.c1));
    const T h0 = ld(a.in_h + y(s.c0)), h1 = ld(a.in_h + y(s.c1));
    const T hl0 = COMP ? ld(a.in_hl + y(s.c0)) : T(0), hl1 = COMP ? ld(a.in_hl + y(s.c1)) : T(0);
    const T K0 = ld(a.ring_k + y(s.c0)), K1 = ld(a.ring_k + y(s.c1));
    return edge_u<T, COMP>(C0, C1, h0, h1, hl0, hl1, K0, K1, s.db, s.rdc, a.g);
}

template <class T, bool COMP, bool LY>
__device__ __forceinline__ T edge_tendency(const DevArgs<T>& a, int e, const DevSeg<T>& seg, int epi,
                                           EpiOps<T>& eo, const Lay<LY>& y) {
    const Ld ld(a.l2);
    EdgeStat<T> s;
    edge_stat(a.t, ld, e, s);
    griddep_wait();
    epi_load<T, COMP, LY>(ld, seg, epi, e, a.in_u, eo, y);
    return edge_value<T, COMP, LY>(a, ld, s, y);
}

template <class T, bool COMP, bool LY>
__device__ __forceinline__ void pointwise(const DevSeg<T>& s, int i, const Lay<LY>& y, const St& st);
template <class T>
__device__ __forceinline__ int find_seg(const DevArgs<T>& a, int blk);

// ----------------------------------------------------------- kind 3: tiles
//
// The fused right-hand side: one block per tile (a band-order range of
// cells inside one band, the edges whose lower cell it owns, a halo of the
// other cells of those edges, and every ring vertex of those cells).
//   pass 1: q_v of the tile's vertices            -> shared memory
//   pass 2: ring pass of own + halo cells         -> C_p, K_c in shared memory;
//           H_c with the stage update / accumulation for own cells
//   pass 3: U_e of the owned edges from shared C and K -> stage update / accumulation
// A vertex or halo cell shared by two tiles is evaluated by both from the
// same inputs with the same code, so the results are bit-identical to the
// three-launch path's.  No intermediate leaves the block.

template <class T>
__device__ __forceinline__ T vertex_value(const DevArgs<T>& a, const Ld& ld, int v) {
    const Tables<T>& t = a.t;
    const int e0 = ld.stat(t.ve0 + v), e1 = ld.stat(t.ve1 + v), e2 = ld.stat(t.ve2 + v);
    const int c0 = ld.stat(t.vc0 + v), c1 = ld.stat(t.vc1 + v), c2 = ld.stat(t.vc2 + v);
    const T d0 = ld.stat(t.vd0 + v), d1 = ld.stat(t.vd1 + v), d2 = ld.stat(t.vd2 + v);
    const T k0 = ld.stat(t.vk0 + v), k1 = ld.stat(t.vk1 + v), k2 = ld.stat(t.vk2 + v);
    const T f = ld.stat(t.f + v);
    const T u0 = ld(a.in_u + e0), u1 = ld(a.in_u + e1), u2 = ld(a.in_u + e2);
    const T h0 = ld(a.in_h + c0), h1 = ld(a.in_h + c1), h2 = ld(a.in_h + c2);
    return q_value(d0, d1, d2, u0, u1, u2, k0, k1, k2, h0, h1, h2, f);
}

// The ring pass of kind 1 with q read from shared memory (local vertex ids
// lsv) and C, K written to shared memory (slot-major over the local cells).
template <class T, bool COMP, int MAXR>
__device__ __forceinline__ T ring_local(const DevArgs<T>& a, const Ld& ld, int c, int k, int nl,
                                        const uint16_t* lsv, const T* q_s, T* rc_s, T* K_s) {
    const Tables<T>& t = a.t;
    const int N = t.nC;
    const int n = ld.stat(t.cn + c);
    const T hc = ld(a.in_h + c);
    T uj[MAXR], hn[MAXR], qv[MAXR], snl[MAXR], Rj[MAXR], sK[MAXR], C[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        if (j < UNCOND || j < n) {
            uj[j] = ld(a.in_u + ld.stat(t.se + j * N + c));
            hn[j] = ld(a.in_h + ld.stat(t.sn + j * N + c));
            qv[j] = q_s[lsv[j * nl + k]];
            snl[j] = ld.stat(t.snl + j * N + c);
            Rj[j] = ld.stat(t.sR + j * N + c);
            sK[j] = ld.stat(t.sK + j * N + c);
        } else {
            uj[j] = hn[j] = qv[j] = snl[j] = Rj[j] = sK[j] = T(0);
        }
    }
    T Kc;
    const T H = ring_core<T, COMP, MAXR>(n, hc, ld.stat(t.rA + c), uj, hn, qv, snl, Rj, sK, C, Kc);
#pragma unroll
    for (int p = 0; p < MAXR; ++p)
        if (p < n) rc_s[p * nl + k] = C[p];
    K_s[k] = Kc;
    return H;
}

// Stage update or accumulation with explicit arrays (fused kernel epilogue).
template <class T, bool COMP>
__device__ __forceinline__ void store_update(const T* oh, const T* ol, const T* xh, const T* xl,
                                             T* outh, T* outl, int i, T a_, T D, T R, bool cell,
                                             int* flag) {
    T yh, yl;
    combine<T, COMP>(oh[i], COMP ? ol[i] : T(0), xh[i], COMP ? xl[i] : T(0), a_, D, R, yh, yl);
    outh[i] = yh;
    if (COMP) outl[i] = yl;
    const bool ok = cell ? finite_pos(yh) : finite_val(yh);
    if (!ok) atomicOr(flag, cell ? 1 : 2);
}

template <class T, bool COMP, int MAXR>
__device__ __forceinline__ void tile_pass(const DevArgs<T>& a, const DevSeg<T>& s, int tile) {
    const Tables<T>& t = a.t;
    const Ld ld(a.l2);
    const int4 ta = t.ta[tile];
    const int4 tb = t.tbk[tile];
    const int c_begin = ta.x, nown = ta.y, halo_begin = ta.z, nl = ta.w;
    const int e_begin = tb.x, e_end = tb.y, v_begin = tb.z, nv = tb.w;
    const uint16_t* lsv = t.lsv + t.tlsv[tile];
    const bool acc = tile >= s.pad;   // tiles from s.pad on accumulate (Steps 3.x.2)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // guard: a tile that would not fit the launch's shared memory is skipped
    // and reported (flag bit 4) instead of touching memory it does not own
    const long need = static_cast<long>(sizeof(T)) * (((nv + 3) & ~3) + (MAXR + 1) * static_cast<long>(nl));
    if (need > a.smem) {
        if (threadIdx.x == 0) atomicOr(a.flag, 4);
        return;
    }
    T* q_s = reinterpret_cast<T*>(smem_raw);
    T* rc_s = q_s + ((nv + 3) & ~3);
    T* K_s = rc_s + MAXR * nl;
    griddep_wait();
    // pass 1: potential vorticity of the tile's vertices
    for (int k = threadIdx.x; k < nv; k += blockDim.x) q_s[k] = vertex_value(a, ld, t.tverts[v_begin + k]);
    __syncthreads();
    // pass 2: rings of own and halo cells; own cells get their update
    for (int k = threadIdx.x; k < nl; k += blockDim.x) {
        const int c = k < nown ? c_begin + k : t.halo[halo_begin + (k - nown)];
        const T H = ring_local<T, COMP, MAXR>(a, ld, c, k, nl, lsv, q_s, rc_s, K_s);
        if (k < nown) {
            if (acc) {
                T* ac = static_cast<T*>(s.p[8]);
                const int q = c - s.base;
                ac[q] = s.flag ? H : ac[q] + H;
            } else {
                store_update<T, COMP>((const T*)s.p[0], (const T*)s.p[1], a.in_h, a.in_hl, (T*)s.p[2],
                                      (T*)s.p[3], c, s.c[0], s.c[1], H, true, a.flag);
            }
        }
    }
    __syncthreads();
    // pass 3: owned edges
    const int N = t.nC;
    for (int e = e_begin + threadIdx.x; e < e_end; e += blockDim.x) {
        const uint32_t l = t.lec[e];
        const int l0 = l & 0xffff, l1 = l >> 16;
        const uint32_t pp = ld.stat(t.ep + e);
        const int p0 = pp & 0xff, p1 = (pp >> 8) & 0xff;
        const int c0 = ld.stat(t.ec0 + e), c1 = ld.stat(t.ec1 + e);
        const T C0 = rc_s[p0 * nl + l0], C1 = rc_s[p1 * nl + l1];
        const T h0 = ld(a.in_h + c0), h1 = ld(a.in_h + c1);
        const T hl0 = COMP ? ld(a.in_hl + c0) : T(0), hl1 = COMP ? ld(a.in_hl + c1) : T(0);
        const T U = edge_u<T, COMP>(C0, C1, h0, h1, hl0, hl1, K_s[l0], K_s[l1], ld.stat(t.db + e),
                                    ld.stat(t.rdc + e), a.g);
        if (acc) {
            T* ac = static_cast<T*>(s.p[9]);
            const int q = e - s.base2;
            ac[q] = s.flag ? U : ac[q] + U;
        } else {
            store_update<T, COMP>((const T*)s.p[4], (const T*)s.p[5], a.in_u, a.in_ul, (T*)s.p[6],
                                  (T*)s.p[7], e, s.c[0], s.c[1], U, false, a.flag);
        }
    }
    (void)N;
}

template <class T, bool COMP, int MAXR>
__global__ void __launch_bounds__(256) kernel_tiles(const __grid_constant__ DevArgs<T> a) {
    griddep_launch_dependents();
    const int sidx = find_seg(a, blockIdx.x);
    const DevSeg<T>& s = a.seg[sidx];
    if (s.type == SEG_TILE) {
        tile_pass<T, COMP, MAXR>(a, s, s.begin + (blockIdx.x - s.block0));
        return;
    }
    const int i = s.begin + (blockIdx.x - s.block0) * blockDim.x + threadIdx.x;
    if (i >= s.end) return;
    griddep_wait();
    pointwise<T, COMP, false>(s, i, Lay<false>{}, St(a.l2));
}

// ------------------------------------------------------------ pointwise parts

// The interface-1 prediction of element i of a SEG_PRED segment.
template <class T, bool COMP, bool LY>
__device__ __forceinline__ void pred_at(const DevSeg<T>& s, int i, const Lay<LY>& y, T& yh, T& yl) {
    const T* oh = (const T*)s.p[0];
    const T* ol = (const T*)s.p[1];
    const T* x1h = (const T*)s.p[2];
    const T* x1l = (const T*)s.p[3];
    const T* x2h = (const T*)s.p[4];
    const T* x2l = (const T*)s.p[5];
    const auto ii = y(i), k = y(i - s.base), k2 = y(i - s.base2);
    predict<T, COMP>(oh[ii], COMP ? ol[ii] : T(0), x1h[k], COMP ? x1l[k] : T(0), x2h[k2],
                     COMP ? x2l[k2] : T(0), s.c[0], s.c[1], s.flag, yh, yl);
}

template <class T, bool COMP, bool LY>
__device__ __forceinline__ void pointwise(const DevSeg<T>& s, int i, const Lay<LY>& y, const St& st) {
    if (s.type == SEG_PRED) {
        T* outh = (T*)s.p[6];
        T* outl = (T*)s.p[7];
        const auto ii = y(i);
        T yh, yl;
        pred_at<T, COMP, LY>(s, i, y, yh, yl);
        st(outh + ii, yh);
        if (COMP) st(outl + ii, yl);
    } else if (s.type == SEG_COPY) {
        const T* sh = (const T*)s.p[0];
        const T* sl = (const T*)s.p[1];
        T* dh = (T*)s.p[2];
        T* dl = (T*)s.p[3];
        st(dh + y(i - s.base), sh[y(i - s.base2)]);
        if (COMP) st(dl + y(i - s.base), sl[y(i - s.base2)]);
    } else if (s.type == SEG_REPLAY) {
        // Step 5 as the replay of the interface stages (reading R5): three
        // stages for LTS3, two for LTS2 (flag 2: x_new = x2).
        const T* oh = (const T*)s.p[0];
        const T* ol = (const T*)s.p[1];
        const T* a1 = (const T*)s.p[2];
        const T* a2 = (const T*)s.p[3];
        T* outh = (T*)s.p[5];
        T* outl = (T*)s.p[6];
        const auto ii = y(i), k = y(i - s.base);
        const T xh = oh[ii], xl = COMP ? ol[ii] : T(0);
        T x1h, x1l, x2h, x2l, yh, yl;
        combine<T, COMP>(xh, xl, xh, xl, T(0), s.c[0], a1[k], x1h, x1l);
        combine<T, COMP>(xh, xl, x1h, x1l, s.c[3], s.c[1], a2[k], x2h, x2l);
        if (s.flag == 2) {
            yh = x2h;
            yl = x2l;
        } else {
            const T* a3 = (const T*)s.p[4];
            combine<T, COMP>(xh, xl, x2h, x2l, s.c[4], s.c[2], a3[k], yh, yl);
        }
        st(outh + ii, yh);
        if (COMP) st(outl + ii, yl);
    }
}

// Stage update (UPD) or correction accumulation (ACC) of a cell or edge
// value from the operands epi_load fetched.
template <class T, bool COMP, bool IS_CELL, bool LY>
__device__ __forceinline__ void epilogue(const DevArgs<T>& a, const DevSeg<T>& s, int epi, int i, T R,
                                         const EpiOps<T>& o, const Lay<LY>& y) {
    const St st(a.l2);
    if (epi == EPI_ACC) {
        T* acc = (T*)s.p[0];
        st(acc + y(i - s.base), s.flag ? R : o.oh + R);
        return;
    }
    T* outh = (T*)s.p[3];
    T* outl = (T*)s.p[4];
    T yh, yl;
    combine<T, COMP>(o.oh, o.ol, o.xh, o.xl, s.c[0], s.c[1], R, yh, yl);
    st(outh + y(i), yh);
    if (COMP) st(outl + y(i), yl);
    const bool ok = IS_CELL ? finite_pos(yh) : finite_val(yh);
    if (!ok) atomicOr(a.flag, IS_CELL ? 1 : 2);
}

// The epilogue of W consecutive layers (y.l .. y.l + W - 1): each layer's
// arithmetic is the single-layer epilogue's, the stores one access per array.
template <class T, bool COMP, bool IS_CELL, int W>
__device__ __forceinline__ void epilogue_group(const DevArgs<T>& a, const DevSeg<T>& s, int epi, int i,
                                               const T (&R)[W], const EpiOps<T> (&o)[W], const Lay<true>& y) {
    const St st(a.l2);
    if (epi == EPI_ACC) {
        Lanes<T, W> v;
#pragma unroll
        for (int k = 0; k < W; ++k) v.v[k] = s.flag ? R[k] : o[k].oh + R[k];
        st.lanes<W>((T*)s.p[0] + y(i - s.base), v);
        return;
    }
    Lanes<T, W> yh, yl;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        combine<T, COMP>(o[k].oh, o[k].ol, o[k].xh, o[k].xl, s.c[0], s.c[1], R[k], yh.v[k], yl.v[k]);
        ok = ok && (IS_CELL ? finite_pos(yh.v[k]) : finite_val(yh.v[k]));
    }
    st.lanes<W>((T*)s.p[3] + y(i), yh);
    if (COMP) st.lanes<W>((T*)s.p[4] + y(i), yl);
    if (!ok) atomicOr(a.flag, IS_CELL ? 1 : 2);
}

template <class T>
__device__ __forceinline__ int find_seg(const DevArgs<T>& a, int blk) {
    int s = 0;
#pragma unroll
    for (int k = 1; k < MAXSEG; ++k)
        if (k < a.nseg && blk >= a.seg[k].block0) s = k;
    return s;
}


__device__ __forceinline__ bool is_ring(int type) {
    return type == SEG_RING || type == SEG_RING_UPD || type == SEG_RING_ACC;
}

// The work of element i (one layer, y) of segment s.
template <class T, bool COMP, int MAXR, int KIND, bool LY>
__device__ __forceinline__ void element_work(const DevArgs<T>& a, const DevSeg<T>& s, int i, const Lay<LY>& y) {
    const int type = s.type;
    if (KIND == 0 && type == SEG_VERT) {
        vertex_pv<T, LY>(a, i, y);
    } else if (KIND == 1 && is_ring(type)) {
        // the cell update's operands are loaded after the ring (the ring pass
        // holds ~40 registers; loading them earlier costs a resident block)
        const int epi = type == SEG_RING ? EPI_NONE : type == SEG_RING_ACC ? EPI_ACC : EPI_UPD;
        const T H = ring_pass<T, COMP, MAXR, LY>(a, i, y);
        if (epi != EPI_NONE) {
            EpiOps<T> o;
            epi_load<T, COMP, LY>(Ld(a.l2), s, epi, i, a.in_h, o, y);
            epilogue<T, COMP, true, LY>(a, s, epi, i, H, o, y);
        }
    } else if (KIND == 2 && (type == SEG_EDGE_UPD || type == SEG_EDGE_ACC)) {
        const int epi = type == SEG_EDGE_ACC ? EPI_ACC : EPI_UPD;
        EpiOps<T> o;
        const T U = edge_tendency<T, COMP, LY>(a, i, s, epi, o, y);
        epilogue<T, COMP, false, LY>(a, s, epi, i, U, o, y);
    } else {
        griddep_wait();
        pointwise<T, COMP, LY>(s, i, y, St(a.l2));
    }
}

// Vertex and edge work of W consecutive layers (y.l .. y.l + W - 1) of a
// multi-layer state: each state word is one aligned W-word access for all
// W layers, all of them out before any layer's arithmetic, so the group
// costs one dependent round trip and one set of table loads; each layer's
// arithmetic is the single-layer code's.
template <class T, bool COMP, int KIND, int W>
__device__ __forceinline__ void group_work(const DevArgs<T>& a, const DevSeg<T>& s, int i, const Lay<true>& y0) {
    using G = Lanes<T, W>;
    const Ld ld(a.l2);
    if (KIND == 0) {
        VertStat<T> vs;
        vertex_stat(a.t, ld, i, vs);
        griddep_wait();
        const G u0 = ld.lanes<W>(a.in_u + y0(vs.e0)), u1 = ld.lanes<W>(a.in_u + y0(vs.e1)),
                u2 = ld.lanes<W>(a.in_u + y0(vs.e2));
        const G h0 = ld.lanes<W>(a.in_h + y0(vs.c0)), h1 = ld.lanes<W>(a.in_h + y0(vs.c1)),
                h2 = ld.lanes<W>(a.in_h + y0(vs.c2));
        G q;
#pragma unroll
        for (int k = 0; k < W; ++k)
            q.v[k] = q_value(vs.d0, vs.d1, vs.d2, u0.v[k], u1.v[k], u2.v[k], vs.k0, vs.k1, vs.k2, h0.v[k], h1.v[k],
                             h2.v[k], vs.f);
        St(a.l2).lanes<W>(a.q + y0(i), q);
    } else {
        const int epi = s.type == SEG_EDGE_ACC ? EPI_ACC : EPI_UPD;
        EdgeStat<T> es;
        edge_stat(a.t, ld, i, es);
        griddep_wait();
        EpiOps<T> o[W];
        epi_load_group<T, COMP, W>(ld, s, epi, i, a.in_u, o, y0);
        const int N = a.t.nC;
        const G C0 = ld.lanes<W>(a.ring_c + y0(es.p0 * N + es.c0)), C1 = ld.lanes<W>(a.ring_c + y0(es.p1 * N + es.c1));
        const G h0 = ld.lanes<W>(a.in_h + y0(es.c0)), h1 = ld.lanes<W>(a.in_h + y0(es.c1));
        G hl0, hl1;
        if (COMP) {
            hl0 = ld.lanes<W>(a.in_hl + y0(es.c0));
            hl1 = ld.lanes<W>(a.in_hl + y0(es.c1));
        } else {
#pragma unroll
            for (int k = 0; k < W; ++k) hl0.v[k] = hl1.v[k] = T(0);
        }
        const G K0 = ld.lanes<W>(a.ring_k + y0(es.c0)), K1 = ld.lanes<W>(a.ring_k + y0(es.c1));
        T U[W];
#pragma unroll
        for (int k = 0; k < W; ++k)
            U[k] = edge_u<T, COMP>(C0.v[k], C1.v[k], h0.v[k], h1.v[k], hl0.v[k], hl1.v[k], K0.v[k], K1.v[k], es.db,
                                   es.rdc, a.g);
        epilogue_group<T, COMP, false, W>(a, s, epi, i, U, o, y0);
    }
}

// The work of (virtual) block `vblk` of segment s.  Multi-layer states run
// one thread per (element, group of lpt consecutive layers), groups fastest.
// Where the host found the groups aligned, the thread runs its layers two
// or four at a time (vertex and edge kinds) or two at a time (FP32 ring),
// each state word one aligned vector access and the mesh table loads issued
// once per pass; otherwise it repeats the single-layer work for each layer.
// Each layer's arithmetic is the single-layer code's.
template <class T, bool COMP, int MAXR, int KIND, bool LY>
__device__ __forceinline__ void phase_block(const DevArgs<T>& a, const DevSeg<T>& s, int vblk) {
    const int local = (vblk - s.block0) * blockDim.x + threadIdx.x;
    if constexpr (LY) {
        const int q = local / a.G;
        const int i = s.begin + q;
        if (i >= s.end) return;
        const int l0 = (local - q * a.G) * a.lpt;
        const int nl = min(a.lpt, a.L - l0);
        Lay<true> y;
        y.L = a.L;
        int k = 0;
        // pairs of layers only where the host found every pair aligned
        // (otherwise each layer runs the single-layer code, the same bits)
        if constexpr (KIND == 1 && sizeof(T) == 4) {
            // FP32 ring segments: two layers per ring pass (packed arithmetic)
            if (a.v2 && is_ring(s.type)) {
                const int epi = s.type == SEG_RING ? EPI_NONE : s.type == SEG_RING_ACC ? EPI_ACC : EPI_UPD;
#pragma unroll 1
                for (; k + 1 < nl; k += 2) {
                    y.l = l0 + k;
                    EpiOps<T> o[2];
                    const float2 H = ring_pass_pair<COMP, MAXR>(a, s, epi, i, y, o);
                    if (epi != EPI_NONE) {
                        const T R[2] = {H.x, H.y};
                        epilogue_group<T, COMP, true, 2>(a, s, epi, i, R, o, y);
                    }
                }
            }
        }
        if constexpr (KIND == 0 || KIND == 2) {
            if (a.v2 && ((KIND == 0 && s.type == SEG_VERT) ||
                         (KIND == 2 && (s.type == SEG_EDGE_UPD || s.type == SEG_EDGE_ACC)))) {
                if constexpr (sizeof(T) == 4) {
                    // four layers in one pass where the host found every
                    // group of four aligned
                    if (a.v4 && nl == 4) {
                        y.l = l0;
                        group_work<T, COMP, KIND, 4>(a, s, i, y);
                        k = 4;
                    }
                }
#pragma unroll 1
                for (; k + 1 < nl; k += 2) {
                    y.l = l0 + k;
                    group_work<T, COMP, KIND, 2>(a, s, i, y);
                }
            }
        }
#pragma unroll 1
        for (; k < nl; ++k) {
            y.l = l0 + k;
            element_work<T, COMP, MAXR, KIND, true>(a, s, i, y);
        }
    } else {
        const int i = s.begin + local;
        if (i >= s.end) return;
        element_work<T, COMP, MAXR, KIND, false>(a, s, i, Lay<false>{});
    }
}

// Resident 256-thread blocks per SM the ring kind is compiled for.  FP32
// single-layer: four (64 registers), which on GB300 beat both five blocks
// (48 registers, with spills) and no limit (80 registers, three blocks) on
// the 655k-cell cap mesh.  Multi-layer states (two layers per ring pass in
// FP32) and FP64: two (up to 128 registers, no spills); their launches run
// many waves, so fewer resident blocks cost little.
template <class T, bool LY>
constexpr int ring_min_blocks() { return (LY || sizeof(T) == 8) ? 2 : 4; }

template <class T, bool COMP, int MAXR, int KIND, bool LY = false>
__global__ void __launch_bounds__(256, (KIND == 1 ? ring_min_blocks<T, LY>() : 1))
    kernel_phase(const __grid_constant__ DevArgs<T> a) {
    griddep_launch_dependents();
    const int sidx = find_seg(a, blockIdx.x);
    phase_block<T, COMP, MAXR, KIND, LY>(a, a.seg[sidx], blockIdx.x);
}

// Two elements per thread (vertex and edge kinds, single-layer states):
// thread t of block b of a segment handles elements 2 b blockDim + t and
// that + blockDim, with the table loads of both before the dependency wait
// and the gathers of both in flight before either value is formed.  Half the
// blocks, so a fine-region launch fits in one wave; each element's
// arithmetic is the one-element code's, so results are bit-identical.
template <class T, bool COMP, int KIND>
__device__ __forceinline__ void phase_block2(const DevArgs<T>& a, const DevSeg<T>& s, int vblk) {
    const int bd = static_cast<int>(blockDim.x);
    const int i0 = s.begin + (vblk - s.block0) * 2 * bd + static_cast<int>(threadIdx.x);
    if (i0 >= s.end) return;
    const bool two = i0 + bd < s.end;
    const int i1 = two ? i0 + bd : i0;   // a lone element repeats its loads and stores once
    const Lay<false> y;
    const Ld ld(a.l2);
    if (KIND == 0 && s.type == SEG_VERT) {
        VertStat<T> s0, s1;
        vertex_stat(a.t, ld, i0, s0);
        vertex_stat(a.t, ld, i1, s1);
        griddep_wait();
        const T q0 = vertex_q<T, false>(a, ld, s0, y);
        const T q1 = vertex_q<T, false>(a, ld, s1, y);
        a.q[i0] = q0;
        if (two) a.q[i1] = q1;
    } else if (KIND == 2 && (s.type == SEG_EDGE_UPD || s.type == SEG_EDGE_ACC)) {
        const int epi = s.type == SEG_EDGE_ACC ? EPI_ACC : EPI_UPD;
        EdgeStat<T> s0, s1;
        edge_stat(a.t, ld, i0, s0);
        edge_stat(a.t, ld, i1, s1);
        griddep_wait();
        EpiOps<T> o0, o1;
        epi_load<T, COMP, false>(ld, s, epi, i0, a.in_u, o0, y);
        epi_load<T, COMP, false>(ld, s, epi, i1, a.in_u, o1, y);
        const T U0 = edge_value<T, COMP, false>(a, ld, s0, y);
        const T U1 = edge_value<T, COMP, false>(a, ld, s1, y);
        epilogue<T, COMP, false, false>(a, s, epi, i0, U0, o0, y);
        if (two) epilogue<T, COMP, false, false>(a, s, epi, i1, U1, o1, y);
    } else {
        griddep_wait();
        pointwise<T, COMP, false>(s, i0, y, St(a.l2));
        if (two) pointwise<T, COMP, false>(s, i1, y, St(a.l2));
    }
}

template <class T, bool COMP, int KIND>
__global__ void __launch_bounds__(256) kernel_phase2(const __grid_constant__ DevArgs<T> a) {
    griddep_launch_dependents();
    const int sidx = find_seg(a, blockIdx.x);
    phase_block2<T, COMP, KIND>(a, a.seg[sidx], blockIdx.x);
}

// The FP32 ring pass compiled for MINB resident 256-thread blocks per SM
// (fewer registers, possibly spills): a fine-region launch then leaves block
// slots free, where the next launch's blocks prefetch their tables.
template <bool COMP, int MINB>
__global__ void __launch_bounds__(256, MINB) kernel_ring_occ(const __grid_constant__ DevArgs<float> a) {
    griddep_launch_dependents();
    const int sidx = find_seg(a, blockIdx.x);
    phase_block<float, COMP, 8, 1, false>(a, a.seg[sidx], blockIdx.x);
}

// Segment-table variant (ensembles of meshes, and states with several fine
// regions: one launch carries more segments than fit in the kernel
// parameters).  Each virtual block finds its segment by a binary search over
// the segments' first virtual block.
template <class T>
__device__ __forceinline__ int find_gseg(const DevArgs<T>& a, int vblk) {
    int lo = 0, hi = a.ngseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.gseg[mid].block0 <= vblk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// PERSIST: a grid of resident blocks walks the virtual blocks in turn;
// otherwise one block per virtual block.  The loop keeps loop-invariant
// values live across its iterations (the persistent ring takes about 110
// registers uncapped and spills under the cap), so the one-shot form is the
// one that compiles like kernel_phase.
template <class T, bool COMP, int MAXR, int KIND, bool PERSIST>
__global__ void __launch_bounds__(256, (KIND == 1 ? ring_min_blocks<T, false>() : 1))
    kernel_phase_table(const __grid_constant__ DevArgs<T> a) {
    griddep_launch_dependents();
    if (PERSIST) {
        for (int vb = blockIdx.x; vb < a.vblocks; vb += gridDim.x)
            phase_block<T, COMP, MAXR, KIND, false>(a, a.gseg[find_gseg(a, vb)], vb);
    } else {
        const int vb = blockIdx.x;
        phase_block<T, COMP, MAXR, KIND, false>(a, a.gseg[find_gseg(a, vb)], vb);
    }
}

template <class K, class A>
cudaError_t launch_kernel(K kernel, int blocks, int block, bool pdl, cudaStream_t st, const A& a,
                          int smem = 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <class T>
DevSeg<T> to_dev(const SegDesc& s, int block0) {
    DevSeg<T> o;
    o.type = s.type;
    o.begin = s.begin;
    o.end = s.end;
    o.base = s.base;
    o.base2 = s.base2;
    o.flag = s.flag;
    o.block0 = block0;
    o.pad = s.type == SEG_TILE ? s.flag2 : 0;
    for (int m = 0; m < 6; ++m) o.c[m] = static_cast<T>(m < 4 ? s.c[m] : 0.0);
    if (s.type == SEG_REPLAY) {   // the weights a of the replayed stages 2 and 3
        o.c[3] = static_cast<T>(s.flag == 2 ? 0.5 : 0.75);
        o.c[4] = static_cast<T>(1.0 / 3.0);
    }
    for (int m = 0; m < 10; ++m) o.p[m] = s.p[m];
    return o;
}

inline int seg_blocks(const SegDesc& s, int block, int layers = 1) {
    return s.type == SEG_TILE ? s.end - s.begin              // one block per tile
                              : static_cast<int>((static_cast<long long>(s.end - s.begin) * layers + block - 1) / block);
}

template <class T>
void fill_args(DevArgs<T>& a, const LaunchDesc& d, const void* tables, int smem, int* flag) {
    a.t = *static_cast<const Tables<T>*>(tables);
    a.in_h = static_cast<const T*>(d.in_h);
    a.in_hl = static_cast<const T*>(d.in_hl);
    a.in_u = static_cast<const T*>(d.in_u);
    a.in_ul = static_cast<const T*>(d.in_ul);
    a.q = static_cast<T*>(d.q);
    a.ring_c = static_cast<T*>(d.ring_c);
    a.ring_k = static_cast<T*>(d.ring_k);
    a.g = static_cast<T>(d.g);
    a.flag = flag;
    a.l2 = d.l2;
    a.smem = smem;
    a.lpt = 1;
    a.G = 1;
    a.v2 = 0;
    a.v4 = 0;
    a.gseg = nullptr;
    a.ngseg = 0;
    a.vblocks = 0;
    a.L = 1;
}

// Multi-layer launches: W consecutive layers (l .. l + W - 1) of element x
// sit at words x L + l .. x L + l + W - 1.  With L and every group's first
// layer multiples of W (L and the layers per thread multiples of W) and
// every array the launch touches aligned to W words, each group is one
// aligned W-word access.
template <class T>
bool groups_aligned(const DevArgs<T>& a, const LaunchDesc& d, int W) {
    if (a.L < W || a.L % W || a.lpt % W) return false;
    const uintptr_t bytes = static_cast<uintptr_t>(W) * sizeof(T);
    auto ok = [bytes](const void* p) { return (reinterpret_cast<uintptr_t>(p) % bytes) == 0; };
    if (!ok(a.in_h) || !ok(a.in_hl) || !ok(a.in_u) || !ok(a.in_ul) || !ok(a.q) || !ok(a.ring_c) || !ok(a.ring_k))
        return false;
    for (int k = 0; k < d.nseg; ++k)
        for (int m = 0; m < 10; ++m)
            if (!ok(d.seg[k].p[m])) return false;
    return true;
}

// A table set without the packed rows a launch kind reads (the ring pass's
// slot rows, the vertex and edge passes' rows) cannot run that kind:
// refused on the host instead of faulting on the device.
template <class T>
bool tables_ok(const Tables<T>& t, int kind) {
    if (kind == 0) return t.vri != nullptr && (sizeof(T) != 4 || (t.vrd != nullptr && t.vrk != nullptr));
    if (kind == 2) return t.erow != nullptr;
    if (kind != 1) return true;
    return t.sidx != nullptr && (sizeof(T) != 4 || t.scf != nullptr);
}

template <class T, bool COMP, int MAXR>
cudaError_t launch_t(const LaunchDesc& d, const void* tables, int block, bool pdl, int smem, int* flag,
                     cudaStream_t st, int layers, int ring_occ, int ept, int lpt) {
    if (!tables_ok(*static_cast<const Tables<T>*>(tables), d.kind)) return cudaErrorInvalidValue;
    DevArgs<T> a;
    fill_args(a, d, tables, smem, flag);
    a.L = layers;
    a.lpt = layers > 1 ? std::max(1, std::min(lpt, layers)) : 1;
    a.G = (layers + a.lpt - 1) / a.lpt;
    a.v2 = groups_aligned(a, d, 2) ? 1 : 0;
    a.v4 = sizeof(T) == 4 && groups_aligned(a, d, 4) ? 1 : 0;
    const bool two = ept == 2 && layers == 1 && (d.kind == 0 || d.kind == 2);
    int blocks = 0, ns = 0;
    for (int k = 0; k < d.nseg; ++k) {
        const SegDesc& s = d.seg[k];
        if (s.end <= s.begin) continue;
        a.seg[ns++] = to_dev<T>(s, blocks);
        blocks += seg_blocks(s, two ? 2 * block : block, a.G);
    }
    a.nseg = ns;
    for (int k = ns; k < MAXSEG; ++k) {
        a.seg[k] = a.seg[0];
        a.seg[k].block0 = 0x7fffffff;
    }
    if (blocks == 0) return cudaSuccess;
    if (d.kind == 3) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kernel_tiles<T, COMP, MAXR>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        return launch_kernel(kernel_tiles<T, COMP, MAXR>, blocks, block, pdl, st, a, smem);
    }
    if (layers > 1) {
        switch (d.kind) {
            case 0: return launch_kernel(kernel_phase<T, COMP, MAXR, 0, true>, blocks, block, pdl, st, a);
            case 1: return launch_kernel(kernel_phase<T, COMP, MAXR, 1, true>, blocks, block, pdl, st, a);
            default: return launch_kernel(kernel_phase<T, COMP, MAXR, 2, true>, blocks, block, pdl, st, a);
        }
    }
    if (two)
        return d.kind == 0 ? launch_kernel(kernel_phase2<T, COMP, 0>, blocks, block, pdl, st, a)
                           : launch_kernel(kernel_phase2<T, COMP, 2>, blocks, block, pdl, st, a);
    if constexpr (sizeof(T) == 4 && MAXR == 8) {
        if (d.kind == 1 && ring_occ == 6) return launch_kernel(kernel_ring_occ<COMP, 6>, blocks, block, pdl, st, a);
        if (d.kind == 1 && ring_occ == 8) return launch_kernel(kernel_ring_occ<COMP, 8>, blocks, block, pdl, st, a);
    }
    switch (d.kind) {
        case 0: return launch_kernel(kernel_phase<T, COMP, MAXR, 0>, blocks, block, pdl, st, a);
        case 1: return launch_kernel(kernel_phase<T, COMP, MAXR, 1>, blocks, block, pdl, st, a);
        default: return launch_kernel(kernel_phase<T, COMP, MAXR, 2>, blocks, block, pdl, st, a);
    }
}

template <class T, bool COMP, int MAXR>
cudaError_t launch_table_t(const LaunchDesc& d, const void* dsegs, int nseg, int vblocks, int grid,
                           const void* tables, int block, bool pdl, int* flag, cudaStream_t st) {
    if (!tables_ok(*static_cast<const Tables<T>*>(tables), d.kind)) return cudaErrorInvalidValue;
    DevArgs<T> a;
    fill_args(a, d, tables, 0, flag);
    a.nseg = 0;
    for (int k = 0; k < MAXSEG; ++k) a.seg[k] = DevSeg<T>{};
    a.gseg = static_cast<const DevSeg<T>*>(dsegs);
    a.ngseg = nseg;
    a.vblocks = vblocks;
    if (vblocks == 0 || nseg == 0) return cudaSuccess;
    if (grid > 0 && grid < vblocks) {
        switch (d.kind) {
            case 0: return launch_kernel(kernel_phase_table<T, COMP, MAXR, 0, true>, grid, block, pdl, st, a);
            case 1: return launch_kernel(kernel_phase_table<T, COMP, MAXR, 1, true>, grid, block, pdl, st, a);
            case 2: return launch_kernel(kernel_phase_table<T, COMP, MAXR, 2, true>, grid, block, pdl, st, a);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (d.kind) {   // the grid covers every virtual block: one block each
        case 0: return launch_kernel(kernel_phase_table<T, COMP, MAXR, 0, false>, vblocks, block, pdl, st, a);
        case 1: return launch_kernel(kernel_phase_table<T, COMP, MAXR, 1, false>, vblocks, block, pdl, st, a);
        case 2: return launch_kernel(kernel_phase_table<T, COMP, MAXR, 2, false>, vblocks, block, pdl, st, a);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------ state I/O

// State I/O: host arrays are [layer][element] in the caller's order, device
// arrays [element * L + layer] in band order (L = 1: a plain permutation).
template <class T, bool COMP>
__global__ void scatter_kernel(int n, int L, const int* perm, const double* src, T* hi, T* lo) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<long long>(n) * L) return;
    const int e = static_cast<int>(i / L), l = static_cast<int>(i - static_cast<long long>(e) * L);
    double x = src[static_cast<long long>(l) * n + perm[e]];
    T h = static_cast<T>(x);
    hi[i] = h;
    if (COMP) lo[i] = static_cast<T>(x - static_cast<double>(h));
}

// snap (may be null): the same FP64 values in band order, for diagnostics
// that run beside the following steps
template <class T, bool COMP>
__global__ void gather_kernel(int n, int L, const int* perm, const T* hi, const T* lo, double* dst,
                              double* snap) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<long long>(n) * L) return;
    const int e = static_cast<int>(i / L), l = static_cast<int>(i - static_cast<long long>(e) * L);
    double x = static_cast<double>(hi[i]);
    if (COMP) x += static_cast<double>(lo[i]);
    dst[static_cast<long long>(l) * n + perm[e]] = x;
    if (snap) snap[i] = x;
}

// ------------------------------------------------------------ FP64 diagnostics
// mass = sum A_i h_i, energy = sum A_i h_i (K_i + g (h_i/2 + b_i)), FP64,
// fixed blocking and a fixed-order tree, so the result is deterministic.
constexpr int DIAG_THREADS = 256;

// (summed over the layers of a multi-layer state: element-major, layers
// innermost)
// TT: the tables' precision; TS: the state's (FP64 for a band-order
// snapshot of an FP32 state, which gives the same values as the state)
template <class TT, class TS, bool COMP>
__global__ void __launch_bounds__(DIAG_THREADS) diag_kernel(const Tables<TT> t, const TS* hh, const TS* hl,
                                                           const TS* uh, const TS* ul, double g,
                                                           double* partial, int L) {
    __shared__ double sm[2][DIAG_THREADS];
    const int N = t.nC;
    const long long NL = static_cast<long long>(N) * L;
    double m = 0.0, en = 0.0;
    for (long long x = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; x < NL;
         x += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(x / L), l = static_cast<int>(x - static_cast<long long>(c) * L);
        double h = static_cast<double>(hh[x]) + (COMP ? static_cast<double>(hl[x]) : 0.0);
        const int n = t.cn[c];
        double K = 0.0;
        // the first 8 slots unrolled, so their index loads and gathers are in
        // flight together; higher degrees continue in order
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < n) {
                const long long e = static_cast<long long>(t.se[j * N + c]) * L + l;
                double u = static_cast<double>(uh[e]) + (COMP ? static_cast<double>(ul[e]) : 0.0);
                K += t.sK64[j * N + c] * u * u;
            }
        }
        for (int j = 8; j < n; ++j) {
            const long long e = static_cast<long long>(t.se[j * N + c]) * L + l;
            double u = static_cast<double>(uh[e]) + (COMP ? static_cast<double>(ul[e]) : 0.0);
            K += t.sK64[j * N + c] * u * u;
        }
        double A = t.area[c];
        m += A * h;
        en += A * h * (K + g * (0.5 * h + t.bd[c]));
    }
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = en;
    __syncthreads();
    for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sm[0][0];
        partial[2 * blockIdx.x + 1] = sm[1][0];
    }
}

// Second stage: one block sums the per-block partials in a fixed-order tree.
__global__ void __launch_bounds__(DIAG_THREADS) diag_final(const double* partial, int nb, double* out) {
    __shared__ double sm[2][DIAG_THREADS];
    double m = 0.0, en = 0.0;
    for (int b = threadIdx.x; b < nb; b += DIAG_THREADS) {
        m += partial[2 * b];
        en += partial[2 * b + 1];
    }
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = en;
    __syncthreads();
    for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sm[0][0];
        out[1] = sm[1][0];
    }
}

template <class T, bool COMP>
cudaError_t launch_any(const LaunchDesc& d, const void* tables, const KernelConfig& kc, int* flag,
                       cudaStream_t s) {
    const int L = kc.layers > 1 ? kc.layers : 1;
    if (kc.maxdeg <= 8)
        return launch_t<T, COMP, 8>(d, tables, kc.block, kc.pdl, kc.tile_smem, flag, s, L, kc.ring_occ, kc.ept,
                                    kc.lpt);
    return launch_t<T, COMP, MAX_DEGREE>(d, tables, kc.block, kc.pdl, kc.tile_smem, flag, s, L, 0, kc.ept,
                                         kc.lpt);
}

}  // namespace

cudaError_t launch_phase(const LaunchDesc& d, const void* tables, const KernelConfig& kc, int* flag,
                         cudaStream_t s) {
    if (kc.precision == 1) return launch_any<double, false>(d, tables, kc, flag, s);
    if (kc.comp) return launch_any<float, true>(d, tables, kc, flag, s);
    return launch_any<float, false>(d, tables, kc, flag, s);
}

namespace {
template <class T, bool COMP>
cudaError_t launch_table_any(const LaunchDesc& d, const void* dsegs, int nseg, int vblocks, int grid,
                             const void* tables, const KernelConfig& kc, int* flag, cudaStream_t s) {
    if (kc.maxdeg <= 8)
        return launch_table_t<T, COMP, 8>(d, dsegs, nseg, vblocks, grid, tables, kc.block, kc.pdl, flag, s);
    return launch_table_t<T, COMP, MAX_DEGREE>(d, dsegs, nseg, vblocks, grid, tables, kc.block, kc.pdl,
                                               flag, s);
}

template <class T>
int encode_t(const SegDesc* segs, int n, int block, std::vector<unsigned char>& out, int* nout) {
    std::vector<DevSeg<T>> v;
    int blocks = 0;
    for (int k = 0; k < n; ++k) {
        const SegDesc& s = segs[k];
        if (s.end <= s.begin) continue;
        if (s.type == SEG_TILE) return -1;
        v.push_back(to_dev<T>(s, blocks));
        blocks += seg_blocks(s, block);
    }
    out.resize(v.size() * sizeof(DevSeg<T>));
    if (!v.empty()) std::memcpy(out.data(), v.data(), out.size());
    *nout = static_cast<int>(v.size());
    return blocks;
}

template <class T, bool COMP, int MAXR>
int table_occupancy_t(int kind, int block) {
    int nb = 0;
    cudaError_t e = kind == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_phase_table<T, COMP, MAXR, 0, true>, block, 0)
                    : kind == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_phase_table<T, COMP, MAXR, 1, true>, block, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_phase_table<T, COMP, MAXR, 2, true>, block, 0);
    return e == cudaSuccess ? nb : -1;
}
}  // namespace

int encode_segment_table(const KernelConfig& kc, const SegDesc* segs, int n,
                         std::vector<unsigned char>& out, int* nseg_out) {
    if (kc.precision == 1) return encode_t<double>(segs, n, kc.block, out, nseg_out);
    return encode_t<float>(segs, n, kc.block, out, nseg_out);
}

cudaError_t launch_phase_table(const LaunchDesc& d, const void* dsegs, int nseg, int vblocks, int grid,
                               const void* tables, const KernelConfig& kc, int* flag, cudaStream_t s) {
    if (kc.precision == 1) return launch_table_any<double, false>(d, dsegs, nseg, vblocks, grid, tables, kc, flag, s);
    if (kc.comp) return launch_table_any<float, true>(d, dsegs, nseg, vblocks, grid, tables, kc, flag, s);
    return launch_table_any<float, false>(d, dsegs, nseg, vblocks, grid, tables, kc, flag, s);
}

int table_blocks_per_sm(const KernelConfig& kc, int kind) {
    const bool big = kc.maxdeg > 8;
    if (kc.precision == 1)
        return big ? table_occupancy_t<double, false, 16>(kind, kc.block) : table_occupancy_t<double, false, 8>(kind, kc.block);
    if (kc.comp)
        return big ? table_occupancy_t<float, true, 16>(kind, kc.block) : table_occupancy_t<float, true, 8>(kind, kc.block);
    return big ? table_occupancy_t<float, false, 16>(kind, kc.block) : table_occupancy_t<float, false, 8>(kind, kc.block);
}

cudaError_t launch_scatter_state(const KernelConfig& kc, int n, const int* perm, const double* src,
                                 void* hi, void* lo, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int L = kc.layers > 1 ? kc.layers : 1;
    const int b = 256;
    const long long g = (static_cast<long long>(n) * L + b - 1) / b;
    if (kc.precision == 1)
        scatter_kernel<double, false><<<g, b, 0, s>>>(n, L, perm, src, (double*)hi, nullptr);
    else if (kc.comp)
        scatter_kernel<float, true><<<g, b, 0, s>>>(n, L, perm, src, (float*)hi, (float*)lo);
    else
        scatter_kernel<float, false><<<g, b, 0, s>>>(n, L, perm, src, (float*)hi, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_gather_state(const KernelConfig& kc, int n, const int* perm, const void* hi,
                                const void* lo, double* dst, cudaStream_t s, double* snap) {
    if (n <= 0) return cudaSuccess;
    const int L = kc.layers > 1 ? kc.layers : 1;
    const int b = 256;
    const long long g = (static_cast<long long>(n) * L + b - 1) / b;
    if (kc.precision == 1)
        gather_kernel<double, false><<<g, b, 0, s>>>(n, L, perm, (const double*)hi, nullptr, dst, snap);
    else if (kc.comp)
        gather_kernel<float, true><<<g, b, 0, s>>>(n, L, perm, (const float*)hi, (const float*)lo, dst, snap);
    else
        gather_kernel<float, false><<<g, b, 0, s>>>(n, L, perm, (const float*)hi, nullptr, dst, snap);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(const KernelConfig& kc, const void* tables, const void* h_hi,
                               const void* h_lo, const void* u_hi, const void* u_lo, double g,
                               double* partial, int nblocks, double* out2, cudaStream_t s) {
    const int L = kc.layers > 1 ? kc.layers : 1;
    if (kc.precision == 1) {
        const Tables<double>& t = *static_cast<const Tables<double>*>(tables);
        diag_kernel<double, double, false><<<nblocks, DIAG_THREADS, 0, s>>>(
            t, (const double*)h_hi, nullptr, (const double*)u_hi, nullptr, g, partial, L);
    } else {
        const Tables<float>& t = *static_cast<const Tables<float>*>(tables);
        if (kc.comp)
            diag_kernel<float, float, true><<<nblocks, DIAG_THREADS, 0, s>>>(
                t, (const float*)h_hi, (const float*)h_lo, (const float*)u_hi, (const float*)u_lo, g,
                partial, L);
        else
            diag_kernel<float, float, false><<<nblocks, DIAG_THREADS, 0, s>>>(
                t, (const float*)h_hi, nullptr, (const float*)u_hi, nullptr, g, partial, L);
    }
    diag_final<<<1, DIAG_THREADS, 0, s>>>(partial, nblocks, out2);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics_snapshot(const KernelConfig& kc, const void* tables, const double* h,
                                        const double* u, double g, double* partial, int nblocks, double* out2,
                                        cudaStream_t s) {
    const int L = kc.layers > 1 ? kc.layers : 1;
    if (kc.precision == 1)
        diag_kernel<double, double, false><<<nblocks, DIAG_THREADS, 0, s>>>(
            *static_cast<const Tables<double>*>(tables), h, nullptr, u, nullptr, g, partial, L);
    else
        diag_kernel<float, double, false><<<nblocks, DIAG_THREADS, 0, s>>>(
            *static_cast<const Tables<float>*>(tables), h, nullptr, u, nullptr, g, partial, L);
    diag_final<<<1, DIAG_THREADS, 0, s>>>(partial, nblocks, out2);
    return cudaGetLastError();
}

template <class T, bool COMP, int MAXR>
int regs_t(int kind) {
    cudaFuncAttributes at{};
    cudaError_t err = kind == 0   ? cudaFuncGetAttributes(&at, kernel_phase<T, COMP, MAXR, 0>)
                      : kind == 1 ? cudaFuncGetAttributes(&at, kernel_phase<T, COMP, MAXR, 1>)
                                  : cudaFuncGetAttributes(&at, kernel_phase<T, COMP, MAXR, 2>);
    return err == cudaSuccess ? at.numRegs : -1;
}

int kernel_registers(const KernelConfig& kc, int kind) {
    if (kc.precision == 1) return kc.maxdeg <= 8 ? regs_t<double, false, 8>(kind) : regs_t<double, false, 16>(kind);
    if (kc.comp) return kc.maxdeg <= 8 ? regs_t<float, true, 8>(kind) : regs_t<float, true, 16>(kind);
    return kc.maxdeg <= 8 ? regs_t<float, false, 8>(kind) : regs_t<float, false, 16>(kind);
}

}  // namespace lts
