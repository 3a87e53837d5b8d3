// lts_api.cpp -- the C ABI of liblts.so (include/lts.h): mesh validation,
// regions, device tables, device state, the phase plans of Algorithm 2.2
// (LTS3) and Algorithm 2.1 (SSPRK3), CUDA-graph capture of one coarse step,
// state I/O and launch statistics.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/lts.h"
#include "lts_error.h"
#include "lts_internal.h"
#include "lts_objects.h"
#include "regions.h"

using namespace lts;

namespace {
constexpr int kDefaultTileCells = 256;   // cells per tile of the fused kernel
}

namespace {

void release_mesh(lts_mesh_s* m) {
    if (m && --m->ref == 0) delete m;
}
void release_regions(lts_regions_s* r) {
    if (r && --r->ref == 0) {
        int dev = -1;
        if (r->device >= 0 && cudaGetDevice(&dev) == cudaSuccess && dev != r->device)
            cudaSetDevice(r->device);
        r->arena[0].reset();
        r->arena[1].reset();
        release_mesh(r->mesh);
        delete r;
    }
}

int check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return set_error(LTS_ENODEV, "no CUDA device: %s", cudaGetErrorString(e));
    }
    return LTS_OK;
}

template <class T>
int build_tables(lts_regions_s* R, int which, Tables<T>& t) {
    const HostMesh& m = R->mesh->m;
    const RegionsHost& r = R->r;
    CoefTables<T> co;
    coefficient_tables<T>(m, r, co);
    auto arena = std::make_unique<DeviceArena>();
    cudaError_t err = cudaSuccess;
    auto up = [&](const auto& v) { return arena->upload(v, err); };
    t.nC = m.nC;
    t.nE = m.nE;
    t.nV = m.nV;
    t.maxE = m.maxE;
    t.cn = up(r.cn);
    t.se = up(r.se);
    t.sn = up(r.sn);
    t.sv = up(r.sv);
    t.snl = up(co.snl);
    t.sR = up(co.sR);
    t.sK = up(co.sK);
    {
        std::vector<int4> sidx;
        std::vector<float2> scf;
        pack_ring_slots<T>(r.se, r.sn, r.sv, co.snl, co.sR, co.sK, sidx, scf);
        t.sidx = up(sidx);
        t.scf = sizeof(T) == 4 ? up(scf) : nullptr;
    }
    {
        std::vector<int4> erow, vri;
        std::vector<float4> vrd, vrk;
        pack_edge_vertex_rows<T>(r.ec0, r.ec1, r.ep, co.rdc, r.vc, r.ve, co.vd, co.vk, co.f, erow, vri, vrd, vrk);
        t.erow = up(erow);
        t.vri = up(vri);
        t.vrd = sizeof(T) == 4 ? up(vrd) : nullptr;
        t.vrk = sizeof(T) == 4 ? up(vrk) : nullptr;
    }
    t.rA = up(co.rA);
    t.b = up(co.b);
    t.ec0 = up(r.ec0);
    t.ec1 = up(r.ec1);
    t.ep = up(r.ep);
    t.rdc = up(co.rdc);
    t.db = up(co.db);
    const int* vc = up(r.vc);
    const int* ve = up(r.ve);
    const T* vk = up(co.vk);
    const T* vd = up(co.vd);
    if (err != cudaSuccess) return set_error(LTS_ECUDA, "table upload: %s", cudaGetErrorString(err));
    const size_t nV = static_cast<size_t>(m.nV);
    t.vc0 = vc; t.vc1 = vc + nV; t.vc2 = vc + 2 * nV;
    t.ve0 = ve; t.ve1 = ve + nV; t.ve2 = ve + 2 * nV;
    t.vk0 = vk; t.vk1 = vk + nV; t.vk2 = vk + 2 * nV;
    t.vd0 = vd; t.vd1 = vd + nV; t.vd2 = vd + 2 * nV;
    t.f = up(co.f);
    t.ta = up(r.tile_a);
    t.tbk = up(r.tile_b);
    t.tlsv = up(r.tile_lsv_off);
    t.halo = up(r.halo);
    t.tverts = up(r.tverts);
    t.lsv = up(r.lsv);
    t.lec = up(r.lec);
    t.area = up(co.area);
    t.bd = up(co.bd);
    t.sK64 = up(co.sK64);
    if (!R->d_perm_c) {
        R->d_perm_c = arena->upload(r.perm_c, err);
        R->d_perm_e = arena->upload(r.perm_e, err);
    }
    if (err != cudaSuccess) return set_error(LTS_ECUDA, "table upload: %s", cudaGetErrorString(err));
    R->arena[which] = std::move(arena);
    return LTS_OK;
}

// ------------------------------------------------------- algorithmic bytes
// Bytes of every array element a launch touches, each counted once (a
// perfect cache): the compulsory traffic of the launch.  Mesh tables are
// read once per element; state and intermediates once per layer.
double launch_bytes(const LaunchDesc& d, const RegionsHost& r, int nC, int nE, int nV, size_t T,
                    bool comp, int layers) {
    std::vector<char> mh(nC, 0), mhl(nC, 0), mu(nE, 0), mq(nV, 0), mk(nC, 0);
    std::vector<char> mrow(nC, 0), mvert(nV, 0);   // fused tiles: ring rows and vertices read
    double tab = 0.0, st = 0.0;   // table bytes, state bytes per layer
    const double c = comp ? 1.0 : 0.0;
    for (int s = 0; s < d.nseg; ++s) {
        const SegDesc& g = d.seg[s];
        const double n = std::max(0, g.end - g.begin);
        switch (g.type) {
            case SEG_VERT:
                tab += n * (24.0 + 7.0 * T);   // vc, ve, vk, vd, f
                st += n * T;                   // q write
                for (int v = g.begin; v < g.end; ++v)
                    for (int q = 0; q < 3; ++q) {
                        mh[r.vc[static_cast<size_t>(q) * nV + v]] = 1;
                        mu[r.ve[static_cast<size_t>(q) * nV + v]] = 1;
                    }
                break;
            case SEG_RING:
            case SEG_RING_UPD:
            case SEG_RING_ACC:
                for (int k = g.begin; k < g.end; ++k) {
                    // cn, rA; per slot se, sn, sv, snl, sR, sK; the C and K writes
                    tab += 1.0 + T + r.cn[k] * (12.0 + 3.0 * T);
                    st += r.cn[k] * T + T;
                    mh[k] = 1;
                    for (int j = 0; j < r.cn[k]; ++j) {
                        mu[r.se[static_cast<size_t>(j) * nC + k]] = 1;
                        mh[r.sn[static_cast<size_t>(j) * nC + k]] = 1;
                        mq[r.sv[static_cast<size_t>(j) * nC + k]] = 1;
                    }
                }
                if (g.type == SEG_RING_UPD) st += n * T * (2.0 + 3.0 * c);
                if (g.type == SEG_RING_ACC) st += n * T * (g.flag ? 1 : 2);
                break;
            case SEG_EDGE_UPD:
            case SEG_EDGE_ACC:
                tab += n * (12.0 + 2.0 * T);                 // ec0, ec1, ep, rdc, db
                for (int e = g.begin; e < g.end; ++e) {
                    mu[e] = 1;
                    for (int cc : {r.ec0[e], r.ec1[e]}) {
                        mh[cc] = mk[cc] = 1;
                        if (comp) mhl[cc] = 1;
                    }
                }
                st += n * 2.0 * T;                           // the two ring shares C (one per edge end)
                st += g.type == SEG_EDGE_UPD ? n * T * (2.0 + 3.0 * c) : n * T * (g.flag ? 1 : 2);
                break;
            case SEG_TILE:
                for (int tl = g.begin; tl < g.end; ++tl) {
                    const int4 ta = r.tile_a[tl], tb = r.tile_b[tl];
                    const bool acc = tl >= g.flag2;
                    // own cells: epilogue; all local cells: ring tables; vertices; edges
                    st += ta.y * T * (acc ? (g.flag ? 1.0 : 2.0) : (2.0 + 3.0 * c));
                    tab += static_cast<double>(tb.y - tb.x) * (12.0 + T + 4.0);
                    st += static_cast<double>(tb.y - tb.x) *
                          (acc ? T * (g.flag ? 1.0 : 2.0) : T * (2.0 + 3.0 * c));
                    tab += 8.0 * 4 + 8.0 * 4;   // tile descriptors
                    for (int k = 0; k < ta.w; ++k) {
                        const int cc = k < ta.y ? ta.x + k : r.halo[ta.z + (k - ta.y)];
                        mrow[cc] = 1;
                    }
                    for (int k = 0; k < tb.w; ++k) mvert[r.tverts[tb.z + k]] = 1;
                    tab += static_cast<double>(tb.y - tb.x) * T;   // db of the owned edges
                    for (int e = tb.x; e < tb.y; ++e) {
                        mu[e] = 1;
                        for (int cc : {r.ec0[e], r.ec1[e]}) {
                            mh[cc] = 1;
                            if (comp) mhl[cc] = 1;
                        }
                    }
                }
                break;
            case SEG_PRED:
                st += n * T * (g.flag ? 2.0 * (1 + c) : 4.0 * (1 + c));
                break;
            case SEG_COPY:
                st += n * T * 2.0 * (1 + c);
                break;
            case SEG_REPLAY:
                st += n * T * ((g.flag == 2 ? 4.0 : 5.0) + 2.0 * c);
                break;
        }
    }
    // fused tiles: ring tables (cn, rA, per slot se, sn, lsv, snl, sR, sK) of every
    // local cell, and the state the rings gather; vertex tables and their gathers
    for (int k = 0; k < nC; ++k) {
        if (!mrow[k]) continue;
        tab += 1.0 + T + r.cn[k] * (10.0 + 3.0 * T);
        mh[k] = 1;
        for (int j = 0; j < r.cn[k]; ++j) {
            mu[r.se[static_cast<size_t>(j) * nC + k]] = 1;
            mh[r.sn[static_cast<size_t>(j) * nC + k]] = 1;
        }
    }
    for (int v = 0; v < nV; ++v) {
        if (!mvert[v]) continue;
        tab += 24.0 + 7.0 * T;
        for (int q = 0; q < 3; ++q) {
            mh[r.vc[static_cast<size_t>(q) * nV + v]] = 1;
            mu[r.ve[static_cast<size_t>(q) * nV + v]] = 1;
        }
    }
    double cnt = 0.0;
    for (int k = 0; k < nC; ++k) cnt += mh[k] + mhl[k] + mk[k];
    for (char x : mu) cnt += x;
    for (char x : mq) cnt += x;
    return tab + layers * (st + cnt * T);
}

// ------------------------------------------------------------ phase plans

struct Planner {
    lts_state_s* S;
    const RegionsHost& r;
    const int* cb;
    const int* eb;
    const int* vb;
    bool comp;

    SegDesc vert(int lo, int hi) const {   // vertex bands lo..hi
        SegDesc s;
        s.type = SEG_VERT;
        s.elem = ELEM_VERT;
        s.begin = vb[lo];
        s.end = vb[hi + 1];
        return s;
    }
    // fused right-hand side over the tiles of bands lo..hi; tiles of bands
    // >= acc_lo accumulate (Steps 3.x.2) instead of updating
    SegDesc tiles(int lo, int hi, int acc_lo, const SV& old, const SV& out, double a, double D,
                  int stage, bool first) const {
        SegDesc s;
        s.type = SEG_TILE;
        s.elem = -1;   // tiles: not placeable in an ensemble
        s.begin = r.tb[lo];
        s.end = r.tb[hi + 1];
        s.flag2 = acc_lo <= hi ? r.tb[acc_lo] : s.end;
        s.flag = first ? 1 : 0;
        s.base = cb[B_I1];
        s.base2 = eb[B_I1];
        s.p[0] = old.hh; s.p[1] = old.hl; s.p[2] = out.hh; s.p[3] = out.hl;
        s.p[4] = old.uh; s.p[5] = old.ul; s.p[6] = out.uh; s.p[7] = out.ul;
        s.p[8] = stage >= 0 ? S->acc_c[stage] : nullptr;
        s.p[9] = stage >= 0 ? S->acc_e[stage] : nullptr;
        s.c[0] = a;
        s.c[1] = D;
        return s;
    }
    SegDesc ring(int lo, int hi) const {   // ring results only, cell bands lo..hi
        SegDesc s;
        s.type = SEG_RING;
        s.elem = ELEM_CELL;
        s.begin = cb[lo];
        s.end = cb[hi + 1];
        return s;
    }
    SegDesc upd(bool cell, int lo, int hi, const SV& old, const SV& in, const SV& out, double a,
                double D) const {
        SegDesc s;
        s.type = cell ? SEG_RING_UPD : SEG_EDGE_UPD;
        s.elem = cell ? ELEM_CELL : ELEM_EDGE;
        const int* ofs = cell ? cb : eb;
        s.begin = ofs[lo];
        s.end = ofs[hi + 1];
        s.p[0] = cell ? old.hh : old.uh;
        s.p[1] = cell ? old.hl : old.ul;
        s.p[2] = cell ? in.hl : in.ul;
        s.p[3] = cell ? out.hh : out.uh;
        s.p[4] = cell ? out.hl : out.ul;
        s.c[0] = a;
        s.c[1] = D;
        return s;
    }
    SegDesc acc(bool cell, int stage, bool first) const {
        SegDesc s;
        s.type = cell ? SEG_RING_ACC : SEG_EDGE_ACC;
        s.elem = cell ? ELEM_CELL : ELEM_EDGE;
        const int* ofs = cell ? cb : eb;
        s.begin = ofs[B_I1];
        s.end = ofs[B_I2 + 1];
        s.base = ofs[B_I1];
        s.cfam = FAM_I;
        s.flag = first ? 1 : 0;
        s.p[0] = cell ? S->acc_c[stage] : S->acc_e[stage];
        return s;
    }
    // x[I1] = prediction (Steps 3.x.1) from x_old (full), P1, P2 (compact).
    // order 2 (LTS2): the tilde coefficients are 0 and P2 is not used (P1
    // stands in for it, multiplied by 0).
    SegDesc pred(bool cell, const SV& old, const SV& out, int k, int M, int which,
                 const SV* x2full = nullptr, int order = 3) const {
        double a, at;
        const double kk = k, MM = M;
        if (which == 1) {          // alpha
            a = kk / MM;
            at = kk * kk / (MM * MM);
        } else if (which == 2) {   // beta
            a = (kk + 1.0) / MM;
            at = kk * (kk + 2.0) / (MM * MM);
        } else {                   // gamma
            a = (2.0 * kk + 1.0) / (2.0 * MM);
            at = (2.0 * kk * kk + 2.0 * kk + 1.0) / (2.0 * MM * MM);
        }
        if (order == 2) at = 0.0;
        const double c1 = a - at, c2 = 2.0 * at;
        SegDesc s;
        s.type = SEG_PRED;
        s.elem = cell ? ELEM_CELL : ELEM_EDGE;
        const int* ofs = cell ? cb : eb;
        s.begin = ofs[B_I1];
        s.end = ofs[B_I1 + 1];
        s.base = ofs[B_I1];
        s.cfam = FAM_I1;
        s.cfam2 = FAM_I1;
        s.flag = (c1 == 0.0 && c2 == 0.0) ? 1 : (c1 == 1.0 && c2 == 0.0) ? 2 : (c1 == 0.0 && c2 == 1.0) ? 3 : 0;
        const SV& p1 = cell ? S->P1c : S->P1e;
        const SV& p2 = order == 2 ? p1 : (cell ? S->P2c : S->P2e);
        s.p[0] = cell ? old.hh : old.uh;
        s.p[1] = cell ? old.hl : old.ul;
        s.p[2] = cell ? p1.hh : p1.uh;
        s.p[3] = cell ? p1.hl : p1.ul;
        s.p[4] = cell ? p2.hh : p2.uh;
        s.p[5] = cell ? p2.hl : p2.ul;
        s.base2 = s.base;
        if (x2full) {   // x_2nd read from its stage array (before Step 3 overwrites I1)
            s.p[4] = cell ? x2full->hh : x2full->uh;
            s.p[5] = cell ? x2full->hl : x2full->ul;
            s.base2 = 0;
            s.cfam2 = FAM_FULL;
        }
        s.p[6] = cell ? out.hh : out.uh;
        s.p[7] = cell ? out.hl : out.ul;
        s.c[0] = c1;
        s.c[1] = c2;
        return s;
    }
    // dst_base = 0: dst is a full array; otherwise dst is the compact I1 array
    // starting at element dst_base (interface snapshots)
    SegDesc copy(bool cell, int lo, int hi, const SV& src, const SV& dst, int dst_base) const {
        SegDesc s;
        s.type = SEG_COPY;
        s.elem = cell ? ELEM_CELL : ELEM_EDGE;
        const int* ofs = cell ? cb : eb;
        s.begin = ofs[lo];
        s.end = ofs[hi + 1];
        s.base = dst_base;
        s.base2 = 0;
        s.cfam = dst_base != 0 ? FAM_I1 : FAM_FULL;
        s.p[0] = cell ? src.hh : src.uh;
        s.p[1] = cell ? src.hl : src.ul;
        s.p[2] = cell ? dst.hh : dst.uh;
        s.p[3] = cell ? dst.hl : dst.ul;
        return s;
    }
    SegDesc replay(bool cell, const SV& old, const SV& out, double dtM, int order = 3) const {
        SegDesc s;
        s.type = SEG_REPLAY;
        s.flag = order == 2 ? 2 : 0;
        s.elem = cell ? ELEM_CELL : ELEM_EDGE;
        const int* ofs = cell ? cb : eb;
        s.begin = ofs[B_I1];
        s.end = ofs[B_I2 + 1];
        s.base = ofs[B_I1];
        s.cfam = FAM_I;
        s.p[0] = cell ? old.hh : old.uh;
        s.p[1] = cell ? old.hl : old.ul;
        for (int k = 0; k < 3; ++k) s.p[2 + k] = cell ? S->acc_c[k] : S->acc_e[k];
        s.p[5] = cell ? out.hh : out.uh;
        s.p[6] = cell ? out.hl : out.ul;
        s.c[0] = dtM;
        s.c[1] = order == 2 ? dtM / 2.0 : dtM / 4.0;
        s.c[2] = 2.0 * dtM / 3.0;
        if (order == 2) s.p[4] = s.p[3];   // no third accumulator (never read)
        return s;
    }
    LaunchDesc launch(int kind, const SV& in, std::initializer_list<SegDesc> segs, int key = -1) const {
        LaunchDesc d;
        d.kind = kind;
        d.key = key;
        d.in_h = in.hh;
        d.in_hl = in.hl;
        d.in_u = in.uh;
        d.in_ul = in.ul;
        d.q = S->q;
        d.ring_c = S->ring_c;
        d.ring_k = S->ring_k;
        d.g = S->p.g;
        for (const SegDesc& s : segs)
            if (s.end > s.begin) d.seg[d.nseg++] = s;
        return d;
    }
};

constexpr double A1 = 0.0, A2 = 0.75, A3 = 1.0 / 3.0;

void plan_lts3(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    const RegionsHost& r = S->reg->r;
    Planner P{S, r, r.cb, r.eb, r.vb, S->kc.comp};
    const SV& X0 = S->buf[parity];
    const SV& XN = S->buf[1 - parity];
    const SV& X1 = S->buf[2];
    const SV& X2 = S->buf[3];
    const double dt = S->p.dt;
    const int M = r.M;
    const double dtM = dt / M;
    const int I1 = r.cb[B_I1];
    const int I1e = r.eb[B_I1];
    const SegDesc none;
    // Coarse phases beside Step 3 (Algorithm 2.2 orders Steps 1, 2 and 4
    // with Step 3 only through data: Step 3 reads the coarse stage values of
    // bands up to C2 and writes none beyond I1).  STEP4: Step 4 on C3+ as a
    // concurrent branch; FAR: Steps 1, 2 and 4 on the far bands as that
    // branch; SERIAL (and the profiling modes): step order.
    const int sched = S->p.profile != 0 ? LTS_COARSE_SERIAL : S->p.coarse_schedule;
    const bool concurrent = sched != LTS_COARSE_SERIAL;
    const bool far = sched == LTS_COARSE_FAR;
    out.clear();
    // Each right-hand side updating bands [lo, hi] is three launches:
    // vertex bands [lo-1, hi+1], ring cells [lo, hi+1] (ring results only on
    // hi+1), edges [lo, hi].  A phase updating [lo, hi] reads [lo-1, hi+2].
    // Step 1 (first stage on Fbar u I1 u I2 u C) and Step 2 (second stage on
    // I1 u I2 u C).  Concurrent: the main stream updates bands up to C4
    // (Step 1) and C2 (Step 2), exactly what Step 3 and Step 2 read.
    const int s1_hi = far ? B_C4 : B_CREST;
    const int s2_hi = far ? B_C2 : B_CREST;
    auto ring_halo = [&](int hi) { return hi < B_CREST ? P.ring(hi + 1, hi + 1) : none; };
    out.push_back(P.launch(0, X0, {P.vert(B_F3, std::min(s1_hi + 1, (int)B_CREST)),
                                   P.copy(true, B_I2, B_C2, X0, XN, 0)}, KEY_STEP1 + 0));
    out.push_back(P.launch(1, X0, {P.upd(true, B_F2, s1_hi, X0, X0, X1, A1, dt), ring_halo(s1_hi)},
                           KEY_STEP1 + 1));
    out.push_back(P.launch(2, X0, {P.upd(false, B_F2, s1_hi, X0, X0, X1, A1, dt),
                                   P.copy(false, B_I2, B_C2, X0, XN, 0),
                                   P.copy(true, B_I1, B_I1, X1, S->P1c, I1)}, KEY_STEP1 + 2));
    out.push_back(P.launch(0, X1, {P.vert(B_F1, std::min(s2_hi + 1, (int)B_CREST)),
                                   P.copy(false, B_I1, B_I1, X1, S->P1e, I1e)}, KEY_STEP2 + 0));
    out.push_back(P.launch(1, X1, {P.upd(true, B_I1, s2_hi, X0, X1, X2, A2, dt / 4.0), ring_halo(s2_hi)},
                           KEY_STEP2 + 1));
    out.push_back(P.launch(2, X1, {P.upd(false, B_I1, s2_hi, X0, X1, X2, A2, dt / 4.0),
                                   P.copy(true, B_I1, B_I1, X2, S->P2c, I1)}, KEY_STEP2 + 2));
    const size_t after_step2 = out.size();
    for (auto& d : out) d.l2 = 2;   // Steps 1 and 2 stream the coarse region
    // Step 3: M fine substeps on F, correction terms on I1 u I2, I1 predicted
    for (int k = 0; k < M; ++k) {
        const SV& old = (k == 0) ? X0 : XN;
        for (int s = 1; s <= 3; ++s) {
            const SV& in = (s == 1) ? old : (s == 2 ? X1 : X2);
            const SV& o = (s == 1) ? X1 : (s == 2 ? X2 : XN);
            const double a = (s == 1) ? A1 : (s == 2 ? A2 : A3);
            const double D = (s == 1) ? dtM : (s == 2 ? dtM / 4.0 : 2.0 * dtM / 3.0);
            // prediction of I1 for the next stage that reads it
            SegDesc pc, pe;
            if (s == 1) {
                pc = P.pred(true, X0, X1, k, M, 2);
                pe = P.pred(false, X0, X1, k, M, 2);
            } else if (s == 2) {
                pc = P.pred(true, X0, X2, k, M, 3);
                pe = P.pred(false, X0, X2, k, M, 3);
            } else if (k + 1 < M) {
                pc = P.pred(true, X0, o, k + 1, M, 1);
                pe = P.pred(false, X0, o, k + 1, M, 1);
            }
            const SegDesc snap = (k == 0 && s == 1) ? P.copy(false, B_I1, B_I1, X2, S->P2e, I1e) : none;
            const int key = KEY_STEP3 + 9 * k + 3 * (s - 1);
            out.push_back(P.launch(0, in, {P.vert(B_FDEEP, B_C1), snap}, key + 0));
            out.push_back(P.launch(1, in, {P.upd(true, B_FDEEP, B_F1, old, in, o, a, D),
                                           P.acc(true, s - 1, k == 0), P.ring(B_C1, B_C1), pc}, key + 1));
            out.push_back(P.launch(2, in, {P.upd(false, B_FDEEP, B_F1, old, in, o, a, D),
                                           P.acc(false, s - 1, k == 0), pe}, key + 2));
        }
    }
    for (size_t k = after_step2; k < out.size(); ++k) out[k].l2 = 1;   // fine substeps stay in L2
    // Step 4 (third stage on C, reading R2) and Step 5 (interface correction).
    std::vector<LaunchDesc> side, tail;
    if (concurrent) {
        // The branch, with its own intermediates.  FAR: Step 1 on C5..C rest,
        // Step 2 on C3..C rest; both: Step 4 on C3..C rest.  It reads stage
        // values of bands >= C2 only, which the main stream finished before
        // the fork, and writes bands Step 3 never reads.
        if (far) {
            side.push_back(P.launch(0, X0, {P.vert(B_C4, B_CREST)}, KEY_SIDE + 0));
            side.push_back(P.launch(1, X0, {P.upd(true, B_C5, B_CREST, X0, X0, X1, A1, dt)}, KEY_SIDE + 1));
            side.push_back(P.launch(2, X0, {P.upd(false, B_C5, B_CREST, X0, X0, X1, A1, dt)}, KEY_SIDE + 2));
            side.push_back(P.launch(0, X1, {P.vert(B_C2, B_CREST)}, KEY_SIDE + 3));
            side.push_back(P.launch(1, X1, {P.upd(true, B_C3, B_CREST, X0, X1, X2, A2, dt / 4.0)}, KEY_SIDE + 4));
            side.push_back(P.launch(2, X1, {P.upd(false, B_C3, B_CREST, X0, X1, X2, A2, dt / 4.0)}, KEY_SIDE + 5));
        }
        side.push_back(P.launch(0, X2, {P.vert(B_C2, B_CREST)}, KEY_SIDE + 6));
        side.push_back(P.launch(1, X2, {P.upd(true, B_C3, B_CREST, X0, X2, XN, A3, 2.0 * dt / 3.0)}, KEY_SIDE + 7));
        side.push_back(P.launch(2, X2, {P.upd(false, B_C3, B_CREST, X0, X2, XN, A3, 2.0 * dt / 3.0)}, KEY_SIDE + 8));
        for (auto& d : side) {
            d.q = S->q_side;
            d.ring_c = S->ring_c_side;
            d.ring_k = S->ring_k_side;
        }
    }
    // the near part of Step 4 (C1..C2 when concurrent, else all of C) and
    // Step 5 after Step 3
    const int s4_hi = concurrent ? B_C2 : B_CREST;
    tail.push_back(P.launch(0, X2, {P.vert(B_I2, std::min(s4_hi + 1, (int)B_CREST))}, KEY_TAIL + 0));
    tail.push_back(P.launch(1, X2, {P.upd(true, B_C1, s4_hi, X0, X2, XN, A3, 2.0 * dt / 3.0),
                                    ring_halo(s4_hi), P.replay(true, X0, XN, dtM)}, KEY_TAIL + 1));
    tail.push_back(P.launch(2, X2, {P.upd(false, B_C1, s4_hi, X0, X2, XN, A3, 2.0 * dt / 3.0),
                                    P.replay(false, X0, XN, dtM)}, KEY_TAIL + 2));
    for (auto& d : side) d.l2 = 2;
    for (auto& d : tail) d.l2 = 2;
    auto drop = [](std::vector<LaunchDesc>& v) {
        v.erase(std::remove_if(v.begin(), v.end(), [](const LaunchDesc& d) { return d.nseg == 0; }),
                v.end());
    };
    drop(side);
    drop(tail);
    if (!side.empty()) {
        // the side branch forks right after Step 2 and joins before the tail
        for (auto& d : side) d.branch = 1;
        side.front().fork = true;
        if (!tail.empty()) tail.front().join = true;
        out.insert(out.begin() + static_cast<long>(after_step2), side.begin(), side.end());
    }
    out.insert(out.end(), tail.begin(), tail.end());
    if (!side.empty() && tail.empty()) {
        LaunchDesc j;   // nothing after Step 3: still join before the step ends
        j.join = true;
        j.key = KEY_TAIL - 1;
        out.push_back(j);
    }
    // empty launches (bands without cells) are dropped, markers are kept
    out.erase(std::remove_if(out.begin(), out.end(),
                             [](const LaunchDesc& d) { return d.nseg == 0 && !d.fork && !d.join; }),
              out.end());
}

// Algorithm 2.2 with its LTS2 branches, three launches per right-hand side.
// Step 1 (first stage) on I1 u I2 u C; Step 3: two stages per substep with
// the linear predictions of I1 and two correction terms; Step 2 (second
// stage on C, x_new = x_2nd there: Step 4) reads only first-stage values
// that Step 3 leaves alone, so it runs after Step 3 or, for the bands C3
// and beyond, as a concurrent branch beside it; Step 5 replays the two
// interface stages.
void plan_lts2(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    const RegionsHost& r = S->reg->r;
    Planner P{S, r, r.cb, r.eb, r.vb, S->kc.comp};
    const SV& X0 = S->buf[parity];
    const SV& XN = S->buf[1 - parity];
    const SV& X1 = S->buf[2];
    const double dt = S->p.dt;
    const int M = r.M;
    const double dtM = dt / M;
    const int I1 = r.cb[B_I1];
    const int I1e = r.eb[B_I1];
    const SegDesc none;
    const int sched = S->p.profile != 0 ? LTS_COARSE_SERIAL : S->p.coarse_schedule;
    const bool concurrent = sched != LTS_COARSE_SERIAL;
    auto ring_halo = [&](int hi) { return hi < B_CREST ? P.ring(hi + 1, hi + 1) : none; };
    out.clear();
    // Step 1 on I1 u I2 u C (bands I1..C rest); x_new on I2..C2 holds x_old
    // while Step 3 reads it as a halo
    out.push_back(P.launch(0, X0, {P.vert(B_F1, B_CREST), P.copy(true, B_I2, B_C2, X0, XN, 0)},
                           KEY_STEP1 + 0));
    out.push_back(P.launch(1, X0, {P.upd(true, B_I1, B_CREST, X0, X0, X1, A1, dt)}, KEY_STEP1 + 1));
    out.push_back(P.launch(2, X0, {P.upd(false, B_I1, B_CREST, X0, X0, X1, A1, dt),
                                   P.copy(false, B_I2, B_C2, X0, XN, 0),
                                   P.copy(true, B_I1, B_I1, X1, S->P1c, I1)}, KEY_STEP1 + 2));
    const size_t after_step1 = out.size();
    for (auto& d : out) d.l2 = 2;
    // Step 3
    for (int k = 0; k < M; ++k) {
        const SV& old = (k == 0) ? X0 : XN;
        for (int s = 1; s <= 2; ++s) {
            const SV& in = (s == 1) ? old : X1;
            const SV& o = (s == 1) ? X1 : XN;
            const double a = (s == 1) ? A1 : 0.5;
            const double D = (s == 1) ? dtM : dtM / 2.0;
            SegDesc pc, pe;
            if (s == 1) {            // I1 at the second stage: beta_k
                pc = P.pred(true, X0, X1, k, M, 2, nullptr, 2);
                pe = P.pred(false, X0, X1, k, M, 2, nullptr, 2);
            } else if (k + 1 < M) {  // I1 at the next substep: alpha_{k+1}
                pc = P.pred(true, X0, XN, k + 1, M, 1, nullptr, 2);
                pe = P.pred(false, X0, XN, k + 1, M, 1, nullptr, 2);
            }
            const SegDesc snap = (k == 0 && s == 1) ? P.copy(false, B_I1, B_I1, X1, S->P1e, I1e) : none;
            const int key = KEY_STEP3 + 9 * k + 3 * (s - 1);
            out.push_back(P.launch(0, in, {P.vert(B_FDEEP, B_C1), snap}, key + 0));
            out.push_back(P.launch(1, in, {P.upd(true, B_FDEEP, B_F1, old, in, o, a, D),
                                           P.acc(true, s - 1, k == 0), P.ring(B_C1, B_C1), pc}, key + 1));
            out.push_back(P.launch(2, in, {P.upd(false, B_FDEEP, B_F1, old, in, o, a, D),
                                           P.acc(false, s - 1, k == 0), pe}, key + 2));
        }
    }
    for (size_t k = after_step1; k < out.size(); ++k) out[k].l2 = 1;
    // Step 2 (= Step 4 for LTS2) on C and Step 5
    std::vector<LaunchDesc> side, tail;
    if (concurrent) {
        side.push_back(P.launch(0, X1, {P.vert(B_C2, B_CREST)}, KEY_SIDE + 6));
        side.push_back(P.launch(1, X1, {P.upd(true, B_C3, B_CREST, X0, X1, XN, 0.5, dt / 2.0)}, KEY_SIDE + 7));
        side.push_back(P.launch(2, X1, {P.upd(false, B_C3, B_CREST, X0, X1, XN, 0.5, dt / 2.0)}, KEY_SIDE + 8));
        for (auto& d : side) {
            d.q = S->q_side;
            d.ring_c = S->ring_c_side;
            d.ring_k = S->ring_k_side;
        }
    }
    const int s2_hi = concurrent ? B_C2 : B_CREST;
    tail.push_back(P.launch(0, X1, {P.vert(B_I2, std::min(s2_hi + 1, (int)B_CREST))}, KEY_TAIL + 0));
    tail.push_back(P.launch(1, X1, {P.upd(true, B_C1, s2_hi, X0, X1, XN, 0.5, dt / 2.0), ring_halo(s2_hi),
                                    P.replay(true, X0, XN, dtM, 2)}, KEY_TAIL + 1));
    tail.push_back(P.launch(2, X1, {P.upd(false, B_C1, s2_hi, X0, X1, XN, 0.5, dt / 2.0),
                                    P.replay(false, X0, XN, dtM, 2)}, KEY_TAIL + 2));
    for (auto& d : side) d.l2 = 2;
    for (auto& d : tail) d.l2 = 2;
    auto drop = [](std::vector<LaunchDesc>& v) {
        v.erase(std::remove_if(v.begin(), v.end(), [](const LaunchDesc& d) { return d.nseg == 0; }),
                v.end());
    };
    drop(side);
    drop(tail);
    if (!side.empty()) {
        for (auto& d : side) d.branch = 1;
        side.front().fork = true;
        if (!tail.empty()) tail.front().join = true;
        out.insert(out.begin() + static_cast<long>(after_step1), side.begin(), side.end());
    }
    out.insert(out.end(), tail.begin(), tail.end());
    if (!side.empty() && tail.empty()) {
        LaunchDesc j;
        j.join = true;
        j.key = KEY_TAIL - 1;
        out.push_back(j);
    }
    out.erase(std::remove_if(out.begin(), out.end(),
                             [](const LaunchDesc& d) { return d.nseg == 0 && !d.fork && !d.join; }),
              out.end());
}

// Algorithm 2.1, SSPRK2 on the whole mesh.
void plan_ssprk2(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    const RegionsHost& r = S->reg->r;
    Planner P{S, r, r.cb, r.eb, r.vb, S->kc.comp};
    const SV& X0 = S->buf[parity];
    const SV& XN = S->buf[1 - parity];
    const SV& X1 = S->buf[2];
    const double dt = S->p.dt;
    out.clear();
    const SV* ins[2] = {&X0, &X1};
    const SV* outs[2] = {&X1, &XN};
    const double as[2] = {A1, 0.5};
    const double Ds[2] = {dt, dt / 2.0};
    for (int s = 0; s < 2; ++s) {
        out.push_back(P.launch(0, *ins[s], {P.vert(B_FDEEP, B_CREST)}, 3 * s + 0));
        out.push_back(P.launch(1, *ins[s], {P.upd(true, B_FDEEP, B_CREST, X0, *ins[s], *outs[s], as[s], Ds[s])}, 3 * s + 1));
        out.push_back(P.launch(2, *ins[s], {P.upd(false, B_FDEEP, B_CREST, X0, *ins[s], *outs[s], as[s], Ds[s])}, 3 * s + 2));
    }
}

// The same plan with one fused tile launch per right-hand side.
void plan_lts3_fused(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    const RegionsHost& r = S->reg->r;
    Planner P{S, r, r.cb, r.eb, r.vb, S->kc.comp};
    const SV& X0 = S->buf[parity];
    const SV& XN = S->buf[1 - parity];
    const SV& X1 = S->buf[2];
    const SV& X2 = S->buf[3];
    const double dt = S->p.dt;
    const int M = r.M;
    const double dtM = dt / M;
    const int I1 = r.cb[B_I1];
    const int I1e = r.eb[B_I1];
    const SegDesc none;
    const int NOACC = NBANDS;   // acc_lo past every band: all tiles update
    out.clear();
    // Step 1 on Fbar u I1 u I2 u C; x_new on I2..C2 prefilled with x_old
    out.push_back(P.launch(3, X0, {P.tiles(B_F2, B_CREST, NOACC, X0, X1, A1, dt, -1, false),
                                   P.copy(true, B_I2, B_C2, X0, XN, 0),
                                   P.copy(false, B_I2, B_C2, X0, XN, 0)}));
    // Step 2 on I1 u I2 u C; snapshots of x_1st on I1
    out.push_back(P.launch(3, X1, {P.tiles(B_I1, B_CREST, NOACC, X0, X2, A2, dt / 4.0, -1, false),
                                   P.copy(true, B_I1, B_I1, X1, S->P1c, I1),
                                   P.copy(false, B_I1, B_I1, X1, S->P1e, I1e)}));
    const size_t after_step2 = out.size();
    for (auto& d : out) d.l2 = 2;
    // Step 3
    for (int k = 0; k < M; ++k) {
        const SV& old = (k == 0) ? X0 : XN;
        for (int s = 1; s <= 3; ++s) {
            const SV& in = (s == 1) ? old : (s == 2 ? X1 : X2);
            const SV& o = (s == 1) ? X1 : (s == 2 ? X2 : XN);
            const double a = (s == 1) ? A1 : (s == 2 ? A2 : A3);
            const double D = (s == 1) ? dtM : (s == 2 ? dtM / 4.0 : 2.0 * dtM / 3.0);
            SegDesc pc, pe, sc, se;
            if (s == 1) {
                // x_2nd on I1 still holds the coarse stage here: read it in place,
                // and take the snapshot for the later predictions
                const bool first = (k == 0);
                pc = P.pred(true, X0, X1, k, M, 2, first ? &X2 : nullptr);
                pe = P.pred(false, X0, X1, k, M, 2, first ? &X2 : nullptr);
                if (first) {
                    sc = P.copy(true, B_I1, B_I1, X2, S->P2c, I1);
                    se = P.copy(false, B_I1, B_I1, X2, S->P2e, I1e);
                }
            } else if (s == 2) {
                pc = P.pred(true, X0, X2, k, M, 3);
                pe = P.pred(false, X0, X2, k, M, 3);
            } else if (k + 1 < M) {
                pc = P.pred(true, X0, XN, k + 1, M, 1);
                pe = P.pred(false, X0, XN, k + 1, M, 1);
            }
            LaunchDesc d = P.launch(3, in, {P.tiles(B_FDEEP, B_I2, B_I1, old, o, a, D, s - 1, k == 0),
                                            pc, pe, sc, se});
            d.l2 = 1;
            out.push_back(d);
        }
    }
    (void)none;
    // Step 4 on C rest concurrently with Step 3; C1, C2 and Step 5 after it
    std::vector<LaunchDesc> side, tail;
    side.push_back(P.launch(3, X2, {P.tiles(B_CREST, B_CREST, NOACC, X0, XN, A3, 2.0 * dt / 3.0, -1, false)}));
    tail.push_back(P.launch(3, X2, {P.tiles(B_C1, B_C5, NOACC, X0, XN, A3, 2.0 * dt / 3.0, -1, false),
                                    P.replay(true, X0, XN, dtM), P.replay(false, X0, XN, dtM)}));
    for (auto& d : side) d.l2 = 2;
    for (auto& d : tail) d.l2 = 2;
    auto drop = [](std::vector<LaunchDesc>& v) {
        v.erase(std::remove_if(v.begin(), v.end(), [](const LaunchDesc& d) { return d.nseg == 0; }),
                v.end());
    };
    drop(side);
    drop(tail);
    const bool concurrent = S->p.profile == 0 && S->p.coarse_schedule != LTS_COARSE_SERIAL && !side.empty();
    size_t at = after_step2;
    if (concurrent) {
        for (auto& d : side) d.branch = 1;
        side.front().fork = true;
        if (!tail.empty()) tail.front().join = true;
        out.insert(out.begin() + static_cast<long>(at), side.begin(), side.end());
    } else {
        out.insert(out.end(), side.begin(), side.end());
    }
    out.insert(out.end(), tail.begin(), tail.end());
    if (concurrent && tail.empty()) {
        LaunchDesc j;
        j.join = true;
        out.push_back(j);
    }
    out.erase(std::remove_if(out.begin(), out.end(),
                             [](const LaunchDesc& d) { return d.nseg == 0 && !d.fork && !d.join; }),
              out.end());
}

void plan_ssprk3_fused(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    const RegionsHost& r = S->reg->r;
    Planner P{S, r, r.cb, r.eb, r.vb, S->kc.comp};
    const SV& X0 = S->buf[parity];
    const SV& XN = S->buf[1 - parity];
    const SV& X1 = S->buf[2];
    const SV& X2 = S->buf[3];
    const double dt = S->p.dt;
    out.clear();
    const SV* ins[3] = {&X0, &X1, &X2};
    const SV* outs[3] = {&X1, &X2, &XN};
    const double as[3] = {A1, A2, A3};
    const double Ds[3] = {dt, dt / 4.0, 2.0 * dt / 3.0};
    for (int s = 0; s < 3; ++s)
        out.push_back(P.launch(3, *ins[s], {P.tiles(B_FDEEP, B_CREST, NBANDS, X0, *outs[s], as[s], Ds[s], -1, false)}));
}

void plan_ssprk3(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    const RegionsHost& r = S->reg->r;
    Planner P{S, r, r.cb, r.eb, r.vb, S->kc.comp};
    const SV& X0 = S->buf[parity];
    const SV& XN = S->buf[1 - parity];
    const SV& X1 = S->buf[2];
    const SV& X2 = S->buf[3];
    const double dt = S->p.dt;
    out.clear();
    const SV* ins[3] = {&X0, &X1, &X2};
    const SV* outs[3] = {&X1, &X2, &XN};
    const double as[3] = {A1, A2, A3};
    const double Ds[3] = {dt, dt / 4.0, 2.0 * dt / 3.0};
    for (int s = 0; s < 3; ++s) {
        out.push_back(P.launch(0, *ins[s], {P.vert(B_FDEEP, B_CREST)}, 3 * s + 0));
        out.push_back(P.launch(1, *ins[s], {P.upd(true, B_FDEEP, B_CREST, X0, *ins[s], *outs[s], as[s], Ds[s])}, 3 * s + 1));
        out.push_back(P.launch(2, *ins[s], {P.upd(false, B_FDEEP, B_CREST, X0, *ins[s], *outs[s], as[s], Ds[s])}, 3 * s + 2));
    }
}

// Enqueues one coarse step: main-stream launches on `st`, side-branch
// launches on `side`, with an event fork before the branch and a join before
// the first launch that needs it.  A launch that follows a fork or join is
// not a programmatic dependent of its stream predecessor.
int enqueue_plan(lts_state_s* S, const std::vector<LaunchDesc>& plan, cudaStream_t st,
                 cudaStream_t side) {
    bool after_event[2] = {false, false};
    for (const LaunchDesc& d : plan) {
        if (d.fork) {
            CUDA_TRY(cudaEventRecord(S->ev_fork, st));
            CUDA_TRY(cudaStreamWaitEvent(side, S->ev_fork, 0));
            after_event[1] = true;
        }
        if (d.join) {
            CUDA_TRY(cudaEventRecord(S->ev_join, side));
            CUDA_TRY(cudaStreamWaitEvent(st, S->ev_join, 0));
            after_event[0] = true;
        }
        if (d.nseg == 0) continue;
        KernelConfig kc = S->kc;
        if (after_event[d.branch]) kc.pdl = false;
        after_event[d.branch] = false;
        cudaError_t e = launch_phase(d, S->tables, kc, S->flag, d.branch ? side : st);
        if (e != cudaSuccess) return set_error(LTS_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    }
    return LTS_OK;
}

// profile == 2: an external event-record node before and after every kernel
// node, so per-kernel times can be read after each graph launch.
int enqueue_plan_timed(lts_state_s* S, const std::vector<LaunchDesc>& plan, cudaStream_t st, int p) {
    for (size_t k = 0; k < plan.size(); ++k) {
        cudaEvent_t* ev = &S->gevents[p][2 * k];
        cudaError_t e = cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_phase(plan[k], S->tables, S->kc, S->flag, st);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
        if (e != cudaSuccess) return set_error(LTS_ECUDA, "timed capture: %s", cudaGetErrorString(e));
    }
    return LTS_OK;
}

// Several fine regions: the plan of every block (one per region with its M
// and its own snapshots and correction terms, one for the far coarse cells),
// each seeing the shared state buffers and its block's band offsets, merged
// launch by launch into segment-table launches.
int build_multi_plan(lts_state_s* S, int parity, int nsm, TablePlanStats* st) {
    const RegionsHost& r = S->reg->r;
    const HostMesh& m = S->reg->mesh->m;
    std::vector<std::vector<LaunchDesc>> plans;
    for (int b = 0; b <= r.nreg; ++b) {
        lts_regions_s view;   // band offsets and M of block b only (planning needs no more)
        for (int k = 0; k <= NBANDS; ++k) {
            view.r.cb[k] = r.mcb[b][k];
            view.r.eb[k] = r.meb[b][k];
            view.r.vb[k] = r.mvb[b][k];
        }
        view.r.M = b < r.nreg ? r.Mr[b] : 1;
        view.r.order = r.order;
        view.r.layers = r.layers;
        lts_state_s F;
        F.reg = &view;
        F.p = S->p;
        F.kc = S->kc;
        F.tsz = S->tsz;
        for (int k = 0; k < 4; ++k) F.buf[k] = S->buf[k];
        const auto& mb = S->mbufs[b];
        F.P1c = mb.P1c;
        F.P1e = mb.P1e;
        F.P2c = mb.P2c;
        F.P2e = mb.P2e;
        for (int k = 0; k < 3; ++k) {
            F.acc_c[k] = mb.acc_c[k];
            F.acc_e[k] = mb.acc_e[k];
        }
        F.q = S->q;
        F.ring_c = S->ring_c;
        F.ring_k = S->ring_k;
        F.q_side = S->q_side;
        F.ring_c_side = S->ring_c_side;
        F.ring_k_side = S->ring_k_side;
        F.flag = S->flag;
        std::vector<LaunchDesc> plan;
        make_plan(&F, parity, plan);
        F.reg = nullptr;
        for (LaunchDesc& d : plan) {
            if (d.nseg == 0) continue;
            if (S->p.no_l2_hints) d.l2 = 0;
            d.bytes = launch_bytes(d, r, m.nC, m.nE, m.nV, S->tsz, S->kc.comp, 1);
        }
        plans.push_back(std::move(plan));
    }
    return merge_table_plan(S->kc, plans, nsm, S->arena, S->tplan[parity], st);
}

int capture_graphs(lts_state_s* S) {
    for (int p = 0; p < 2; ++p) {
        if (S->p.profile == 2) {
            S->gevents[p].resize(2 * S->plan[p].size());
            for (auto& ev : S->gevents[p]) CUDA_TRY(cudaEventCreate(&ev));
        }
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(S->capture_stream, cudaStreamCaptureModeThreadLocal));
        int rc = S->multi ? enqueue_table_plan(S->tplan[p], S->tables, S->kc, S->flag, S->capture_stream,
                                               S->capture_side, S->ev_fork, S->ev_join)
                 : S->p.profile == 2 ? enqueue_plan_timed(S, S->plan[p], S->capture_stream, p)
                                     : enqueue_plan(S, S->plan[p], S->capture_stream, S->capture_side);
        cudaError_t e = cudaStreamEndCapture(S->capture_stream, &g);
        if (rc != LTS_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CUDA_TRY(e);
        e = cudaGraphInstantiate(&S->exec[p], g, 0);
        cudaGraphDestroy(g);
        CUDA_TRY(e);
    }
    return LTS_OK;
}

int state_alloc(lts_state_s* S) {
    const RegionsHost& r = S->reg->r;
    const HostMesh& m = S->reg->mesh->m;
    const size_t T = S->tsz;
    const bool comp = S->kc.comp;
    cudaError_t err = cudaSuccess;
    // state-sized arrays hold every layer ([element * L + layer])
    const size_t Ly = static_cast<size_t>(S->kc.layers);
    auto A = [&](size_t n) { return S->arena.alloc(n * Ly * T, err); };
    for (int k = 0; k < 4; ++k) {
        S->buf[k].hh = A(m.nC);
        S->buf[k].uh = A(m.nE);
        if (comp) {
            S->buf[k].hl = A(m.nC);
            S->buf[k].ul = A(m.nE);
        }
    }
    if (S->multi) {
        // one set of interface snapshots and correction terms per region
        S->mbufs.assign(r.nreg + 1, lts_state_s::MemberBufs{});
        for (int b = 0; b < r.nreg; ++b) {
            auto& mb = S->mbufs[b];
            const auto &cb = r.mcb[b], &eb = r.meb[b];
            const int n1c = cb[B_I1 + 1] - cb[B_I1], n1e = eb[B_I1 + 1] - eb[B_I1];
            const int nic = cb[B_I2 + 1] - cb[B_I1], nie = eb[B_I2 + 1] - eb[B_I1];
            for (SV* p : {&mb.P1c, &mb.P2c}) {
                p->hh = A(n1c);
                if (comp) p->hl = A(n1c);
            }
            for (SV* p : {&mb.P1e, &mb.P2e}) {
                p->uh = A(n1e);
                if (comp) p->ul = A(n1e);
            }
            for (int k = 0; k < 3; ++k) {
                mb.acc_c[k] = A(nic);
                mb.acc_e[k] = A(nie);
            }
        }
    }
    const int nI1c = r.cb[B_I1 + 1] - r.cb[B_I1], nI1e = r.eb[B_I1 + 1] - r.eb[B_I1];
    const int nIc = r.cb[B_I2 + 1] - r.cb[B_I1], nIe = r.eb[B_I2 + 1] - r.eb[B_I1];
    for (SV* p : {&S->P1c, &S->P2c}) {
        p->hh = A(nI1c);
        if (comp) p->hl = A(nI1c);
    }
    for (SV* p : {&S->P1e, &S->P2e}) {
        p->uh = A(nI1e);
        if (comp) p->ul = A(nI1e);
    }
    for (int k = 0; k < 3; ++k) {
        S->acc_c[k] = A(nIc);
        S->acc_e[k] = A(nIe);
    }
    S->q = A(m.nV);
    S->ring_c = A(static_cast<size_t>(m.maxE) * m.nC);
    S->ring_k = A(m.nC);
    if (S->p.mode == LTS_MODE_LTS) {
        S->q_side = A(m.nV);
        S->ring_c_side = A(static_cast<size_t>(m.maxE) * m.nC);
        S->ring_k_side = A(m.nC);
    }
    S->flag = static_cast<int*>(S->arena.alloc(sizeof(int), err));
    S->stage_c = static_cast<double*>(S->arena.alloc(sizeof(double) * m.nC * Ly, err));
    S->stage_e = static_cast<double*>(S->arena.alloc(sizeof(double) * m.nE * Ly, err));
    S->out_c = static_cast<double*>(S->arena.alloc(sizeof(double) * m.nC * Ly, err));
    S->out_e = static_cast<double*>(S->arena.alloc(sizeof(double) * m.nE * Ly, err));
    S->snap_c = static_cast<double*>(S->arena.alloc(sizeof(double) * m.nC * Ly, err));
    S->snap_e = static_cast<double*>(S->arena.alloc(sizeof(double) * m.nE * Ly, err));
    // one (cell, layer) per thread up to 8192 blocks, then grid-stride
    S->diag_blocks = static_cast<int>(std::max<size_t>(1, std::min<size_t>(8192, (m.nC * Ly + 255) / 256)));
    S->diag_partial = static_cast<double*>(S->arena.alloc(sizeof(double) * 2 * S->diag_blocks, err));
    S->diag_out = static_cast<double*>(S->arena.alloc(sizeof(double) * 2, err));
    if (err != cudaSuccess)
        return set_error(err == cudaErrorMemoryAllocation ? LTS_ENOMEM : LTS_ECUDA,
                         "state allocation: %s", cudaGetErrorString(err));
    // the zero fills ran on the legacy stream; the state's stream does not wait for it
    CUDA_TRY(cudaDeviceSynchronize());
    return LTS_OK;
}

int write_state(lts_state_s* S, const double* h, const double* u) {
    const HostMesh& m = S->reg->mesh->m;
    const SV& X = S->buf[S->parity];
    const size_t Ly = static_cast<size_t>(S->kc.layers);
    // The copies wait only until the input staging is free (the previous
    // write's scatters have run), so they overlap whatever the state's stream
    // is still doing; the scatters replace the state in stream order, and the
    // h scatter overlaps the u copy.
    CUDA_TRY(cudaStreamWaitEvent(S->h2d_stream, S->ev_in_free, 0));
    CUDA_TRY(cudaMemcpyAsync(S->stage_c, h, sizeof(double) * m.nC * Ly, cudaMemcpyHostToDevice, S->h2d_stream));
    CUDA_TRY(cudaEventRecord(S->ev_in_h, S->h2d_stream));
    CUDA_TRY(cudaMemcpyAsync(S->stage_e, u, sizeof(double) * m.nE * Ly, cudaMemcpyHostToDevice, S->h2d_stream));
    CUDA_TRY(cudaEventRecord(S->ev_in_u, S->h2d_stream));
    CUDA_TRY(cudaStreamWaitEvent(S->stream, S->ev_in_h, 0));
    CUDA_TRY(launch_scatter_state(S->kc, m.nC, S->reg->d_perm_c, S->stage_c, X.hh, X.hl, S->stream));
    CUDA_TRY(cudaStreamWaitEvent(S->stream, S->ev_in_u, 0));
    CUDA_TRY(launch_scatter_state(S->kc, m.nE, S->reg->d_perm_e, S->stage_e, X.uh, X.ul, S->stream));
    CUDA_TRY(cudaEventRecord(S->ev_in_free, S->stream));
    return LTS_OK;
}

// Enqueues the copy of the current state (and its diagnostics) to the host:
// gathers into the output staging on the state's stream once the previous
// read's copies are done, then the device-to-host copies on d2h_stream.
int read_state(lts_state_s* S, double* h, double* u, lts_diag* d) {
    const HostMesh& m = S->reg->mesh->m;
    const SV& X = S->buf[S->parity];
    const size_t Ly = static_cast<size_t>(S->kc.layers);
    if (d && static_cast<int>(S->pending_diag.size()) >= lts_state_s::kDiagSlots)
        return set_error(LTS_EINVAL, "more than %d reads with diagnostics before lts_sync",
                         lts_state_s::kDiagSlots);
    CUDA_TRY(cudaStreamWaitEvent(S->stream, S->ev_out_free, 0));
    if (d) CUDA_TRY(cudaStreamWaitEvent(S->stream, S->ev_snap_free, 0));
    // with diagnostics both fields are gathered (for the snapshot), whether
    // or not the caller copies them
    if (h || d) {
        CUDA_TRY(launch_gather_state(S->kc, m.nC, S->reg->d_perm_c, X.hh, X.hl, S->out_c, S->stream,
                                     d ? S->snap_c : nullptr));
        CUDA_TRY(cudaEventRecord(S->ev_out_h, S->stream));
        CUDA_TRY(cudaStreamWaitEvent(S->d2h_stream, S->ev_out_h, 0));
        if (h)
            CUDA_TRY(cudaMemcpyAsync(h, S->out_c, sizeof(double) * m.nC * Ly, cudaMemcpyDeviceToHost,
                                     S->d2h_stream));
    }
    if (u || d)
        CUDA_TRY(launch_gather_state(S->kc, m.nE, S->reg->d_perm_e, X.uh, X.ul, S->out_e, S->stream,
                                     d ? S->snap_e : nullptr));
    CUDA_TRY(cudaEventRecord(S->ev_out_u, S->stream));
    CUDA_TRY(cudaStreamWaitEvent(S->d2h_stream, S->ev_out_u, 0));
    if (u)
        CUDA_TRY(cudaMemcpyAsync(u, S->out_e, sizeof(double) * m.nE * Ly, cudaMemcpyDeviceToHost, S->d2h_stream));
    CUDA_TRY(cudaEventRecord(S->ev_out_free, S->d2h_stream));
    if (d) {
        const int slot = static_cast<int>(S->pending_diag.size());
        CUDA_TRY(cudaStreamWaitEvent(S->diag_stream, S->ev_out_u, 0));
        CUDA_TRY(launch_diagnostics_snapshot(S->kc, S->tables, S->snap_c, S->snap_e, S->p.g, S->diag_partial,
                                             S->diag_blocks, S->diag_out, S->diag_stream));
        CUDA_TRY(cudaMemcpyAsync(S->diag_host + 2 * slot, S->diag_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                 S->diag_stream));
        CUDA_TRY(cudaEventRecord(S->ev_snap_free, S->diag_stream));
        S->pending_diag.push_back({d, S->time, S->steps});
    }
    return LTS_OK;
}

// Waits for everything enqueued on the state and its copy streams, fills
// the pending diagnostics and reports (and clears) the error flag.
int sync_state(lts_state_s* S) {
    // the callers' records are filled only on success; on any error they are
    // dropped, so no later call writes through a pointer the caller may have
    // released
    std::vector<lts_state_s::PendingDiag> pending;
    pending.swap(S->pending_diag);
    CUDA_TRY(cudaMemcpyAsync(S->flag_host, S->flag, sizeof(int), cudaMemcpyDeviceToHost, S->stream));
    CUDA_TRY(cudaMemsetAsync(S->flag, 0, sizeof(int), S->stream));
    CUDA_TRY(cudaStreamSynchronize(S->stream));
    CUDA_TRY(cudaStreamSynchronize(S->h2d_stream));
    CUDA_TRY(cudaStreamSynchronize(S->d2h_stream));
    CUDA_TRY(cudaStreamSynchronize(S->diag_stream));
    for (size_t k = 0; k < pending.size(); ++k) {
        lts_diag* d = pending[k].d;
        d->mass = S->diag_host[2 * k];
        d->energy = S->diag_host[2 * k + 1];
        d->time = pending[k].time;
        d->steps = pending[k].steps;
    }
    const int flag = *S->flag_host;
    if (flag & 4) return set_error(LTS_ECUDA, "internal error: a tile exceeded its shared memory (skipped)");
    if (flag)
        return set_error(LTS_ENONFINITE, "a stage produced %s",
                         (flag & 1) ? "a thickness <= 0 or non-finite" : "a non-finite velocity");
    return LTS_OK;
}

}  // namespace

namespace lts {
int device_check() { return check_device(); }
void make_plan(lts_state_s* S, int parity, std::vector<LaunchDesc>& out) {
    if (S->p.mode == LTS_MODE_LTS) {
        if (S->reg->r.order == 2) plan_lts2(S, parity, out);
        else plan_lts3(S, parity, out);
    } else if (S->p.mode == LTS_MODE_SSPRK2) {
        plan_ssprk2(S, parity, out);
    } else {
        plan_ssprk3(S, parity, out);
    }
}
double plan_launch_bytes(const LaunchDesc& d, const RegionsHost& r, int nC, int nE, int nV, size_t T,
                         bool comp) {
    return launch_bytes(d, r, nC, nE, nV, T, comp, 1);
}
}  // namespace lts

lts_state_s::~lts_state_s() {
    // copies may still be in flight into pinned or caller memory: finish them
    // before anything they use is released.  Only the library's own streams
    // are waited for (a caller's stream may already be gone); the copy
    // streams wait on the caller's stream through events, and the device
    // buffers are freed by calls that synchronise.
    if (own_stream && stream) cudaStreamSynchronize(stream);
    for (cudaStream_t st : {side_stream, h2d_stream, d2h_stream, diag_stream})
        if (st) cudaStreamSynchronize(st);
    for (auto& e : exec)
        if (e) cudaGraphExecDestroy(e);
    for (auto ev : events) cudaEventDestroy(ev);
    for (auto& v : gevents)
        for (auto ev : v) cudaEventDestroy(ev);
    if (own_stream && stream) cudaStreamDestroy(stream);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (side_stream) cudaStreamDestroy(side_stream);
    if (h2d_stream) cudaStreamDestroy(h2d_stream);
    if (d2h_stream) cudaStreamDestroy(d2h_stream);
    if (diag_stream) cudaStreamDestroy(diag_stream);
    for (auto ev : {ev_in_h, ev_in_u, ev_in_free, ev_out_h, ev_out_u, ev_out_free, ev_snap_free})
        if (ev) cudaEventDestroy(ev);
    if (flag_host) cudaFreeHost(flag_host);
    if (diag_host) cudaFreeHost(diag_host);
    if (capture_side) cudaStreamDestroy(capture_side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
}

// ---------------------------------------------------------------- the C ABI

extern "C" {

int lts_mesh_create(const lts_mesh_desc* d, lts_mesh* out) {
    if (!d || !out) return set_error(LTS_EINVAL, "null argument");
    *out = nullptr;
    const int nC = d->nCells, nE = d->nEdges, nV = d->nVertices, W = d->maxEdges;
    if (nC < 3 || nE < 3 || nV < 2 || W < 3 || W > MAX_DEGREE)
        return set_error(LTS_EINVAL, "bad mesh sizes (nCells %d, nEdges %d, nVertices %d, maxEdges %d)",
                         nC, nE, nV, W);
    if (!d->nEdgesOnCell || !d->edgesOnCell || !d->cellsOnCell || !d->verticesOnCell ||
        !d->cellsOnEdge || !d->verticesOnEdge || !d->edgesOnVertex || !d->cellsOnVertex ||
        !d->areaCell || !d->areaTriangle || !d->kiteAreasOnVertex || !d->dcEdge || !d->dvEdge ||
        !d->fVertex)
        return set_error(LTS_EINVAL, "a required mesh array is NULL");
    std::unique_ptr<lts_mesh_s> M(new (std::nothrow) lts_mesh_s);
    if (!M) return set_error(LTS_ENOMEM, "out of host memory");
    HostMesh& m = M->m;
    m.nC = nC; m.nE = nE; m.nV = nV; m.maxE = W;
    m.sphere = d->on_sphere != 0;
    m.R = d->radius; m.Lx = d->period_x; m.Ly = d->period_y;
    auto cp = [](auto* p, size_t n, auto& v) { v.assign(p, p + n); };
    try {
        if (d->xCell && d->yCell && d->zCell) {
            cp(d->xCell, nC, m.xc); cp(d->yCell, nC, m.yc); cp(d->zCell, nC, m.zc);
        } else {
            m.xc.assign(nC, 0.0); m.yc.assign(nC, 0.0); m.zc.assign(nC, 0.0);
        }
        cp(d->nEdgesOnCell, nC, m.nEoC);
        cp(d->edgesOnCell, (size_t)nC * W, m.EoC);
        cp(d->cellsOnCell, (size_t)nC * W, m.CoC);
        cp(d->verticesOnCell, (size_t)nC * W, m.VoC);
        cp(d->cellsOnEdge, 2 * (size_t)nE, m.CoE);
        cp(d->verticesOnEdge, 2 * (size_t)nE, m.VoE);
        cp(d->edgesOnVertex, 3 * (size_t)nV, m.EoV);
        cp(d->cellsOnVertex, 3 * (size_t)nV, m.CoV);
        cp(d->areaCell, nC, m.A);
        cp(d->areaTriangle, nV, m.Av);
        cp(d->kiteAreasOnVertex, 3 * (size_t)nV, m.kite);
        cp(d->dcEdge, nE, m.dc);
        cp(d->dvEdge, nE, m.dv);
        cp(d->fVertex, nV, m.f);
        if (d->bottom) cp(d->bottom, nC, m.b);
        else m.b.assign(nC, 0.0);
    } catch (const std::bad_alloc&) {
        return set_error(LTS_ENOMEM, "out of host memory");
    }
    // ---- validation
    for (int i = 0; i < nC; ++i) {
        int n = m.nEoC[i];
        if (n < 3 || n > W) return set_error(LTS_EINVAL, "cell %d has %d edges", i, n);
        if (!(m.A[i] > 0.0)) return set_error(LTS_EINVAL, "areaCell[%d] <= 0", i);
        for (int j = 0; j < n; ++j) {
            int e = m.EoC[(size_t)i * W + j], nb = m.CoC[(size_t)i * W + j], v = m.VoC[(size_t)i * W + j];
            if (e < 0 || e >= nE || nb < 0 || nb >= nC || v < 0 || v >= nV)
                return set_error(LTS_EINVAL, "cell %d slot %d: index out of range", i, j);
        }
    }
    for (int e = 0; e < nE; ++e) {
        for (int k = 0; k < 2; ++k) {
            if (m.CoE[2 * e + k] < 0 || m.CoE[2 * e + k] >= nC || m.VoE[2 * e + k] < 0 ||
                m.VoE[2 * e + k] >= nV)
                return set_error(LTS_EINVAL, "edge %d: index out of range", e);
        }
        if (m.CoE[2 * e] == m.CoE[2 * e + 1]) return set_error(LTS_EINVAL, "edge %d joins a cell to itself", e);
        if (!(m.dc[e] > 0.0) || !(m.dv[e] >= 0.0)) return set_error(LTS_EINVAL, "edge %d: bad lengths", e);
    }
    for (int v = 0; v < nV; ++v) {
        if (!(m.Av[v] > 0.0)) return set_error(LTS_EINVAL, "areaTriangle[%d] <= 0", v);
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
            if (m.EoV[3 * v + k] < 0 || m.EoV[3 * v + k] >= nE || m.CoV[3 * v + k] < 0 || m.CoV[3 * v + k] >= nC)
                return set_error(LTS_EINVAL, "vertex %d: index out of range", v);
            s += m.kite[3 * v + k];
        }
        if (std::fabs(s - m.Av[v]) > 1e-9 * m.Av[v])
            return set_error(LTS_EINVAL, "kites of vertex %d do not sum to areaTriangle", v);
    }
    // rings: slot j joins cell i and cellsOnCell[j]; vertex j is shared by
    // slots j and j+1; the ring is counter-clockwise (t_{e_j, v_j} = n_{e_j, i})
    std::vector<double> ksum(nC, 0.0);
    for (int v = 0; v < nV; ++v)
        for (int k = 0; k < 3; ++k) ksum[m.CoV[3 * v + k]] += m.kite[3 * v + k];
    for (int i = 0; i < nC; ++i) {
        if (std::fabs(ksum[i] - m.A[i]) > 1e-9 * m.A[i])
            return set_error(LTS_EINVAL, "kites of cell %d do not sum to areaCell", i);
        int n = m.nEoC[i];
        for (int j = 0; j < n; ++j) {
            int e = m.EoC[(size_t)i * W + j], nb = m.CoC[(size_t)i * W + j];
            int v = m.VoC[(size_t)i * W + j];
            int e2 = m.EoC[(size_t)i * W + (j + 1) % n];
            bool has_i = m.CoE[2 * e] == i || m.CoE[2 * e + 1] == i;
            bool has_nb = m.CoE[2 * e] == nb || m.CoE[2 * e + 1] == nb;
            if (!has_i || !has_nb) return set_error(LTS_EINVAL, "cell %d slot %d: edge/neighbour mismatch", i, j);
            bool v_on_e = m.VoE[2 * e] == v || m.VoE[2 * e + 1] == v;
            bool v_on_e2 = m.VoE[2 * e2] == v || m.VoE[2 * e2 + 1] == v;
            if (!v_on_e || !v_on_e2) return set_error(LTS_EINVAL, "cell %d slot %d: vertex not between slots", i, j);
            bool left = m.VoE[2 * e + 1] == v;
            bool out = m.CoE[2 * e] == i;
            if (left != out) return set_error(LTS_EINVAL, "cell %d: ring is not counter-clockwise", i);
        }
    }
    // optional MPAS weights: compare with the kite-derived ones
    if (d->weightsOnEdge && d->edgesOnEdge && d->nEdgesOnEdge) {
        for (int e = 0; e < nE; ++e) {
            int cnt = d->nEdgesOnEdge[e];
            for (int q = 0; q < cnt; ++q) {
                int ep = d->edgesOnEdge[(size_t)e * 2 * W + q];
                double w = d->weightsOnEdge[(size_t)e * 2 * W + q];
                double best = 1e300;
                for (int s = 0; s < 2; ++s) {
                    int c = m.CoE[2 * e + s];
                    int jp = -1, je = -1;
                    for (int j = 0; j < m.nEoC[c]; ++j) {
                        if (m.EoC[(size_t)c * W + j] == ep) jp = j;
                        if (m.EoC[(size_t)c * W + j] == e) je = j;
                    }
                    if (jp >= 0 && je >= 0) best = std::min(best, std::fabs(derived_weight(m, c, jp, je) - w));
                }
                if (best > 1e-9)
                    return set_error(LTS_EINVAL, "weightsOnEdge[%d][%d] disagrees with the kite areas", e, q);
            }
        }
    }
    *out = M.release();
    return LTS_OK;
}

void lts_mesh_destroy(lts_mesh m) { release_mesh(m); }

int lts_regions_set(lts_mesh m, const int8_t* fine_mask, int32_t order, int32_t M, int32_t layers,
                    lts_regions* out) {
    if (!m || !fine_mask || !out) return set_error(LTS_EINVAL, "null argument");
    *out = nullptr;
    if (order != 2 && order != 3) return set_error(LTS_EINVAL, "order %d not supported (2 = LTS2, 3 = LTS3)", order);
    if (M < 1 || M > 4096) return set_error(LTS_EINVAL, "M must be in [1, 4096]");
    std::unique_ptr<lts_regions_s> R(new (std::nothrow) lts_regions_s);
    if (!R) return set_error(LTS_ENOMEM, "out of host memory");
    int rc;
    try {
        rc = compute_regions(m->m, fine_mask, layers, 0, R->r);
        if (rc == LTS_OK) rc = build_tiles(m->m, R->r, kDefaultTileCells);
    } catch (const std::bad_alloc&) {
        return set_error(LTS_ENOMEM, "out of host memory");
    }
    if (rc != LTS_OK) return rc;
    R->r.M = M;
    R->r.order = order;
    m->ref++;
    R->mesh = m;
    *out = R.release();
    return LTS_OK;
}

int lts_regions_set_multi(lts_mesh m, const int8_t* region_of_cell, int32_t nregions, const int32_t* M,
                          int32_t order, int32_t layers, lts_regions* out) {
    if (!m || !region_of_cell || !M || !out) return set_error(LTS_EINVAL, "null argument");
    *out = nullptr;
    if (order != 3) return set_error(LTS_EINVAL, "several fine regions run LTS3 only (order 3)");
    if (nregions < 1 || nregions > 64) return set_error(LTS_EINVAL, "nregions must be in [1, 64]");
    for (int k = 0; k < nregions; ++k)
        if (M[k] < 1 || M[k] > 4096) return set_error(LTS_EINVAL, "M of region %d must be in [1, 4096]", k + 1);
    std::unique_ptr<lts_regions_s> R(new (std::nothrow) lts_regions_s);
    if (!R) return set_error(LTS_ENOMEM, "out of host memory");
    int rc;
    try {
        rc = compute_regions_multi(m->m, region_of_cell, nregions, layers, 0, R->r);
        if (rc == LTS_OK && nregions == 1) rc = build_tiles(m->m, R->r, kDefaultTileCells);
    } catch (const std::bad_alloc&) {
        return set_error(LTS_ENOMEM, "out of host memory");
    }
    if (rc != LTS_OK) return rc;
    R->r.M = M[0];
    R->r.Mr.assign(M, M + nregions);
    R->r.order = order;
    m->ref++;
    R->mesh = m;
    *out = R.release();
    return LTS_OK;
}

void lts_regions_destroy(lts_regions r) { release_regions(r); }

int lts_regions_labels(lts_regions r, int8_t* cl, int8_t* el) {
    if (!r) return set_error(LTS_EINVAL, "null regions");
    static const int8_t cmap[NBANDS] = {0, 0, 1, 2, 3, 4, 5, 5, 5, 5, 5, 5};
    static const int8_t emap[NBANDS] = {0, 0, 1, 1, 3, 4, 5, 5, 5, 5, 5, 5};
    if (cl)
        for (size_t i = 0; i < r->r.cband.size(); ++i) cl[i] = cmap[r->r.cband[i]];
    if (el)
        for (size_t e = 0; e < r->r.eband.size(); ++e) el[e] = emap[r->r.eband[e]];
    return LTS_OK;
}

int lts_regions_tiling(lts_regions r, int32_t tile_cells) {
    if (!r) return set_error(LTS_EINVAL, "null regions");
    if (r->r.nreg > 1) return set_error(LTS_EINVAL, "several fine regions have no tiles (three-launch path)");
    if (r->ref.load() != 1) return set_error(LTS_EINVAL, "regions are in use by a state");
    int rc;
    try {
        rc = build_tiles(r->mesh->m, r->r, tile_cells);
    } catch (const std::bad_alloc&) {
        return set_error(LTS_ENOMEM, "out of host memory");
    }
    if (rc != LTS_OK) return rc;
    r->arena[0].reset();   // device tables are rebuilt on the next state creation
    r->arena[1].reset();
    r->d_perm_c = r->d_perm_e = nullptr;
    return LTS_OK;
}

int lts_regions_ordering(lts_regions r, int32_t ordering) {
    if (!r) return set_error(LTS_EINVAL, "null regions");
    if (r->ref.load() != 1) return set_error(LTS_EINVAL, "regions are in use by a state");
    if (ordering == r->r.ordering) return LTS_OK;
    RegionsHost nr;
    int rc;
    try {
        if (r->r.nreg > 1) {
            const std::vector<int8_t> rid = r->r.rid;
            rc = compute_regions_multi(r->mesh->m, rid.data(), r->r.nreg, r->r.layers, ordering, nr);
        } else {
            const std::vector<int8_t> fine = r->r.fine;
            rc = compute_regions(r->mesh->m, fine.data(), r->r.layers, ordering, nr);
            if (rc == LTS_OK) rc = build_tiles(r->mesh->m, nr, r->r.tile_cells);
        }
    } catch (const std::bad_alloc&) {
        return set_error(LTS_ENOMEM, "out of host memory");
    }
    if (rc != LTS_OK) return rc;
    nr.M = r->r.M;
    nr.Mr = r->r.Mr;
    nr.order = r->r.order;
    r->r = std::move(nr);
    r->arena[0].reset();   // device tables are rebuilt on the next state creation
    r->arena[1].reset();
    r->d_perm_c = r->d_perm_e = nullptr;
    return LTS_OK;
}

int lts_regions_counts(lts_regions r, int64_t* cells, int64_t* edges, int64_t* vertices) {
    if (!r) return set_error(LTS_EINVAL, "null regions");
    for (int k = 0; k < NBANDS; ++k) {
        if (cells) cells[k] = r->r.cb[k + 1] - r->r.cb[k];
        if (edges) edges[k] = r->r.eb[k + 1] - r->r.eb[k];
        if (vertices) vertices[k] = r->r.vb[k + 1] - r->r.vb[k];
    }
    return LTS_OK;
}

int lts_regions_permutation(lts_regions r, int32_t* pc, int32_t* pe, int32_t* pv) {
    if (!r) return set_error(LTS_EINVAL, "null regions");
    if (pc) std::copy(r->r.perm_c.begin(), r->r.perm_c.end(), pc);
    if (pe) std::copy(r->r.perm_e.begin(), r->r.perm_e.end(), pe);
    if (pv) std::copy(r->r.perm_v.begin(), r->r.perm_v.end(), pv);
    return LTS_OK;
}

int lts_state_create(lts_mesh mesh, lts_regions reg, const double* h0, const double* u0,
                     const lts_params* p, lts_state* out) {
    if (!mesh || !reg || !h0 || !u0 || !p || !out) return set_error(LTS_EINVAL, "null argument");
    *out = nullptr;
    if (reg->mesh != mesh) return set_error(LTS_EINVAL, "regions belong to another mesh");
    if (!(p->dt > 0.0) || !(p->g > 0.0)) return set_error(LTS_EINVAL, "dt and g must be > 0");
    if (p->precision != LTS_FP32 && p->precision != LTS_FP64)
        return set_error(LTS_EINVAL, "precision must be LTS_FP32 or LTS_FP64");
    if (p->mode != LTS_MODE_LTS && p->mode != LTS_MODE_SSPRK3 && p->mode != LTS_MODE_SSPRK2)
        return set_error(LTS_EINVAL, "mode must be LTS_MODE_LTS, LTS_MODE_SSPRK3 or LTS_MODE_SSPRK2");
    if (p->kernel_path == 1 && (p->mode == LTS_MODE_SSPRK2 || (p->mode == LTS_MODE_LTS && reg->r.order == 2)))
        return set_error(LTS_EINVAL, "the fused tile kernel runs LTS3 and SSPRK3 only");
    const bool multi = reg->r.nreg > 1 && p->mode == LTS_MODE_LTS;
    if (multi && (p->kernel_path != 0 || p->profile != 0 || (p->layers > 1)))
        return set_error(LTS_EINVAL,
                         "several fine regions run the three-launch path, single layer, without profiling");
    int bs = p->block_size ? p->block_size : 256;
    if (bs < 32 || bs > 256 || bs % 32) return set_error(LTS_EINVAL, "block_size must be 32..256, multiple of 32");
    int rc = check_device();
    if (rc != LTS_OK) return rc;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (reg->device >= 0 && reg->device != dev) return set_error(LTS_EINVAL, "regions live on another device");
    reg->device = dev;
    const int which = p->precision == LTS_FP64 ? 1 : 0;
    if (!reg->arena[which]) {
        rc = which ? build_tables<double>(reg, 1, reg->t64) : build_tables<float>(reg, 0, reg->t32);
        if (rc != LTS_OK) return rc;
    }
    std::unique_ptr<lts_state_s> S(new (std::nothrow) lts_state_s);
    if (!S) return set_error(LTS_ENOMEM, "out of host memory");
    S->p = *p;
    S->kc.precision = which;
    S->kc.comp = (which == 0) && p->compensated;
    S->kc.block = bs;
    S->tsz = which ? 8 : 4;
    S->kc.maxdeg = mesh->m.maxE <= 8 ? 8 : MAX_DEGREE;
    const int layers = p->layers > 0 ? p->layers : 1;
    if (layers > 65536) return set_error(LTS_EINVAL, "layers must be in [1, 65536]");
    if (layers > 1 && p->kernel_path != 0)
        return set_error(LTS_EINVAL, "multi-layer states run the three-launch path only (kernel_path 0)");
    if (static_cast<long long>(mesh->m.maxE) * mesh->m.nC * layers > 0x7fffffffLL * 8LL ||
        static_cast<long long>(mesh->m.nE) * layers > 0x7fffffffLL ||
        static_cast<long long>(slot_rows(mesh->m.maxE)) * mesh->m.nC > 0x7fffffffLL)
        return set_error(LTS_EINVAL, "mesh x layers too large");
    if (p->coarse_schedule < LTS_COARSE_FAR || p->coarse_schedule > LTS_COARSE_SERIAL)
        return set_error(LTS_EINVAL, "coarse_schedule must be LTS_COARSE_FAR, _STEP4 or _SERIAL");
    if (p->kernel_path != 0 && p->kernel_path != 1)
        return set_error(LTS_EINVAL, "kernel_path must be 0 (three launches) or 1 (fused tiles)");
    {
        const int nv = (reg->r.max_local_verts + 3) & ~3;
        S->kc.tile_smem = static_cast<int>(S->tsz) * (nv + (S->kc.maxdeg + 1) * reg->r.max_local_cells);
        if (S->kc.tile_smem > 227 * 1024) return set_error(LTS_EINVAL, "tiles need too much shared memory");
    }
    S->kc.mindeg = *std::min_element(mesh->m.nEoC.begin(), mesh->m.nEoC.end());
    S->kc.pdl = p->pdl != 0 && p->profile == 0;
    S->kc.layers = layers;
    S->kc.lpt = std::min(kLayersPerThread, layers);
    if (p->ring_occupancy != 0 && p->ring_occupancy != 6 && p->ring_occupancy != 8)
        return set_error(LTS_EINVAL, "ring_occupancy must be 0, 6 or 8");
    S->kc.ring_occ = p->ring_occupancy;
    if (p->elems_per_thread < 0 || p->elems_per_thread > 2)
        return set_error(LTS_EINVAL, "elems_per_thread must be 0, 1 or 2");
    S->kc.ept = p->elems_per_thread == 0 ? LTS_DEFAULT_EPT : p->elems_per_thread;
    S->tables = which ? static_cast<const void*>(&reg->t64) : static_cast<const void*>(&reg->t32);
    if (p->stream) {
        S->stream = static_cast<cudaStream_t>(p->stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
        S->own_stream = true;
    }
    CUDA_TRY(cudaStreamCreateWithFlags(&S->capture_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&S->capture_side, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&S->side_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&S->h2d_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&S->d2h_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&S->diag_stream, cudaStreamNonBlocking));
    for (cudaEvent_t* ev : {&S->ev_in_h, &S->ev_in_u, &S->ev_in_free, &S->ev_out_h, &S->ev_out_u, &S->ev_out_free,
                            &S->ev_snap_free})
        CUDA_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&S->flag_host), sizeof(int), cudaHostAllocDefault));
    CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&S->diag_host), sizeof(double) * 2 * lts_state_s::kDiagSlots,
                           cudaHostAllocDefault));
    CUDA_TRY(cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&S->ev_join, cudaEventDisableTiming));
    reg->ref++;
    S->reg = reg;
    S->multi = multi;
    rc = state_alloc(S.get());
    if (rc != LTS_OK) {
        release_regions(reg);
        S->reg = nullptr;
        return rc;
    }
    if (multi) {
        // one block per virtual block: on the 2.6M-cell two-cap mesh 2.55 ms
        // per coarse step against 2.79 ms for a persistent grid, whose loop
        // costs the ring its register budget
        for (int par = 0; par < 2 && rc == LTS_OK; ++par) {
            TablePlanStats st;
            rc = build_multi_plan(S.get(), par, 0, &st);
            if (par == 0)
                for (int k = 0; k < NKINDS; ++k) {
                    S->bytes[k] = st.bytes[k];
                    S->launches[k] = 0;
                }
            if (par == 0)
                for (const auto& L : S->tplan[0])
                    if (L.nseg) S->launches[L.d.kind] += 1;
        }
        if (rc != LTS_OK) {
            lts_regions_s* keep = S->reg;
            S.reset();
            release_regions(keep);
            return rc;
        }
    }
    for (int par = 0; par < 2 && !multi; ++par) {
        if (p->kernel_path == 1) {
            if (p->mode == LTS_MODE_LTS) plan_lts3_fused(S.get(), par, S->plan[par]);
            else plan_ssprk3_fused(S.get(), par, S->plan[par]);
        } else {
            make_plan(S.get(), par, S->plan[par]);
        }
    }
    if (p->no_l2_hints)
        for (auto& plan : S->plan)
            for (LaunchDesc& d : plan) d.l2 = 0;
    // launch statistics of one step (both parities have the same sizes)
    const HostMesh& m = mesh->m;
    for (LaunchDesc& d : S->plan[0]) {
        if (d.nseg == 0) continue;
        d.bytes = launch_bytes(d, reg->r, m.nC, m.nE, m.nV, S->tsz, S->kc.comp, S->kc.layers);
        S->bytes[d.kind] += d.bytes;
        S->launches[d.kind] += 1;
    }
    rc = write_state(S.get(), h0, u0);
    if (rc == LTS_OK && ((p->use_graph && p->profile != 1) || p->profile == 2)) rc = capture_graphs(S.get());
    if (rc == LTS_OK) {
        cudaError_t e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) rc = set_error(LTS_ECUDA, "state upload: %s", cudaGetErrorString(e));
    }
    if (rc != LTS_OK) {
        lts_regions_s* keep = S->reg;
        S.reset();
        release_regions(keep);
        return rc;
    }
    *out = S.release();
    return LTS_OK;
}

void lts_state_destroy(lts_state s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    lts_regions_s* r = s->reg;
    delete s;
    release_regions(r);
}

int lts_step(lts_state s, int32_t n) {
    if (!s) return set_error(LTS_EINVAL, "null state");
    if (n < 0) return set_error(LTS_EINVAL, "n_coarse must be >= 0");
    if (s->p.profile == 2) {
        // graph launches with event nodes; per-kernel times summed over the call
        for (double& x : s->prof_ms) x = 0.0;
        for (int i = 0; i < n; ++i) {
            const int par = s->parity;
            CUDA_TRY(cudaGraphLaunch(s->exec[par], s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
            const auto& plan = s->plan[par];
            for (size_t k = 0; k < plan.size(); ++k) {
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, s->gevents[par][2 * k], s->gevents[par][2 * k + 1]));
                s->prof_ms[plan[k].kind] += ms;
            }
            s->parity ^= 1;
            s->steps++;
            s->time += s->p.dt;
        }
        return LTS_OK;
    }
    if (s->p.profile == 1) {
        const size_t L = s->plan[0].size();
        if (s->events.size() < 2 * L) {
            for (size_t k = s->events.size(); k < 2 * L; ++k) {
                cudaEvent_t ev;
                CUDA_TRY(cudaEventCreate(&ev));
                s->events.push_back(ev);
            }
        }
        for (double& x : s->prof_ms) x = 0.0;
        for (int i = 0; i < n; ++i) {
            const auto& plan = s->plan[s->parity];
            for (size_t k = 0; k < plan.size(); ++k) {
                CUDA_TRY(cudaEventRecord(s->events[2 * k], s->stream));
                cudaError_t e = launch_phase(plan[k], s->tables, s->kc, s->flag, s->stream);
                if (e != cudaSuccess) return set_error(LTS_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
                CUDA_TRY(cudaEventRecord(s->events[2 * k + 1], s->stream));
            }
            CUDA_TRY(cudaStreamSynchronize(s->stream));
            for (size_t k = 0; k < plan.size(); ++k) {
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, s->events[2 * k], s->events[2 * k + 1]));
                s->prof_ms[plan[k].kind] += ms;
            }
            s->parity ^= 1;
            s->steps++;
            s->time += s->p.dt;
        }
        return LTS_OK;
    }
    for (int i = 0; i < n; ++i) {
        if (s->exec[s->parity]) {
            CUDA_TRY(cudaGraphLaunch(s->exec[s->parity], s->stream));
        } else {
            int rc = s->multi ? enqueue_table_plan(s->tplan[s->parity], s->tables, s->kc, s->flag, s->stream,
                                                   s->side_stream, s->ev_fork, s->ev_join)
                              : enqueue_plan(s, s->plan[s->parity], s->stream, s->side_stream);
            if (rc != LTS_OK) return rc;
        }
        s->parity ^= 1;
        s->steps++;
        s->time += s->p.dt;
    }
    return LTS_OK;
}

int lts_read(lts_state s, double* h, double* u, lts_diag* d) {
    if (!s) return set_error(LTS_EINVAL, "null state");
    int rc = read_state(s, h, u, d);
    const int rs = sync_state(s);
    return rc != LTS_OK ? rc : rs;
}

int lts_read_async(lts_state s, double* h, double* u, lts_diag* d) {
    if (!s) return set_error(LTS_EINVAL, "null state");
    return read_state(s, h, u, d);
}

int lts_sync(lts_state s) {
    if (!s) return set_error(LTS_EINVAL, "null state");
    return sync_state(s);
}

int lts_write(lts_state s, const double* h, const double* u, double time, int64_t steps) {
    if (!s || !h || !u) return set_error(LTS_EINVAL, "null argument");
    int rc = write_state(s, h, u);
    if (rc != LTS_OK) return rc;
    s->time = time;
    s->steps = steps;
    return LTS_OK;
}

}  // extern "C"

namespace lts {
int state_view(lts_state s, StateView* v) {
    if (!s || !v) return set_error(LTS_EINVAL, "null argument");
    const SV& X = s->buf[s->parity];
    v->kc = s->kc;
    v->tables = s->tables;
    v->h_hi = X.hh;
    v->h_lo = X.hl;
    v->u_hi = X.uh;
    v->u_lo = X.ul;
    v->g = s->p.g;
    v->nC = s->reg->mesh->m.nC;
    v->device = s->reg->device;
    v->stream = s->stream;
    return LTS_OK;
}
}  // namespace lts

extern "C" {

int lts_step_stats(lts_state s, int32_t* launches_per_step, double* bytes, double* ms,
                   int32_t* launches_per_kind) {
    if (!s) return set_error(LTS_EINVAL, "null state");
    if (launches_per_step) {
        *launches_per_step = 0;
        for (int k = 0; k < NKINDS; ++k) *launches_per_step += s->launches[k];
    }
    for (int k = 0; k < NKINDS; ++k) {
        if (bytes) bytes[k] = s->bytes[k];
        if (ms) ms[k] = s->prof_ms[k];
        if (launches_per_kind) launches_per_kind[k] = s->launches[k];
    }
    return LTS_OK;
}

}  // extern "C"
