// lts_internal.h -- structures shared by the host runtime (C++) and the
// CUDA kernels of liblts.so.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace lts {

// Bands of the band ordering (cells; an edge takes the smaller band of its
// two cells, a vertex the smallest band of its three cells).  C1..C5 are the
// coarse layers at edge distance 1..5 from I2: the halos the near-interface
// coarse phases read, so the far coarse bands can run concurrently.
enum Band : int {
    B_FDEEP = 0, B_F3 = 1, B_F2 = 2, B_F1 = 3, B_I1 = 4, B_I2 = 5, B_C1 = 6, B_C2 = 7,
    B_C3 = 8, B_C4 = 9, B_C5 = 10, B_CREST = 11, NBANDS = 12
};

// Device tables in band order.  Cell "slot" arrays are slot-major:
// element (slot j, cell c) is at [j * nC + c]; slot j of cell c holds the
// j-th edge of c counter-clockwise, the neighbour across it, and the vertex
// between slot j and slot j+1.  Slots j >= nEdgesOnCell repeat slot 0 (valid
// indices, never used in a sum), so they may be loaded unconditionally.
template <class T>
struct Tables {
    int nC, nE, nV, maxE;
    // cells
    const uint8_t* cn;   // [nC]       number of edges
    const int* se;       // [maxE*nC]  edge of slot j
    const int* sn;       // [maxE*nC]  neighbour cell across slot j
    const int* sv;       // [maxE*nC]  vertex between slot j and j+1
    const T* snl;        // [maxE*nC]  n_{e,c} l_e      (signed primal length)
    const T* sR;         // [maxE*nC]  A_{c,v_j} / A_c  (kite fraction)
    const T* sK;         // [maxE*nC]  l_e d_e / (4 A_c)
    // the same slots packed for the ring pass's vector loads: {se, sn, sv,
    // the bits of snl in FP32 (0 in FP64)} and, in FP32, {sR, sK}
    const int4* sidx;    // [maxE*nC]
    const float2* scf;   // [maxE*nC]  (FP32 tables only)
    const T* rA;         // [nC]       1 / A_c
    const T* b;          // [nC]       bottom topography
    // edges
    const int* ec0;      // [nE]       cell n_e points out of
    const int* ec1;      // [nE]       cell n_e points into
    const uint32_t* ep;  // [nE]       slot of e in ec0 (bits 0-7) and in ec1 (bits 8-15)
    const T* rdc;        // [nE]       1 / d_e
    const T* db;         // [nE]       b_{c1} - b_{c0}, formed in T from the T copies of b
    // vertices
    const int* vc0; const int* vc1; const int* vc2;   // [nV] cells on vertex
    const int* ve0; const int* ve1; const int* ve2;   // [nV] edges on vertex
    const T* vk0; const T* vk1; const T* vk2;         // [nV] A_{c,v} / A_v
    const T* vd0; const T* vd1; const T* vd2;         // [nV] t_{e,v} d_e / A_v
    const T* f;                                        // [nV] Coriolis parameter
    // the edge and vertex operands packed for the vector loads of the edge
    // and vertex passes: {ec0, ec1, ep, the bits of rdc in FP32 (0 in FP64)},
    // {ve0, ve1, ve2, vc0} and, in FP32 only, {vd0, vd1, vd2, f} and
    // {vk0, vk1, vk2, the bits of vc1} (vc2 stays a plain array)
    const int4* erow;    // [nE]
    const int4* vri;     // [nV]
    const float4* vrd;   // [nV]  (FP32 tables only)
    const float4* vrk;   // [nV]  (FP32 tables only)
    // tiles of the fused kernel (kind 3)
    const int4* ta;      // [ntiles] {cell begin, own cells, halo begin, local cells}
    const int4* tbk;     // [ntiles] {edge begin, edge end, vertex-list begin, local vertices}
    const int* tlsv;     // [ntiles] start of the tile's local-slot-vertex block
    const int* halo;     // halo cells of all tiles
    const int* tverts;   // local vertex lists of all tiles
    const uint16_t* lsv; // local vertex of (slot, local cell), slot-major per tile
    const uint32_t* lec; // [nE] local cells of the owning tile: c0 | c1 << 16
    // diagnostics
    const double* area;  // [nC] A_c (FP64 master copy)
    const double* bd;    // [nC] b   (FP64 master copy)
    const double* sK64;  // [maxE*nC] l_e d_e / (4 A_c) in FP64
};

// Segment kinds of a phase launch.  One right-hand side is three launches:
// kind 0 (vertex): q_v; kind 1 (ring, one thread per cell): K_i, the
// per-slot potential-vorticity contributions and H_i with its stage update;
// kind 2 (edge): U_e from the ring results, with its stage update.
// Pointwise segments (PRED, COPY, REPLAY) may ride in any launch.
enum SegType : int {
    SEG_VERT = 0,       // q_v from the launch's input state
    SEG_RING = 1,       // ring results only (halo cells of the updated edges)
    SEG_RING_UPD = 2,   // ring results + H_i, then x_out = combine(x_old, x_in, a, D, H)
    SEG_RING_ACC = 3,   // ring results + H_i, then acc (+)= H
    SEG_EDGE_UPD = 4,   // U_e, then combine
    SEG_EDGE_ACC = 5,   // U_e, then acc (+)= U
    SEG_PRED = 6,       // out = x_old + c1 (x1 - x_old) + c2 (x2 - x_old)   (I1 prediction)
    SEG_COPY = 7,       // dst[i - base_dst] = src[i - base_src]   (hi and lo)
    SEG_REPLAY = 8,     // Step 5: three stage combinations from the accumulated RHS
    SEG_TILE = 9,       // fused right-hand side over tiles [begin, end) (one block per tile)
};

// Largest cell degree the ring kernel is compiled for (variants 8 and 16).
constexpr int MAX_DEGREE = 16;

constexpr int MAXSEG = 8;

// Host description of one segment.  Pointers index element arrays of the
// right kind (cells or edges); "lo" pointers may be null when the state
// carries no compensation word.
struct SegDesc {
    int type = 0;
    int begin = 0, end = 0;   // element range [begin, end)
    int base = 0;             // compact-array offset (acc, snapshots): compact index = i - base
    int base2 = 0;            // second offset (COPY source)
    int flag = 0;             // ACC: 1 = first term (store); PRED: 0 general, 1/2/3 select old/x1/x2
    int flag2 = 0;            // TILE: first tile that accumulates instead of updating
    double c[4] = {0, 0, 0, 0};  // UPD: a, D; PRED: c1, c2; REPLAY: D1, D2, D3
    void* p[10] = {};         // see kernels.cu for the meaning per type
    // host-only: element kind of [begin, end) and the compact family that
    // `base` / `base2` index (used to place a member's segments in an ensemble)
    int elem = 0;             // ELEM_CELL, ELEM_EDGE or ELEM_VERT
    int cfam = 0, cfam2 = 0;  // FAM_FULL, FAM_I1 or FAM_I
};
enum : int { ELEM_CELL = 0, ELEM_EDGE = 1, ELEM_VERT = 2 };
// Compact arrays: FAM_I1 holds band I1 (interface snapshots), FAM_I holds
// bands I1..I2 (correction accumulators); FAM_FULL = a full-length array.
enum : int { FAM_FULL = 0, FAM_I1 = 1, FAM_I = 2 };

struct LaunchDesc {
    int kind = 0;             // 0 = vertex, 1 = ring, 2 = edge, 3 = fused tiles
    int nseg = 0;
    SegDesc seg[MAXSEG];
    const void* in_h = nullptr;   // input state (hi words) of the RHS
    const void* in_hl = nullptr;  // compensation words of the input thickness (or null)
    const void* in_ul = nullptr;  // compensation words of the input velocity (or null)
    const void* in_u = nullptr;
    void* q = nullptr;            // vertex potential vorticity buffer
    void* ring_c = nullptr;       // [maxE*nC] per-slot PV contributions (slot-major)
    void* ring_k = nullptr;       // [nC] kinetic energy K_i
    double g = 9.81;
    double bytes = 0.0;           // algorithmic bytes (filled by the planner)
    int branch = 0;               // 0 = main stream, 1 = side branch (concurrent work)
    int l2 = 0;                   // L2 policy of read-only loads: 0 none, 1 keep, 2 stream
    bool fork = false;            // side branch starts here (waits for the main stream)
    bool join = false;            // main stream waits for the side branch before this launch
    int key = -1;                 // position in the step's phase structure (same key = same
                                  // phase, input buffers and kind in every plan)
};

// Launch keys of the LTS3 plan: the phase of a launch (Step 1, Step 2, the
// Step 4 side branch, Step 3 substep k stage s, the tail) plus its kind.
// Plans of different meshes have equal keys for the same phase, so an
// ensemble merges them launch by launch in key order.  SSPRK3 plans use
// 3 * stage + kind.
constexpr int KEY_STEP1 = 0, KEY_STEP2 = 3, KEY_SIDE = 10, KEY_STEP3 = 100, KEY_TAIL = 1000000;

// Slot-major cell tables (ring slots, their coefficients, the tiles' local
// vertex ids) hold at least this many rows, the extra rows repeating slot 0
// (indices) or zero (coefficients), so the ring kernels may load their first
// slots without knowing the cell's degree.
constexpr int kSlotRowsMin = 8;
inline int slot_rows(int maxE) { return maxE > kSlotRowsMin ? maxE : kSlotRowsMin; }

// Consecutive layers of one element per thread in multi-layer states.
constexpr int kLayersPerThread = 4;

// Elements per thread of the vertex and edge launches when the caller
// leaves the choice to the library.
constexpr int LTS_DEFAULT_EPT = 1;

struct KernelConfig {
    int precision;   // 0 FP32, 1 FP64
    bool comp;       // FP32 compensated
    int block;       // threads per block
    int maxdeg;      // ring kernel variant: 8 or 16
    int tile_smem;   // dynamic shared memory of the fused kernel (bytes)
    int mindeg;      // smallest cell degree of the mesh (slots loaded unconditionally)
    bool pdl;        // programmatic dependent launch
    int layers = 1;  // layers per element (multi-layer states)
    int ring_occ = 0;  // FP32 ring pass built for 6 or 8 resident blocks per SM (0: default)
    int ept = 1;       // elements per thread of the vertex and edge kinds (1 or 2)
    int lpt = 1;       // multi-layer states: consecutive layers of an element per thread
};

// kernels.cu
cudaError_t launch_phase(const LaunchDesc& d, const void* tables, const KernelConfig& kc,
                         int* flag, cudaStream_t s);
cudaError_t launch_scatter_state(const KernelConfig& kc, int n, const int* perm, const double* src,
                                 void* hi, void* lo, cudaStream_t s);
cudaError_t launch_gather_state(const KernelConfig& kc, int n, const int* perm, const void* hi,
                                const void* lo, double* dst, cudaStream_t s, double* snap = nullptr);
cudaError_t launch_diagnostics(const KernelConfig& kc, const void* tables, const void* h_hi,
                               const void* h_lo, const void* u_hi, const void* u_lo, double g,
                               double* partial, int nblocks, double* out2, cudaStream_t s);
// The same reduction over a band-order FP64 snapshot of the state (written
// by launch_gather_state), equal to the state's own to the last bit.
cudaError_t launch_diagnostics_snapshot(const KernelConfig& kc, const void* tables, const double* h,
                                        const double* u, double g, double* partial, int nblocks, double* out2,
                                        cudaStream_t s);
int kernel_registers(const KernelConfig& kc, int kind);
// Segment-table launches (ensembles).  encode_segment_table converts the
// non-empty segments of `segs` into the device records of kc's precision
// (bytes in `out`, count in *nseg_out) and returns the number of virtual
// blocks, or -1 for a segment kind the table kernel does not run (tiles).
int encode_segment_table(const KernelConfig& kc, const SegDesc* segs, int n,
                         std::vector<unsigned char>& out, int* nseg_out);
// One launch of kind d.kind (0..2) over a device segment table; d supplies
// the input state and intermediate buffers (its own segments are ignored).
// grid = number of resident blocks (persistent) or <= 0 for one block per
// virtual block.
cudaError_t launch_phase_table(const LaunchDesc& d, const void* dsegs, int nseg, int vblocks, int grid,
                               const void* tables, const KernelConfig& kc, int* flag, cudaStream_t s);
int table_blocks_per_sm(const KernelConfig& kc, int kind);

// Device view of a state's current solution, for entry points defined in
// other translation units (lts_api.cpp fills it).
struct StateView {
    KernelConfig kc;
    const void* tables;
    const void *h_hi, *h_lo, *u_hi, *u_lo;
    double g;
    int nC;
    int device;
    cudaStream_t stream;
};
constexpr int NKINDS = 4;

}  // namespace lts
