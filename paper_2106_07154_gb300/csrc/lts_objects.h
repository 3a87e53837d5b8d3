// lts_objects.h -- host objects behind the opaque handles of include/lts.h
// (mesh, regions, state), shared by the translation units of liblts.so.
// Not part of the public ABI.
#pragma once
#include <algorithm>
#include <atomic>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lts.h"
#include "lts_error.h"
#include "lts_internal.h"
#include "regions.h"

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess)                                                                \
            return lts::set_error(_e == cudaErrorMemoryAllocation ? LTS_ENOMEM : LTS_ECUDA,        \
                             "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
    } while (0)


// Device allocations freed together.  `err` records the first failure of a
// sequence of calls and is never reset to success, so a caller may check it
// once after many uploads.
struct DeviceArena {
    std::vector<void*> blocks;
    ~DeviceArena() {
        for (void* p : blocks) cudaFree(p);
    }
    template <class T>
    T* upload(const std::vector<T>& v, cudaError_t& err) {
        void* p = nullptr;
        size_t n = std::max<size_t>(1, v.size()) * sizeof(T);
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            if (err == cudaSuccess) err = e;
            return nullptr;
        }
        blocks.push_back(p);
        if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        return static_cast<T*>(p);
    }
    void* alloc(size_t bytes, cudaError_t& err) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            if (err == cudaSuccess) err = e;
            return nullptr;
        }
        blocks.push_back(p);
        e = cudaMemset(p, 0, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        return p;
    }
};

struct lts_mesh_s {
    std::atomic<int> ref{1};
    lts::HostMesh m;
};

struct lts_regions_s {
    std::atomic<int> ref{1};
    lts_mesh_s* mesh = nullptr;
    lts::RegionsHost r;
    // device tables per precision (built on first use)
    std::unique_ptr<DeviceArena> arena[2];
    lts::Tables<float> t32{};
    lts::Tables<double> t64{};
    int* d_perm_c = nullptr;
    int* d_perm_e = nullptr;
    int device = -1;
};

// One launch of a segment-table plan (ensembles, several fine regions): the
// segments live in device memory, any number per launch.
struct TableLaunch {
    lts::LaunchDesc d;            // kind, buffers, L2 policy, branch, fork, join, bytes
    const void* dsegs = nullptr;  // device segment records
    int nseg = 0, vblocks = 0, grid = 0;
};
struct SV {   // one state vector (h, u) with optional compensation words
    void* hh = nullptr;
    void* hl = nullptr;
    void* uh = nullptr;
    void* ul = nullptr;
};

struct lts_state_s {
    lts_regions_s* reg = nullptr;
    lts_params p{};
    lts::KernelConfig kc{};
    size_t tsz = 4;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t side_stream = nullptr;          // concurrent branch (direct launches)
    cudaStream_t capture_side = nullptr;         // concurrent branch during capture
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // host I/O: host-to-device copies run on h2d_stream, device-to-host
    // copies on d2h_stream, so they overlap the kernels on the state's stream
    // (and, with lts_write_async / lts_read_async, the coarse steps).  Input
    // staging (stage_c, stage_e) is free again once its scatter has run
    // (ev_in_free); output staging (out_c, out_e, diag_out) once its copy to
    // the host is done (ev_out_free).
    // The diagnostics of a read run on diag_stream over a band-order FP64
    // snapshot (snap_c, snap_e) that the gathers write, so they too overlap
    // the following steps; the snapshot is free again after them
    // (ev_snap_free).
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr, diag_stream = nullptr;
    cudaEvent_t ev_in_h = nullptr, ev_in_u = nullptr, ev_in_free = nullptr;
    cudaEvent_t ev_out_h = nullptr, ev_out_u = nullptr, ev_out_free = nullptr;
    cudaEvent_t ev_snap_free = nullptr;
    // pinned host words: the error flag and the diagnostics of the reads
    // since the last lts_sync, with the caller's lts_diag each belongs to
    static constexpr int kDiagSlots = 16;
    int* flag_host = nullptr;
    double* diag_host = nullptr;     // [kDiagSlots][2]
    struct PendingDiag {
        lts_diag* d;
        double time;
        int64_t steps;
    };
    std::vector<PendingDiag> pending_diag;
    DeviceArena arena;
    const void* tables = nullptr;
    SV buf[4];            // [parity] = x_old, [1-parity] = x_new, [2] = x_1st, [3] = x_2nd
    SV P1c, P1e, P2c, P2e;   // interface-1 snapshots of the coarse 1st / 2nd stage
    void* acc_c[3] = {};  // correction terms on I1 u I2 cells (Steps 3.x.2)
    void* acc_e[3] = {};
    void* q = nullptr;
    void* ring_c = nullptr;   // [maxE*nC] per-slot PV contributions
    void* ring_k = nullptr;   // [nC] K_i
    // intermediates of the concurrent far-coarse branch (its own, so the two
    // branches never share a buffer)
    void* q_side = nullptr;
    void* ring_c_side = nullptr;
    void* ring_k_side = nullptr;
    int* flag = nullptr;
    double* stage_c = nullptr;   // FP64 input staging (original order)
    double* stage_e = nullptr;
    double* out_c = nullptr;     // FP64 output staging (original order)
    double* out_e = nullptr;
    double* snap_c = nullptr;    // FP64 snapshot of the state (band order)
    double* snap_e = nullptr;
    double* diag_partial = nullptr;
    double* diag_out = nullptr;
    int diag_blocks = 0;
    std::vector<lts::LaunchDesc> plan[2];
    // several fine regions: one plan per region (and one for the far coarse
    // cells), merged launch by launch into segment-table launches; each
    // region keeps its own interface snapshots and correction terms
    bool multi = false;
    std::vector<TableLaunch> tplan[2];
    struct MemberBufs {
        SV P1c, P1e, P2c, P2e;
        void* acc_c[3] = {};
        void* acc_e[3] = {};
    };
    std::vector<MemberBufs> mbufs;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int parity = 0;
    int64_t steps = 0;
    double time = 0.0;
    // statistics
    double bytes[lts::NKINDS] = {};
    int launches[lts::NKINDS] = {};
    double prof_ms[lts::NKINDS] = {};
    std::vector<cudaEvent_t> events;
    std::vector<cudaEvent_t> gevents[2];   // profile == 2: per kernel node, per parity
    ~lts_state_s();
};

namespace lts {

struct TablePlanStats {
    double bytes[NKINDS] = {};
    int launches = 0, segments = 0;
};
// Merges plans whose segments already index the shared arrays, launch by
// launch in key order (d.bytes of every member launch summed per launch);
// nsm > 0: persistent grids of resident blocks x nsm.  ensemble.cpp.
int merge_table_plan(const KernelConfig& kc, const std::vector<std::vector<LaunchDesc>>& plans, int nsm,
                     DeviceArena& arena, std::vector<TableLaunch>& out, TablePlanStats* stats);
int enqueue_table_plan(const std::vector<TableLaunch>& plan, const void* tables, const KernelConfig& kc,
                       int* flag, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join);

// Internal planning API used by the ensemble (ensemble.cpp).
int device_check();
// Three-launch plan of one coarse step of S (LTS3 or SSPRK3 by S->p.mode)
// for the given parity, launch keys set (LaunchDesc::key).
void make_plan(lts_state_s* S, int parity, std::vector<LaunchDesc>& out);
double plan_launch_bytes(const LaunchDesc& d, const RegionsHost& r, int nC, int nE, int nV, size_t T,
                         bool comp);

}  // namespace lts
