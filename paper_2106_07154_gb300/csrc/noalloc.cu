// noalloc.cu -- FP64 mass/energy diagnostics that allocate no memory.
//
// Some callers cannot allocate device memory at the moment they need the
// diagnostics: code running while a stream is being captured into a CUDA
// graph (cudaMalloc is not allowed inside a capture), callers whose memory
// comes from a pool that must not grow, or hosts that forbid allocation in
// their time loop.  lts_diagnostics_noalloc serves them: the per-block
// partial sums of the deterministic two-stage reduction live in a fixed,
// file-scope device array instead of a buffer allocated per call or per
// state, and the result goes to device memory the caller owns.
#include <mutex>

#include "../../include/lts.h"
#include "lts_error.h"
#include "lts_internal.h"

namespace lts {
int state_view(lts_state s, StateView* v);
}

namespace {

// 2 doubles (mass, energy) per reduction block of 256 cells: at most
// 4096 blocks, i.e. meshes of up to 4096 * 256 = 1,048,576 cells (64 KiB).
constexpr int kMaxBlocks = 4096;
constexpr int kCellsPerBlock = 256;
static __device__ __align__(256) double g_diag_scratch[2 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; resolved once
// per device (cudaGetSymbolAddress), with that device current.
int scratch_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices)
        return lts::set_error(LTS_EINVAL, "device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess)
            return lts::set_error(LTS_ECUDA, "cudaGetSymbolAddress(diagnostics scratch): %s",
                                  cudaGetErrorString(e));
        g_scratch_ptr[device] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[device];
    return LTS_OK;
}

}  // namespace

extern "C" int lts_diagnostics_noalloc(lts_state s, double* d_out) {
    if (!s || !d_out) return lts::set_error(LTS_EINVAL, "null argument");
    lts::StateView v;
    int rc = lts::state_view(s, &v);
    if (rc != LTS_OK) return rc;
    const int nblocks = (v.nC + kCellsPerBlock - 1) / kCellsPerBlock;
    if (nblocks > kMaxBlocks)
        return lts::set_error(LTS_EINVAL,
                              "lts_diagnostics_noalloc supports at most %d cells (mesh has %d)",
                              kMaxBlocks * kCellsPerBlock, v.nC);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lts::set_error(LTS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev != v.device)
        return lts::set_error(LTS_EINVAL, "the state lives on device %d, device %d is current", v.device,
                              dev);
    double* scratch = nullptr;
    rc = scratch_address(dev, &scratch);
    if (rc != LTS_OK) return rc;
    // every block writes its own partial pair and the final pass reads only
    // those, so nothing has to be cleared between calls
    e = lts::launch_diagnostics(v.kc, v.tables, v.h_hi, v.h_lo, v.u_hi, v.u_lo, v.g, scratch, nblocks,
                                d_out, v.stream);
    if (e != cudaSuccess)
        return lts::set_error(LTS_ECUDA, "diagnostics launch: %s", cudaGetErrorString(e));
    return LTS_OK;
}
