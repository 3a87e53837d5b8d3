// noalloc.cu -- FP64 mass/energy diagnostics that allocate no memory.
//
// Some callers cannot allocate device memory at the moment they need the
// diagnostics: hosts whose device memory comes from a fixed pool that must
// not grow, or time loops that forbid allocation because cudaMalloc may
// synchronise the device and stall the work in flight.
// lts_diagnostics_noalloc serves them: the per-block partial sums of the
// deterministic two-stage reduction live in a fixed, file-scope device array
// instead of a buffer allocated per call or per state, and the result goes
// to device memory the caller owns.
#include <mutex>

#include "../../include/lts.h"
#include "lts_error.h"
#include "lts_internal.h"

namespace lts {
int state_view(lts_state s, StateView* v);
}

namespace {

// 2 doubles (mass, energy) per reduction block of 256 (cell, layer) pairs:
// at most 4096 blocks, i.e. states of up to 4096 * 256 = 1,048,576 cells x
// layers (64 KiB).
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
    // the blocking of lts_read's reduction (one (cell, layer) pair per
    // thread), so both give the same sums to the last bit
    const long long L = v.kc.layers > 1 ? v.kc.layers : 1;
    const long long nblocks = (static_cast<long long>(v.nC) * L + kCellsPerBlock - 1) / kCellsPerBlock;
    if (nblocks > kMaxBlocks)
        return lts::set_error(LTS_EINVAL,
                              "lts_diagnostics_noalloc supports at most %d cells x layers (state has %lld)",
                              kMaxBlocks * kCellsPerBlock, static_cast<long long>(v.nC) * L);
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
    e = lts::launch_diagnostics(v.kc, v.tables, v.h_hi, v.h_lo, v.u_hi, v.u_lo, v.g, scratch, static_cast<int>(nblocks),
                                d_out, v.stream);
    if (e != cudaSuccess)
        return lts::set_error(LTS_ECUDA, "diagnostics launch: %s", cudaGetErrorString(e));
    return LTS_OK;
}
