// hylu_solve_static: the substitution of hylu_solve for one right-hand side,
// with its two work vectors in a file-scope device array instead of memory
// the library allocates.  For callers that cannot have a library call
// cudaMalloc (a caller-owned memory pool that holds the whole device, or a
// loop that cannot take cudaMalloc's device-wide synchronization).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hylu.h"

struct hylu_handle;

namespace hylu {
int32_t handle_n(const hylu_handle* h);
int static_solve_ready(const hylu_handle* h);
int solve_into(hylu_handle* h, const double* d_b, double* d_x, double* z, double* xh, cudaStream_t st);
}  // namespace hylu

namespace {

constexpr int64_t kMaxN = HYLU_STATIC_SOLVE_MAX_N;
constexpr int kMaxDevices = 128;

// [0, kMaxN): forward-substitution vector z; [kMaxN, 2 kMaxN): solution by
// column label.  Every device that loads the library holds these 4 MiB.
static __device__ __align__(256) double g_scratch[2 * kMaxN];

// Device address of g_scratch per device.  In host code the name g_scratch
// is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached for the life of the process; a
// cudaDeviceReset of the device ends every handle on it and this cache too.
double* g_addr[kMaxDevices] = {};
std::mutex g_mu;

int scratch_address(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HYLU_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HYLU_ERR_CUDA;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return HYLU_OK;
}

}  // namespace

extern "C" int hylu_solve_static(hylu_handle* h, const double* d_b, double* d_x, void* stream) {
    if (!h) return HYLU_ERR_ARG;
    const int32_t n = hylu::handle_n(h);
    if ((int64_t)n > kMaxN) return HYLU_ERR_TOO_LARGE;
    // state, precision and current device first: the array is looked up on
    // the current device, which must be the handle's
    const int ready = hylu::static_solve_ready(h);
    if (ready < 0) return ready;
    if (ready == 1) return HYLU_OK;              // factored empty system
    if (!d_b || !d_x) return HYLU_ERR_ARG;
    double* base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != HYLU_OK) return rc;
    return hylu::solve_into(h, d_b, d_x, base, base + kMaxN, static_cast<cudaStream_t>(stream));
}
