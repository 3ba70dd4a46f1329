// fame_apply_Ar_static: the A_r apply with its 3 m n complex workspace in a
// statically reserved device array instead of the context's grown buffer, so
// the call allocates no device memory at all.
//
// The workspace needs no initial contents: the Z-in pass writes every entry
// before the XY and Z-out passes read it, so nothing is cleared.  The array is
// one per device and per process, shared by every context: two calls that
// overlap in time (different streams, different host threads) race on it.
#include <mutex>
#include <string>

#include "fame_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_ws[FAME_STATIC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_ws_mu;
void* g_ws_addr[kMaxDevices] = {};   // device address of g_static_ws, looked up once per device

fame_status static_workspace(fame_ctx* c, void** out) {
    int dev = 0;
    FAME_CUDA_TRY(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_err(c, FAME_E_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (!g_ws_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_err(c, FAME_E_CUDA, std::string("cudaGetSymbolAddress(static workspace): ") +
                                               cudaGetErrorString(e));
        }
        g_ws_addr[dev] = p;
    }
    *out = g_ws_addr[dev];
    return FAME_OK;
}

}  // namespace

extern "C" FAME_API fame_status fame_apply_Ar_static(fame_ctx* c, const void* y, void* Ay, int m, int dtype,
                                                     void* stream) {
    if (!c) return FAME_E_ARG;
    c->err.clear();
    if (!y || !Ay || m < 1) return set_err(c, FAME_E_ARG, "bad y/Ay/m");
    if (y == Ay) return set_err(c, FAME_E_ARG, "y and Ay must not overlap");
    if (!c->eps_set) return set_err(c, FAME_E_STATE, "fame_set_eps has not been called");
    if (dtype != FAME_C64 && dtype != FAME_C128)
        return set_err(c, FAME_E_ARG, "dtype must be FAME_C64 or FAME_C128");
    const size_t elem = dtype == FAME_C64 ? sizeof(float2) : sizeof(double2);
    const size_t need = (size_t)m * 3 * (size_t)c->n * elem;
    if (need > (size_t)FAME_STATIC_WORKSPACE_BYTES)
        return set_err(c, FAME_E_ARG,
                       "fame_apply_Ar_static: workspace of " + std::to_string(need) +
                           " bytes (3 m n complex) exceeds the static maximum of " +
                           std::to_string((size_t)FAME_STATIC_WORKSPACE_BYTES) + " bytes");
    void* ws = nullptr;
    const fame_status s = static_workspace(c, &ws);
    if (s != FAME_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == FAME_C64)
        return run_apply_into<float>(c, static_cast<const float2*>(y), static_cast<float2*>(Ay), m,
                                     static_cast<float2*>(ws), st);
    return run_apply_into<double>(c, static_cast<const double2*>(y), static_cast<double2*>(Ay), m,
                                  static_cast<double2*>(ws), st);
}
