// B^{-1} tables (Section 3: B = diag(vec B1, vec B2, vec B3)) in both precisions.
#include <algorithm>

#include "fame_internal.h"

namespace {
// 1/B in both precisions; per block the sum, minimum and maximum of 1/B
__global__ void k_invB(const double* __restrict__ B, float* __restrict__ f, double* __restrict__ d,
                       size_t N, double* __restrict__ part) {
    __shared__ double red[3][32];
    double s = 0.0, lo = 1e300, hi = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const double v = 1.0 / B[i];
        d[i] = v;
        f[i] = (float)v;
        s += v;
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s;
        red[1][threadIdx.x >> 5] = lo;
        red[2][threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < (blockDim.x >> 5);
        s = in ? red[0][threadIdx.x] : 0.0;
        lo = in ? red[1][threadIdx.x] : 1e300;
        hi = in ? red[2][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xffffffffu, s, o);
            lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
        }
        if (threadIdx.x == 0) {
            part[3 * blockIdx.x] = s;
            part[3 * blockIdx.x + 1] = lo;
            part[3 * blockIdx.x + 2] = hi;
        }
    }
}
}  // namespace

fame_status eps_from_device(fame_ctx* c, const double* B, cudaStream_t st, double* mean_invB) {
    const size_t N = 3 * (size_t)c->n;
    const int nblk = 608;
    fame_status s = grow(c, c->partial, 3 * nblk * sizeof(double));
    if (s != FAME_OK) return s;
    double* part = static_cast<double*>(c->partial.p);
    k_invB<<<nblk, 256, 0, st>>>(B, c->tf.invB, c->td.invB, N, part);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    double h[3 * nblk];
    FAME_CUDA_TRY(c, cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    double sum = 0.0, lo = 1e300, hi = 0.0;
    for (int i = 0; i < nblk; ++i) {
        sum += h[3 * i];
        lo = std::min(lo, h[3 * i + 1]);
        hi = std::max(hi, h[3 * i + 2]);
    }
    *mean_invB = sum / (double)N;
    c->min_invB = lo;
    c->max_invB = hi;
    return FAME_OK;
}
