// B^{-1} tables (Section 3: B = diag(vec B1, vec B2, vec B3)) in both precisions.
#include "fame_internal.h"

namespace {
__global__ void k_invB(const double* __restrict__ B, float* __restrict__ f, double* __restrict__ d,
                       size_t N, double* __restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const double v = 1.0 / B[i];
        d[i] = v;
        f[i] = (float)v;
        s += v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}
}  // namespace

fame_status eps_from_device(fame_ctx* c, const double* B, cudaStream_t st, double* mean_invB) {
    const size_t N = 3 * (size_t)c->n;
    const int nblk = 608;
    fame_status s = grow(c, c->partial, nblk * sizeof(double));
    if (s != FAME_OK) return s;
    double* part = static_cast<double*>(c->partial.p);
    k_invB<<<nblk, 256, 0, st>>>(B, c->tf.invB, c->td.invB, N, part);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    double h[nblk];
    FAME_CUDA_TRY(c, cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    double sum = 0.0;
    for (int i = 0; i < nblk; ++i) sum += h[i];
    *mean_invB = sum / (double)N;
    return FAME_OK;
}
