// Tall-skinny block operations of the block eigensolver: Gram matrices with
// FP64 accumulation, block linear combinations, residuals with the
// preconditioner, and precision conversion.  Vectors are 2n complex, stored
// vector-major ([m][2n]).
#include <cstdint>
#include <type_traits>

#include "blockops.h"

namespace {

// per-thread register tile of the Gram kernel
constexpr int TI = 4;
constexpr int TJ = 4;
constexpr int TROWS = 32;          // rows staged in shared memory per step
constexpr int FLUSH_TILES = 4;     // FP32 partial sums flushed to FP64 every 4 x 32 rows

template <typename C> struct Acc;
template <> struct Acc<float2> { using T = float; };
template <> struct Acc<double2> { using T = double; };

template <typename C>
__device__ __forceinline__ const C* col_ptr(const BlockList<C>& L, int i, size_t ld) {
#pragma unroll
    for (int b = 0; b < BlockList<C>::kMax - 1; ++b) {
        if (i < L.cols[b]) return L.ptr[b] + (size_t)i * ld;
        i -= L.cols[b];
    }
    return L.ptr[BlockList<C>::kMax - 1] + (size_t)i * ld;
}

// partial[blk][j][i] = sum over this block's rows of conj(U_i) V_j  (column-major ku x kv).
// Each thread owns a TI x TJ tile of (i, j) pairs; blockIdx.y picks a group of
// at most kGramThreads tiles.  Complex64 inputs: FP32 products summed in FP32
// over FLUSH_TILES x TROWS rows, then added into FP64 accumulators kept in
// shared memory.  Complex128 inputs: FP64 throughout.
constexpr int kGramThreads = 512;

template <typename CU, typename CV>
__global__ void __launch_bounds__(kGramThreads) k_gram(BlockList<CU> U, BlockList<CV> V, size_t ld,
                                                      size_t rows_per_blk,
                                                      double2* __restrict__ partial) {
    // products in FP64 when either side is complex128
    using R = typename std::conditional<(sizeof(CU) == 16 || sizeof(CV) == 16), double, float>::type;
    using C = typename cpx<R>::T;
    using RU = typename Acc<CU>::T;
    using RV = typename Acc<CV>::T;
    constexpr bool kSplit = sizeof(R) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ku = U.total, kv = V.total;
    CU* su = reinterpret_cast<CU*>(smem_raw);                        // [TROWS][ku]
    CV* sv = reinterpret_cast<CV*>(su + TROWS * ku);                 // [TROWS][kv]
    double2* acc64 = reinterpret_cast<double2*>(sv + TROWS * kv);    // [TI*TJ][blockDim]
    const int tiles_i = (ku + TI - 1) / TI, tiles_j = (kv + TJ - 1) / TJ;
    const int tile = blockIdx.y * blockDim.x + threadIdx.x;
    const int ti = tile / tiles_j, tj = tile % tiles_j;
    const bool active = ti < tiles_i;
    const size_t r0 = blockIdx.x * rows_per_blk;
    const size_t r1 = min(ld, r0 + rows_per_blk);
    R accr[TI][TJ], acci[TI][TJ];
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) accr[a][b] = acci[a][b] = 0;
    if (kSplit)
        for (int q = 0; q < TI * TJ; ++q) acc64[q * blockDim.x + threadIdx.x] = make_double2(0.0, 0.0);
    int tiles_done = 0;
    for (size_t rb = r0; rb < r1; rb += TROWS) {
        const int nr = (int)min((size_t)TROWS, r1 - rb);
        for (int e = threadIdx.x; e < TROWS * ku; e += blockDim.x) {
            const int i = e / TROWS, t = e % TROWS;
            su[t * ku + i] = (t < nr) ? col_ptr(U, i, ld)[rb + t] : mk((RU)0, (RU)0);
        }
        for (int e = threadIdx.x; e < TROWS * kv; e += blockDim.x) {
            const int j = e / TROWS, t = e % TROWS;
            sv[t * kv + j] = (t < nr) ? col_ptr(V, j, ld)[rb + t] : mk((RV)0, (RV)0);
        }
        __syncthreads();
        if (active) {
#pragma unroll 2
            for (int t = 0; t < TROWS; ++t) {
                C u[TI], w[TJ];
#pragma unroll
                for (int a = 0; a < TI; ++a) {
                    const int i = ti * TI + a;
                    const CU x = (i < ku) ? su[t * ku + i] : mk((RU)0, (RU)0);
                    u[a] = mk((R)x.x, (R)x.y);
                }
#pragma unroll
                for (int b = 0; b < TJ; ++b) {
                    const int j = tj * TJ + b;
                    const CV x = (j < kv) ? sv[t * kv + j] : mk((RV)0, (RV)0);
                    w[b] = mk((R)x.x, (R)x.y);
                }
#pragma unroll
                for (int a = 0; a < TI; ++a)
#pragma unroll
                    for (int b = 0; b < TJ; ++b) {
                        accr[a][b] = fma(u[a].x, w[b].x, fma(u[a].y, w[b].y, accr[a][b]));
                        acci[a][b] = fma(u[a].x, w[b].y, fma(-u[a].y, w[b].x, acci[a][b]));
                    }
            }
        }
        __syncthreads();
        if (kSplit && ++tiles_done == FLUSH_TILES) {
            tiles_done = 0;
#pragma unroll
            for (int a = 0; a < TI; ++a)
#pragma unroll
                for (int b = 0; b < TJ; ++b) {
                    double2& d = acc64[(a * TJ + b) * blockDim.x + threadIdx.x];
                    d.x += (double)accr[a][b];
                    d.y += (double)acci[a][b];
                    accr[a][b] = acci[a][b] = 0;
                }
        }
    }
    if (!active) return;
    double2* out = partial + (size_t)blockIdx.x * ku * kv;
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) {
            const int i = ti * TI + a, j = tj * TJ + b;
            if (i < ku && j < kv) {
                double xr = (double)accr[a][b], xi = (double)acci[a][b];
                if (kSplit) {
                    const double2 d = acc64[(a * TJ + b) * blockDim.x + threadIdx.x];
                    xr += d.x;
                    xi += d.y;
                }
                out[(size_t)j * ku + i] = make_double2(xr, xi);
            }
        }
}

// G = sum over blocks of partial (fixed order, deterministic)
// One warp per entry: lanes take blocks lane, lane+32, ...; fixed shuffle tree.
__global__ void k_gram_reduce(const double2* __restrict__ partial, int nblk, int kk,
                              double2* __restrict__ G) {
    const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (e >= kk) return;
    double sr = 0.0, si = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = partial[(size_t)b * kk + e];
        sr += v.x;
        si += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) G[e] = make_double2(sr, si);
}

// out1_j = sum_{i<k} S_i M[i][j];  out2_j = sum_{i>=i0} S_i M[i][j]   (j < m)
// M column-major k x m double2 in device memory, rounded once into shared memory
// in the block's precision; accumulation in that precision.
template <typename C, typename Co>
__global__ void k_combine(BlockList<C> S, size_t ld, const double2* __restrict__ M, int m, int i0,
                          Co* __restrict__ out1, Co* __restrict__ out2) {
    using R = typename Acc<C>::T;
    using Ro = decltype(Co().x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = S.total;
    C* sm = reinterpret_cast<C*>(smem_raw);
    for (int e = threadIdx.x; e < k * m; e += blockDim.x) sm[e] = mk((R)M[e].x, (R)M[e].y);
    __syncthreads();
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        constexpr int JC = sizeof(R) == 4 ? 16 : 8;   // output columns per pass over S
        for (int j0 = 0; j0 < m; j0 += JC) {
            const int jn = min(JC, m - j0);
            C a1[JC], a2[JC];
#pragma unroll
            for (int b = 0; b < JC; ++b) { a1[b] = mk((R)0, (R)0); a2[b] = a1[b]; }
            for (int i = 0; i < k; ++i) {
                const C s = col_ptr(S, i, ld)[row];
#pragma unroll
                for (int b = 0; b < JC; ++b) {
                    if (b < jn) {
                        const C p = cmul(s, sm[(size_t)(j0 + b) * k + i]);
                        a1[b] = a1[b] + p;
                        if (i >= i0) a2[b] = a2[b] + p;
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < JC; ++b) {
                if (b < jn) {
                    if (out1) out1[(size_t)(j0 + b) * ld + row] = mk((Ro)a1[b].x, (Ro)a1[b].y);
                    if (out2) out2[(size_t)(j0 + b) * ld + row] = mk((Ro)a2[b].x, (Ro)a2[b].y);
                }
            }
        }
    }
}

// R_j = AX_j - theta_j X_j;  W_j = tinv .* R_j (tinv indexed by frequency, both coordinates);
// part[j][blk] = sum |R_j|^2 over the block's rows
template <typename C>
__global__ void k_resid(const C* __restrict__ X, const C* __restrict__ AX,
                        const double* __restrict__ theta, const typename Acc<C>::T* __restrict__ tinv,
                        size_t n, C* __restrict__ W, double* __restrict__ part) {
    using R = typename Acc<C>::T;
    __shared__ double red[32];
    const int j = blockIdx.y;
    const size_t ld = 2 * n;
    const R th = (R)theta[j];
    double s = 0.0;
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        const C x = X[(size_t)j * ld + row], ax = AX[(size_t)j * ld + row];
        const C r = mk(ax.x - th * x.x, ax.y - th * x.y);
        s += (double)r.x * r.x + (double)r.y * r.y;
        const R t = tinv[row < n ? row : row - n];
        if (W) W[(size_t)j * ld + row] = mk(t * r.x, t * r.y);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
}

// Refinement residual: R_j = AX_j - theta_j X_j in FP64 from complex128 X, AX;
// W_j = tinv .* R_j rounded to complex64; part[j][blk] = partial ||R_j||^2.
__global__ void k_resid_mixed(const double2* __restrict__ X, const double2* __restrict__ AX,
                              const double* __restrict__ theta, const float* __restrict__ tinv,
                              size_t n, float2* __restrict__ W, float2* __restrict__ R32,
                              double* __restrict__ part) {
    __shared__ double red[32];
    const int j = blockIdx.y;
    const size_t ld = 2 * n;
    const double th = theta[j];
    double s = 0.0;
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        const double2 x = X[(size_t)j * ld + row], ax = AX[(size_t)j * ld + row];
        const double rx = ax.x - th * x.x, ry = ax.y - th * x.y;
        s += rx * rx + ry * ry;
        const float t = tinv[row < n ? row : row - n];
        W[(size_t)j * ld + row] = make_float2(t * (float)rx, t * (float)ry);
        if (R32) R32[(size_t)j * ld + row] = make_float2((float)rx, (float)ry);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
}

// Refinement update of one of (X, AX):
//   Xn_j  = sum_{i<m} X_i M[i][j] (FP64) + Dn_j,   Dn_j = sum_{i<nq} Q_i M[m+i][j] (FP32),
//   X32n_j = Xn_j rounded to complex64, and Pn_j = Dn_j (complex64).
// The FP32 part carries the search-direction correction, whose size shrinks with the residual.
__global__ void k_combine_mixed(const double2* __restrict__ X, int m, BlockList<float2> Q, size_t ld,
                                const double2* __restrict__ M, double2* __restrict__ Xn,
                                float2* __restrict__ X32n, float2* __restrict__ Pn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nq = Q.total, k = m + nq;
    double2* sd = reinterpret_cast<double2*>(smem_raw);          // M rows 0..m-1, FP64
    float2* sf = reinterpret_cast<float2*>(sd + (size_t)m * m);  // M rows m..k-1, FP32
    for (int e = threadIdx.x; e < k * m; e += blockDim.x) {
        const int j = e / k, i = e % k;
        if (i < m) sd[(size_t)j * m + i] = M[e];
        else sf[(size_t)j * nq + (i - m)] = make_float2((float)M[e].x, (float)M[e].y);
    }
    __syncthreads();
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        constexpr int JC = 8;    // output columns per pass (register budget of the FP64 part)
        for (int j0 = 0; j0 < m; j0 += JC) {
            const int jn = min(JC, m - j0);
            double2 a[JC];
            float2 d[JC];
#pragma unroll
            for (int b = 0; b < JC; ++b) { a[b] = make_double2(0.0, 0.0); d[b] = make_float2(0.f, 0.f); }
            for (int i = 0; i < m; ++i) {
                const double2 x = X[(size_t)i * ld + row];
#pragma unroll
                for (int b = 0; b < JC; ++b)
                    if (b < jn) a[b] = a[b] + cmul(x, sd[(size_t)(j0 + b) * m + i]);
            }
            for (int i = 0; i < nq; ++i) {
                const float2 q = col_ptr(Q, i, ld)[row];
#pragma unroll
                for (int b = 0; b < JC; ++b)
                    if (b < jn) d[b] = d[b] + cmul(q, sf[(size_t)(j0 + b) * nq + i]);
            }
#pragma unroll
            for (int b = 0; b < JC; ++b) {
                if (b < jn) {
                    const size_t o = (size_t)(j0 + b) * ld + row;
                    const double2 v = make_double2(a[b].x + (double)d[b].x, a[b].y + (double)d[b].y);
                    Xn[o] = v;
                    X32n[o] = make_float2((float)v.x, (float)v.y);
                    if (Pn) Pn[o] = d[b];
                }
            }
        }
    }
}

// Q_j <- Q_j - sum_i X_i c[i][j] for the nq columns of Q (in place), c m x nq
// column-major.  Arithmetic in FP64 when X is complex128, else FP32.
template <typename CX, typename CQ>
__global__ void k_orth(const CX* __restrict__ X, int m, BlockList<CQ> Q, size_t ld,
                       const double2* __restrict__ cfs) {
    using R = typename Acc<CX>::T;
    using C = CX;
    using RQ = typename Acc<CQ>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nq = Q.total;
    C* sc = reinterpret_cast<C*>(smem_raw);
    for (int e = threadIdx.x; e < m * nq; e += blockDim.x) sc[e] = mk((R)cfs[e].x, (R)cfs[e].y);
    __syncthreads();
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        constexpr int JC = sizeof(R) == 4 ? 16 : 8;   // output columns per pass over X
        for (int j0 = 0; j0 < nq; j0 += JC) {
            const int jn = min(JC, nq - j0);
            C a[JC];
#pragma unroll
            for (int b = 0; b < JC; ++b) a[b] = mk((R)0, (R)0);
            for (int i = 0; i < m; ++i) {
                const C x = X[(size_t)i * ld + row];
#pragma unroll
                for (int b = 0; b < JC; ++b)
                    if (b < jn) a[b] = a[b] + cmul(x, sc[(size_t)(j0 + b) * m + i]);
            }
#pragma unroll
            for (int b = 0; b < JC; ++b) {
                if (b < jn) {
                    CQ* q = const_cast<CQ*>(col_ptr(Q, j0 + b, ld)) + row;
                    const CQ v = *q;
                    *q = mk((RQ)((R)v.x - a[b].x), (RQ)((R)v.y - a[b].y));
                }
            }
        }
    }
}

template <typename Ci, typename Co>
__global__ void k_convert(const Ci* __restrict__ in, Co* __restrict__ out, size_t N) {
    using Ro = decltype(Co().x);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = mk((Ro)in[i].x, (Ro)in[i].y);
}

// zero the coordinates whose preconditioner entry is 0 (the Gamma zero modes)
template <typename C>
__global__ void k_mask(C* __restrict__ X, const typename Acc<C>::T* __restrict__ tinv, size_t n,
                       int m) {
    const size_t ld = 2 * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ld * m;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i % ld;
        if (tinv[row < n ? row : row - n] == 0) X[i] = mk(decltype(X[0].x)(0), decltype(X[0].x)(0));
    }
}

// counter-based uniform deviates (SplitMix64) for reproducible start blocks
__device__ __forceinline__ uint64_t splitmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
template <typename C>
__global__ void k_random(C* __restrict__ X, size_t N, uint64_t seed) {
    using R = decltype(X[0].x);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix(seed ^ (2 * i)), b = splitmix(seed ^ (2 * i + 1));
        const double u = (double)(a >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        const double v = (double)(b >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        X[i] = mk((R)u, (R)v);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
template <typename CU, typename CV>
fame_status gram(fame_ctx* c, const BlockList<CU>& U, const BlockList<CV>& V, size_t ld,
                 double2* G, cudaStream_t st) {
    const int ku = U.total, kv = V.total;
    const int tiles = ((ku + TI - 1) / TI) * ((kv + TJ - 1) / TJ);
    const int groups = (tiles + kGramThreads - 1) / kGramThreads;
    int threads = (((tiles + groups - 1) / groups + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    const bool dbl = sizeof(CU) == 16 || sizeof(CV) == 16;
    const size_t smem = (size_t)TROWS * (ku * sizeof(CU) + kv * sizeof(CV)) +
                        (dbl ? 0 : (size_t)TI * TJ * threads * sizeof(double2));
    int nblk = 152 * 4;
    size_t rpb = (ld + nblk - 1) / nblk;
    rpb = ((rpb + TROWS - 1) / TROWS) * TROWS;
    nblk = (int)((ld + rpb - 1) / rpb);
    fame_status s = grow(c, c->partial, (size_t)nblk * ku * kv * sizeof(double2));
    if (s != FAME_OK) return s;
    if (smem > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute((const void*)k_gram<CU, CV>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    double2* part = reinterpret_cast<double2*>(c->partial.p);
    {
        ProfScope ps(K_GRAM, dbl, st, (double)ld * (ku * sizeof(CU) + kv * sizeof(CV)),
                     8.0 * ku * kv * (double)ld);
        k_gram<CU, CV><<<dim3(nblk, groups), threads, smem, st>>>(U, V, ld, rpb, part);
    }
    const int kk = ku * kv;
    {
        ProfScope ps(K_GRAM_RED, dbl, st, (double)nblk * kk * sizeof(double2), 2.0 * nblk * kk);
        k_gram_reduce<<<(kk + 7) / 8, 256, 0, st>>>(part, nblk, kk, G);
    }
    count_launch(2);
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename C, typename Co>
fame_status combine(fame_ctx* c, const BlockList<C>& S, size_t ld, const double2* M, int m, int i0,
                    Co* out1, Co* out2, cudaStream_t st) {
    const size_t smem = (size_t)S.total * m * sizeof(C);
    if (smem > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute((const void*)k_combine<C, Co>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        const double outs = (out1 ? m : 0) + (out2 ? m : 0);
        ProfScope ps(K_COMBINE, sizeof(C) == sizeof(double2), st,
                     (double)S.total * ld * sizeof(C) + outs * ld * sizeof(Co), 8.0 * S.total * outs * (double)ld);
        k_combine<C, Co><<<152 * 8, 256, smem, st>>>(S, ld, M, m, i0, out1, out2);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename C>
fame_status residual(fame_ctx* c, const C* X, const C* AX, const double* theta_dev,
                     const typename RealOf<C>::T* tinv, int m, C* W, double* part, int nblk,
                     cudaStream_t st) {
    dim3 grid(nblk, m);
    {
        const double ld = 2.0 * c->n;
        ProfScope ps(K_RESID, sizeof(C) == sizeof(double2), st, (W ? 3.0 : 2.0) * m * ld * sizeof(C),
                     8.0 * m * ld);
        k_resid<C><<<grid, 256, 0, st>>>(X, AX, theta_dev, tinv, (size_t)c->n, W, part);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

fame_status residual_mixed(fame_ctx* c, const double2* X, const double2* AX, const double* theta_dev,
                           int m, float2* W, float2* R32, double* part, int nblk, cudaStream_t st) {
    dim3 grid(nblk, m);
    {
        const double ld = 2.0 * c->n;
        ProfScope ps(K_RESID, true, st, m * ld * (2 * sizeof(double2) + (R32 ? 2 : 1) * sizeof(float2)), 8.0 * m * ld);
        k_resid_mixed<<<grid, 256, 0, st>>>(X, AX, theta_dev, c->tf.tinv, (size_t)c->n, W, R32, part);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

fame_status combine_mixed(fame_ctx* c, const double2* X, int m, const BlockList<float2>& Q, size_t ld,
                          const double2* M, double2* Xn, float2* X32n, float2* Pn, cudaStream_t st) {
    const int nq = Q.total;
    const size_t smem = (size_t)m * m * sizeof(double2) + (size_t)nq * m * sizeof(float2);
    if (smem > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute((const void*)k_combine_mixed,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        ProfScope ps(K_COMBINE, true, st,
                     (double)ld * (m * sizeof(double2) + nq * sizeof(float2) +
                                   m * (sizeof(double2) + sizeof(float2) + (Pn ? sizeof(float2) : 0))),
                     8.0 * (double)ld * m * (m + nq));
        k_combine_mixed<<<152 * 8, 256, smem, st>>>(X, m, Q, ld, M, Xn, X32n, Pn);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename CX, typename CQ>
fame_status orth_against(fame_ctx* c, const CX* X, int m, const BlockList<CQ>& Q, size_t ld,
                         const double2* cfs, cudaStream_t st) {
    const int nq = Q.total;
    if (nq == 0) return FAME_OK;
    const size_t smem = (size_t)m * nq * sizeof(CX);
    if (smem > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute((const void*)k_orth<CX, CQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        ProfScope ps(K_COMBINE, sizeof(CX) == 16, st, (double)ld * (m * sizeof(CX) + 2 * nq * sizeof(CQ)),
                     8.0 * (double)ld * m * nq);
        k_orth<CX, CQ><<<152 * 8, 256, smem, st>>>(X, m, Q, ld, cfs);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template fame_status orth_against<float2, float2>(fame_ctx*, const float2*, int, const BlockList<float2>&, size_t, const double2*, cudaStream_t);
template fame_status orth_against<double2, float2>(fame_ctx*, const double2*, int, const BlockList<float2>&, size_t, const double2*, cudaStream_t);
template fame_status orth_against<double2, double2>(fame_ctx*, const double2*, int, const BlockList<double2>&, size_t, const double2*, cudaStream_t);

template <typename Ci, typename Co>
fame_status convert(fame_ctx* c, const Ci* in, Co* out, size_t N, cudaStream_t st) {
    k_convert<Ci, Co><<<152 * 8, 256, 0, st>>>(in, out, N);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename C>
fame_status random_block(fame_ctx* c, C* X, int m, uint64_t seed, const typename RealOf<C>::T* tinv,
                         cudaStream_t st) {
    const size_t N = (size_t)m * 2 * c->n;
    k_random<C><<<152 * 8, 256, 0, st>>>(X, N, seed);
    k_mask<C><<<152 * 8, 256, 0, st>>>(X, tinv, (size_t)c->n, m);
    count_launch(2);
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename C>
fame_status mask_block(fame_ctx* c, C* X, int m, const typename RealOf<C>::T* tinv, cudaStream_t st) {
    k_mask<C><<<152 * 8, 256, 0, st>>>(X, tinv, (size_t)c->n, m);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template fame_status gram<float2, float2>(fame_ctx*, const BlockList<float2>&, const BlockList<float2>&, size_t, double2*, cudaStream_t);
template fame_status gram<double2, double2>(fame_ctx*, const BlockList<double2>&, const BlockList<double2>&, size_t, double2*, cudaStream_t);
template fame_status gram<double2, float2>(fame_ctx*, const BlockList<double2>&, const BlockList<float2>&, size_t, double2*, cudaStream_t);
template fame_status combine<float2, float2>(fame_ctx*, const BlockList<float2>&, size_t, const double2*, int, int, float2*, float2*, cudaStream_t);
template fame_status combine<double2, double2>(fame_ctx*, const BlockList<double2>&, size_t, const double2*, int, int, double2*, double2*, cudaStream_t);
template fame_status residual<float2>(fame_ctx*, const float2*, const float2*, const double*, const float*, int, float2*, double*, int, cudaStream_t);
template fame_status residual<double2>(fame_ctx*, const double2*, const double2*, const double*, const double*, int, double2*, double*, int, cudaStream_t);
template fame_status convert<float2, double2>(fame_ctx*, const float2*, double2*, size_t, cudaStream_t);
template fame_status convert<double2, float2>(fame_ctx*, const double2*, float2*, size_t, cudaStream_t);
template fame_status random_block<float2>(fame_ctx*, float2*, int, uint64_t, const float*, cudaStream_t);
template fame_status random_block<double2>(fame_ctx*, double2*, int, uint64_t, const double*, cudaStream_t);
template fame_status mask_block<float2>(fame_ctx*, float2*, int, const float*, cudaStream_t);
template fame_status mask_block<double2>(fame_ctx*, double2*, int, const double*, cudaStream_t);
