// Tall-skinny block operations of the block eigensolver: Gram matrices (FP64
// sums across row blocks), block linear combinations, residuals with the
// preconditioner, and precision conversion.  Vectors are 2n complex, stored
// vector-major ([m][2n]).
#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <type_traits>

#include "blockops.h"
#include "bounds.cuh"
#include "df64.cuh"

// FP64 arithmetic on the FP64 units instead of double-float on the FP32 units (the
// environment variable FAME_FP64_NATIVE=1; for comparisons)
bool fp64_native() {
    const char* v = std::getenv("FAME_FP64_NATIVE");
    return v && v[0] == '1';
}

FAME_BOUNDS_READER(blockops)

namespace {

// Complex64 Grams whose wider side has at least this many vectors run on the tensor
// cores (tc_gram.cu); narrower ones on the FP32 ring kernel, which is faster there
// (measured at 64^3 and 96^3: 15 x 30 vectors 116 against 187 us; 30 x 75: 356 against
// 250 us; 45 x 90: 556 against 408 us).
// The environment variable FAME_TC_MIN_WIDTH overrides the threshold (e.g. 1: every shape
// the tensor-core kernel takes).
int tc_min_width() {
    const char* v = std::getenv("FAME_TC_MIN_WIDTH");
    return v ? std::max(1, std::atoi(v)) : 64;
}

// Gram kernel: GT x GT complex outputs per thread, GROWS rows per shared-memory stage
constexpr int GT = 4;
constexpr int GROWS = 32;
// ring-staged complex64 combine / orthogonalisation: rows per tile, columns per
// stage, stages in flight, outputs per thread group
constexpr int kStRows = 128, kStCols = 8, kStStages = 4, kStOut = 16;
static_assert(kStOut % kStCols == 0, "a group's outputs span whole stages");

// Refinement form of the ring-staged combine (k_combine_st<.., RF = true>): the inputs
// are [X32 | Q] with X32 the complex64 copy of the complex128 block X64 (its first mx
// columns); for each output j the entries M[i][j] of j's block (blk[j] = count, then
// the columns i) are taken from X64 in double-float arithmetic, all other entries
// from the complex64 inputs in FP32.  Outputs Xn64 (complex128) and X32n (its
// complex64 copy, may be null).
constexpr int kRefBlk = kRefineBlock;
struct RefineEpi {
    const double2* X64 = nullptr;
    int mx = 0;
    const int* blk = nullptr;       // device [m][kRefBlk + 1]
    double2* Xn64 = nullptr;
    float2* X32n = nullptr;
};

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

// asynchronous 8- or 16-byte global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async_c(float2* dst, const float2* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_c(double2* dst, const double2* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
// 16-byte global -> shared copy (both addresses 16-byte aligned); valid = false writes zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory row strides of the Gram stages: room for the padded tile columns,
// odd (in elements) so that the row-wise staging stores are conflict-free.
__host__ __device__ inline int gram_stride(int k) {
    const int s = ((k + GT - 1) / GT) * GT;
    return s | 1;
}

// partial[blk][j][i] = sum over this block's rows of conj(U_i) V_j  (column-major ku x kv).
// Thread (ti, tj) owns outputs i = ti + TIN a, j = tj + TJN b (a, b < GT), so a warp
// reads consecutive V columns and few U columns of each staged row.  Rows arrive in
// stages of GROWS by cp.async, double-buffered.  Complex64 inputs: FP32 products
// summed in FP32 over the block's rows (about a thousand), the blocks then summed
// in FP64 by k_gram_reduce.  Complex128 inputs: FP64 throughout.
constexpr int kGramThreads = 512;

template <typename CU, typename CV>
__global__ void __launch_bounds__(kGramThreads) k_gram(BlockList<CU> U, BlockList<CV> V, size_t ld,
                                                      size_t rows_per_blk,
                                                      double2* __restrict__ partial) {
    using R = typename std::conditional<(sizeof(CU) == 16 || sizeof(CV) == 16), double, float>::type;
    using RU = typename Acc<CU>::T;
    using RV = typename Acc<CV>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ku = U.total, kv = V.total;
    const int SU = gram_stride(ku), SV = gram_stride(kv);
    const int TIN = (ku + GT - 1) / GT, TJN = (kv + GT - 1) / GT;
    CU* su = reinterpret_cast<CU*>(smem_raw);                  // [2][GROWS][SU]
    CV* sv = reinterpret_cast<CV*>(su + 2 * GROWS * SU);       // [2][GROWS][SV]
    const CU** pu = reinterpret_cast<const CU**>(sv + 2 * GROWS * SV);   // column bases [ku]
    const CV** pv = reinterpret_cast<const CV**>(pu + ku);               // [kv]
    for (int i = threadIdx.x; i < ku; i += blockDim.x) pu[i] = col_ptr(U, i, ld);
    for (int j = threadIdx.x; j < kv; j += blockDim.x) pv[j] = col_ptr(V, j, ld);
    const int tile = blockIdx.y * blockDim.x + threadIdx.x;
    const int ti = tile / TJN, tj = tile - ti * TJN;
    const bool active = ti < TIN;
    const size_t r0 = blockIdx.x * rows_per_blk;
    const size_t r1 = min(ld, r0 + rows_per_blk);
    // padding columns (never loaded) stay zero
    for (int e = threadIdx.x; e < 2 * GROWS; e += blockDim.x) {
        for (int i = ku; i < SU; ++i) su[e * SU + i] = mk((RU)0, (RU)0);
        for (int j = kv; j < SV; ++j) sv[e * SV + j] = mk((RV)0, (RV)0);
    }
    __syncthreads();
    const auto stage = [su, sv, pu, pv, ku, kv, SU, SV, r1](size_t rb, int buf) {
        const int nr = (int)min((size_t)GROWS, r1 - rb);
        CU* du = su + buf * GROWS * SU;
        CV* dv = sv + buf * GROWS * SV;
        for (int e = threadIdx.x; e < GROWS * ku; e += blockDim.x) {
            const int i = e / GROWS, t = e - i * GROWS;
            cp_async_c(&du[t * SU + i], pu[i] + rb + (t < nr ? t : 0), t < nr);
        }
        for (int e = threadIdx.x; e < GROWS * kv; e += blockDim.x) {
            const int j = e / GROWS, t = e - j * GROWS;
            cp_async_c(&dv[t * SV + j], pv[j] + rb + (t < nr ? t : 0), t < nr);
        }
        cp_async_commit();
    };
    R accr[GT][GT], acci[GT][GT];
#pragma unroll
    for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) accr[a][b] = acci[a][b] = 0;
    const int nst = (int)((r1 - r0 + GROWS - 1) / GROWS);
    if (nst > 0) stage(r0, 0);
    for (int s = 0; s < nst; ++s) {
        if (s + 1 < nst) {
            stage(r0 + (size_t)(s + 1) * GROWS, (s + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (active) {
            const CU* bu = su + (s & 1) * GROWS * SU + ti;
            const CV* bv = sv + (s & 1) * GROWS * SV + tj;
#pragma unroll 1
            for (int t = 0; t < GROWS; ++t) {   // not unrolled: 83 registers, two 288-thread blocks per SM
                R ur[GT], ui[GT], wr[GT], wi[GT];
#pragma unroll
                for (int a = 0; a < GT; ++a) {
                    const CU x = bu[t * SU + TIN * a];
                    ur[a] = (R)x.x;
                    ui[a] = (R)x.y;
                }
#pragma unroll
                for (int b = 0; b < GT; ++b) {
                    const CV x = bv[t * SV + TJN * b];
                    wr[b] = (R)x.x;
                    wi[b] = (R)x.y;
                }
#pragma unroll
                for (int a = 0; a < GT; ++a)
#pragma unroll
                    for (int b = 0; b < GT; ++b) {
                        accr[a][b] = fma(ur[a], wr[b], fma(ui[a], wi[b], accr[a][b]));
                        acci[a][b] = fma(ur[a], wi[b], fma(-ui[a], wr[b], acci[a][b]));
                    }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    double2* out = partial + (size_t)blockIdx.x * ku * kv;
#pragma unroll
    for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) {
            const int i = ti + TIN * a, j = tj + TJN * b;
            if (i < ku && j < kv) out[(size_t)j * ku + i] = make_double2((double)accr[a][b], (double)acci[a][b]);
        }
}

// Complex64 Gram partials through a cp.async ring: same outputs and tile ownership
// as k_gram (FP32 products and sums within a block, partial[blk * nsl + slice]),
// for blocks that own whole kGRows-row tiles, kGStages tiles in flight.  The block
// runs nsl slices of the thread tiles; slice s takes the rows t = s (mod nsl) of
// every staged tile, so one stage feeds all warps with one pair of barriers.
// Shared memory: per stage, the U and V columns padded to multiples of GT (the
// padding columns stay zero), each column kGRows + 2 elements long (16-byte
// aligned, and columns four banks apart).
constexpr int kGRows = 64, kGStages = 3, kGStride = kGRows + 2;

__global__ void __launch_bounds__(512) k_gram_st(BlockList<float2> U, BlockList<float2> V, size_t ld, int nsl,
                                                  double2* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ku = U.total, kv = V.total, tid = threadIdx.x;
    const int TIN = (ku + GT - 1) / GT, TJN = (kv + GT - 1) / GT, KU = TIN * GT, KV = TJN * GT;
    const int ncol = KU + KV, ts = blockDim.x / nsl;
    float2* ring = reinterpret_cast<float2*>(smem_raw);             // [kGStages][ncol][kGStride]
    const float2** pc = reinterpret_cast<const float2**>(ring + (size_t)kGStages * ncol * kGStride);
    for (int c = tid; c < ncol; c += blockDim.x) {
        const float2* p = nullptr;
        if (c < ku) p = col_ptr(U, c, ld);
        else if (c >= KU && c - KU < kv) p = col_ptr(V, c - KU, ld);
        pc[c] = p;
    }
    for (int e = tid; e < kGStages * ncol * kGStride; e += blockDim.x) ring[e] = make_float2(0.f, 0.f);
    __syncthreads();
    const int slice = tid / ts, lt = tid - slice * ts;
    const int ti = lt / TJN, tj = lt - ti * TJN;
    const bool active = slice < nsl && ti < TIN;
    const size_t ntiles = (ld + kGRows - 1) / kGRows;
    size_t p_tile = blockIdx.x;
    int p_buf = 0;
    auto issue = [&]() {
        if (p_tile < ntiles) {
            float2* dst = ring + (size_t)p_buf * ncol * kGStride;
            for (int e = tid; e < ncol * (kGRows / 2); e += blockDim.x) {
                const int c = e / (kGRows / 2), rp = e - c * (kGRows / 2);
                const float2* col = pc[c];
                if (!col) continue;                                    // padding column
                const size_t row = p_tile * kGRows + 2 * (size_t)rp;
                const bool ok = row < ld;
                cp_async16(dst + c * kGStride + 2 * rp, ok ? col + row : col, ok);
            }
        }
        cp_async_commit();
        p_tile += gridDim.x;
        p_buf = p_buf + 1 == kGStages ? 0 : p_buf + 1;
    };
#pragma unroll
    for (int st = 0; st < kGStages - 1; ++st) issue();
    float accr[GT][GT], acci[GT][GT];
#pragma unroll
    for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) accr[a][b] = acci[a][b] = 0.f;
    int c_buf = 0;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        issue();
        cp_async_wait<kGStages - 1>();
        __syncthreads();
        if (active) {
            const float2* bu = ring + (size_t)c_buf * ncol * kGStride + (size_t)ti * kGStride;
            const float2* bv = ring + (size_t)c_buf * ncol * kGStride + (size_t)(KU + tj) * kGStride;
#pragma unroll 2
            for (int t = slice; t < kGRows; t += nsl) {
                float ur[GT], ui[GT], wr[GT], wi[GT];
#pragma unroll
                for (int a = 0; a < GT; ++a) {
                    const float2 x = bu[(size_t)TIN * a * kGStride + t];
                    ur[a] = x.x;
                    ui[a] = x.y;
                }
#pragma unroll
                for (int b = 0; b < GT; ++b) {
                    const float2 x = bv[(size_t)TJN * b * kGStride + t];
                    wr[b] = x.x;
                    wi[b] = x.y;
                }
#pragma unroll
                for (int a = 0; a < GT; ++a)
#pragma unroll
                    for (int b = 0; b < GT; ++b) {
                        accr[a][b] = fmaf(ur[a], wr[b], fmaf(ui[a], wi[b], accr[a][b]));
                        acci[a][b] = fmaf(ur[a], wi[b], fmaf(-ui[a], wr[b], acci[a][b]));
                    }
            }
        }
        c_buf = c_buf + 1 == kGStages ? 0 : c_buf + 1;
        __syncthreads();
    }
    cp_async_wait<0>();
    if (!active) return;
    double2* out = partial + ((size_t)blockIdx.x * nsl + slice) * ku * kv;
#pragma unroll
    for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) {
            const int i = ti + TIN * a, j = tj + TJN * b;
            if (i < ku && j < kv) out[(size_t)j * ku + i] = make_double2((double)accr[a][b], (double)acci[a][b]);
        }
}

// the ring-staged complex64 kernels apply: m <= 2 kStOut outputs, ld even, every
// column 16-byte aligned
template <typename C>
bool combine_st_ok(const BlockList<C>& S, size_t ld, int m) {
    if (!std::is_same<C, float2>::value || m > 2 * kStOut || (ld & 1) || S.total < 1) return false;
    for (int b = 0; b < BlockList<C>::kMax; ++b)
        if (S.cols[b] > 0 && (reinterpret_cast<uintptr_t>(S.ptr[b]) & 15)) return false;
    return true;
}

size_t gram_st_smem(int ku, int kv) {
    const int ncol = ((ku + GT - 1) / GT + (kv + GT - 1) / GT) * GT;
    return (size_t)kGStages * ncol * kGStride * sizeof(float2) + (size_t)ncol * sizeof(void*);
}

// Hermitian pair of Gram blocks of LOBPCG: partial[blk] = [U^H U | U^H V] over the
// block's rows (ku x 2ku, column-major), V = A U, for the entries on or below the
// diagonal of each block only (both are Hermitian; the consumer rebuilds the upper
// triangles from the lower ones).  Thread: one contiguous GT x GT tile of one
// block, tiles of the lower triangle enumerated row by row.  Same staging and
// precision as k_gram.
__host__ __device__ inline int herm_stride(int ku) {
    // row stride of the staged rows in elements: 16-byte aligned, 16 mod 128 bytes
    const int s = ((ku + GT - 1) / GT) * GT;
    return s + ((2 - s % 16) + 16) % 16;
}

// four consecutive complex values from 16-byte aligned shared memory, in 16-byte loads
__device__ __forceinline__ void load4(const float2* p, float2* v) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2* v) {
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = p[a];
}

template <typename C>
__global__ void __launch_bounds__(kGramThreads) k_gram_herm(BlockList<C> U, BlockList<C> V, size_t ld,
                                                           size_t rows_per_blk, double2* __restrict__ partial) {
    using R = typename Acc<C>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ku = U.total, SP = herm_stride(ku);
    const int T = (ku + GT - 1) / GT, ntri = T * (T + 1) / 2;
    C* su = reinterpret_cast<C*>(smem_raw);                    // [2][GROWS][SP]
    C* sv = su + 2 * GROWS * SP;                               // [2][GROWS][SP]
    const C** pu = reinterpret_cast<const C**>(sv + 2 * GROWS * SP);
    const C** pv = pu + ku;
    for (int i = threadIdx.x; i < ku; i += blockDim.x) {
        pu[i] = col_ptr(U, i, ld);
        pv[i] = col_ptr(V, i, ld);
    }
    for (int e = threadIdx.x; e < 2 * GROWS; e += blockDim.x)
        for (int i = ku; i < SP; ++i) su[e * SP + i] = sv[e * SP + i] = mk((R)0, (R)0);
    const int tile = blockIdx.y * blockDim.x + threadIdx.x;
    const bool active = tile < 2 * ntri;
    const int sblk = active ? tile / ntri : 0, tr = active ? tile - sblk * ntri : 0;
    int ti = (int)((sqrtf(8.0f * tr + 1.0f) - 1.0f) * 0.5f);
    while (ti * (ti + 1) / 2 > tr) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= tr) ++ti;
    const int tj = tr - ti * (ti + 1) / 2;
    const size_t r0 = blockIdx.x * rows_per_blk;
    const size_t r1 = min(ld, r0 + rows_per_blk);
    __syncthreads();
    const auto stage = [su, sv, pu, pv, ku, SP, r1](size_t rb, int buf) {
        const int nr = (int)min((size_t)GROWS, r1 - rb);
        C* du = su + buf * GROWS * SP;
        C* dv = sv + buf * GROWS * SP;
        for (int e = threadIdx.x; e < GROWS * ku; e += blockDim.x) {
            const int i = e / GROWS, t = e - i * GROWS;
            const size_t off = rb + (t < nr ? t : 0);
            cp_async_c(&du[t * SP + i], pu[i] + off, t < nr);
            cp_async_c(&dv[t * SP + i], pv[i] + off, t < nr);
        }
        cp_async_commit();
    };
    R accr[GT][GT], acci[GT][GT];
#pragma unroll
    for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) accr[a][b] = acci[a][b] = 0;
    const int nst = (int)((r1 - r0 + GROWS - 1) / GROWS);
    if (nst > 0) stage(r0, 0);
    for (int st = 0; st < nst; ++st) {
        if (st + 1 < nst) {
            stage(r0 + (size_t)(st + 1) * GROWS, (st + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (active) {
            const C* bu = su + (st & 1) * GROWS * SP + ti * GT;
            const C* bw = (sblk == 0 ? su : sv) + (st & 1) * GROWS * SP + tj * GT;
#pragma unroll 1
            for (int t = 0; t < GROWS; ++t) {
                static_assert(GT == 4, "load4 stages four columns");
                C u[GT], w[GT];
                load4(bu + t * SP, u);
                load4(bw + t * SP, w);
#pragma unroll
                for (int a = 0; a < GT; ++a)
#pragma unroll
                    for (int b = 0; b < GT; ++b) {
                        accr[a][b] = fma(u[a].x, w[b].x, fma(u[a].y, w[b].y, accr[a][b]));
                        acci[a][b] = fma(u[a].x, w[b].y, fma(-u[a].y, w[b].x, acci[a][b]));
                    }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    double2* out = partial + (size_t)blockIdx.x * ku * 2 * ku + (size_t)sblk * ku * ku;
#pragma unroll
    for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) {
            const int i = ti * GT + a, j = tj * GT + b;
            if (i < ku && j < ku) out[(size_t)j * ku + i] = make_double2((double)accr[a][b], (double)acci[a][b]);
        }
}

// The Hermitian Gram pair of k_gram_herm for complex128 blocks in double-float
// arithmetic on the FP32 units (df64.cuh: Dekker's exact products with FMA, Knuth's
// two-sum; about 2^-47 relative per sum), where the FP64 units of this GPU run at a
// small fraction of the FP32 rate.  Same staging as k_gram_herm; after each stage
// lands, every staged double is split once into a float pair (h, l) in shared
// memory, then each thread accumulates a 2 x 2 tile of entries.
constexpr int GT2 = 2;

__global__ void __launch_bounds__(kGramThreads) k_gram_herm_df(BlockList<double2> U, BlockList<double2> V,
                                                               size_t ld, size_t rows_per_blk,
                                                               double2* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ku = U.total, SP = herm_stride(ku);
    const int T = (ku + GT2 - 1) / GT2, ntri = T * (T + 1) / 2;
    double2* su = reinterpret_cast<double2*>(smem_raw);              // [2][GROWS][SP]
    double2* sv = su + 2 * GROWS * SP;                               // [2][GROWS][SP]
    float4* hu = reinterpret_cast<float4*>(sv + 2 * GROWS * SP);     // [GROWS][SP]: (re h, re l, im h, im l)
    float4* hv = hu + GROWS * SP;                                    // [GROWS][SP]
    const double2** pu = reinterpret_cast<const double2**>(hv + GROWS * SP);
    const double2** pv = pu + ku;
    for (int i = threadIdx.x; i < ku; i += blockDim.x) {
        pu[i] = col_ptr(U, i, ld);
        pv[i] = col_ptr(V, i, ld);
    }
    for (int e = threadIdx.x; e < 2 * GROWS; e += blockDim.x)
        for (int i = ku; i < SP; ++i) su[e * SP + i] = sv[e * SP + i] = make_double2(0.0, 0.0);
    const int tile = blockIdx.y * blockDim.x + threadIdx.x;
    const bool active = tile < 2 * ntri;
    const int sblk = active ? tile / ntri : 0, tr = active ? tile - sblk * ntri : 0;
    int ti = (int)((sqrtf(8.0f * tr + 1.0f) - 1.0f) * 0.5f);
    while (ti * (ti + 1) / 2 > tr) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= tr) ++ti;
    const int tj = tr - ti * (ti + 1) / 2;
    const size_t r0 = blockIdx.x * rows_per_blk;
    const size_t r1 = min(ld, r0 + rows_per_blk);
    __syncthreads();
    const auto stage = [su, sv, pu, pv, ku, SP, r1](size_t rb, int buf) {
        const int nr = (int)min((size_t)GROWS, r1 - rb);
        double2* du = su + buf * GROWS * SP;
        double2* dv = sv + buf * GROWS * SP;
        for (int e = threadIdx.x; e < GROWS * ku; e += blockDim.x) {
            const int i = e / GROWS, t = e - i * GROWS;
            const size_t off = rb + (t < nr ? t : 0);
            cp_async_c(&du[t * SP + i], pu[i] + off, t < nr);
            cp_async_c(&dv[t * SP + i], pv[i] + off, t < nr);
        }
        cp_async_commit();
    };
    float Sr[GT2][GT2], Er[GT2][GT2], Si[GT2][GT2], Ei[GT2][GT2];
#pragma unroll
    for (int a = 0; a < GT2; ++a)
#pragma unroll
        for (int b = 0; b < GT2; ++b) Sr[a][b] = Er[a][b] = Si[a][b] = Ei[a][b] = 0.f;
    const int nst = (int)((r1 - r0 + GROWS - 1) / GROWS);
    if (nst > 0) stage(r0, 0);
    for (int st = 0; st < nst; ++st) {
        if (st + 1 < nst) {
            stage(r0 + (size_t)(st + 1) * GROWS, (st + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        {
            const double2* bu = su + (st & 1) * GROWS * SP;
            const double2* bv = sv + (st & 1) * GROWS * SP;
            for (int e = threadIdx.x; e < GROWS * SP; e += blockDim.x) {
                const double2 x = bu[e], y = bv[e];
                const df64::Split a = df64::split(x.x), b = df64::split(x.y);
                const df64::Split c = df64::split(y.x), d = df64::split(y.y);
                hu[e] = make_float4(a.h, a.l, b.h, b.l);
                hv[e] = make_float4(c.h, c.l, d.h, d.l);
            }
        }
        __syncthreads();
        if (active) {
            const float4* bu = hu + ti * GT2;
            const float4* bw = (sblk == 0 ? hu : hv) + tj * GT2;
#pragma unroll 1
            for (int t = 0; t < GROWS; ++t) {
                float4 u[GT2], w[GT2];
#pragma unroll
                for (int a = 0; a < GT2; ++a) {
                    u[a] = bu[t * SP + a];
                    w[a] = bw[t * SP + a];
                }
#pragma unroll
                for (int a = 0; a < GT2; ++a)
#pragma unroll
                    for (int b = 0; b < GT2; ++b) {
                        // conj(u) w: re = ur wr + ui wi, im = ur wi - ui wr
                        df64::mac(Sr[a][b], Er[a][b], u[a].x, u[a].y, w[b].x, w[b].y);
                        df64::mac(Sr[a][b], Er[a][b], u[a].z, u[a].w, w[b].z, w[b].w);
                        df64::mac(Si[a][b], Ei[a][b], u[a].x, u[a].y, w[b].z, w[b].w);
                        df64::mac(Si[a][b], Ei[a][b], -u[a].z, -u[a].w, w[b].x, w[b].y);
                    }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    double2* out = partial + (size_t)blockIdx.x * ku * 2 * ku + (size_t)sblk * ku * ku;
#pragma unroll
    for (int a = 0; a < GT2; ++a)
#pragma unroll
        for (int b = 0; b < GT2; ++b) {
            const int i = ti * GT2 + a, j = tj * GT2 + b;
            if (i < ku && j < ku)
                out[(size_t)j * ku + i] = make_double2(df64::widen(Sr[a][b]) + df64::widen(Er[a][b]),
                                                       df64::widen(Si[a][b]) + df64::widen(Ei[a][b]));
        }
}

// G = sum over blocks of partial (fixed order, deterministic)
// One warp per entry: lanes take blocks lane, lane+32, ...; fixed shuffle tree.
// herm_k > 0: the Hermitian pair layout of k_gram_herm (k x 2k); entries above the
// diagonal of either block were not computed and are set to zero.
__global__ void k_gram_reduce(const double2* __restrict__ partial, int nblk, int kk,
                              double2* __restrict__ G, int herm_k) {
    const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (e >= kk) return;
    if (herm_k > 0 && (e / herm_k) % herm_k > e % herm_k) {
        if (lane == 0) G[e] = make_double2(0.0, 0.0);
        return;
    }
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
// ([i][j], outputs padded to a multiple of CJ) in the block's precision;
// accumulation in that precision.  A thread owns CR rows (r, r + 32) by CJ
// consecutive outputs; a warp covers 64 consecutive rows of one output group,
// so its loads of S are coalesced and its coefficient reads are broadcasts.
constexpr int CR = 2, CJ = 8, kCombineThreads = 256, kCombineSlots = 2;

template <typename C, typename Co>
__global__ void __launch_bounds__(kCombineThreads) k_combine(BlockList<C> S, size_t ld, const double2* __restrict__ M,
                                                             int m, int i0, Co* __restrict__ out1,
                                                             Co* __restrict__ out2) {
    using R = typename Acc<C>::T;
    using Ro = decltype(Co().x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = S.total, ng = (m + CJ - 1) / CJ, MP = ng * CJ;
    C* sm = reinterpret_cast<C*>(smem_raw);                        // [k][MP]
    const C** ps = reinterpret_cast<const C**>(sm + (size_t)k * MP); // column bases [k]
    for (int e = threadIdx.x; e < k * MP; e += blockDim.x) {
        const int i = e / MP, j = e - i * MP;
        sm[e] = j < m ? mk((R)M[(size_t)j * k + i].x, (R)M[(size_t)j * k + i].y) : mk((R)0, (R)0);
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) ps[i] = col_ptr(S, i, ld);
    __syncthreads();
    constexpr int TPS = kCombineThreads / kCombineSlots;         // threads per output-group slot
    const int slot = threadIdx.x / TPS, lt = threadIdx.x % TPS;
    const size_t span = (size_t)TPS * CR;                         // rows per block step
    for (size_t base = blockIdx.x * span; base < ld; base += (size_t)gridDim.x * span) {
        const size_t ra = base + (size_t)(lt >> 5) * 64 + (lt & 31), rb = ra + 32;
        // rows past the end load a valid row and are never stored: unconditional loads
        const size_t la = min(ra, ld - 1), lb = min(rb, ld - 1);
        for (int g = slot; g < ng; g += kCombineSlots) {
            C a1[CR][CJ], a2[CR][CJ];
#pragma unroll
            for (int r = 0; r < CR; ++r)
#pragma unroll
                for (int j = 0; j < CJ; ++j) a1[r][j] = a2[r][j] = mk((R)0, (R)0);
            const C* cf = sm + g * CJ;
#pragma unroll 4
            for (int i = 0; i < i0 && i < k; ++i) {
                const C xa = ps[i][la];
                const C xb = ps[i][lb];
#pragma unroll
                for (int j = 0; j < CJ; ++j) {
                    const C w = cf[(size_t)i * MP + j];
                    a1[0][j] = a1[0][j] + cmul(xa, w);
                    a1[1][j] = a1[1][j] + cmul(xb, w);
                }
            }
#pragma unroll 4
            for (int i = i0; i < k; ++i) {
                const C xa = ps[i][la];
                const C xb = ps[i][lb];
#pragma unroll
                for (int j = 0; j < CJ; ++j) {
                    const C w = cf[(size_t)i * MP + j];
                    a2[0][j] = a2[0][j] + cmul(xa, w);
                    a2[1][j] = a2[1][j] + cmul(xb, w);
                }
            }
#pragma unroll
            for (int j = 0; j < CJ; ++j) {
                const int jj = g * CJ + j;
                if (jj >= m) break;
#pragma unroll
                for (int r = 0; r < CR; ++r) {
                    const size_t row = r == 0 ? ra : rb;
                    if (row >= ld) continue;
                    const C t = a1[r][j] + a2[r][j];
                    if (out1) out1[(size_t)jj * ld + row] = mk((Ro)t.x, (Ro)t.y);
                    if (out2) out2[(size_t)jj * ld + row] = mk((Ro)a2[r][j].x, (Ro)a2[r][j].y);
                }
            }
        }
    }
}

// Complex64 combine with the inputs streamed through shared memory.  Same result as
// k_combine<float2, Co> (out1_j = sum_{i<k} S_i M[i][j], out2_j = sum_{i>=i0} S_i M[i][j],
// FP32 products and sums) for m <= 2 kStOut outputs.  A block owns kStRows-row tiles
// and has one kStRows-thread group per kStOut outputs (one row per thread, the
// group's outputs in registers); it streams the k input columns in chunks of
// kStCols through a kStStages-deep ring of cp.async copies, so the loads of later
// chunks (and of the next tile) are in flight while a chunk is consumed.  Columns
// are visited in the order i0..k-1, 0..i0-1 with one accumulator: out2 is stored
// when the first group of columns is complete, out1 at the end.
template <typename Co, int G, bool RF = false>
__global__ void __launch_bounds__(G * kStRows, (G == 1 ? 1 : 2)) k_combine_st(BlockList<float2> S, size_t ld,
                                                             const double2* __restrict__ M, int m, int i0,
                                                             Co* __restrict__ out1, Co* __restrict__ out2,
                                                             RefineEpi rf = RefineEpi{}) {
    using Ro = decltype(Co().x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nthr = G * kStRows, mo = G * kStOut;
    const int k = S.total, tid = threadIdx.x;
    const int g = tid / kStRows, rl = tid - g * kStRows, j0 = g * kStOut;
    const int first = i0 < k ? i0 : k;                         // columns i0..k-1 come first
    const int nchunk = (k + kStCols - 1) / kStCols, kp = nchunk * kStCols;
    // coefficients [kp][mo] in visiting order, zero past k and past m
    float4* cf = reinterpret_cast<float4*>(smem_raw);
    float2* stage = reinterpret_cast<float2*>(cf + (size_t)kp * (mo / 2));   // [stages][cols][rows]
    const float2** ps = reinterpret_cast<const float2**>(stage + kStStages * kStCols * kStRows);
    // refinement form: the double-float coefficients of each output's block, [mo][kRefBlk]
    // as (re h, re l, im h, im l), and the block table [mo][kRefBlk + 1]
    float4* cfd = reinterpret_cast<float4*>(ps + ((k + 1) & ~1));
    int* blk = reinterpret_cast<int*>(cfd + (RF ? mo * kRefBlk : 0));
    // refinement form: the tile's rows of the complex128 X, [mx][kStRows], copied when the
    // tile starts so that the epilogue finds them in shared memory
    double2* xs = reinterpret_cast<double2*>(blk + (RF ? mo * (kRefBlk + 1) : 0));
    if constexpr (RF) {
        for (int e = tid; e < mo * (kRefBlk + 1); e += nthr) {
            const int j = e / (kRefBlk + 1);
            blk[e] = j < m ? rf.blk[e] : 0;
        }
        __syncthreads();
        for (int e = tid; e < mo * kRefBlk; e += nthr) {
            const int j = e / kRefBlk, t = e - j * kRefBlk;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < blk[j * (kRefBlk + 1)]) {
                const double2 v = M[(size_t)j * k + blk[j * (kRefBlk + 1) + 1 + t]];
                const df64::Split a = df64::split(v.x), b = df64::split(v.y);
                w = make_float4(a.h, a.l, b.h, b.l);
            }
            cfd[e] = w;
        }
    }
    for (int e = tid; e < kp * mo; e += nthr) {
        const int pos = e / mo, j = e - pos * mo;
        const int i = pos < k - first ? first + pos : pos - (k - first);
        double2 v = (j < m && pos < k) ? M[(size_t)j * k + i] : make_double2(0.0, 0.0);
        if constexpr (RF) {
            // entries of an output's own block are summed in double-float below
            if (j < m && i < rf.mx)
                for (int t = 0; t < blk[j * (kRefBlk + 1)]; ++t)
                    if (blk[j * (kRefBlk + 1) + 1 + t] == i) v = make_double2(0.0, 0.0);
        }
        reinterpret_cast<float2*>(cf)[e] = make_float2((float)v.x, (float)v.y);
    }
    for (int pos = tid; pos < k; pos += nthr) {
        const int i = pos < k - first ? first + pos : pos - (k - first);
        ps[pos] = col_ptr(S, i, ld);
    }
    __syncthreads();
    const size_t ntiles = (ld + kStRows - 1) / kStRows;
    // out2 is complete after visiting position k - first - 1
    const int split = k - first - 1, split_chunk = split >= 0 ? split / kStCols : -1;
    const int split_c = split >= 0 ? split - split_chunk * kStCols : -1;
    // producer: the next (tile, chunk) stage to request; every call commits one group
    size_t p_tile = blockIdx.x;
    int p_chunk = 0, p_buf = 0;
    auto issue = [&]() {
        if (p_tile < ntiles) {
            float2* dst = stage + p_buf * (kStCols * kStRows);
            for (int e = tid; e < kStCols * kStRows / 2; e += nthr) {
                const int c = e / (kStRows / 2), rp = e - c * (kStRows / 2);
                const int pos = p_chunk * kStCols + c;
                const size_t row = p_tile * kStRows + 2 * (size_t)rp;
                // a 16-byte copy takes rows row and row + 1
                const bool ok = pos < k && row < ld && bounds_ok(row + 2 <= ld, kBndRing, (long long)row);
                cp_async16(dst + c * kStRows + 2 * rp, ok ? ps[pos] + row : ps[0], ok);
            }
        }
        cp_async_commit();
        if (++p_chunk == nchunk) {
            p_chunk = 0;
            p_tile += gridDim.x;
        }
        p_buf = p_buf + 1 == kStStages ? 0 : p_buf + 1;
    };
#pragma unroll
    for (int st = 0; st < kStStages - 1; ++st) issue();
    int c_buf = 0;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t row = tile * kStRows + rl;
        if constexpr (RF) {
            // one more copy group, older than the tile's nchunk stages: complete by the
            // last chunk's wait when nchunk >= kStStages - 1, else waited for below
            __syncthreads();                                   // the previous epilogue has read xs
            const size_t rbase = tile * kStRows;
            for (int e = tid; e < rf.mx * kStRows; e += nthr) {
                const int i = e / kStRows, r = e - i * kStRows;
                const bool ok = rbase + r < ld;
                cp_async16(xs + e, ok ? rf.X64 + (size_t)i * ld + rbase + r : rf.X64, ok);
            }
            cp_async_commit();
        }
        float2 acc[kStOut];
#pragma unroll
        for (int j = 0; j < kStOut; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int chunk = 0; chunk < nchunk; ++chunk) {
            issue();
            cp_async_wait<kStStages - 1>();
            __syncthreads();
            const float2* X = stage + c_buf * (kStCols * kStRows);
            const float4* w = cf + (size_t)chunk * kStCols * (mo / 2) + g * (kStOut / 2);
            const int store_c = (out2 && chunk == split_chunk) ? split_c : -1;
#pragma unroll
            for (int c = 0; c < kStCols; ++c) {
                const float2 x = X[c * kStRows + rl];
#pragma unroll
                for (int q = 0; q < kStOut / 2; ++q) {
                    const float4 c2 = w[c * (mo / 2) + q];
                    acc[2 * q].x = fmaf(x.x, c2.x, fmaf(-x.y, c2.y, acc[2 * q].x));
                    acc[2 * q].y = fmaf(x.x, c2.y, fmaf(x.y, c2.x, acc[2 * q].y));
                    acc[2 * q + 1].x = fmaf(x.x, c2.z, fmaf(-x.y, c2.w, acc[2 * q + 1].x));
                    acc[2 * q + 1].y = fmaf(x.x, c2.w, fmaf(x.y, c2.z, acc[2 * q + 1].y));
                }
                if (c == store_c && row < ld) {
#pragma unroll
                    for (int j = 0; j < kStOut; ++j) {
                        if (j0 + j >= m) break;
                        out2[(size_t)(j0 + j) * ld + row] = mk((Ro)acc[j].x, (Ro)acc[j].y);
                    }
                }
            }
            c_buf = c_buf + 1 == kStStages ? 0 : c_buf + 1;
            __syncthreads();
        }
        if constexpr (RF) {
            static_assert(kStStages == 4, "the waits below cover nchunk < kStStages - 1");
            if (nchunk < kStStages - 1) {
                if (nchunk == 1) cp_async_wait<1>();
                else cp_async_wait<2>();
                __syncthreads();
            }
        }
        if (row < ld) {
#pragma unroll
            for (int j = 0; j < kStOut; ++j) {
                if (j0 + j >= m) break;
                if (out1) out1[(size_t)(j0 + j) * ld + row] = mk((Ro)acc[j].x, (Ro)acc[j].y);
                if (out2 && first == k) out2[(size_t)(j0 + j) * ld + row] = mk((Ro)0, (Ro)0);   // empty second sum
            }
            if constexpr (RF) {
                // Xn_j = sum over the block of j of X_i M[i][j] (complex128 inputs, double-float
                // sums) + the FP32 sum of everything else
#pragma unroll
                for (int j = 0; j < kStOut; ++j) {
                    const int jj = j0 + j;
                    if (jj >= m) break;
                    const int* b = blk + jj * (kRefBlk + 1);
                    float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f;
                    for (int t = 0; t < b[0]; ++t) {
                        if (!bounds_ok(b[1 + t] >= 0 && b[1 + t] < rf.mx, kBndXRows, b[1 + t])) continue;
                        const double2 x = xs[b[1 + t] * kStRows + rl];
                        const df64::Split xr = df64::split(x.x), xi = df64::split(x.y);
                        const float4 w = cfd[jj * kRefBlk + t];
                        df64::mac(Sr, Er, xr.h, xr.l, w.x, w.y);
                        df64::mac(Sr, Er, -xi.h, -xi.l, w.z, w.w);
                        df64::mac(Si, Ei, xr.h, xr.l, w.z, w.w);
                        df64::mac(Si, Ei, xi.h, xi.l, w.x, w.y);
                    }
                    const float er = Er + acc[j].x, ei = Ei + acc[j].y;
                    const size_t o = (size_t)jj * ld + row;
                    rf.Xn64[o] = make_double2(df64::widen(Sr) + df64::widen(er), df64::widen(Si) + df64::widen(ei));
                    if (rf.X32n) rf.X32n[o] = make_float2(Sr + er, Si + ei);
                }
            }
        }
    }
    cp_async_wait<0>();
}

// Complex64 Q_j <- Q_j - sum_i X_i c[i][j] (in place, m <= 2 kStOut, nq <= 4 kStOut) with
// the same cp.async ring as k_combine_st.  A row tile's stream is the Q columns
// (chunks of kStCols; they initialise the accumulators) followed by the X columns.
// The block has one 128-thread group per kStOut output columns; every group reads
// each X chunk, and each group takes only its own Q chunks.
template <int G>
__global__ void __launch_bounds__(G * kStRows) k_orth_st(const float2* __restrict__ X, int m, BlockList<float2> Q,
                                                          size_t ld, const double2* __restrict__ cfs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nthr = G * kStRows, nqo = G * kStOut;
    const int nq = Q.total, tid = threadIdx.x;
    const int g = tid / kStRows, rl = tid - g * kStRows;
    const int nqc = (nq + kStCols - 1) / kStCols, nxc = (m + kStCols - 1) / kStCols, nchunk = nqc + nxc;
    const int mp = nxc * kStCols;
    float4* cf = reinterpret_cast<float4*>(smem_raw);              // [mp][nqo / 2]: (c[i][2q], c[i][2q+1])
    float2* stage = reinterpret_cast<float2*>(cf + (size_t)mp * (nqo / 2));
    float2** qp = reinterpret_cast<float2**>(stage + kStStages * kStCols * kStRows);   // [nqo]
    for (int e = tid; e < mp * nqo; e += nthr) {
        const int i = e / nqo, j = e - i * nqo;
        const double2 v = (i < m && j < nq) ? cfs[(size_t)j * m + i] : make_double2(0.0, 0.0);
        reinterpret_cast<float2*>(cf)[e] = make_float2((float)v.x, (float)v.y);
    }
    for (int j = tid; j < nqo; j += nthr) qp[j] = j < nq ? const_cast<float2*>(col_ptr(Q, j, ld)) : nullptr;
    __syncthreads();
    const size_t ntiles = (ld + kStRows - 1) / kStRows;
    size_t p_tile = blockIdx.x;
    int p_chunk = 0, p_buf = 0;
    auto issue = [&]() {
        if (p_tile < ntiles) {
            float2* dst = stage + p_buf * (kStCols * kStRows);
            for (int e = tid; e < kStCols * kStRows / 2; e += nthr) {
                const int c = e / (kStRows / 2), rp = e - c * (kStRows / 2);
                const size_t row = p_tile * kStRows + 2 * (size_t)rp;
                const float2* src = nullptr;
                if (p_chunk < nqc) {
                    const int j = p_chunk * kStCols + c;
                    if (j < nq) src = qp[j] + row;
                } else {
                    const int i = (p_chunk - nqc) * kStCols + c;
                    if (i < m) src = X + (size_t)i * ld + row;
                }
                const bool ok = src != nullptr && row < ld && bounds_ok(row + 2 <= ld, kBndRing, (long long)row);
                cp_async16(dst + c * kStRows + 2 * rp, ok ? src : X, ok);
            }
        }
        cp_async_commit();
        if (++p_chunk == nchunk) {
            p_chunk = 0;
            p_tile += gridDim.x;
        }
        p_buf = p_buf + 1 == kStStages ? 0 : p_buf + 1;
    };
#pragma unroll
    for (int s = 0; s < kStStages - 1; ++s) issue();
    int c_buf = 0;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t row = tile * kStRows + rl;
        float2 acc[kStOut];
#pragma unroll
        for (int j = 0; j < kStOut; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int ch = 0; ch < nchunk; ++ch) {
            issue();
            cp_async_wait<kStStages - 1>();
            __syncthreads();
            const float2* B = stage + c_buf * (kStCols * kStRows);
            if (ch < nqc) {
                const int lo = ch * kStCols - g * kStOut;            // offset in this group's outputs
#pragma unroll
                for (int s0 = 0; s0 < kStOut; s0 += kStCols) {
                    if (lo == s0) {
#pragma unroll
                        for (int c = 0; c < kStCols; ++c) acc[s0 + c] = B[c * kStRows + rl];
                    }
                }
            } else {
                const float4* w = cf + (size_t)(ch - nqc) * kStCols * (nqo / 2) + g * (kStOut / 2);
#pragma unroll
                for (int c = 0; c < kStCols; ++c) {
                    const float2 x = B[c * kStRows + rl];
#pragma unroll
                    for (int q = 0; q < kStOut / 2; ++q) {
                        const float4 c2 = w[c * (nqo / 2) + q];
                        acc[2 * q].x = fmaf(-x.x, c2.x, fmaf(x.y, c2.y, acc[2 * q].x));
                        acc[2 * q].y = fmaf(-x.x, c2.y, fmaf(-x.y, c2.x, acc[2 * q].y));
                        acc[2 * q + 1].x = fmaf(-x.x, c2.z, fmaf(x.y, c2.w, acc[2 * q + 1].x));
                        acc[2 * q + 1].y = fmaf(-x.x, c2.w, fmaf(-x.y, c2.z, acc[2 * q + 1].y));
                    }
                }
            }
            c_buf = c_buf + 1 == kStStages ? 0 : c_buf + 1;
            __syncthreads();
        }
        if (row < ld) {
#pragma unroll
            for (int j = 0; j < kStOut; ++j) {
                const int col = g * kStOut + j;
                if (col < nq) qp[col][row] = acc[j];
            }
        }
    }
    cp_async_wait<0>();
}

size_t orth_st_smem(int m, int groups) {
    const int mp = (m + kStCols - 1) / kStCols * kStCols;
    return (size_t)mp * groups * kStOut * sizeof(float2) +
           (size_t)kStStages * kStCols * kStRows * sizeof(float2) + (size_t)groups * kStOut * sizeof(void*);
}

size_t combine_st_smem(int k, int groups, bool refine = false) {
    const int kp = (k + kStCols - 1) / kStCols * kStCols;
    return (size_t)kp * groups * kStOut * sizeof(float2) +
           (size_t)kStStages * kStCols * kStRows * sizeof(float2) + (size_t)((k + 1) & ~1) * sizeof(void*) +
           (refine ? (size_t)groups * kStOut *
                         (kRefBlk * sizeof(float4) + (kRefBlk + 1) * sizeof(int) + kStRows * sizeof(double2))
                   : 0);
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
    R sr = 0;                       // a thread's few rows summed in the block's precision
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        const C x = X[(size_t)j * ld + row], ax = AX[(size_t)j * ld + row];
        const C r = mk(ax.x - th * x.x, ax.y - th * x.y);
        sr += r.x * r.x + r.y * r.y;
        const R t = tinv[row < n ? row : row - n];
        if (W) W[(size_t)j * ld + row] = mk(t * r.x, t * r.y);
    }
    double s = (double)sr;
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
    float sf = 0.0f;                // |R|^2 of a thread's few rows from R rounded to float
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        const double2 x = X[(size_t)j * ld + row], ax = AX[(size_t)j * ld + row];
        const float rx = df64::narrow(ax.x - th * x.x), ry = df64::narrow(ax.y - th * x.y);
        sf += rx * rx + ry * ry;
        const float t = tinv[row < n ? row : row - n];
        W[(size_t)j * ld + row] = make_float2(t * rx, t * ry);
        if (R32) R32[(size_t)j * ld + row] = make_float2(rx, ry);
    }
    double s = (double)sf;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
}

// Refinement update Xn = X M[:m] + Q M[m:] with X complex128.  The X part is
// summed in double-float arithmetic (df64.cuh: FP64-accurate, FP32 instructions;
// the native FP64 rate of this GPU is a small fraction of its FP32 rate), the Q
// part (a correction orthogonal to X) in FP32.  Outputs: Xn (complex128), its
// complex64 copy X32n (may be null), and Pn = Q M[m:] (complex64, may be null).  M column-major
// k x m, k = m + nq; its X rows are split into float pairs once per block.
constexpr int MJ = 8;   // output columns per pass over the inputs

__global__ void __launch_bounds__(256) k_combine_mixed(const double2* __restrict__ X, int m, BlockList<float2> Q,
                                                       size_t ld, const double2* __restrict__ M,
                                                       double2* __restrict__ Xn, float2* __restrict__ X32n,
                                                       float2* __restrict__ Pn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nq = Q.total, k = m + nq, ng = (m + MJ - 1) / MJ, MP = ng * MJ;
    float4* cx = reinterpret_cast<float4*>(smem_raw);               // [m][MP]: (re h, re l, im h, im l)
    float2* cq = reinterpret_cast<float2*>(cx + (size_t)m * MP);     // [nq][MP]
    const float2** qp = reinterpret_cast<const float2**>(cq + (size_t)nq * MP);
    for (int e = threadIdx.x; e < k * MP; e += blockDim.x) {
        const int i = e / MP, j = e - i * MP;
        const double2 v = j < m ? M[(size_t)j * k + i] : make_double2(0.0, 0.0);
        if (i < m) {
            const float rh = (float)v.x, ih = (float)v.y;
            cx[e] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
        } else {
            cq[e - (size_t)m * MP] = make_float2((float)v.x, (float)v.y);
        }
    }
    for (int i = threadIdx.x; i < nq; i += blockDim.x) qp[i] = col_ptr(Q, i, ld);
    __syncthreads();
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < ld;
         row += (size_t)gridDim.x * blockDim.x) {
        for (int g = 0; g < ng; ++g) {
            float Sr[MJ], Er[MJ], Si[MJ], Ei[MJ];
            float2 d[MJ];
#pragma unroll
            for (int j = 0; j < MJ; ++j) {
                Sr[j] = Er[j] = Si[j] = Ei[j] = 0.0f;
                d[j] = make_float2(0.0f, 0.0f);
            }
            for (int i = 0; i < m; ++i) {
                const double2 x = X[(size_t)i * ld + row];
                const df64::Split xr = df64::split(x.x), xi = df64::split(x.y);
                const float4* c = cx + (size_t)i * MP + g * MJ;
#pragma unroll
                for (int j = 0; j < MJ; ++j) {
                    const float4 w = c[j];
                    // (xr + i xi)(wr + i wi): re = xr wr - xi wi, im = xr wi + xi wr
                    df64::mac(Sr[j], Er[j], xr.h, xr.l, w.x, w.y);
                    df64::mac(Sr[j], Er[j], -xi.h, -xi.l, w.z, w.w);
                    df64::mac(Si[j], Ei[j], xr.h, xr.l, w.z, w.w);
                    df64::mac(Si[j], Ei[j], xi.h, xi.l, w.x, w.y);
                }
            }
            for (int i = 0; i < nq; ++i) {
                const float2 q = qp[i][row];
                const float2* c = cq + (size_t)i * MP + g * MJ;
#pragma unroll
                for (int j = 0; j < MJ; ++j) d[j] = d[j] + cmul(q, c[j]);
            }
#pragma unroll
            for (int j = 0; j < MJ; ++j) {
                const int jj = g * MJ + j;
                if (jj >= m) break;
                const size_t o = (size_t)jj * ld + row;
                const float er = Er[j] + d[j].x, ei = Ei[j] + d[j].y;
                Xn[o] = make_double2(df64::widen(Sr[j]) + df64::widen(er), df64::widen(Si[j]) + df64::widen(ei));
                if (X32n) X32n[o] = make_float2(Sr[j] + er, Si[j] + ei);
                if (Pn) Pn[o] = d[j];
            }
        }
    }
}

// Q_j <- Q_j - sum_i X_i c[i][j] for the nq columns of Q (in place), c m x nq
// column-major.  Arithmetic in FP64 when X is complex128, else FP32.  Same thread
// layout as k_combine: CR rows (r, r + 32) by CJ consecutive columns of Q.
template <typename CX, typename CQ>
__global__ void __launch_bounds__(kCombineThreads) k_orth(const CX* __restrict__ X, int m, BlockList<CQ> Q,
                                                          size_t ld, const double2* __restrict__ cfs) {
    using R = typename Acc<CX>::T;
    using C = CX;
    using RQ = typename Acc<CQ>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nq = Q.total, ng = (nq + CJ - 1) / CJ, MP = ng * CJ;
    C* sc = reinterpret_cast<C*>(smem_raw);                          // [m][MP]
    CQ** qp = reinterpret_cast<CQ**>(sc + (size_t)m * MP);           // [nq]
    for (int e = threadIdx.x; e < m * MP; e += blockDim.x) {
        const int i = e / MP, j = e - i * MP;
        sc[e] = j < nq ? mk((R)cfs[(size_t)j * m + i].x, (R)cfs[(size_t)j * m + i].y) : mk((R)0, (R)0);
    }
    for (int j = threadIdx.x; j < nq; j += blockDim.x) qp[j] = const_cast<CQ*>(col_ptr(Q, j, ld));
    __syncthreads();
    constexpr int TPS = kCombineThreads / kCombineSlots;
    const int slot = threadIdx.x / TPS, lt = threadIdx.x % TPS;
    const size_t span = (size_t)TPS * CR;
    for (size_t base = blockIdx.x * span; base < ld; base += (size_t)gridDim.x * span) {
        const size_t ra = base + (size_t)(lt >> 5) * 64 + (lt & 31), rb = ra + 32;
        const size_t la = min(ra, ld - 1), lb = min(rb, ld - 1);   // as in k_combine
        for (int g = slot; g < ng; g += kCombineSlots) {
            // start from Q (loads in flight while the products accumulate)
            C a[CR][CJ];
#pragma unroll
            for (int j = 0; j < CJ; ++j) {
                const int jj = g * CJ + j;
#pragma unroll
                for (int r = 0; r < CR; ++r) {
                    const size_t row = r == 0 ? ra : rb;
                    if (jj < nq && row < ld) {
                        const CQ v = qp[jj][row];
                        a[r][j] = mk((R)v.x, (R)v.y);
                    } else {
                        a[r][j] = mk((R)0, (R)0);
                    }
                }
            }
            const C* cf = sc + g * CJ;
#pragma unroll 4
            for (int i = 0; i < m; ++i) {
                const C xa = X[(size_t)i * ld + la];
                const C xb = X[(size_t)i * ld + lb];
#pragma unroll
                for (int j = 0; j < CJ; ++j) {
                    const C w = cf[(size_t)i * MP + j];
                    a[0][j] = a[0][j] - cmul(xa, w);
                    a[1][j] = a[1][j] - cmul(xb, w);
                }
            }
#pragma unroll
            for (int j = 0; j < CJ; ++j) {
                const int jj = g * CJ + j;
                if (jj >= nq) break;
#pragma unroll
                for (int r = 0; r < CR; ++r) {
                    const size_t row = r == 0 ? ra : rb;
                    if (row < ld) qp[jj][row] = mk((RQ)a[r][j].x, (RQ)a[r][j].y);
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
// Dynamic shared memory limit above the 48 KB default, and the largest shared-memory
// carveout (so that several blocks fit per SM), set once per kernel.
fame_status kernel_smem(fame_ctx* c, const void* fn, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(fn);
    if (it != done.end() && it->second >= smem) return FAME_OK;
    if (smem > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FAME_CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
    done[fn] = std::max(smem, it != done.end() ? it->second : (size_t)0);
    return FAME_OK;
}

template <typename CU, typename CV>
fame_status gram(fame_ctx* c, const BlockList<CU>& U, const BlockList<CV>& V, size_t ld,
                 double2* G, cudaStream_t st) {
    const int ku = U.total, kv = V.total;
    if constexpr (std::is_same<CU, float2>::value && std::is_same<CV, float2>::value) {
        if (tensor_cores_enabled() && std::max(ku, kv) >= tc_min_width()) {
            // the wider side on the 128-row MMA operand
            const fame_status s = kv >= ku ? gram_tc(c, V, U, ld, 1, G, st) : gram_tc(c, U, V, ld, 0, G, st);
            if (s != FAME_E_ARG) return s;
        }
        const int tiles = ((ku + GT - 1) / GT) * ((kv + GT - 1) / GT);
        const int ts = (tiles + 31) / 32 * 32;
        const size_t smem = gram_st_smem(ku, kv);
        if (ts <= 512 && smem <= 200u * 1024u && combine_st_ok(U, ld, 1) && combine_st_ok(V, ld, 1)) {
            const int nsl = std::min(8, 512 / ts);
            const void* fn = (const void*)k_gram_st;
            fame_status s = kernel_smem(c, fn, smem);
            if (s != FAME_OK) return s;
            int per_sm = 0;
            FAME_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ts * nsl, smem));
            const size_t ntiles = (ld + kGRows - 1) / kGRows;
            const int nblk = (int)std::max<size_t>(1, std::min<size_t>((size_t)152 * std::max(per_sm, 1), ntiles));
            const int nparts = nblk * nsl;
            if ((s = grow(c, c->partial, (size_t)nparts * ku * kv * sizeof(double2))) != FAME_OK) return s;
            double2* part = reinterpret_cast<double2*>(c->partial.p);
            {
                ProfScope ps(K_GRAM, false, st, (double)ld * (ku + kv) * sizeof(float2), 8.0 * ku * kv * (double)ld);
                k_gram_st<<<nblk, ts * nsl, smem, st>>>(U, V, ld, nsl, part);
            }
            const int kk = ku * kv;
            {
                ProfScope ps(K_GRAM_RED, false, st, (double)nparts * kk * sizeof(double2), 2.0 * nparts * kk);
                k_gram_reduce<<<(kk + 7) / 8, 256, 0, st>>>(part, nparts, kk, G, 0);
            }
            count_launch(2);
            FAME_CUDA_TRY(c, cudaGetLastError());
            return FAME_OK;
        }
    }
    const int tiles = ((ku + GT - 1) / GT) * ((kv + GT - 1) / GT);
    const int groups = (tiles + kGramThreads - 1) / kGramThreads;
    int threads = (((tiles + groups - 1) / groups + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    const bool dbl = sizeof(CU) == 16 || sizeof(CV) == 16;
    const size_t smem = (size_t)2 * GROWS * (gram_stride(ku) * sizeof(CU) + gram_stride(kv) * sizeof(CV)) +
                        (size_t)(ku + kv) * sizeof(void*);
    // enough blocks for about 24 resident warps per SM (small Grams have small blocks),
    // within what shared memory allows; each block's rows summed in the block's precision
    const int warps = threads / 32;
    const int by_smem = std::max(1, (int)((200u * 1024u) / std::max<size_t>(smem, 1)));
    int nblk = 152 * std::max(2, std::min({8, 24 / std::max(1, warps), by_smem}));
    size_t rpb = (ld + nblk - 1) / nblk;
    rpb = ((rpb + GROWS - 1) / GROWS) * GROWS;
    nblk = (int)((ld + rpb - 1) / rpb);
    fame_status s = grow(c, c->partial, (size_t)nblk * ku * kv * sizeof(double2));
    if (s != FAME_OK) return s;
    if ((s = kernel_smem(c, (const void*)k_gram<CU, CV>, smem)) != FAME_OK) return s;
    double2* part = reinterpret_cast<double2*>(c->partial.p);
    {
        ProfScope ps(K_GRAM, dbl, st, (double)ld * (ku * sizeof(CU) + kv * sizeof(CV)),
                     8.0 * ku * kv * (double)ld);
        k_gram<CU, CV><<<dim3(nblk, groups), threads, smem, st>>>(U, V, ld, rpb, part);
    }
    const int kk = ku * kv;
    {
        ProfScope ps(K_GRAM_RED, dbl, st, (double)nblk * kk * sizeof(double2), 2.0 * nblk * kk);
        k_gram_reduce<<<(kk + 7) / 8, 256, 0, st>>>(part, nblk, kk, G, 0);
    }
    count_launch(2);
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename C>
fame_status block_gram(fame_ctx* c, const C* U, int ku, const C* V, int kv, size_t ld, double2* G,
                       cudaStream_t st) {
    fame_status s = gram<C, C>(c, blocks<C>(U, ku), blocks<C>(V, kv), ld, G, st);
    if (s != FAME_OK) return s;
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}
template fame_status block_gram<float2>(fame_ctx*, const float2*, int, const float2*, int, size_t, double2*, cudaStream_t);
template fame_status block_gram<double2>(fame_ctx*, const double2*, int, const double2*, int, size_t, double2*, cudaStream_t);

template <typename C>
fame_status gram_herm(fame_ctx* c, const BlockList<C>& U, const BlockList<C>& V, size_t ld, double2* G,
                      cudaStream_t st) {
    const int ku = U.total;
    if (V.total != ku) return set_err(c, FAME_E_ARG, "gram_herm: U and V differ in width");
    if constexpr (std::is_same<C, float2>::value) {
        if (tensor_cores_enabled() && 2 * ku >= tc_min_width()) {
            const fame_status s = gram_tc(c, concat(U, V), U, ld, 2, G, st);
            if (s != FAME_E_ARG) return s;
        }
    }
    const int T = (ku + GT - 1) / GT, tiles = T * (T + 1);
    const int groups = (tiles + kGramThreads - 1) / kGramThreads;
    int threads = (((tiles + groups - 1) / groups + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    const bool dbl = sizeof(C) == 16;
    const size_t smem = (size_t)4 * GROWS * herm_stride(ku) * sizeof(C) + (size_t)2 * ku * sizeof(void*);
    int nblk = 152 * 4;
    size_t rpb = (ld + nblk - 1) / nblk;
    rpb = ((rpb + GROWS - 1) / GROWS) * GROWS;
    nblk = (int)((ld + rpb - 1) / rpb);
    const int kk = ku * 2 * ku;
    fame_status s = grow(c, c->partial, (size_t)nblk * kk * sizeof(double2));
    if (s != FAME_OK) return s;
    if ((s = kernel_smem(c, (const void*)k_gram_herm<C>, smem)) != FAME_OK) return s;
    double2* part = reinterpret_cast<double2*>(c->partial.p);
    {
        // algorithmic work: the ku (ku + 1) entries on or below the two diagonals
        ProfScope ps(K_GRAM_HERM, dbl, st, (double)ld * 2 * ku * sizeof(C), 8.0 * ku * (ku + 1) * (double)ld);
        k_gram_herm<C><<<dim3(nblk, groups), threads, smem, st>>>(U, V, ld, rpb, part);
    }
    {
        ProfScope ps(K_GRAM_RED, dbl, st, (double)nblk * kk * sizeof(double2), 2.0 * nblk * kk);
        k_gram_reduce<<<(kk + 7) / 8, 256, 0, st>>>(part, nblk, kk, G, ku);
    }
    count_launch(2);
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

// The Hermitian pair of Grams of complex128 blocks in double-float arithmetic on
// the FP32 units (k_gram_herm_df): about 2^-47 relative per product against the
// 2^-53 of native FP64, so only for blocks whose Gram is well conditioned -- the
// Ritz confirmation of near-eigenvectors X, where AX ~ X Theta -- and never for the
// LOBPCG blocks [X W P], whose W^H A W entries carry ||A|| / lambda amplification.
// Native FP64 (k_gram_herm<double2>) where the double-float stages do not fit in
// shared memory or FAME_FP64_NATIVE is set.
fame_status gram_herm_df(fame_ctx* c, const BlockList<double2>& U, const BlockList<double2>& V, size_t ld,
                         double2* G, cudaStream_t st) {
    using C = double2;
    const int ku = U.total;
    if (V.total != ku) return set_err(c, FAME_E_ARG, "gram_herm_df: U and V differ in width");
    if (!fp64_native()) {
        const int T = (ku + GT2 - 1) / GT2, tiles = T * (T + 1);
        const int groups = (tiles + kGramThreads - 1) / kGramThreads;
        int threads = (((tiles + groups - 1) / groups + 31) / 32) * 32;
        if (threads < 64) threads = 64;
        const int SP = herm_stride(ku);
        const size_t smem = (size_t)4 * GROWS * SP * sizeof(double2) + (size_t)2 * GROWS * SP * sizeof(float4) +
                            (size_t)2 * ku * sizeof(void*);
        if (smem <= 200u * 1024u) {
            int nblk = 152 * 4;
            size_t rpb = (ld + nblk - 1) / nblk;
            rpb = ((rpb + GROWS - 1) / GROWS) * GROWS;
            nblk = (int)((ld + rpb - 1) / rpb);
            const int kk = ku * 2 * ku;
            fame_status s = grow(c, c->partial, (size_t)nblk * kk * sizeof(double2));
            if (s != FAME_OK) return s;
            if ((s = kernel_smem(c, (const void*)k_gram_herm_df, smem)) != FAME_OK) return s;
            double2* part = reinterpret_cast<double2*>(c->partial.p);
            {
                ProfScope ps(K_GRAM_HERM, true, st, (double)ld * 2 * ku * sizeof(C), 8.0 * ku * (ku + 1) * (double)ld);
                k_gram_herm_df<<<dim3(nblk, groups), threads, smem, st>>>(U, V, ld, rpb, part);
            }
            {
                ProfScope ps(K_GRAM_RED, true, st, (double)nblk * kk * sizeof(double2), 2.0 * nblk * kk);
                k_gram_reduce<<<(kk + 7) / 8, 256, 0, st>>>(part, nblk, kk, G, ku);
            }
            count_launch(2);
            FAME_CUDA_TRY(c, cudaGetLastError());
            return FAME_OK;
        }
    }
    return gram_herm<double2>(c, U, V, ld, G, st);
}

template <typename C, typename Co>
fame_status combine(fame_ctx* c, const BlockList<C>& S, size_t ld, const double2* M, int m, int i0,
                    Co* out1, Co* out2, cudaStream_t st) {
    if constexpr (std::is_same<C, float2>::value) {
        if (combine_st_ok(S, ld, m)) {
            const int groups = (m + kStOut - 1) / kStOut, threads = groups * kStRows;
            const size_t smem = combine_st_smem(S.total, groups);
            const void* fn = groups == 1 ? (const void*)k_combine_st<Co, 1> : (const void*)k_combine_st<Co, 2>;
            fame_status s = kernel_smem(c, fn, smem);
            if (s != FAME_OK) return s;
            int per_sm = 0;
            FAME_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
            const size_t ntiles = (ld + kStRows - 1) / kStRows;
            const unsigned nblk = (unsigned)std::max<size_t>(1, std::min<size_t>((size_t)152 * std::max(per_sm, 1), ntiles));
            const double outs = (out1 ? m : 0) + (out2 ? m : 0);
            ProfScope ps(K_COMBINE, false, st, (double)S.total * ld * sizeof(C) + outs * ld * sizeof(Co),
                         8.0 * S.total * m * (double)ld);
            if (groups == 1)
                k_combine_st<Co, 1><<<nblk, threads, smem, st>>>(S, ld, M, m, i0, out1, out2);
            else
                k_combine_st<Co, 2><<<nblk, threads, smem, st>>>(S, ld, M, m, i0, out1, out2);
            count_launch();
            FAME_CUDA_TRY(c, cudaGetLastError());
            return FAME_OK;
        }
    }
    const int MP = ((m + CJ - 1) / CJ) * CJ;
    const size_t smem = (size_t)S.total * MP * sizeof(C) + (size_t)S.total * sizeof(void*);
    fame_status s = kernel_smem(c, (const void*)k_combine<C, Co>, smem);
    if (s != FAME_OK) return s;
    {
        const double outs = (out1 ? m : 0) + (out2 ? m : 0);
        ProfScope ps(K_COMBINE, sizeof(C) == sizeof(double2), st,
                     (double)S.total * ld * sizeof(C) + outs * ld * sizeof(Co), 8.0 * S.total * m * (double)ld);
        const size_t span = (size_t)(kCombineThreads / kCombineSlots) * CR;
        const unsigned nblk = (unsigned)std::min<size_t>(152 * 4, (ld + span - 1) / span);
        k_combine<C, Co><<<nblk, kCombineThreads, smem, st>>>(S, ld, M, m, i0, out1, out2);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

fame_status combine_refine(fame_ctx* c, const double2* X64, const float2* X32, int m, const BlockList<float2>& Q,
                           size_t ld, const double2* M, const int* blk, double2* Xn, float2* X32n, float2* Pn,
                           cudaStream_t st) {
    const BlockList<float2> S = concat(blocks<float2>(X32, m), Q);
    if (!combine_st_ok(S, ld, m) || m < 1)
        return set_err(c, FAME_E_ARG, "combine_refine: block layout not supported");
    const int groups = (m + kStOut - 1) / kStOut, threads = groups * kStRows;
    const size_t smem = combine_st_smem(S.total, groups, true);
    const void* fn = groups == 1 ? (const void*)k_combine_st<float2, 1, true> : (const void*)k_combine_st<float2, 2, true>;
    fame_status s = kernel_smem(c, fn, smem);
    if (s != FAME_OK) return s;
    int per_sm = 0;
    FAME_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    const size_t ntiles = (ld + kStRows - 1) / kStRows;
    const unsigned nblk = (unsigned)std::max<size_t>(1, std::min<size_t>((size_t)152 * std::max(per_sm, 1), ntiles));
    RefineEpi rf;
    rf.X64 = X64;
    rf.mx = m;
    rf.blk = blk;
    rf.Xn64 = Xn;
    rf.X32n = X32n;
    {
        // algorithmic bytes: X64 and [X32 Q] read, Xn64, X32n, Pn written; 8 flops per complex MAC
        const int nq = Q.total;
        ProfScope ps(K_COMBINE_DF, true, st,
                     (double)ld * (m * sizeof(double2) + (m + nq) * sizeof(float2) + m * sizeof(double2) +
                                   (X32n ? m * sizeof(float2) : 0) + (Pn ? m * sizeof(float2) : 0)),
                     8.0 * (double)ld * m * (m + nq));
        if (groups == 1)
            k_combine_st<float2, 1, true><<<nblk, threads, smem, st>>>(S, ld, M, m, m, nullptr, Pn, rf);
        else
            k_combine_st<float2, 2, true><<<nblk, threads, smem, st>>>(S, ld, M, m, m, nullptr, Pn, rf);
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
    const int nq = Q.total;   // may be 0: Xn = X M only
    const int MP = ((m + MJ - 1) / MJ) * MJ;
    const size_t smem = (size_t)m * MP * sizeof(float4) + (size_t)nq * MP * sizeof(float2) + (size_t)nq * sizeof(void*);
    fame_status s = kernel_smem(c, (const void*)k_combine_mixed, smem);
    if (s != FAME_OK) return s;
    {
        // algorithmic work: 8 flops per complex multiply-add, for the X and the Q part
        // alike (the double-float arithmetic of the X part spends about 60 FP32
        // operations per complex coefficient, which is how it is computed, not how much)
        ProfScope ps(K_COMBINE_DF, true, st,
                     (double)ld * (m * sizeof(double2) + nq * sizeof(float2) +
                                   m * (sizeof(double2) + (X32n ? sizeof(float2) : 0) + (Pn ? sizeof(float2) : 0))),
                     (double)ld * m * (8.0 * m + 8.0 * nq));
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
    if constexpr (std::is_same<CX, float2>::value && std::is_same<CQ, float2>::value) {
        if (m <= 2 * kStOut && nq <= 4 * kStOut && combine_st_ok(Q, ld, 1) &&
            !(reinterpret_cast<uintptr_t>(X) & 15)) {
            const int groups = (nq + kStOut - 1) / kStOut, threads = groups * kStRows;
            const size_t smem = orth_st_smem(m, groups);
            const void* fn = groups == 1   ? (const void*)k_orth_st<1>
                             : groups == 2 ? (const void*)k_orth_st<2>
                             : groups == 3 ? (const void*)k_orth_st<3>
                                           : (const void*)k_orth_st<4>;
            fame_status s = kernel_smem(c, fn, smem);
            if (s != FAME_OK) return s;
            int per_sm = 0;
            FAME_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
            const size_t ntiles = (ld + kStRows - 1) / kStRows;
            const unsigned nblk =
                (unsigned)std::max<size_t>(1, std::min<size_t>((size_t)152 * std::max(per_sm, 1), ntiles));
            ProfScope ps(K_ORTH, false, st, (double)ld * (m * sizeof(CX) + 2 * nq * sizeof(CQ)),
                         8.0 * (double)ld * m * nq);
            switch (groups) {
                case 1: k_orth_st<1><<<nblk, threads, smem, st>>>(X, m, Q, ld, cfs); break;
                case 2: k_orth_st<2><<<nblk, threads, smem, st>>>(X, m, Q, ld, cfs); break;
                case 3: k_orth_st<3><<<nblk, threads, smem, st>>>(X, m, Q, ld, cfs); break;
                default: k_orth_st<4><<<nblk, threads, smem, st>>>(X, m, Q, ld, cfs); break;
            }
            count_launch();
            FAME_CUDA_TRY(c, cudaGetLastError());
            return FAME_OK;
        }
    }
    const int MP = ((nq + CJ - 1) / CJ) * CJ;
    const size_t smem = (size_t)m * MP * sizeof(CX) + (size_t)nq * sizeof(void*);
    fame_status s = kernel_smem(c, (const void*)k_orth<CX, CQ>, smem);
    if (s != FAME_OK) return s;
    {
        ProfScope ps(K_ORTH, sizeof(CX) == 16, st, (double)ld * (m * sizeof(CX) + 2 * nq * sizeof(CQ)),
                     8.0 * (double)ld * m * nq);
        const size_t span = (size_t)(kCombineThreads / kCombineSlots) * CR;
        const unsigned nblk = (unsigned)std::min<size_t>(152 * 4, (ld + span - 1) / span);
        k_orth<CX, CQ><<<nblk, kCombineThreads, smem, st>>>(X, m, Q, ld, cfs);
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

template fame_status gram_herm<float2>(fame_ctx*, const BlockList<float2>&, const BlockList<float2>&, size_t, double2*, cudaStream_t);
template fame_status gram_herm<double2>(fame_ctx*, const BlockList<double2>&, const BlockList<double2>&, size_t, double2*, cudaStream_t);
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
