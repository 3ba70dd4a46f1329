// Block operations used by the eigensolver (definitions in blockops.cu).
#pragma once
#include "fame_internal.h"

// Up to three column blocks of vectors (each column = 2n complex, leading dim ld).
template <typename C>
struct BlockList {
    static constexpr int kMax = 6;
    const C* ptr[kMax];
    int cols[kMax];
    int total;
};

template <typename C>
inline BlockList<C> blocks(const C* a, int na, const C* b = nullptr, int nb = 0,
                           const C* c = nullptr, int nc = 0) {
    BlockList<C> L;
    for (int i = 0; i < BlockList<C>::kMax; ++i) { L.ptr[i] = nullptr; L.cols[i] = 0; }
    L.ptr[0] = a; L.cols[0] = na;
    L.ptr[1] = b; L.cols[1] = nb;
    L.ptr[2] = c; L.cols[2] = nc;
    L.total = na + nb + nc;
    return L;
}

// concatenation of two block lists (at most kMax blocks in total)
template <typename C>
inline BlockList<C> concat(const BlockList<C>& a, const BlockList<C>& b) {
    BlockList<C> L = a;
    int k = 0;
    while (k < BlockList<C>::kMax && L.cols[k] > 0) ++k;
    for (int i = 0; i < BlockList<C>::kMax && b.cols[i] > 0 && k < BlockList<C>::kMax; ++i, ++k) {
        L.ptr[k] = b.ptr[i];
        L.cols[k] = b.cols[i];
    }
    L.total = a.total + b.total;
    return L;
}

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

// G (column-major ku x kv, double2, device) = U^H V; FP64 products when either side is
// complex128, else FP32 products summed in FP32 over row blocks of about a thousand
// rows and in FP64 across the blocks
template <typename CU, typename CV>
fame_status gram(fame_ctx* c, const BlockList<CU>& U, const BlockList<CV>& V, size_t ld, double2* G,
                 cudaStream_t st);
// Tensor-core Gram (tc_gram.cu): P = A^H B for complex64 blocks with at most 128 columns
// on each side, written to G as P (mode 0, MA x NB), P^H (mode 1, NB x MA) or, for
// A = [U | V] and B = U with k = NB, [P[:k] | P[k:]^H] (mode 2, k x 2k).  FAME_E_ARG
// (nothing launched) when the shapes, the alignment or the driver do not allow it.
fame_status gram_tc(fame_ctx* c, const BlockList<float2>& A, const BlockList<float2>& B, size_t ld, int mode,
                    double2* G, cudaStream_t st);
// false when the environment sets FAME_NO_TC=1 (the FP32 CUDA-core kernels are used)
bool tensor_cores_enabled();
// G (column-major k x 2k) = [U^H U | U^H V] for V = A U with A Hermitian: only the
// entries on or below the diagonal of each k x k block are computed (the others are 0)
template <typename C>
fame_status gram_herm(fame_ctx* c, const BlockList<C>& U, const BlockList<C>& V, size_t ld, double2* G,
                      cudaStream_t st);
// The same for complex128 blocks in double-float arithmetic on the FP32 units (about
// 2^-47 relative per product): for well-conditioned Grams only, i.e. near-eigenvectors
// U with V = A U ~ U Theta
fame_status gram_herm_df(fame_ctx* c, const BlockList<double2>& U, const BlockList<double2>& V, size_t ld,
                         double2* G, cudaStream_t st);
// out1 = S M[:, :m], out2 = S[:, i0:] M[i0:, :m]  (either output may be null)
template <typename C, typename Co>
fame_status combine(fame_ctx* c, const BlockList<C>& S, size_t ld, const double2* M, int m, int i0,
                    Co* out1, Co* out2, cudaStream_t st);
// W = tinv .* (AX - X theta) (W may be null), part[j][blk] = partial ||R_j||^2
template <typename C>
fame_status residual(fame_ctx* c, const C* X, const C* AX, const double* theta_dev,
                     const typename RealOf<C>::T* tinv, int m, C* W, double* part, int nblk,
                     cudaStream_t st);
// refinement: R = AX - X theta from complex128 X, AX (FP64), W = tinv .* R as complex64,
// R32 = R as complex64 (may be null)
fame_status residual_mixed(fame_ctx* c, const double2* X, const double2* AX, const double* theta_dev,
                           int m, float2* W, float2* R32, double* part, int nblk, cudaStream_t st);
// refinement update: Xn = X M[:m] (FP64 accuracy, double-float sums) + Q M[m:] (FP32),
// X32n = complex64 copy of Xn (may be null), Pn = Q M[m:] (may be null); Q may be empty
fame_status combine_mixed(fame_ctx* c, const double2* X, int m, const BlockList<float2>& Q, size_t ld,
                          const double2* M, double2* Xn, float2* X32n, float2* Pn, cudaStream_t st);
// The same update with the FP64-accurate part confined to blocks of outputs: for output j
// the entries M[i][j] with i in j's block (blk: device int [m][kRefineBlock + 1] = count,
// then the columns i) multiply the complex128 X64 in double-float arithmetic; every other
// entry multiplies X32 (the complex64 copy of X64) or Q in FP32.  Exact to the FP32
// rounding of the off-block terms, so the blocks must hold every entry of M[:m] that is
// not small.  Xn (complex128), X32n (complex64 copy, may be null), Pn = Q M[m:] (may be null).
constexpr int kRefineBlock = 6;
fame_status combine_refine(fame_ctx* c, const double2* X64, const float2* X32, int m, const BlockList<float2>& Q,
                           size_t ld, const double2* M, const int* blk, double2* Xn, float2* X32n, float2* Pn,
                           cudaStream_t st);
// Q <- Q - X cfs (cfs m x nq), in place; FP64 arithmetic when X is complex128
template <typename CX, typename CQ>
fame_status orth_against(fame_ctx* c, const CX* X, int m, const BlockList<CQ>& Q, size_t ld,
                         const double2* cfs, cudaStream_t st);
template <typename Ci, typename Co>
fame_status convert(fame_ctx* c, const Ci* in, Co* out, size_t N, cudaStream_t st);
template <typename C>
fame_status random_block(fame_ctx* c, C* X, int m, uint64_t seed,
                         const typename RealOf<C>::T* tinv, cudaStream_t st);
template <typename C>
fame_status mask_block(fame_ctx* c, C* X, int m, const typename RealOf<C>::T* tinv,
                       cudaStream_t st);
