// Preconditioner of the block eigensolver: an inexact A_r^{-1} built from the
// factorisation A_r = Sigma_r M Sigma_r, M = Q_r^* B^{-1} Q_r (eq. NFSEP).
//
// The paper solves with M by an unpreconditioned inner CG (Section 5.2: M is
// Hermitian positive definite with spectrum inside [min 1/B, max 1/B], since Q_r
// has orthonormal columns, so kappa(M) <= max B / min B).  Here M^{-1} is replaced
// by the degree-K Chebyshev polynomial for that interval (the Chebyshev
// semi-iteration, e.g. Saad, Iterative Methods for Sparse Linear Systems, Section
// 12.1): a fixed linear, Hermitian positive definite operator -- as LOBPCG wants of
// a preconditioner -- that needs no inner products, only K - 1 applies of M per
// block.  With S = Sigma_r^{-1} (0 on the zero frequencies of the Gamma point),
//   T R = S P_K(M) S R,   M v = S A_r (S v),
// so each application of M is one fused A_r apply with diagonal scalings around it.
// The previous preconditioner Sigma_r^{-2} / mean(1/B) is the degree-1 member of the
// family (up to a scale).  Arithmetic is complex64: T only has to be a good, fixed
// approximation of A_r^{-1}.
#include <cmath>
#include <cstdlib>
#include <type_traits>

#include "blockops.h"

namespace {

// S = sqrt(tinv mean(1/B)) at frequency f, from the diagonal preconditioner table
// tinv = 1 / (Lambda_q mean(1/B)) (0 where Lambda_q = 0)
__device__ __forceinline__ float sinv_of(const float* __restrict__ tinv, size_t f, float mean) {
    const float t = tinv[f];
    return t > 0.f ? sqrtf(t * mean) : 0.f;
}

// Start: b = S R = W mean / S (W = tinv .* R on entry), d0 = b / theta;
// r = b, x = d0, v = S d0.
__global__ void k_cheb_init(const float2* __restrict__ W, const float* __restrict__ tinv, size_t n, size_t total,
                            float mean, float inv_theta, float2* __restrict__ r, float2* __restrict__ x,
                            float2* __restrict__ v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float s = sinv_of(tinv, i % n, mean);
        const float2 w = W[i];
        const float g = s > 0.f ? mean / s : 0.f;
        const float2 b = make_float2(w.x * g, w.y * g);
        const float2 d = make_float2(b.x * inv_theta, b.y * inv_theta);
        r[i] = b;
        x[i] = d;
        v[i] = make_float2(s * d.x, s * d.y);
    }
}

// One step after Av = A_r v (v = S d_k):
//   r <- r - S Av;  d_{k+1} = c1 d_k + c2 r (d_k = v / S);  x <- x + d_{k+1};
//   v <- S d_{k+1}, or on the last step out = S x.
__global__ void k_cheb_step(const float2* __restrict__ Av, const float* __restrict__ tinv, size_t n, size_t total,
                            float mean, float c1, float c2, float2* __restrict__ r, float2* __restrict__ x,
                            float2* __restrict__ v, float2* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float s = sinv_of(tinv, i % n, mean);
        if (!(s > 0.f)) {
            if (out) out[i] = make_float2(0.f, 0.f);
            else v[i] = make_float2(0.f, 0.f);
            continue;
        }
        const float2 a = Av[i];
        float2 rr = r[i];
        rr.x -= s * a.x;
        rr.y -= s * a.y;
        const float2 vo = v[i];
        const float is = 1.f / s;
        const float2 d = make_float2(c1 * vo.x * is + c2 * rr.x, c1 * vo.y * is + c2 * rr.y);
        float2 xx = x[i];
        xx.x += d.x;
        xx.y += d.y;
        if (out) {
            out[i] = make_float2(s * xx.x, s * xx.y);
        } else {
            r[i] = rr;
            x[i] = xx;
            v[i] = make_float2(s * d.x, s * d.y);
        }
    }
}

template <typename Ci, typename Co>
__global__ void k_cheb_convert(const Ci* __restrict__ in, Co* __restrict__ out, size_t N) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
        out[i] = mk((decltype(Co().x))in[i].x, (decltype(Co().x))in[i].y);
}

constexpr int kGrid = 152 * 8, kBlock = 256;

}  // namespace

// Degree of the Chebyshev polynomial (environment FAME_CHEB_DEGREE, default 3: two
// applies of M per preconditioned block; 1 gives the diagonal preconditioner).
int cheb_degree() {
    const char* v = std::getenv("FAME_CHEB_DEGREE");
    const int k = v ? std::atoi(v) : 3;
    return k < 1 ? 1 : (k > 16 ? 16 : k);
}

template <typename C>
fame_status precond_cheb(fame_ctx* c, C* W, int ncols, cudaStream_t st) {
    const int K = cheb_degree();
    const double a = c->min_invB, b = c->max_invB;
    // K = 1, or a (numerically) homogeneous medium, where M is a multiple of I and the
    // diagonal preconditioner already in W is exact
    if (K <= 1 || ncols < 1 || !(b - a > 1e-6 * b)) return FAME_OK;
    const size_t n = (size_t)c->n, ld = 2 * n, total = (size_t)ncols * ld;
    const bool dbl = std::is_same<C, double2>::value;
    fame_status s = grow(c, c->cheb, (dbl ? 4 : 3) * total * sizeof(float2));
    if (s != FAME_OK) return s;
    float2* r = static_cast<float2*>(c->cheb.p);
    float2* v = r + total;
    float2* Av = v + total;
    float2* x = dbl ? Av + total : reinterpret_cast<float2*>(W);
    const float* tinv = c->tf.tinv;
    const float mean = (float)c->mean_invB;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma1 = theta / delta;
    const float2* Win = reinterpret_cast<const float2*>(W);
    if (dbl) {
        k_cheb_convert<double2, float2><<<kGrid, kBlock, 0, st>>>(reinterpret_cast<const double2*>(W), x, total);
        count_launch();
        Win = x;
    }
    {
        ProfScope ps(K_PRECOND, false, st, (double)total * 4 * sizeof(float2), 6.0 * total);
        k_cheb_init<<<kGrid, kBlock, 0, st>>>(Win, tinv, n, total, mean, (float)(1.0 / theta), r, x, v);
    }
    count_launch();
    double rho = 1.0 / sigma1;
    for (int k = 0; k + 1 < K; ++k) {
        c->stats.applies_c64 += ncols;
        if ((s = run_apply<float>(c, v, Av, ncols, st)) != FAME_OK) return s;
        const double rho1 = 1.0 / (2.0 * sigma1 - rho);
        const float c1 = (float)(rho1 * rho), c2 = (float)(2.0 * rho1 / delta);
        rho = rho1;
        const bool last = k + 2 == K;
        float2* out = last ? (dbl ? v : reinterpret_cast<float2*>(W)) : nullptr;
        // the last step writes S x over W (complex64) or into v, converted below (complex128)
        {
            ProfScope ps(K_PRECOND, false, st, (double)total * (last ? 5 : 8) * sizeof(float2), 12.0 * total);
            k_cheb_step<<<kGrid, kBlock, 0, st>>>(Av, tinv, n, total, mean, c1, c2, r, x, v, out);
        }
        count_launch();
    }
    if (dbl) {
        k_cheb_convert<float2, double2><<<kGrid, kBlock, 0, st>>>(v, reinterpret_cast<double2*>(W), total);
        count_launch();
    }
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template fame_status precond_cheb<float2>(fame_ctx*, float2*, int, cudaStream_t);
template fame_status precond_cheb<double2>(fame_ctx*, double2*, int, cudaStream_t);
