// The paper's eigensolver (Section 5.2, with the settings of Section 6): Lanczos on
// A_r^{-1}, whose largest eigenvalues 1/lambda belong to the smallest eigenvalues
// lambda of A_r, with every product A_r^{-1} q formed by an inner conjugate-gradient
// solve.  Since A_r = Sigma_r M Sigma_r with M = Q_r^* B^{-1} Q_r Hermitian positive
// definite and kappa(M) <= max B / min B,
//   A_r^{-1} q = S M^{-1} (S q),  S = Sigma_r^{-1},
// and M is solved by plain CG, as in the paper (no preconditioner: the condition
// number is that of B).  Everything is complex128; M v = S A_r (S v) is one fused
// complex128 A_r apply between two diagonal scalings.  The zero frequencies of the
// Gamma point (Sigma_r = 0) carry the two zero eigenvalues of A_r and are kept out
// of every vector (S = 0 there).
//
// Lanczos keeps all its vectors and reorthogonalises each new one against them
// twice (classical Gram-Schmidt on the block Gram kernels), so no spurious copies
// of converged values appear; the Ritz values come from the tridiagonal matrix on
// the host.  Convergence: the Ritz estimate beta_j |s_ji| <= tol theta_i for the nev
// largest Ritz values theta_i of A_r^{-1} (the paper's outer tolerance is 1e-12; the
// inner CG stops at min(tol, 1e-13) relative residual).  The explicit residuals
// ||A_r y - lambda y|| / lambda of the returned pairs are measured afterwards with a
// complex128 apply and reported in the solve statistics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "blockops.h"

namespace {

constexpr int kRedBlocks = 512, kThr = 256, kResid = 256;

__device__ __forceinline__ double sinv64(const double* __restrict__ tinv, size_t f, double mean) {
    const double t = tinv[f];
    return t > 0.0 ? sqrt(t * mean) : 0.0;
}

// per-block partial sums in a fixed order (deterministic)
__device__ __forceinline__ void block_sum(double v, double* __restrict__ part) {
    __shared__ double red[kThr / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kThr / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// scal[slot] = sum of the kRedBlocks partials (one warp, fixed order)
__global__ void k_reduce(const double* __restrict__ part, double* __restrict__ scal, int slot) {
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += 32) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) scal[slot] = s;
}

// CG start for M x = b with b = S q:  x = 0, r = p = b, v = S p, partial |r|^2
__global__ void k_cg_start(const double2* __restrict__ q, const double* __restrict__ tinv, double mean, size_t n,
                           size_t N, double2* __restrict__ x, double2* __restrict__ r, double2* __restrict__ p,
                           double2* __restrict__ v, double* __restrict__ part) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double s = sinv64(tinv, i % n, mean);
        const double2 b = make_double2(s * q[i].x, s * q[i].y);
        x[i] = make_double2(0.0, 0.0);
        r[i] = b;
        p[i] = b;
        v[i] = make_double2(s * b.x, s * b.y);
        acc += b.x * b.x + b.y * b.y;
    }
    block_sum(acc, part);
}

// w = S (A_r v) = M p, partial p^H w (real: M is Hermitian)
__global__ void k_cg_mp(const double2* __restrict__ Av, const double* __restrict__ tinv, double mean, size_t n,
                        size_t N, const double2* __restrict__ p, double2* __restrict__ w, double* __restrict__ part) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double s = sinv64(tinv, i % n, mean);
        const double2 a = make_double2(s * Av[i].x, s * Av[i].y);
        w[i] = a;
        acc += p[i].x * a.x + p[i].y * a.y;
    }
    block_sum(acc, part);
}

// alpha = rr / pw:  x += alpha p, r -= alpha w, partial |r|^2
__global__ void k_cg_xr(const double* __restrict__ scal, int rr_slot, size_t N, const double2* __restrict__ p,
                        const double2* __restrict__ w, double2* __restrict__ x, double2* __restrict__ r,
                        double* __restrict__ part) {
    const double alpha = scal[rr_slot] / scal[0];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        x[i] = make_double2(x[i].x + alpha * p[i].x, x[i].y + alpha * p[i].y);
        const double2 rn = make_double2(r[i].x - alpha * w[i].x, r[i].y - alpha * w[i].y);
        r[i] = rn;
        acc += rn.x * rn.x + rn.y * rn.y;
    }
    block_sum(acc, part);
}

// beta = rr_new / rr:  p = r + beta p, v = S p
__global__ void k_cg_p(const double* __restrict__ scal, int rr_slot, int rr_new_slot, const double* __restrict__ tinv,
                       double mean, size_t n, size_t N, const double2* __restrict__ r, double2* __restrict__ p,
                       double2* __restrict__ v) {
    const double beta = scal[rr_new_slot] / scal[rr_slot];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double s = sinv64(tinv, i % n, mean);
        const double2 pn = make_double2(r[i].x + beta * p[i].x, r[i].y + beta * p[i].y);
        p[i] = pn;
        v[i] = make_double2(s * pn.x, s * pn.y);
    }
}

// out = f * S x  (f: a host scale)
__global__ void k_scale_s(const double2* __restrict__ x, const double* __restrict__ tinv, double mean, size_t n,
                          size_t N, double f, double2* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double s = f * sinv64(tinv, i % n, mean);
        out[i] = make_double2(s * x[i].x, s * x[i].y);
    }
}

// random start vector (counter-based hash), zero on the masked frequencies
__global__ void k_lanczos_start(double2* __restrict__ q, const double* __restrict__ tinv, size_t n, size_t N,
                                unsigned long long seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double a = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        const double b = (double)((z * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        q[i] = tinv[i % n] > 0.0 ? make_double2(a, b) : make_double2(0.0, 0.0);
    }
}

}  // namespace

// A_r^{-1} q by CG on M (see the file comment); z may not alias q.
static fame_status inv_apply(fame_ctx* c, const double2* q, double2* z, double2* buf, double* part, double* scal,
                             double* hscal, double cg_tol, int max_cg, int* iters, cudaStream_t st) {
    const size_t n = (size_t)c->n, N = 2 * n;
    const double* tinv = c->td.tinv;
    const double mean = c->mean_invB;
    double2 *x = buf, *r = buf + N, *p = buf + 2 * N, *v = buf + 3 * N, *Av = buf + 4 * N, *w = buf + 5 * N;
    fame_status s;
    k_cg_start<<<kRedBlocks, kThr, 0, st>>>(q, tinv, mean, n, N, x, r, p, v, part);
    k_reduce<<<1, 32, 0, st>>>(part, scal, 2);
    count_launch(2);
    FAME_CUDA_TRY(c, cudaMemcpyAsync(hscal, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    const double rr0 = hscal[0];
    int it = 0;
    if (rr0 > 0.0) {
        for (it = 0; it < max_cg; ++it) {
            const int cur = 2 + (it & 1), nxt = 2 + ((it + 1) & 1);
            c->stats.applies_c128 += 1;
            if ((s = run_apply<double>(c, v, Av, 1, st)) != FAME_OK) return s;
            k_cg_mp<<<kRedBlocks, kThr, 0, st>>>(Av, tinv, mean, n, N, p, w, part);
            k_reduce<<<1, 32, 0, st>>>(part, scal, 0);
            k_cg_xr<<<kRedBlocks, kThr, 0, st>>>(scal, cur, N, p, w, x, r, part);
            k_reduce<<<1, 32, 0, st>>>(part, scal, nxt);
            k_cg_p<<<kRedBlocks, kThr, 0, st>>>(scal, cur, nxt, tinv, mean, n, N, r, p, v);
            count_launch(5);
            if ((it & 7) == 7 || it + 1 == max_cg) {
                FAME_CUDA_TRY(c, cudaMemcpyAsync(hscal, scal + nxt, sizeof(double), cudaMemcpyDeviceToHost, st));
                FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
                if (!(hscal[0] > cg_tol * cg_tol * rr0)) {
                    ++it;
                    break;
                }
            }
        }
    }
    k_scale_s<<<kRedBlocks, kThr, 0, st>>>(x, tinv, mean, n, N, 1.0, z);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    *iters += it;
    return FAME_OK;
}

fame_status run_inv_lanczos(fame_ctx* c, int nev, double tol, int max_iter, double* lambda_out, void* Y_out,
                            int* iters_out, cudaStream_t st) {
    const size_t n = (size_t)c->n, N = 2 * n;
    // at most 160 Lanczos vectors: the reorthogonalisation Gram of the whole basis then
    // still fits the FP64 Gram kernel's shared-memory stages
    const int jmax = std::max(nev + 2, std::min(max_iter, 160));
    const double cg_tol = std::min(tol, 1e-13);
    c->stats = fame_solve_stats{};
    c->stats_rr_ms = 0.0;
    fame_status s;
    // device: Lanczos basis [jmax + 1][N], CG vectors [6][N], Ritz block and its image
    // [2 nev][N], partial sums, scalars, small coefficient matrices
    const size_t bytes = ((size_t)(jmax + 1) * N + 6 * N + 2 * (size_t)nev * N) * sizeof(double2) +
                         (kRedBlocks + (size_t)nev * kResid) * sizeof(double) + 128 * sizeof(double) +
                         2 * (size_t)(jmax + 1) * std::max(nev, 2) * sizeof(double2) + 4096;
    if ((s = grow(c, c->solver2, bytes)) != FAME_OK) return s;
    char* base = static_cast<char*>(c->solver2.p);
    double2* Q = reinterpret_cast<double2*>(base);
    double2* buf = Q + (size_t)(jmax + 1) * N;
    double2* Y = buf + 6 * N;
    double2* AY = Y + (size_t)nev * N;
    double* part = reinterpret_cast<double*>(AY + (size_t)nev * N);
    double* rpart = part + kRedBlocks;                             // [nev][kResid] residual partials
    double* scal = rpart + (size_t)nev * kResid;                   // CG scalars; [8, 8 + nev): lambda
    double2* G = reinterpret_cast<double2*>(scal + 128);           // [jmax + 1] x max(nev, 2)
    if ((s = grow_pinned(c, c->pinned, 2 * (size_t)(jmax + 1) * std::max(nev, 2) * sizeof(double2) + 4096)) != FAME_OK)
        return s;
    double2* hG = static_cast<double2*>(c->pinned.p);
    double* hscal = reinterpret_cast<double*>(hG + (size_t)(jmax + 1) * std::max(nev, 2));
    const size_t ld = N;
    // q_1: random, masked, unit
    k_lanczos_start<<<kRedBlocks, kThr, 0, st>>>(Q, c->td.tinv, n, N, 0x1A5C205ull ^ (unsigned long long)c->n);
    count_launch();
    auto norm_of = [&](const double2* v, double* out) -> fame_status {
        fame_status e = gram<double2, double2>(c, blocks<double2>(v, 1), blocks<double2>(v, 1), ld, G, st);
        if (e != FAME_OK) return e;
        FAME_CUDA_TRY(c, cudaMemcpyAsync(hG, G, sizeof(double2), cudaMemcpyDeviceToHost, st));
        FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
        *out = std::sqrt(std::max(hG[0].x, 0.0));
        return FAME_OK;
    };
    double nrm = 0.0;
    if ((s = norm_of(Q, &nrm)) != FAME_OK) return s;
    if (!(nrm > 0.0)) return set_err(c, FAME_E_STATE, "inverse Lanczos: start vector vanished");
    {
        // q_1 /= ||q_1||, as a one-column combination
        hG[0] = make_double2(1.0 / nrm, 0.0);
        FAME_CUDA_TRY(c, cudaMemcpyAsync(G, hG, sizeof(double2), cudaMemcpyHostToDevice, st));
        if ((s = combine<double2, double2>(c, blocks<double2>(Q, 1), ld, G, 1, 1, buf, nullptr, st)) != FAME_OK) return s;
        FAME_CUDA_TRY(c, cudaMemcpyAsync(Q, buf, N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    std::vector<double> alpha, beta;
    std::vector<double> theta;
    std::vector<double2> V;
    int cg_iters = 0, j = 0;
    bool converged = false;
    double2* zt = Y;                 // A_r^{-1} q_j lands here (Y is free until the end)
    for (j = 0; j < jmax; ++j) {
        double2* qj = Q + (size_t)j * N;
        if ((s = inv_apply(c, qj, zt, buf, part, scal, hscal, cg_tol, 4000, &cg_iters, st)) != FAME_OK) return s;
        // two passes of classical Gram-Schmidt against q_1..q_j; alpha_j = q_j^H z from the first
        double a_j = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            const BlockList<double2> Qb = blocks<double2>(Q, j + 1);
            if ((s = gram<double2, double2>(c, Qb, blocks<double2>(zt, 1), ld, G, st)) != FAME_OK) return s;
            if (pass == 0) {
                FAME_CUDA_TRY(c, cudaMemcpyAsync(hG, G + j, sizeof(double2), cudaMemcpyDeviceToHost, st));
            }
            if ((s = orth_against<double2, double2>(c, Q, j + 1, blocks<double2>(zt, 1), ld, G, st)) != FAME_OK)
                return s;
            if (pass == 0) {
                FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
                a_j = hG[0].x;
            }
        }
        double b_j = 0.0;
        if ((s = norm_of(zt, &b_j)) != FAME_OK) return s;
        alpha.push_back(a_j);
        beta.push_back(b_j);
        // Ritz values of the (j+1) x (j+1) tridiagonal matrix (host, FP64)
        const int k = j + 1;
        std::vector<double> T(2 * (size_t)k * k, 0.0), w(k), Z(2 * (size_t)k * k);
        for (int i = 0; i < k; ++i) {
            T[2 * ((size_t)i * k + i)] = alpha[i];
            if (i + 1 < k) {
                T[2 * ((size_t)i * k + i + 1)] = beta[i];
                T[2 * ((size_t)(i + 1) * k + i)] = beta[i];
            }
        }
        if (!herm_eig(k, T.data(), w.data(), Z.data())) return set_err(c, FAME_E_NOCONV, "inverse Lanczos: tridiagonal QR");
        if (k >= nev) {
            // the nev largest Ritz values (ascending order from herm_eig: take the top)
            bool ok = true;
            for (int i = 0; i < nev; ++i) {
                const int col = k - 1 - i;
                const double last = std::hypot(Z[2 * ((size_t)col * k + k - 1)], Z[2 * ((size_t)col * k + k - 1) + 1]);
                if (!(b_j * last <= tol * w[col])) ok = false;
            }
            if (ok || b_j == 0.0) {
                converged = true;
                theta.assign(nev, 0.0);
                V.assign((size_t)k * nev, make_double2(0.0, 0.0));
                for (int i = 0; i < nev; ++i) {
                    const int col = k - 1 - i;
                    theta[i] = w[col];
                    for (int t = 0; t < k; ++t)
                        V[(size_t)i * k + t] = make_double2(Z[2 * ((size_t)col * k + t)], Z[2 * ((size_t)col * k + t) + 1]);
                }
                ++j;
                break;
            }
        }
        if (!(b_j > 0.0)) return set_err(c, FAME_E_NOCONV, "inverse Lanczos: breakdown");
        // q_{j+1} = z / beta_j
        hG[0] = make_double2(1.0 / b_j, 0.0);
        FAME_CUDA_TRY(c, cudaMemcpyAsync(G, hG, sizeof(double2), cudaMemcpyHostToDevice, st));
        if ((s = combine<double2, double2>(c, blocks<double2>(zt, 1), ld, G, 1, 1, Q + (size_t)(j + 1) * N, nullptr,
                                           st)) != FAME_OK)
            return s;
    }
    const int k = j;
    if (!converged) {
        // best values so far from the last tridiagonal matrix
        theta.assign(nev, 0.0);
        std::vector<double> T(2 * (size_t)k * k, 0.0), w(k), Z(2 * (size_t)k * k);
        for (int i = 0; i < k; ++i) {
            T[2 * ((size_t)i * k + i)] = alpha[i];
            if (i + 1 < k) {
                T[2 * ((size_t)i * k + i + 1)] = beta[i];
                T[2 * ((size_t)(i + 1) * k + i)] = beta[i];
            }
        }
        herm_eig(k, T.data(), w.data(), Z.data());
        V.assign((size_t)k * nev, make_double2(0.0, 0.0));
        for (int i = 0; i < nev && i < k; ++i) {
            const int col = k - 1 - i;
            theta[i] = w[col];
            for (int t = 0; t < k; ++t)
                V[(size_t)i * k + t] = make_double2(Z[2 * ((size_t)col * k + t)], Z[2 * ((size_t)col * k + t) + 1]);
        }
    }
    // Ritz vectors Y = Q_k V (ascending lambda = 1 / theta, theta descending already)
    std::memcpy(hG, V.data(), V.size() * sizeof(double2));
    FAME_CUDA_TRY(c, cudaMemcpyAsync(G, hG, V.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    if ((s = combine<double2, double2>(c, blocks<double2>(Q, k), ld, G, nev, k, Y, nullptr, st)) != FAME_OK) return s;
    // explicit residuals with a complex128 apply
    c->stats.applies_c128 += nev;
    if ((s = run_apply<double>(c, Y, AY, nev, st)) != FAME_OK) return s;
    std::vector<double> lam(nev);
    for (int i = 0; i < nev; ++i) lam[i] = 1.0 / theta[i];
    FAME_CUDA_TRY(c, cudaMemcpyAsync(scal + 8, lam.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
    if ((s = residual<double2>(c, Y, AY, scal + 8, c->td.tinv, nev, nullptr, rpart, kResid, st)) != FAME_OK)
        return s;
    std::vector<double> pr((size_t)nev * kResid);
    FAME_CUDA_TRY(c, cudaMemcpyAsync(pr.data(), rpart, pr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int i = 0; i < nev; ++i) {
        double ss = 0.0;
        for (int b = 0; b < kResid; ++b) ss += pr[(size_t)i * kResid + b];
        worst = std::max(worst, std::sqrt(ss) / lam[i]);
    }
    c->stats.max_residual = worst;
    c->stats.iters_fp64 = k;
    c->lambda.assign(lam.begin(), lam.end());
    if (c->Y_nev < nev) {
        if (c->Y) cudaFree(c->Y);
        c->Y = nullptr;
        c->Y_nev = 0;
        if (cudaMalloc((void**)&c->Y, (size_t)nev * N * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, FAME_E_NOMEM, "cudaMalloc eigenvectors");
        }
        c->Y_nev = nev;
    }
    FAME_CUDA_TRY(c, cudaMemcpyAsync(c->Y, Y, (size_t)nev * N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    if (Y_out) FAME_CUDA_TRY(c, cudaMemcpyAsync(Y_out, Y, (size_t)nev * N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    for (int i = 0; i < nev; ++i) lambda_out[i] = lam[i];
    if (iters_out) *iters_out = k;
    c->stats.iters_mixed = cg_iters;      // inner CG iterations (all Lanczos steps together)
    if (!converged) return set_err(c, FAME_E_NOCONV, "inverse Lanczos reached its step limit");
    return FAME_OK;
}
