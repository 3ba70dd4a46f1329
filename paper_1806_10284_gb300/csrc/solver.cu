// Block LOBPCG (Knyazev 2001) for the smallest eigenvalues of A_r (eq. NFSEP).
//
// The paper solves the NFSEP by inverse Lanczos with an inner CG (Section 5.2);
// this library uses the block form, whose only operator access is a block of
// A_r applies, so every FFT pass runs on m vectors at once.
//
// Per iteration, on the GPU: R = AX - X Theta and W = T R with the
// preconditioner T = Sigma_r^{-2} / mean(B^{-1}) (exact for constant B);
// AW = A_r W; the Gram matrices [X W P]^H [X W P] and [X W P]^H [AX AW AP]
// accumulated in FP64; on the host: the FP64 Rayleigh-Ritz problem on the
// GB-orthonormal basis; on the GPU: X <- S C, P <- S_{WP} C_{WP} and the
// same combinations of AS, so each iteration needs one block apply.
//
// FAME_MIXED runs this on complex64 blocks until the residual reaches the
// complex64 floor, then continues on complex128 blocks (refinement) until
// ||A_r y - lambda y|| <= tol lambda with complex128 applies; FAME_FP64 uses
// complex128 blocks throughout.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "blockops.h"

namespace {

constexpr int kResidBlocks = 256;

template <typename C>
struct Workspace {
    // two copies of S = [X W P] and AS = [AX AW AP], each 3m columns
    C* S[2];
    C* AS[2];
    double2* G;       // [k][2k]
    double2* Cd;      // [k][m]
    double* theta;    // [m]
    double* part;     // [m][kResidBlocks]
};

template <typename C>
size_t ws_bytes(size_t ld, int m) {
    const int k = 3 * m;
    return 4 * (size_t)k * ld * sizeof(C) + (size_t)k * 2 * k * sizeof(double2) +
           (size_t)k * m * sizeof(double2) + m * sizeof(double) + (size_t)m * kResidBlocks * sizeof(double) +
           16 * 256;   // each of the 12 carve-outs below rounds up to 256 bytes
}

template <typename C>
Workspace<C> ws_carve(void* base, size_t ld, int m) {
    const int k = 3 * m;
    char* p = static_cast<char*>(base);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    Workspace<C> w;
    for (int i = 0; i < 2; ++i) {
        w.S[i] = reinterpret_cast<C*>(take((size_t)k * ld * sizeof(C)));
        w.AS[i] = reinterpret_cast<C*>(take((size_t)k * ld * sizeof(C)));
    }
    w.G = reinterpret_cast<double2*>(take((size_t)k * 2 * k * sizeof(double2)));
    w.Cd = reinterpret_cast<double2*>(take((size_t)k * m * sizeof(double2)));
    w.theta = reinterpret_cast<double*>(take(m * sizeof(double)));
    w.part = reinterpret_cast<double*>(take((size_t)m * kResidBlocks * sizeof(double)));
    return w;
}

template <typename R>
const R* tinv_of(const fame_ctx* c);
template <> const float* tinv_of<float>(const fame_ctx* c) { return c->tf.tinv; }
template <> const double* tinv_of<double>(const fame_ctx* c) { return c->td.tinv; }

template <typename C>
fame_status apply_block(fame_ctx* c, const C* y, C* Ay, int m, cudaStream_t st);
template <>
fame_status apply_block<float2>(fame_ctx* c, const float2* y, float2* Ay, int m, cudaStream_t st) {
    c->stats.applies_c64 += m;
    return run_apply<float>(c, y, Ay, m, st);
}
template <>
fame_status apply_block<double2>(fame_ctx* c, const double2* y, double2* Ay, int m, cudaStream_t st) {
    c->stats.applies_c128 += m;
    return run_apply<double>(c, y, Ay, m, st);
}

// Result of one phase.
struct PhaseOut {
    int iters = 0;
    bool converged = false;
    std::vector<double> theta;
    std::vector<double> res;
};

// LOBPCG on blocks of type C, starting from the m columns already in w.S[0][X]
// (masked).  Stops when the first nev residuals are <= tol, or after max_iter,
// or (stall_check) when the largest of them has not improved by 10% over
// 8 iterations.
template <typename C>
fame_status lobpcg(fame_ctx* c, Workspace<C>& w, int m, int nev, double tol, int max_iter,
                   bool stall_check, double drop, cudaStream_t st, PhaseOut& out) {
    using R = typename RealOf<C>::T;
    const size_t n = (size_t)c->n, ld = 2 * n;
    const R* tinv = tinv_of<R>(c);
    int cur = 0;
    int np = 0;       // columns of P
    int nw = 0;       // columns of W
    fame_status s;
    std::vector<double2> G, Cm;
    std::vector<double> theta(m), part((size_t)m * kResidBlocks), res(m, 1e300);
    std::vector<double> best_hist;
    // initial Rayleigh-Ritz on X
    C* X = w.S[cur];
    C* AX = w.AS[cur];
    if ((s = apply_block<C>(c, X, AX, m, st)) != FAME_OK) return s;
    for (int it = 0; it <= max_iter; ++it) {
        X = w.S[cur];
        AX = w.AS[cur];
        C* Wb = X + (size_t)m * ld;
        C* AWb = AX + (size_t)m * ld;
        C* Pb = X + (size_t)2 * m * ld;
        C* APb = AX + (size_t)2 * m * ld;
        const int k = m + nw + np;
        BlockList<C> U = blocks<C>(X, m, Wb, nw, Pb, np);
        BlockList<C> V;
        // G = [X W P]^H [X W P | AX AW AP]: two Gram launches into one k x 2k buffer
        s = gram<C>(c, U, U, ld, w.G, st);
        if (s != FAME_OK) return s;
        V = blocks<C>(AX, m, AWb, nw, APb, np);
        s = gram<C>(c, U, V, ld, w.G + (size_t)k * k, st);
        if (s != FAME_OK) return s;
        G.resize((size_t)2 * k * k);
        FAME_CUDA_TRY(c, cudaMemcpyAsync(G.data(), w.G, G.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
        std::vector<double> GB(2 * (size_t)k * k), GA(2 * (size_t)k * k);
        std::memcpy(GB.data(), G.data(), GB.size() * sizeof(double));
        std::memcpy(GA.data(), G.data() + (size_t)k * k, GA.size() * sizeof(double));
        Cm.assign((size_t)k * m, make_double2(0, 0));
        const int got = rayleigh_ritz(k, GA.data(), GB.data(), m, drop, theta.data(),
                                      reinterpret_cast<double*>(Cm.data()));
        if (got < m) {
            // basis lost rank: restart the search directions from X alone
            if (np == 0 && nw == 0) return set_err(c, FAME_E_NOCONV, "block lost rank");
            np = 0;
            nw = 0;
            continue;
        }
        FAME_CUDA_TRY(c, cudaMemcpyAsync(w.Cd, Cm.data(), Cm.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        FAME_CUDA_TRY(c, cudaMemcpyAsync(w.theta, theta.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
        // X' = S C, P' = S[m:] C[m:]   (and the same for AS) into the other buffers
        const int nxt = cur ^ 1;
        C* Xn = w.S[nxt];
        C* AXn = w.AS[nxt];
        const bool have_p = (nw + np) > 0;
        if ((s = combine<C, C>(c, U, ld, w.Cd, m, m, Xn, have_p ? Xn + (size_t)2 * m * ld : nullptr, st)) != FAME_OK) return s;
        if ((s = combine<C, C>(c, V, ld, w.Cd, m, m, AXn, have_p ? AXn + (size_t)2 * m * ld : nullptr, st)) != FAME_OK) return s;
        np = have_p ? m : 0;
        cur = nxt;
        X = Xn;
        AX = AXn;
        Wb = X + (size_t)m * ld;
        AWb = AX + (size_t)m * ld;
        // residuals and preconditioned directions
        if ((s = residual<C>(c, X, AX, w.theta, tinv, m, Wb, w.part, kResidBlocks, st)) != FAME_OK) return s;
        FAME_CUDA_TRY(c, cudaMemcpyAsync(part.data(), w.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int j = 0; j < m; ++j) {
            double ss = 0.0;
            for (int b = 0; b < kResidBlocks; ++b) ss += part[(size_t)j * kResidBlocks + b];
            res[j] = std::sqrt(ss) / std::fabs(theta[j]);
            if (j < nev) worst = std::max(worst, res[j]);
        }
        out.iters = it + 1;
        out.theta.assign(theta.begin(), theta.end());
        out.res.assign(res.begin(), res.end());
        if (worst <= tol) { out.converged = true; break; }
        if (stall_check) {
            best_hist.push_back(worst);
            const size_t h = best_hist.size();
            if (h > 8 && worst > 0.9 * best_hist[h - 9]) break;
        }
        if (it == max_iter) break;
        nw = m;
        if ((s = apply_block<C>(c, Wb, AWb, nw, st)) != FAME_OK) return s;
    }
    // leave the result in w.S[0] / w.AS[0]
    if (cur != 0) {
        FAME_CUDA_TRY(c, cudaMemcpyAsync(w.S[0], w.S[cur], (size_t)m * ld * sizeof(C), cudaMemcpyDeviceToDevice, st));
        FAME_CUDA_TRY(c, cudaMemcpyAsync(w.AS[0], w.AS[cur], (size_t)m * ld * sizeof(C), cudaMemcpyDeviceToDevice, st));
    }
    return FAME_OK;
}

}  // namespace

fame_status run_eigs(fame_ctx* c, int nev, double tol, int max_iter, int flags, double* lambda_out,
                     void* Y_out, int* iters_out, cudaStream_t st) {
    const size_t n = (size_t)c->n, ld = 2 * n;
    const int m = std::min<long long>(nev + std::max(4, (nev + 1) / 2), ld);
    const bool mixed = (flags & FAME_MIXED) && !(flags & FAME_FP64);
    c->stats = fame_solve_stats{};
    fame_status s;
    const size_t b32 = mixed ? ws_bytes<float2>(ld, m) : 0;
    const size_t b64 = ws_bytes<double2>(ld, m);
    if ((s = grow(c, c->solver, std::max(b32, b64))) != FAME_OK) return s;
    const uint64_t seed = 0x5eedF00Dull ^ ((uint64_t)c->n << 20) ^ (uint64_t)nev;
    PhaseOut ph1, ph2;
    Workspace<double2> w64 = ws_carve<double2>(c->solver.p, ld, m);
    const bool warm = (flags & FAME_WARM_START) && c->Y && c->Y_nev >= 1;
    if (mixed) {
        Workspace<float2> w32 = ws_carve<float2>(c->solver.p, ld, m);
        if ((s = random_block<float2>(c, w32.S[0], m, seed, c->tf.tinv, st)) != FAME_OK) return s;
        if (warm) {
            const int nw = std::min(c->Y_nev, m);
            if ((s = convert<double2, float2>(c, reinterpret_cast<const double2*>(c->Y), w32.S[0], (size_t)nw * ld, st)) != FAME_OK) return s;
        }
        // complex64 phase: stop at the complex64 floor (stall) or well below tol
        const double tol32 = std::max(tol, 2e-5);
        if ((s = lobpcg<float2>(c, w32, m, nev, tol32, max_iter, true, 1e-6, st, ph1)) != FAME_OK) return s;
        c->stats.iters_mixed = ph1.iters;
        // promote X to complex128 for refinement (w64.S[0] overlaps w32 buffers: stage through AS[1])
        float2* stage = reinterpret_cast<float2*>(w64.AS[1]);
        FAME_CUDA_TRY(c, cudaMemcpyAsync(stage, w32.S[0], (size_t)m * ld * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        if ((s = convert<float2, double2>(c, stage, w64.S[0], (size_t)m * ld, st)) != FAME_OK) return s;
    } else {
        if ((s = random_block<double2>(c, w64.S[0], m, seed, c->td.tinv, st)) != FAME_OK) return s;
        if (warm) {
            const int nw = std::min(c->Y_nev, m);
            FAME_CUDA_TRY(c, cudaMemcpyAsync(w64.S[0], c->Y, (size_t)nw * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        }
    }
    const int left = std::max(1, max_iter - ph1.iters);
    if ((s = lobpcg<double2>(c, w64, m, nev, tol, left, false, 1e-12, st, ph2)) != FAME_OK) return s;
    c->stats.iters_fp64 = ph2.iters;
    // keep eigenpairs; lambda from the last Rayleigh-Ritz (complex128 basis)
    c->lambda.assign(ph2.theta.begin(), ph2.theta.begin() + nev);
    double worst = 0.0;
    for (int j = 0; j < nev; ++j) worst = std::max(worst, ph2.res[j]);
    c->stats.max_residual = worst;
    if (c->Y_nev < nev) {
        if (c->Y) cudaFree(c->Y);
        c->Y = nullptr;
        c->Y_nev = 0;
        if (cudaMalloc((void**)&c->Y, (size_t)nev * ld * sizeof(double2)) != cudaSuccess)
            return set_err(c, FAME_E_NOMEM, "cudaMalloc eigenvectors");
        c->Y_nev = nev;
    }
    FAME_CUDA_TRY(c, cudaMemcpyAsync(c->Y, w64.S[0], (size_t)nev * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    if (Y_out)
        FAME_CUDA_TRY(c, cudaMemcpyAsync(Y_out, w64.S[0], (size_t)nev * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    for (int j = 0; j < nev; ++j) lambda_out[j] = c->lambda[j];
    if (iters_out) *iters_out = ph1.iters + ph2.iters;
    if (!ph2.converged)
        return set_err(c, FAME_E_NOCONV, "eigensolver reached max_iter; max residual " + std::to_string(worst));
    return FAME_OK;
}

fame_status run_eigs_batched(fame_ctx* const* ctxs, int nprob, int nev, double tol, int max_iter,
                             int flags, double* lambda_out, int* iters_out, cudaStream_t st) {
    fame_status worst = FAME_OK;
    for (int i = 0; i < nprob; ++i) {
        int it = 0;
        fame_status s = fame_eigs(ctxs[i], nev, tol, max_iter, flags, lambda_out + (size_t)i * nev,
                                  nullptr, &it, st);
        if (iters_out) iters_out[i] = it;
        if (s == FAME_E_NOCONV) worst = s;
        else if (s != FAME_OK) return s;
    }
    return worst;
}
