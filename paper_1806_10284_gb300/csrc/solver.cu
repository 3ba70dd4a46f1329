// Block LOBPCG (Knyazev 2001) for the smallest eigenvalues of A_r (eq. NFSEP).
//
// The paper solves the NFSEP by inverse Lanczos with an inner CG (Section 5.2);
// this library uses the block form, whose only operator access is a block of
// A_r applies, so every FFT pass runs on m vectors at once.
//
// One iteration: R = AX - X Theta and W = T R with T = S P_K(M) S, the Chebyshev
// approximation of A_r^{-1} (precond.cu; degree 1 is Sigma_r^{-2} / mean(B^{-1}),
// exact for constant B); AW = A_r W for the columns not yet converged (soft
// locking of the leading converged ones); Gram matrices of [X W P] against
// [X W P | AX AW AP] accumulated in FP64; the FP64 Rayleigh-Ritz problem on a
// GB-orthonormal basis (host); X <- S C, P <- S_{WP} C_{WP} and the same
// combinations of AS, so an iteration costs one block apply.
//
// FAME_MIXED:
//   phase 1  complex64 blocks throughout until the residual reaches the
//            complex64 floor;
//   phase 2  refinement: X and AX held in complex128 and updated in FP64 from
//            the complex64 search directions W, P (whose coefficients shrink
//            with the residual).  The Gram matrices are formed from complex64
//            copies; their X-X blocks are the identity and Theta of the
//            previous Rayleigh-Ritz step.  A complex128 apply starts the phase
//            and confirms convergence.
//   end      explicit FP64 Rayleigh-Ritz on the nev wanted columns of X with a
//            complex128 apply; the reported residuals ||A_r y - lambda y|| / lambda
//            come from it.
// FAME_FP64: complex128 blocks throughout, explicit FP64 Gram matrices.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <utility>
#include <vector>

#include "blockops.h"

namespace {

constexpr int kResidBlocks = 256;

// per-iteration log on stderr when the environment sets FAME_LOG=1
bool log_on() {
    static const bool on = [] {
        const char* v = std::getenv("FAME_LOG");
        return v && v[0] == '1';
    }();
    return on;
}

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
    return run_apply_c128(c, y, Ay, m, c->df128, st);
}

// Requested residuals of at least this size take the complex128 applies in
// double-float arithmetic: their rounding, about 2^-47 relative per operation and
// amplified by roughly sqrt(||A_r|| / lambda) through Sigma_r at both ends, stays
// one to two orders of magnitude below the residual up to 192^3 grids.
constexpr double kDf128MinTol = 1e-10;

template <typename R>
const R* tinv_of(const fame_ctx* c);
template <> const float* tinv_of<float>(const fame_ctx* c) { return c->tf.tinv; }
template <> const double* tinv_of<double>(const fame_ctx* c) { return c->td.tinv; }

// Carves one device allocation into 256-byte aligned pieces.
struct Carver {
    char* p;
    size_t used = 0;
    explicit Carver(void* base) : p(static_cast<char*>(base)) {}
    template <typename T>
    T* take(size_t count) {
        T* r = reinterpret_cast<T*>(p + used);
        used += (count * sizeof(T) + 255) & ~(size_t)255;
        return r;
    }
};

// Small device buffers shared by the phases, and their page-locked host mirror
// (read-backs and uploads go through it, so they are direct DMA transfers).
struct Small {
    double2* G;      // [k][2k]
    double2* Cd;     // [k][m]
    double* theta;   // [m]
    double* part;    // [m][kResidBlocks]
    int* blk;        // [m][kRefineBlock + 1] blocks of the refinement update
    double2* hG = nullptr;
    double2* hC = nullptr;
    double* htheta = nullptr;
    double* hpart = nullptr;
    int* hblk = nullptr;
};

size_t small_bytes(int m) {
    const int k = 3 * m;
    return ((size_t)k * 2 * k * sizeof(double2) + 255) + ((size_t)k * m * sizeof(double2) + 255) +
           (m * sizeof(double) + 255) + ((size_t)m * kResidBlocks * sizeof(double) + 255) +
           ((size_t)m * (kRefineBlock + 1) * sizeof(int) + 255);
}

Small carve_small(Carver& cv, int m) {
    const int k = 3 * m;
    Small s;
    s.G = cv.take<double2>((size_t)k * 2 * k);
    s.Cd = cv.take<double2>((size_t)k * m);
    s.theta = cv.take<double>(m);
    s.part = cv.take<double>((size_t)m * kResidBlocks);
    s.blk = cv.take<int>((size_t)m * (kRefineBlock + 1));
    return s;
}

// Blocks of the refinement update X_new = X C_X + Q C_Q (C_X the leading m rows of the
// k x m Ritz coefficients Cm): outputs i and j share a block when |C_X[i][j]| or
// |C_X[j][i]| exceeds kCouple.  Inside a block the complex128 X is combined in
// FP64-accurate arithmetic; the remaining entries of C_X are below kCouple, so their
// FP32 products carry errors below kCouple * 2^-24 relative.  Writes the table
// [m][kRefineBlock + 1] (count, then the columns); false if a block is too large.
constexpr double kCouple = 1e-4;
bool refine_blocks(const std::vector<double2>& Cm, int k, int m, int* tab) {
    std::vector<int> parent(m);
    for (int i = 0; i < m; ++i) parent[i] = i;
    auto find = [&](int i) {
        while (parent[i] != i) i = parent[i] = parent[parent[i]];
        return i;
    };
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            const double2 v = Cm[(size_t)j * k + i];
            if (i != j && std::hypot(v.x, v.y) > kCouple) parent[find(i)] = find(j);
        }
    std::vector<std::vector<int>> members(m);
    for (int i = 0; i < m; ++i) members[find(i)].push_back(i);
    for (int j = 0; j < m; ++j) {
        const std::vector<int>& b = members[find(j)];
        if ((int)b.size() > kRefineBlock) return false;
        int* row = tab + (size_t)j * (kRefineBlock + 1);
        row[0] = (int)b.size();
        for (int t = 0; t < kRefineBlock; ++t) row[1 + t] = t < (int)b.size() ? b[t] : 0;
    }
    return true;
}

bool gram_finite(const double2* G, size_t cnt) {
    for (size_t i = 0; i < cnt; ++i)
        if (!std::isfinite(G[i].x) || !std::isfinite(G[i].y)) return false;
    return true;
}

// a non-finite Gram matrix: a tensor-core wait that gave up (reported as such), or
// non-finite vectors
fame_status gram_failure(fame_ctx* c) {
    if (tc_wait_failed(c))
        return set_err(c, FAME_E_TIMEOUT, "a bounded wait of the tensor-core Gram kernel gave up");
    return set_err(c, FAME_E_NOCONV, "non-finite Gram matrix");
}

struct PhaseOut {
    int iters = 0;
    bool converged = false;
    std::vector<double> theta;
    std::vector<double> res;
};

// Host Rayleigh-Ritz on the device Gram buffer G = [GB | GA] (each k x k).
// If implicit_xx > 0 the leading implicit_xx x implicit_xx blocks are replaced by
// the identity (GB) and diag(theta_prev) (GA).
int host_rr(fame_ctx* c, const Small& sm, int k, int m, int implicit_xx, const std::vector<double>& theta_prev,
            double drop, std::vector<double>& theta, std::vector<double2>& Cm, cudaStream_t st, fame_status* err,
            bool try_cholesky = true) {
    const double2* G = sm.hG;
    cudaError_t e = cudaMemcpyAsync(sm.hG, sm.G, (size_t)2 * k * k * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = set_err(c, FAME_E_CUDA, std::string("Gram readback: ") + cudaGetErrorString(e));
        return -1;
    }
    if (!gram_finite(G, (size_t)2 * k * k)) {
        *err = gram_failure(c);
        return -1;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<double> GB(2 * (size_t)k * k), GA(2 * (size_t)k * k);
    std::memcpy(GB.data(), G, GB.size() * sizeof(double));
    std::memcpy(GA.data(), G + (size_t)k * k, GA.size() * sizeof(double));
    // Hermitise from the lower triangle: entry (i > j) is [W P]^H [AX ...] against the
    // leading X columns, i.e. built from the accurate AX rather than from AW.
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < j; ++i) {
            const size_t up = 2 * ((size_t)j * k + i), lo = 2 * ((size_t)i * k + j);
            GA[up] = GA[lo];
            GA[up + 1] = -GA[lo + 1];
            GB[up] = GB[lo];
            GB[up + 1] = -GB[lo + 1];
        }
    for (int j = 0; j < implicit_xx; ++j)
        for (int i = 0; i < implicit_xx; ++i) {
            const size_t o = 2 * ((size_t)j * k + i);
            GB[o] = (i == j) ? 1.0 : 0.0;
            GB[o + 1] = 0.0;
            GA[o] = (i == j) ? theta_prev[i] : 0.0;
            GA[o + 1] = 0.0;
        }
    Cm.assign((size_t)k * m, make_double2(0, 0));
    theta.assign(m, 0.0);
    const int got = rayleigh_ritz(k, GA.data(), GB.data(), m, drop, theta.data(),
                                  reinterpret_cast<double*>(Cm.data()), try_cholesky);
    c->stats_rr_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (got == kRRNoConv) {
        *err = set_err(c, FAME_E_NOCONV, "Rayleigh-Ritz: the implicit QR of the small eigenproblem did not converge");
        return -1;
    }
    *err = FAME_OK;
    return got;
}

// Refinement Rayleigh-Ritz.  The basis is [X Q], X the complex128 Ritz block of
// the previous step (X^H X = I, X^H A X = Theta) and Q = [W P] (nq complex64
// columns orthogonalised against X, so X^H Q = 0 and Q^H A X = Q^H R).  Device G
// holds the nq x (2 nq + m) matrix Q^H [Q | AQ | R], column-major.
int host_rr_refine(fame_ctx* c, const Small& sm, int m, int nq, const std::vector<double>& theta_prev,
                   double drop, std::vector<double>& theta, std::vector<double2>& Cm, cudaStream_t st,
                   fame_status* err) {
    const size_t cnt = (size_t)nq * (2 * nq + m);
    const double2* G = sm.hG;
    cudaError_t e = cudaMemcpyAsync(sm.hG, sm.G, cnt * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = set_err(c, FAME_E_CUDA, std::string("Gram readback: ") + cudaGetErrorString(e));
        return -1;
    }
    if (!gram_finite(G, cnt)) {
        *err = gram_failure(c);
        return -1;
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int k = m + nq;
    auto g = [&](int row, int col) { return G[(size_t)col * nq + row]; };
    std::vector<double> GB(2 * (size_t)k * k, 0.0), GA(2 * (size_t)k * k, 0.0);
    auto set = [&](std::vector<double>& M, int i, int j, double re, double im) {
        M[2 * ((size_t)j * k + i)] = re;
        M[2 * ((size_t)j * k + i) + 1] = im;
    };
    for (int i = 0; i < m; ++i) {
        set(GB, i, i, 1.0, 0.0);
        set(GA, i, i, theta_prev[i], 0.0);
    }
    for (int q = 0; q < nq; ++q) {
        for (int i = 0; i < m; ++i) {
            const double2 r = g(q, 2 * nq + i);          // Q_q^H R_i = Q_q^H A X_i
            set(GA, m + q, i, r.x, r.y);
        }
        for (int p = 0; p < nq; ++p) {
            const double2 b = g(p, q), a = g(p, nq + q);
            set(GB, m + p, m + q, b.x, b.y);
            set(GA, m + p, m + q, a.x, a.y);
        }
    }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < j; ++i) {
            const size_t up = 2 * ((size_t)j * k + i), lo = 2 * ((size_t)i * k + j);
            GA[up] = GA[lo];
            GA[up + 1] = -GA[lo + 1];
            GB[up] = GB[lo];
            GB[up + 1] = -GB[lo + 1];
        }
    Cm.assign((size_t)k * m, make_double2(0, 0));
    theta.assign(m, 0.0);
    const int got = rayleigh_ritz(k, GA.data(), GB.data(), m, drop, theta.data(),
                                  reinterpret_cast<double*>(Cm.data()));
    c->stats_rr_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (got == kRRNoConv) {
        *err = set_err(c, FAME_E_NOCONV, "Rayleigh-Ritz: the implicit QR of the small eigenproblem did not converge");
        return -1;
    }
    *err = FAME_OK;
    return got;
}

fame_status upload_rr(fame_ctx* c, const Small& sm, const std::vector<double2>& Cm,
                      const std::vector<double>& theta, cudaStream_t st) {
    // the previous upload has completed: every upload follows a stream synchronisation
    std::memcpy(sm.hC, Cm.data(), Cm.size() * sizeof(double2));
    std::memcpy(sm.htheta, theta.data(), theta.size() * sizeof(double));
    FAME_CUDA_TRY(c, cudaMemcpyAsync(sm.Cd, sm.hC, Cm.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    FAME_CUDA_TRY(c, cudaMemcpyAsync(sm.theta, sm.htheta, theta.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    return FAME_OK;
}

fame_status read_norms(fame_ctx* c, const Small& sm, int m, const std::vector<double>& theta,
                       std::vector<double>& res, cudaStream_t st) {
    const double* part = sm.hpart;
    FAME_CUDA_TRY(c, cudaMemcpyAsync(sm.hpart, sm.part, (size_t)m * kResidBlocks * sizeof(double),
                                     cudaMemcpyDeviceToHost, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    res.assign(m, 0.0);
    for (int j = 0; j < m; ++j) {
        double ss = 0.0;
        for (int b = 0; b < kResidBlocks; ++b) ss += part[(size_t)j * kResidBlocks + b];
        res[j] = std::sqrt(ss) / std::fabs(theta[j]);
    }
    return FAME_OK;
}

int leading_converged(const std::vector<double>& res, int nev, double tol) {
    int j0 = 0;
    while (j0 < nev && res[j0] <= tol) ++j0;
    return j0;
}

// ---------------------------------------------------------------------------
// LOBPCG with explicit Gram matrices on blocks of type C.  X starts in S[0]
// (first m columns).  Result left in S[0] / AS[0].
// ---------------------------------------------------------------------------
template <typename C>
fame_status lob_explicit(fame_ctx* c, C* const S[2], C* const AS[2], const Small& sm, int m, int nev,
                         double tol, int max_iter, bool stall_check, double drop, cudaStream_t st,
                         PhaseOut& out) {
    using R = typename RealOf<C>::T;
    const size_t ld = 2 * (size_t)c->n;
    const R* tinv = tinv_of<R>(c);
    int cur = 0, np = 0, nw = 0, j0 = 0;
    fame_status s;
    std::vector<double> theta(m, 0.0), res(m, 1e300), hist;
    std::vector<double2> Cm;
    if ((s = apply_block<C>(c, S[0], AS[0], m, st)) != FAME_OK) return s;
    for (int it = 0; it <= max_iter; ++it) {
        C* X = S[cur];
        C* AX = AS[cur];
        C* Wb = X + (size_t)m * ld + (size_t)j0 * ld;
        C* AWb = AX + (size_t)m * ld + (size_t)j0 * ld;
        C* Pb = X + (size_t)2 * m * ld;
        C* APb = AX + (size_t)2 * m * ld;
        const int k = m + nw + np;
        const BlockList<C> U = blocks<C>(X, m, Wb, nw, Pb, np);
        const BlockList<C> V = blocks<C>(AX, m, AWb, nw, APb, np);
        // [GB | GA] = U^H [U | V] in one pass over U; lower triangles only (both Hermitian)
        if ((s = gram_herm<C>(c, U, V, ld, sm.G, st)) != FAME_OK) return s;
        std::vector<double> th;
        const int got = host_rr(c, sm, k, m, 0, theta, drop, th, Cm, st, &s);
        if (got < 0) return s;
        if (got < m) {
            if (np == 0 && nw == 0) return set_err(c, FAME_E_NOCONV, "block lost rank");
            np = nw = 0;
            continue;
        }
        theta = th;
        if ((s = upload_rr(c, sm, Cm, theta, st)) != FAME_OK) return s;
        const int nxt = cur ^ 1;
        const bool have_p = (nw + np) > 0;
        if ((s = combine<C, C>(c, U, ld, sm.Cd, m, m, S[nxt], have_p ? S[nxt] + (size_t)2 * m * ld : nullptr, st)) != FAME_OK) return s;
        if ((s = combine<C, C>(c, V, ld, sm.Cd, m, m, AS[nxt], have_p ? AS[nxt] + (size_t)2 * m * ld : nullptr, st)) != FAME_OK) return s;
        np = have_p ? m : 0;
        cur = nxt;
        X = S[cur];
        AX = AS[cur];
        if ((s = residual<C>(c, X, AX, sm.theta, tinv, m, X + (size_t)m * ld, sm.part, kResidBlocks, st)) != FAME_OK) return s;
        if ((s = read_norms(c, sm, m, theta, res, st)) != FAME_OK) return s;
        double worst = 0.0;
        for (int j = 0; j < nev; ++j) worst = std::max(worst, res[j]);
        out.iters = it + 1;
        out.theta = theta;
        out.res = res;
        if (log_on())
            std::fprintf(stderr, "[fame] %s it %d k %d worst %.3e theta0 %.10g theta%d %.10g\n",
                         sizeof(C) == 8 ? "c64" : "c128", it, k, worst, theta[0], nev - 1, theta[nev - 1]);
        if (worst <= tol) { out.converged = true; break; }
        if (stall_check) {
            // the complex64 floor: after 20 iterations, no 30% gain over the last 10
            hist.push_back(worst);
            const size_t h = hist.size();
            if (h > 20 && worst < 1e-3) {
                double best_old = *std::min_element(hist.begin(), hist.end() - 10);
                if (worst > 0.7 * best_old) break;
            }
        }
        if (it == max_iter) break;
        j0 = leading_converged(res, nev, tol);
        nw = m - j0;
        {
            // ortho-LOBPCG (Hetmaniuk and Lehoucq 2006): W and P orthogonalised against X
            // (AP alongside), then AW for the orthogonalised W
            C* Wn = X + (size_t)m * ld + (size_t)j0 * ld;
            if ((s = precond_cheb<C>(c, Wn, nw, st)) != FAME_OK) return s;
            C* Pn = X + (size_t)2 * m * ld;
            C* APn = AX + (size_t)2 * m * ld;
            const BlockList<C> Q = blocks<C>(Wn, nw, Pn, np);
            const BlockList<C> Xl = blocks<C>(X, m);
            if ((s = gram<C, C>(c, Xl, Q, ld, sm.G, st)) != FAME_OK) return s;
            if ((s = orth_against<C, C>(c, X, m, Q, ld, sm.G, st)) != FAME_OK) return s;
            if (np > 0 && (s = orth_against<C, C>(c, AX, m, blocks<C>(APn, np), ld, sm.G + (size_t)m * nw, st)) != FAME_OK) return s;
            if ((s = apply_block<C>(c, Wn, AX + (size_t)m * ld + (size_t)j0 * ld, nw, st)) != FAME_OK) return s;
        }
    }
    if (cur != 0) {
        FAME_CUDA_TRY(c, cudaMemcpyAsync(S[0], S[cur], (size_t)m * ld * sizeof(C), cudaMemcpyDeviceToDevice, st));
        FAME_CUDA_TRY(c, cudaMemcpyAsync(AS[0], AS[cur], (size_t)m * ld * sizeof(C), cudaMemcpyDeviceToDevice, st));
    }
    return FAME_OK;
}

// ---------------------------------------------------------------------------
// Explicit FP64 Rayleigh-Ritz of the complex128 block X (m columns) with a
// complex128 apply: X <- X C, AX <- (A X) C; residual norms from them.
// X, AX in buffers a/aa; results in b/ab.
// ---------------------------------------------------------------------------
fame_status rr64(fame_ctx* c, double2* a, double2* aa, double2* b, double2* ab, const Small& sm, int m,
                 bool do_apply, std::vector<double>& theta, std::vector<double>& res, cudaStream_t st) {
    const size_t ld = 2 * (size_t)c->n;
    fame_status s;
    if (do_apply && (s = apply_block<double2>(c, a, aa, m, st)) != FAME_OK) return s;
    const BlockList<double2> U = blocks<double2>(a, m), V = blocks<double2>(aa, m);
    // X is a near-eigenbasis here (A X ~ X Theta): the double-float Gram suffices
    if ((s = gram_herm_df(c, U, V, ld, sm.G, st)) != FAME_OK) return s;
    std::vector<double2> Cm;
    std::vector<double> th;
    // the final FP64 step reduces through the eigen-decomposition of X^H X
    const int got = host_rr(c, sm, m, m, 0, theta, 1e-14, th, Cm, st, &s, false);
    if (got < 0) return s;
    if (got < m) return set_err(c, FAME_E_NOCONV, "refined block lost rank");
    theta = th;
    if ((s = upload_rr(c, sm, Cm, theta, st)) != FAME_OK) return s;
    // X C and (AX) C in double-float arithmetic (no complex64 part)
    const BlockList<float2> none = blocks<float2>(nullptr, 0);
    if ((s = combine_mixed(c, a, m, none, ld, sm.Cd, b, nullptr, nullptr, st)) != FAME_OK) return s;
    if ((s = combine_mixed(c, aa, m, none, ld, sm.Cd, ab, nullptr, nullptr, st)) != FAME_OK) return s;
    if ((s = residual<double2>(c, b, ab, sm.theta, c->td.tinv, m, nullptr, sm.part, kResidBlocks, st)) != FAME_OK) return s;
    return read_norms(c, sm, m, theta, res, st);
}

// ---------------------------------------------------------------------------
// Mixed refinement.  X32 (complex64 copy of X) starts in S32[0]; on return the
// refined complex128 X is in X64[0] with AX in AX64[0].
// ---------------------------------------------------------------------------
fame_status lob_refine(fame_ctx* c, float2* const S[2], float2* const AS[2], double2* const X64[2],
                       double2* const AX64[2], float2* R32, const Small& sm, int m, int nev, double tol,
                       int max_iter, cudaStream_t st, PhaseOut& out) {
    const size_t ld = 2 * (size_t)c->n;
    fame_status s;
    std::vector<double> theta(m, 0.0), res;
    // start: promote X, complex128 apply, explicit FP64 Rayleigh-Ritz
    if ((s = convert<float2, double2>(c, S[0], X64[1], (size_t)m * ld, st)) != FAME_OK) return s;
    if ((s = rr64(c, X64[1], AX64[1], X64[0], AX64[0], sm, m, true, theta, res, st)) != FAME_OK) return s;
    int cur = 0, np = 0, nw = 0, j0 = 0;
    // complex64 copies of X, AX in the X slots of S[0], AS[0]
    if ((s = convert<double2, float2>(c, X64[0], S[0], (size_t)m * ld, st)) != FAME_OK) return s;
    if ((s = convert<double2, float2>(c, AX64[0], AS[0], (size_t)m * ld, st)) != FAME_OK) return s;
    std::vector<double2> Cm;
    std::vector<double> hist;
    for (int it = 0; it <= max_iter; ++it) {
        // residuals of the tracked pair; W for every column
        float2* X32 = S[cur];
        float2* AX32 = AS[cur];
        if ((s = residual_mixed(c, X64[cur], AX64[cur], sm.theta, m, X32 + (size_t)m * ld, R32, sm.part, kResidBlocks, st)) != FAME_OK) return s;
        if ((s = read_norms(c, sm, m, theta, res, st)) != FAME_OK) return s;
        double worst = 0.0;
        for (int j = 0; j < nev; ++j) worst = std::max(worst, res[j]);
        out.iters = it;
        if (log_on())
            std::fprintf(stderr, "[fame] refine it %d np %d worst %.3e theta0 %.14g\n", it, np, worst, theta[0]);
        hist.push_back(worst);
        if (hist.size() > 8 && worst > 0.5 * *std::min_element(hist.begin(), hist.end() - 4)) {
            // no factor-2 gain over the last 4 iterations: the complex64 directions no
            // longer resolve the residual; hand over to the complex128 solver
            out.theta = theta;
            out.res = res;
            break;
        }
        if (worst <= 0.5 * tol) {
            // confirm the nev wanted pairs with a complex128 apply and an explicit FP64
            // Rayleigh-Ritz on their span (a rotation inside span(X[:nev]), which stays
            // orthogonal to the other columns; those keep their tracked X, AX and theta)
            const int mc = nev;
            std::vector<double> th2(theta.begin(), theta.begin() + mc), r2;
            if ((s = rr64(c, X64[cur], AX64[cur ^ 1], X64[cur ^ 1], AX64[cur], sm, mc, true, th2, r2, st)) != FAME_OK) return s;
            // rr64 left X in X64[cur^1], AX in AX64[cur] (first mc columns): move X back
            FAME_CUDA_TRY(c, cudaMemcpyAsync(X64[cur], X64[cur ^ 1], (size_t)mc * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            for (int j = 0; j < mc; ++j) {
                theta[j] = th2[j];
                res[j] = r2[j];
            }
            worst = 0.0;
            for (int j = 0; j < nev; ++j) worst = std::max(worst, res[j]);
            out.theta = theta;
            out.res = res;
            if (worst <= tol) { out.converged = true; break; }
            if ((s = convert<double2, float2>(c, X64[cur], X32, (size_t)m * ld, st)) != FAME_OK) return s;
            if ((s = convert<double2, float2>(c, AX64[cur], AX32, (size_t)m * ld, st)) != FAME_OK) return s;
            if ((s = residual_mixed(c, X64[cur], AX64[cur], sm.theta, m, X32 + (size_t)m * ld, R32, sm.part, kResidBlocks, st)) != FAME_OK) return s;
            np = 0;
        }
        out.theta = theta;
        out.res = res;
        if (it == max_iter) break;
        j0 = leading_converged(res, nev, 0.5 * tol);
        nw = m - j0;
        float2* Wb = X32 + (size_t)m * ld + (size_t)j0 * ld;
        if ((s = precond_cheb<float2>(c, Wb, nw, st)) != FAME_OK) return s;
        float2* AWb = AX32 + (size_t)m * ld + (size_t)j0 * ld;
        float2* Pb = X32 + (size_t)2 * m * ld;
        float2* APb = AX32 + (size_t)2 * m * ld;
        const int nq = nw + np;
        const BlockList<float2> Q = blocks<float2>(Wb, nw, Pb, np);
        const BlockList<float2> AQ = blocks<float2>(AWb, nw, APb, np);
        // Orthogonalise the complex64 directions against X (c = X^H Q, Q <- Q - X c,
        // AP <- AP - AX c_P) so that no direction carries a large component along X
        // whose complex64 rounding the Rayleigh-Ritz step would amplify; then AW for
        // the orthogonalised W.  With Q orthogonal to X, the coupling Q^H A X equals
        // Q^H R (R = AX - X Theta, small), so every Gram block is an FP32-product
        // Gram: Q^H [Q | AQ | R].
        const BlockList<float2> Xl = blocks<float2>(X32, m);
        if ((s = gram<float2, float2>(c, Xl, Q, ld, sm.G, st)) != FAME_OK) return s;
        if ((s = orth_against<float2, float2>(c, X32, m, Q, ld, sm.G, st)) != FAME_OK) return s;
        if (np > 0 && (s = orth_against<float2, float2>(c, AX32, m, blocks<float2>(APb, np), ld, sm.G + (size_t)m * nw, st)) != FAME_OK) return s;
        if ((s = apply_block<float2>(c, Wb, AWb, nw, st)) != FAME_OK) return s;
        const BlockList<float2> V = concat(concat(Q, AQ), blocks<float2>(R32, m));
        if ((s = gram<float2, float2>(c, Q, V, ld, sm.G, st)) != FAME_OK) return s;
        std::vector<double> th;
        const int got = host_rr_refine(c, sm, m, nq, theta, 1e-6, th, Cm, st, &s);
        if (got < 0) return s;
        if (got < m) { np = 0; continue; }
        theta = th;
        if ((s = upload_rr(c, sm, Cm, theta, st)) != FAME_OK) return s;
        const int nxt = cur ^ 1;
        if (refine_blocks(Cm, m + nq, m, sm.hblk)) {
            // FP64-accurate sums only inside the blocks of strongly coupled outputs; the
            // complex64 copies X32 = S[cur], AX32 = AS[cur] carry the small remainder
            FAME_CUDA_TRY(c, cudaMemcpyAsync(sm.blk, sm.hblk, (size_t)m * (kRefineBlock + 1) * sizeof(int),
                                             cudaMemcpyHostToDevice, st));
            if ((s = combine_refine(c, X64[cur], S[cur], m, Q, ld, sm.Cd, sm.blk, X64[nxt], S[nxt], S[nxt] + (size_t)2 * m * ld, st)) != FAME_OK) return s;
            if ((s = combine_refine(c, AX64[cur], AS[cur], m, AQ, ld, sm.Cd, sm.blk, AX64[nxt], AS[nxt], AS[nxt] + (size_t)2 * m * ld, st)) != FAME_OK) return s;
        } else {
            if ((s = combine_mixed(c, X64[cur], m, Q, ld, sm.Cd, X64[nxt], S[nxt], S[nxt] + (size_t)2 * m * ld, st)) != FAME_OK) return s;
            if ((s = combine_mixed(c, AX64[cur], m, AQ, ld, sm.Cd, AX64[nxt], AS[nxt], AS[nxt] + (size_t)2 * m * ld, st)) != FAME_OK) return s;
        }
        np = m;
        cur = nxt;
    }
    if (cur != 0) {
        FAME_CUDA_TRY(c, cudaMemcpyAsync(X64[0], X64[cur], (size_t)m * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        FAME_CUDA_TRY(c, cudaMemcpyAsync(AX64[0], AX64[cur], (size_t)m * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    return FAME_OK;
}

}  // namespace

fame_status run_eigs(fame_ctx* c, int nev, double tol, int max_iter, int flags, double* lambda_out,
                     void* Y_out, int* iters_out, cudaStream_t st) {
    const size_t n = (size_t)c->n, ld = 2 * n;
    const int m = (int)std::min<long long>(nev + std::max(4, (nev + 1) / 2), (long long)ld / 3);
    const bool mixed = (flags & FAME_MIXED) && !(flags & FAME_FP64);
    c->stats = fame_solve_stats{};
    c->stats_rr_ms = 0.0;
    c->df128 = !fp64_native() && tol >= kDf128MinTol;
    fame_status s;
    if ((s = tc_reset_err(c, st)) != FAME_OK) return s;
    const int k = 3 * m;
    size_t bytes = small_bytes(m) + 256;
    if (mixed)
        bytes += 4 * (((size_t)k * ld * sizeof(float2) + 255)) + 4 * (((size_t)m * ld * sizeof(double2) + 255)) +
                 (((size_t)m * ld * sizeof(float2) + 255));
    else
        bytes += 4 * (((size_t)k * ld * sizeof(double2) + 255));
    if ((s = grow(c, c->solver, bytes)) != FAME_OK) return s;
    Carver cv(c->solver.p);
    Small sm = carve_small(cv, m);
    {
        if ((s = grow_pinned(c, c->pinned, small_bytes(m) + 256)) != FAME_OK) return s;
        Carver hcv(c->pinned.p);
        const Small h = carve_small(hcv, m);
        sm.hG = h.G;
        sm.hC = h.Cd;
        sm.htheta = h.theta;
        sm.hpart = h.part;
        sm.hblk = h.blk;
    }
    const uint64_t seed = 0x5eedF00Dull ^ ((uint64_t)c->n << 20) ^ (uint64_t)nev;
    const bool warm = (flags & FAME_WARM_START) && c->Y && c->Y_nev >= 1;
    const int nwarm = warm ? std::min(c->Y_nev, m) : 0;
    PhaseOut ph1, ph2;
    double2* Xfinal = nullptr;
    if (mixed) {
        float2* S[2];
        float2* AS[2];
        double2* X64[2];
        double2* AX64[2];
        for (int i = 0; i < 2; ++i) { S[i] = cv.take<float2>((size_t)k * ld); AS[i] = cv.take<float2>((size_t)k * ld); }
        for (int i = 0; i < 2; ++i) { X64[i] = cv.take<double2>((size_t)m * ld); AX64[i] = cv.take<double2>((size_t)m * ld); }
        float2* R32 = cv.take<float2>((size_t)m * ld);
        if ((s = random_block<float2>(c, S[0], m, seed, c->tf.tinv, st)) != FAME_OK) return s;
        if (warm && (s = convert<double2, float2>(c, reinterpret_cast<const double2*>(c->Y), S[0], (size_t)nwarm * ld, st)) != FAME_OK) return s;
        const double tol32 = std::max(tol, 2e-5);
        if ((s = lob_explicit<float2>(c, S, AS, sm, m, nev, tol32, max_iter, true, 1e-6, st, ph1)) != FAME_OK) return s;
        c->stats.iters_mixed = ph1.iters;
        const int left = std::max(2, max_iter - ph1.iters);
        if ((s = lob_refine(c, S, AS, X64, AX64, R32, sm, m, nev, tol, left, st, ph2)) != FAME_OK) return s;
        c->stats.iters_fp64 = ph2.iters;
        Xfinal = X64[0];
        const int left2 = max_iter - ph1.iters - ph2.iters;
        if (!ph2.converged && left2 > 0) {
            // refinement stalled above tol: complex128 blocks from the refined X
            if ((s = grow(c, c->solver2, 4 * (((size_t)k * ld * sizeof(double2) + 255)) + 256)) != FAME_OK) return s;
            Carver cv2(c->solver2.p);
            double2* S2[2];
            double2* AS2[2];
            for (int i = 0; i < 2; ++i) { S2[i] = cv2.take<double2>((size_t)k * ld); AS2[i] = cv2.take<double2>((size_t)k * ld); }
            FAME_CUDA_TRY(c, cudaMemcpyAsync(S2[0], X64[0], (size_t)m * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            PhaseOut ph3;
            if ((s = lob_explicit<double2>(c, S2, AS2, sm, m, nev, tol, left2, false, 1e-12, st, ph3)) != FAME_OK) return s;
            c->stats.iters_fp64 += ph3.iters;
            ph2.iters += ph3.iters;
            ph2.converged = ph3.converged;
            ph2.theta = ph3.theta;
            ph2.res = ph3.res;
            Xfinal = S2[0];
        }
    } else {
        double2* S[2];
        double2* AS[2];
        for (int i = 0; i < 2; ++i) { S[i] = cv.take<double2>((size_t)k * ld); AS[i] = cv.take<double2>((size_t)k * ld); }
        if ((s = random_block<double2>(c, S[0], m, seed, c->td.tinv, st)) != FAME_OK) return s;
        if (warm) FAME_CUDA_TRY(c, cudaMemcpyAsync(S[0], c->Y, (size_t)nwarm * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        if ((s = lob_explicit<double2>(c, S, AS, sm, m, nev, tol, max_iter, false, 1e-12, st, ph2)) != FAME_OK) return s;
        c->stats.iters_fp64 = ph2.iters;
        Xfinal = S[0];
    }
    c->lambda.assign(ph2.theta.begin(), ph2.theta.begin() + nev);
    double worst = 0.0;
    for (int j = 0; j < nev; ++j) worst = std::max(worst, ph2.res[j]);
    c->stats.max_residual = worst;
    if (c->Y_nev < nev) {
        if (c->Y) cudaFree(c->Y);
        c->Y = nullptr;
        c->Y_nev = 0;
        if (cudaMalloc((void**)&c->Y, (size_t)nev * ld * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, FAME_E_NOMEM, "cudaMalloc eigenvectors");
        }
        c->Y_nev = nev;
    }
    FAME_CUDA_TRY(c, cudaMemcpyAsync(c->Y, Xfinal, (size_t)nev * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    if (Y_out)
        FAME_CUDA_TRY(c, cudaMemcpyAsync(Y_out, Xfinal, (size_t)nev * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    for (int j = 0; j < nev; ++j) lambda_out[j] = c->lambda[j];
    if (iters_out) *iters_out = ph1.iters + ph2.iters;
    c->stats.rr_host_ms = c->stats_rr_ms;
    if (!ph2.converged)
        return set_err(c, FAME_E_NOCONV, "eigensolver reached max_iter; max residual " + std::to_string(worst));
    return FAME_OK;
}

// Several problems in flight at once: kBatchWorkers host threads, each with its own
// non-blocking stream, take problems from a shared counter.  While one problem waits
// for its host Rayleigh-Ritz step the GPU runs the others' kernels.  A worker lends
// its own workspace to each problem it solves, so device memory grows with the
// number of workers, not with the number of problems.
namespace {
constexpr int kBatchWorkers = 4;

struct BatchWorkspace {
    GrowBuf work, solver, solver2, partial;
};

void lend(fame_ctx* c, BatchWorkspace& w) {
    std::swap(c->work, w.work);
    std::swap(c->solver, w.solver);
    std::swap(c->solver2, w.solver2);
    std::swap(c->partial, w.partial);
}

// The eigenvectors of problem src as the start block of problem dst (same grid).
fame_status seed_from(fame_ctx* dst, const fame_ctx* src, int nev, cudaStream_t st) {
    if (!src->Y || src->Y_nev < 1) return FAME_E_STATE;
    const int k = std::min(nev, src->Y_nev);
    const size_t ld = 2 * (size_t)dst->n;
    if (dst->Y_nev < k) {
        if (dst->Y) cudaFree(dst->Y);
        dst->Y = nullptr;
        dst->Y_nev = 0;
        if (cudaMalloc((void**)&dst->Y, (size_t)nev * ld * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return FAME_E_NOMEM;
        }
        dst->Y_nev = nev;
    }
    if (cudaMemcpyAsync(dst->Y, src->Y, (size_t)k * ld * sizeof(double2), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return FAME_E_CUDA;
    }
    return FAME_OK;
}

void release(BatchWorkspace& w) {
    for (GrowBuf* b : {&w.work, &w.solver, &w.solver2, &w.partial})
        if (b->p) cudaFree(b->p);
}
}  // namespace

fame_status run_eigs_batched(fame_ctx* const* ctxs, int nprob, int nev, double tol, int max_iter,
                             int flags, double* lambda_out, int* iters_out, cudaStream_t st) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_err(nullptr, FAME_E_CUDA, "cudaGetDevice");
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, st) != cudaSuccess) {
        cudaGetLastError();
        if (ready) cudaEventDestroy(ready);
        return set_err(nullptr, FAME_E_CUDA, "batch: event on the caller's stream");
    }
    const int workers = std::min(nprob, kBatchWorkers);
    // Work items: single problems, or with FAME_WARM_START segments of band paths --
    // consecutive contexts on the same grid form a path, cut into segments of at most
    // ceil(nprob / (2 workers)) problems; inside a segment each problem starts from its
    // predecessor's eigenvectors (neighbouring Bloch vectors of a path have nearby
    // eigenvectors in the frequency coordinates), the first one from random vectors.
    const bool warm = (flags & FAME_WARM_START) != 0;
    std::vector<std::pair<int, int>> items;     // [first, last) problems
    if (warm) {
        const int seg = std::max(1, (nprob + 2 * workers - 1) / (2 * workers));
        int i = 0;
        while (i < nprob) {
            int j = i + 1;
            while (j < nprob && j - i < seg && ctxs[j]->plan.n[0] == ctxs[i]->plan.n[0] &&
                   ctxs[j]->plan.n[1] == ctxs[i]->plan.n[1] && ctxs[j]->plan.n[2] == ctxs[i]->plan.n[2] &&
                   ctxs[j]->device == ctxs[i]->device)
                ++j;
            items.emplace_back(i, j);
            i = j;
        }
    } else {
        for (int i = 0; i < nprob; ++i) items.emplace_back(i, i + 1);
    }
    const int nitems = (int)items.size();
    std::atomic<int> next(0);
    std::vector<fame_status> status(nprob, FAME_OK);
    std::vector<fame_status> wstatus(workers, FAME_OK);
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w) {
        pool.emplace_back([&, w] {
            cudaStream_t ws = nullptr;
            if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) {
                cudaGetLastError();
                wstatus[w] = FAME_E_CUDA;
                if (ws) cudaStreamDestroy(ws);
                return;
            }
            BatchWorkspace bw;
            for (;;) {
                const int t = next.fetch_add(1);
                if (t >= nitems) break;
                for (int i = items[t].first; i < items[t].second; ++i) {
                    fame_ctx* c = ctxs[i];
                    int f = flags & ~FAME_WARM_START;
                    if (i > items[t].first && status[i - 1] == FAME_OK &&
                        seed_from(c, ctxs[i - 1], nev, ws) == FAME_OK)
                        f |= FAME_WARM_START;
                    lend(c, bw);
                    int it = 0;
                    status[i] = fame_eigs(c, nev, tol, max_iter, f, lambda_out + (size_t)i * nev, nullptr, &it, ws);
                    lend(c, bw);              // the context gets its own buffers back
                    if (iters_out) iters_out[i] = it;
                }
            }
            if (cudaStreamSynchronize(ws) != cudaSuccess) wstatus[w] = FAME_E_CUDA;
            release(bw);
            cudaStreamDestroy(ws);
        });
    }
    for (auto& t : pool) t.join();
    cudaEventDestroy(ready);
    for (int w = 0; w < workers; ++w)
        if (wstatus[w] != FAME_OK) return set_err(nullptr, wstatus[w], "batch: worker stream setup failed");
    fame_status worst = FAME_OK;
    for (int i = 0; i < nprob; ++i) {
        if (status[i] == FAME_E_NOCONV) worst = FAME_E_NOCONV;
        else if (status[i] != FAME_OK) return status[i];
    }
    return worst;
}
