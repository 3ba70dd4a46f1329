// Small dense FP64 Hermitian eigenproblems for the Rayleigh-Ritz step of the
// block eigensolver.  Householder reduction of a Hermitian matrix to real
// symmetric tridiagonal form (with a diagonal unitary phase), then implicit
// symmetric QR with the Wilkinson shift (Golub and Van Loan, Matrix
// Computations, Sections 8.3.1-8.3.3).  The generalized pair (GA, GB) is
// reduced to a standard problem on a GB-orthonormal basis built from the
// Cholesky factor of the diagonally scaled GB when it is well conditioned, else
// from the eigen-decomposition of the scaled GB, dropping numerically dependent
// directions (the SVQB step of Stathopoulos and Wu, 2002).
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "fame_internal.h"

using cd = std::complex<double>;

namespace {

// column-major k x k complex matrix helpers
inline cd& at(std::vector<cd>& A, int k, int i, int j) { return A[(size_t)j * k + i]; }

void tridiag_qr(int k, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Z) {
    // d[0..k-1] diagonal, e[0..k-2] off-diagonal; Z (k x k, column-major) accumulates rotations
    const double eps = 2.220446049250313e-16;
    int hi = k - 1;
    int guard = 0;
    while (hi > 0 && guard < 60 * k) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
        ++guard;
        // Wilkinson shift from the trailing 2x2 block
        const double delta = 0.5 * (d[hi - 1] - d[hi]);
        const double b2 = e[hi - 1] * e[hi - 1];
        const double sgn = (delta >= 0.0) ? 1.0 : -1.0;
        const double mu = d[hi] - b2 / (delta + sgn * std::sqrt(delta * delta + b2));
        double x = d[lo] - mu, z = e[lo];
        for (int i = lo; i < hi; ++i) {
            const double r = std::hypot(x, z);
            const double c = (r == 0.0) ? 1.0 : x / r;
            const double s = (r == 0.0) ? 0.0 : z / r;
            if (i > lo) e[i - 1] = r;
            const double a = d[i], b = e[i], dd = d[i + 1];
            d[i] = c * c * a + 2.0 * c * s * b + s * s * dd;
            d[i + 1] = s * s * a - 2.0 * c * s * b + c * c * dd;
            e[i] = c * s * (dd - a) + (c * c - s * s) * b;
            if (i + 1 < hi) {
                z = s * e[i + 1];
                e[i + 1] = c * e[i + 1];
            }
            x = e[i];
            double* zi = &Z[(size_t)i * k];
            double* zj = &Z[(size_t)(i + 1) * k];
            for (int t = 0; t < k; ++t) {
                const double u = zi[t], v = zj[t];
                zi[t] = c * u + s * v;
                zj[t] = -s * u + c * v;
            }
        }
    }
}

}  // namespace

void herm_eig_n(int k, const double* Ain, double* w, double* Vout, int nvec);

void herm_eig(int k, const double* Ain, double* w, double* Vout) { herm_eig_n(k, Ain, w, Vout, k); }

// as herm_eig, eigenvectors of the nvec smallest eigenvalues only (all k eigenvalues)
void herm_eig_n(int k, const double* Ain, double* w, double* Vout, int nvec) {
    std::vector<cd> A((size_t)k * k), Q((size_t)k * k, cd(0.0));
    for (size_t i = 0; i < (size_t)k * k; ++i) A[i] = cd(Ain[2 * i], Ain[2 * i + 1]);
    // Hermitise (use the lower triangle as given)
    for (int j = 0; j < k; ++j) {
        at(A, k, j, j) = cd(at(A, k, j, j).real(), 0.0);
        for (int i = j + 1; i < k; ++i) at(A, k, j, i) = std::conj(at(A, k, i, j));
    }
    for (int i = 0; i < k; ++i) at(Q, k, i, i) = 1.0;
    std::vector<cd> v(k), p(k), qv(k);
    for (int j = 0; j + 2 < k; ++j) {
        const int len = k - j - 1;
        double alpha = 0.0;
        for (int i = 0; i < len; ++i) alpha += std::norm(at(A, k, j + 1 + i, j));
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        const cd x0 = at(A, k, j + 1, j);
        const cd ph = (std::abs(x0) == 0.0) ? cd(1.0) : x0 / std::abs(x0);
        for (int i = 0; i < len; ++i) v[i] = at(A, k, j + 1 + i, j);
        v[0] += ph * alpha;
        double vv = 0.0;
        for (int i = 0; i < len; ++i) vv += std::norm(v[i]);
        if (vv == 0.0) continue;
        const double beta = 2.0 / vv;
        // p = beta * A22 v
        for (int i = 0; i < len; ++i) {
            cd s = 0.0;
            for (int t = 0; t < len; ++t) s += at(A, k, j + 1 + i, j + 1 + t) * v[t];
            p[i] = beta * s;
        }
        cd K = 0.0;
        for (int i = 0; i < len; ++i) K += std::conj(v[i]) * p[i];
        K *= 0.5 * beta;
        for (int i = 0; i < len; ++i) qv[i] = p[i] - K * v[i];
        for (int t = 0; t < len; ++t)
            for (int i = 0; i < len; ++i)
                at(A, k, j + 1 + i, j + 1 + t) -= v[i] * std::conj(qv[t]) + qv[i] * std::conj(v[t]);
        at(A, k, j + 1, j) = -ph * alpha;
        at(A, k, j, j + 1) = std::conj(-ph * alpha);
        for (int i = 1; i < len; ++i) { at(A, k, j + 1 + i, j) = 0.0; at(A, k, j, j + 1 + i) = 0.0; }
        // Q <- Q H on columns j+1..k-1
        for (int r = 0; r < k; ++r) {
            cd s = 0.0;
            for (int t = 0; t < len; ++t) s += at(Q, k, r, j + 1 + t) * v[t];
            s *= beta;
            for (int t = 0; t < len; ++t) at(Q, k, r, j + 1 + t) -= s * std::conj(v[t]);
        }
    }
    // real tridiagonal through the diagonal phase D: T_real = D^H T D
    std::vector<double> d(k), e(std::max(k - 1, 1));
    std::vector<cd> ph(k);
    ph[0] = 1.0;
    for (int i = 0; i < k; ++i) d[i] = at(A, k, i, i).real();
    for (int i = 0; i + 1 < k; ++i) {
        const cd ec = at(A, k, i + 1, i);
        const double m = std::abs(ec);
        e[i] = m;
        ph[i + 1] = (m == 0.0) ? ph[i] : ph[i] * ec / m;
    }
    std::vector<double> Z((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) Z[(size_t)i * k + i] = 1.0;
    if (k > 1) tridiag_qr(k, d, e, Z);
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
    // V = Q D Z
    for (int jj = 0; jj < k; ++jj) w[jj] = d[order[jj]];
    for (int jj = 0; jj < nvec; ++jj) {
        const int j = order[jj];
        for (int r = 0; r < k; ++r) {
            cd s = 0.0;
            for (int t = 0; t < k; ++t) s += at(Q, k, r, t) * ph[t] * Z[(size_t)j * k + t];
            Vout[2 * ((size_t)jj * k + r)] = s.real();
            Vout[2 * ((size_t)jj * k + r) + 1] = s.imag();
        }
    }
}

namespace {

// Rayleigh-Ritz through the Cholesky factor of the diagonally scaled GB (unit
// diagonal): Bs = L L^H, M = L^{-1} As L^{-H}, C = D L^{-H} Y.  Declines (returns
// false) when a pivot falls below kMinPivot, i.e. when GB is too close to singular
// for the factor to be trusted; the caller then takes the SVQB route.
bool rr_cholesky(int k, const double* GA, const double* GB, const std::vector<double>& dsc, int nwant,
                 double* theta, double* C, int* nout) {
    constexpr double kMinPivot = 1e-4;
    auto el = [k](const double* G, const std::vector<double>& s, int i, int j) {
        const size_t o = 2 * ((size_t)j * k + i);
        return cd(G[o], G[o + 1]) * (s[i] * s[j]);
    };
    std::vector<cd> L((size_t)k * k, cd(0.0));         // column-major lower triangle
    for (int j = 0; j < k; ++j) {
        double djj = el(GB, dsc, j, j).real();
        for (int t = 0; t < j; ++t) djj -= std::norm(L[(size_t)t * k + j]);
        if (!(djj > kMinPivot)) return false;
        const double ljj = std::sqrt(djj);
        L[(size_t)j * k + j] = ljj;
        for (int i = j + 1; i < k; ++i) {
            cd sum = el(GB, dsc, i, j);                    // lower triangle as given (i > j)
            for (int t = 0; t < j; ++t) sum -= L[(size_t)t * k + i] * std::conj(L[(size_t)t * k + j]);
            L[(size_t)j * k + i] = sum / ljj;
        }
    }
    // X = L^{-1} As (As Hermitian from its lower triangle), column by column
    std::vector<cd> X((size_t)k * k);
    for (int c = 0; c < k; ++c) {
        for (int i = 0; i < k; ++i) {
            cd v = (i >= c) ? el(GA, dsc, i, c) : std::conj(el(GA, dsc, c, i));
            if (i == c) v = cd(v.real(), 0.0);
            for (int t = 0; t < i; ++t) v -= L[(size_t)t * k + i] * X[(size_t)c * k + t];
            X[(size_t)c * k + i] = v / L[(size_t)i * k + i].real();
        }
    }
    // M = X L^{-H} = (L^{-1} X^H)^H; only the lower triangle is read by herm_eig
    std::vector<double> M(2 * (size_t)k * k, 0.0);
    std::vector<cd> col(k);
    for (int r = 0; r < k; ++r) {                          // column r of L^{-1} X^H
        for (int i = 0; i < k; ++i) {
            cd v = std::conj(X[(size_t)i * k + r]);
            for (int t = 0; t < i; ++t) v -= L[(size_t)t * k + i] * col[t];
            col[i] = v / L[(size_t)i * k + i].real();
        }
        for (int i = r; i < k; ++i) {                      // M(i, r) = conj(col[i]) ... row r of the product
            const cd m = std::conj(col[i]);
            M[2 * ((size_t)i * k + r)] = m.real();         // entry (r, i): upper; mirror to (i, r)
            M[2 * ((size_t)i * k + r) + 1] = m.imag();
            M[2 * ((size_t)r * k + i)] = m.real();
            M[2 * ((size_t)r * k + i) + 1] = -m.imag();
        }
    }
    const int nv = std::min(nwant, k);
    std::vector<double> th(k), Y(2 * (size_t)k * k);
    herm_eig_n(k, M.data(), th.data(), Y.data(), nv);
    // C = D L^{-H} Y (back substitution with L^H)
    std::vector<cd> z(k);
    for (int j = 0; j < nv; ++j) {
        theta[j] = th[j];
        for (int i = k - 1; i >= 0; --i) {
            cd v(Y[2 * ((size_t)j * k + i)], Y[2 * ((size_t)j * k + i) + 1]);
            for (int t = i + 1; t < k; ++t) v -= std::conj(L[(size_t)i * k + t]) * z[t];
            z[i] = v / L[(size_t)i * k + i].real();
        }
        for (int i = 0; i < k; ++i) {
            const cd v = z[i] * dsc[i];
            C[2 * ((size_t)j * k + i)] = v.real();
            C[2 * ((size_t)j * k + i) + 1] = v.imag();
        }
    }
    *nout = nv;
    return true;
}

}  // namespace

int rayleigh_ritz(int k, const double* GA, const double* GB, int nwant, double drop, double* theta,
                  double* C, bool try_cholesky) {
    std::vector<double> dsc(k);
    for (int i = 0; i < k; ++i) {
        const double b = GB[2 * ((size_t)i * k + i)];
        dsc[i] = (b > 0.0) ? 1.0 / std::sqrt(b) : 0.0;
    }
    int nout = 0;
    if (try_cholesky && rr_cholesky(k, GA, GB, dsc, nwant, theta, C, &nout)) return nout;
    std::vector<double> Bs(2 * (size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            const size_t o = 2 * ((size_t)j * k + i);
            Bs[o] = GB[o] * dsc[i] * dsc[j];
            Bs[o + 1] = GB[o + 1] * dsc[i] * dsc[j];
        }
    std::vector<double> mu(k), U(2 * (size_t)k * k);
    herm_eig(k, Bs.data(), mu.data(), U.data());
    const double mmax = std::max(mu[k - 1], 1e-300);
    std::vector<int> keep;
    for (int i = 0; i < k; ++i)
        if (mu[i] > drop * mmax) keep.push_back(i);
    const int kk = (int)keep.size();
    // Z = D U_keep diag(mu^{-1/2})   (k x kk)
    std::vector<cd> Zm((size_t)k * kk);
    for (int jj = 0; jj < kk; ++jj) {
        const int j = keep[jj];
        const double sc = 1.0 / std::sqrt(mu[j]);
        for (int i = 0; i < k; ++i)
            Zm[(size_t)jj * k + i] = cd(U[2 * ((size_t)j * k + i)], U[2 * ((size_t)j * k + i) + 1]) * (dsc[i] * sc);
    }
    // M = Z^H GA Z
    std::vector<cd> T((size_t)k * kk);
    for (int jj = 0; jj < kk; ++jj)
        for (int i = 0; i < k; ++i) {
            cd s = 0.0;
            for (int t = 0; t < k; ++t)
                s += cd(GA[2 * ((size_t)t * k + i)], GA[2 * ((size_t)t * k + i) + 1]) * Zm[(size_t)jj * k + t];
            T[(size_t)jj * k + i] = s;
        }
    std::vector<double> M(2 * (size_t)kk * kk);
    for (int jj = 0; jj < kk; ++jj)
        for (int ii = 0; ii < kk; ++ii) {
            cd s = 0.0;
            for (int t = 0; t < k; ++t) s += std::conj(Zm[(size_t)ii * k + t]) * T[(size_t)jj * k + t];
            M[2 * ((size_t)jj * kk + ii)] = s.real();
            M[2 * ((size_t)jj * kk + ii) + 1] = s.imag();
        }
    std::vector<double> th(kk), V(2 * (size_t)kk * kk);
    nout = std::min(nwant, kk);
    herm_eig_n(kk, M.data(), th.data(), V.data(), nout);
    for (int j = 0; j < nout; ++j) {
        theta[j] = th[j];
        for (int i = 0; i < k; ++i) {
            cd s = 0.0;
            for (int t = 0; t < kk; ++t)
                s += Zm[(size_t)t * k + i] * cd(V[2 * ((size_t)j * kk + t)], V[2 * ((size_t)j * kk + t) + 1]);
            C[2 * ((size_t)j * k + i)] = s.real();
            C[2 * ((size_t)j * k + i) + 1] = s.imag();
        }
    }
    return nout;
}
