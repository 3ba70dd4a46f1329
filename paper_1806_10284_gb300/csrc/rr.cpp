// Small dense FP64 Hermitian eigenproblems for the Rayleigh-Ritz step of the
// block eigensolver.  Householder reduction of a Hermitian matrix to real
// symmetric tridiagonal form (with a diagonal unitary phase), then implicit
// symmetric QR with the Wilkinson shift (Golub and Van Loan, Matrix
// Computations, Sections 8.3.1-8.3.3).  The reflectors are kept rather than
// multiplied out, and only the wanted eigenvectors are carried back through
// them: the Rayleigh-Ritz step needs the m smallest of 3m.  The generalized pair (GA, GB) is
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

// Sweep limit of the implicit QR: 60 per matrix order by default (each eigenvalue
// deflates after a few sweeps, so this is far more than convergence takes); a
// positive value set for tests replaces it by that total.
static int g_qr_sweep_total = 0;
void rr_set_qr_sweep_limit(int total) { g_qr_sweep_total = total > 0 ? total : 0; }

namespace {

// sum_i conj(a_i) b_i and sum_i a_i b_i over split complex vectors, with four
// independent partial sums so that the additions pipeline
inline void dot_conj(int n, const double* ar, const double* ai, const double* br, const double* bi, double& sr,
                     double& si) {
    double r0 = 0, r1 = 0, r2 = 0, r3 = 0, i0 = 0, i1 = 0, i2 = 0, i3 = 0;
    int t = 0;
    for (; t + 1 < n; t += 2) {
        r0 += ar[t] * br[t];
        r1 += ai[t] * bi[t];
        i0 += ar[t] * bi[t];
        i1 -= ai[t] * br[t];
        r2 += ar[t + 1] * br[t + 1];
        r3 += ai[t + 1] * bi[t + 1];
        i2 += ar[t + 1] * bi[t + 1];
        i3 -= ai[t + 1] * br[t + 1];
    }
    if (t < n) {
        r0 += ar[t] * br[t] + ai[t] * bi[t];
        i0 += ar[t] * bi[t] - ai[t] * br[t];
    }
    sr = (r0 + r1) + (r2 + r3);
    si = (i0 + i1) + (i2 + i3);
}
inline void dot_plain(int n, const double* ar, const double* ai, const double* br, const double* bi, double& sr,
                      double& si) {
    double r0 = 0, r1 = 0, r2 = 0, r3 = 0, i0 = 0, i1 = 0, i2 = 0, i3 = 0;
    int t = 0;
    for (; t + 1 < n; t += 2) {
        r0 += ar[t] * br[t];
        r1 -= ai[t] * bi[t];
        i0 += ar[t] * bi[t];
        i1 += ai[t] * br[t];
        r2 += ar[t + 1] * br[t + 1];
        r3 -= ai[t + 1] * bi[t + 1];
        i2 += ar[t + 1] * bi[t + 1];
        i3 += ai[t + 1] * br[t + 1];
    }
    if (t < n) {
        r0 += ar[t] * br[t] - ai[t] * bi[t];
        i0 += ar[t] * bi[t] + ai[t] * br[t];
    }
    sr = (r0 + r1) + (r2 + r3);
    si = (i0 + i1) + (i2 + i3);
}

// implicit symmetric QR on the tridiagonal (d, e) with the Wilkinson shift from the
// trailing 2 x 2 block, deflation where |e_i| <= eps (|d_i| + |d_i+1|); the
// rotations are accumulated into Z.  Returns false if the sweep limit ran out
// before every off-diagonal entry was deflated.
bool tridiag_qr(int k, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Z) {
    // d[0..k-1] diagonal, e[0..k-2] off-diagonal; Z (k x k, column-major) accumulates rotations
    const double eps = 2.220446049250313e-16;
    int hi = k - 1;
    int guard = 0;
    const int limit = g_qr_sweep_total > 0 ? g_qr_sweep_total : 60 * k;
    while (hi > 0) {
        if (guard >= limit) return false;
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
            // |(x, z)|: the plain root where the squares neither overflow nor underflow
            double r = std::sqrt(x * x + z * z);
            if (!(r > 1e-150 && r < 1e150)) r = std::hypot(x, z);
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
            double* __restrict__ zi = &Z[(size_t)i * k];
            double* __restrict__ zj = &Z[(size_t)(i + 1) * k];
            for (int t = 0; t < k; ++t) {
                const double u = zi[t], v = zj[t];
                zi[t] = c * u + s * v;
                zj[t] = -s * u + c * v;
            }
        }
    }
    return true;
}

}  // namespace

bool herm_eig_n(int k, const double* Ain, double* w, double* Vout, int nvec);

bool herm_eig(int k, const double* Ain, double* w, double* Vout) { return herm_eig_n(k, Ain, w, Vout, k); }

// as herm_eig, eigenvectors of the nvec smallest eigenvalues only (all k eigenvalues);
// false if the tridiagonal QR did not converge (the outputs are then not eigenpairs)
bool herm_eig_n(int k, const double* Ain, double* w, double* Vout, int nvec) {
    // real and imaginary parts, column-major, lower triangle used; the reflector
    // H_j = I - beta_j v_j v_j^H maps column j below the diagonal onto -phase alpha e_1
    std::vector<double> ar((size_t)k * k), ai((size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = j; i < k; ++i) {
            ar[(size_t)j * k + i] = Ain[2 * ((size_t)j * k + i)];
            ai[(size_t)j * k + i] = (i == j) ? 0.0 : Ain[2 * ((size_t)j * k + i) + 1];
        }
    auto AR = [&](int i, int j) -> double& { return ar[(size_t)j * k + i]; };
    auto AI = [&](int i, int j) -> double& { return ai[(size_t)j * k + i]; };
    std::vector<double> vr((size_t)k * k, 0.0), vi((size_t)k * k, 0.0), betas(k, 0.0);   // reflectors
    std::vector<double> pr(k), pi(k);
    for (int j = 0; j + 2 < k; ++j) {
        const int o = j + 1;
        double alpha = 0.0;
        for (int i = o; i < k; ++i) alpha += AR(i, j) * AR(i, j) + AI(i, j) * AI(i, j);
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        const double x0r = AR(o, j), x0i = AI(o, j), ax0 = std::hypot(x0r, x0i);
        const double phr = (ax0 == 0.0) ? 1.0 : x0r / ax0, phi = (ax0 == 0.0) ? 0.0 : x0i / ax0;
        double* v_r = &vr[(size_t)j * k];
        double* v_i = &vi[(size_t)j * k];
        for (int i = o; i < k; ++i) { v_r[i] = AR(i, j); v_i[i] = AI(i, j); }
        v_r[o] += phr * alpha;
        v_i[o] += phi * alpha;
        double vv = 0.0;
        for (int i = o; i < k; ++i) vv += v_r[i] * v_r[i] + v_i[i] * v_i[i];
        if (vv == 0.0) continue;
        const double beta = 2.0 / vv;
        betas[j] = beta;
        // p = beta A22 v, A22 Hermitian from its lower triangle
        for (int i = o; i < k; ++i) { pr[i] = 0.0; pi[i] = 0.0; }
        for (int t = o; t < k; ++t) {
            const double vtr = v_r[t], vti = v_i[t];
            // diagonal
            pr[t] += AR(t, t) * vtr;
            pi[t] += AR(t, t) * vti;
            const double* cr = &ar[(size_t)t * k];
            const double* ci = &ai[(size_t)t * k];
            for (int i = t + 1; i < k; ++i) {                // p_i += A(i,t) v_t
                pr[i] += cr[i] * vtr - ci[i] * vti;
                pi[i] += cr[i] * vti + ci[i] * vtr;
            }
            double sr, si;                                    // p_t += sum_i conj(A(i,t)) v_i
            dot_conj(k - t - 1, cr + t + 1, ci + t + 1, v_r + t + 1, v_i + t + 1, sr, si);
            pr[t] += sr;
            pi[t] += si;
        }
        double Kr = 0.0, Ki = 0.0;                          // K = (beta/2) v^H p (p before scaling by beta)
        for (int i = o; i < k; ++i) {
            pr[i] *= beta;
            pi[i] *= beta;
            Kr += v_r[i] * pr[i] + v_i[i] * pi[i];
            Ki += v_r[i] * pi[i] - v_i[i] * pr[i];
        }
        Kr *= 0.5 * beta;
        Ki *= 0.5 * beta;
        for (int i = o; i < k; ++i) {                       // q = p - K v (stored in p)
            const double qr = pr[i] - (Kr * v_r[i] - Ki * v_i[i]);
            const double qi = pi[i] - (Kr * v_i[i] + Ki * v_r[i]);
            pr[i] = qr;
            pi[i] = qi;
        }
        for (int t = o; t < k; ++t) {                       // lower triangle: A -= v q^H + q v^H
            const double vtr = v_r[t], vti = v_i[t], qtr = pr[t], qti = pi[t];
            double* cr = &ar[(size_t)t * k];
            double* ci = &ai[(size_t)t * k];
            for (int i = t; i < k; ++i) {
                cr[i] -= (v_r[i] * qtr + v_i[i] * qti) + (pr[i] * vtr + pi[i] * vti);
                ci[i] -= (v_i[i] * qtr - v_r[i] * qti) + (pi[i] * vtr - pr[i] * vti);
            }
        }
        AR(o, j) = -phr * alpha;
        AI(o, j) = -phi * alpha;
    }
    // real tridiagonal through the diagonal phase: T_real = D^H T D
    std::vector<double> d(k), e(std::max(k - 1, 1), 0.0), phr(k), phi(k);
    phr[0] = 1.0;
    phi[0] = 0.0;
    for (int i = 0; i < k; ++i) d[i] = AR(i, i);
    for (int i = 0; i + 1 < k; ++i) {
        const double er = AR(i + 1, i), ei = AI(i + 1, i), m = std::hypot(er, ei);
        e[i] = m;
        if (m == 0.0) { phr[i + 1] = phr[i]; phi[i + 1] = phi[i]; }
        else {
            phr[i + 1] = (phr[i] * er - phi[i] * ei) / m;
            phi[i + 1] = (phr[i] * ei + phi[i] * er) / m;
        }
    }
    std::vector<double> Z((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) Z[(size_t)i * k + i] = 1.0;
    bool converged = true;
    if (k > 1) converged = tridiag_qr(k, d, e, Z);
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
    for (int i = 0; i < k; ++i) w[i] = d[order[i]];
    // V = H_0 ... H_{k-3} D Z: phase, then the reflectors in reverse order
    std::vector<double> yr(k), yi(k);
    for (int c = 0; c < nvec; ++c) {
        const double* z = &Z[(size_t)order[c] * k];
        for (int i = 0; i < k; ++i) { yr[i] = phr[i] * z[i]; yi[i] = phi[i] * z[i]; }
        for (int j = k - 3; j >= 0; --j) {
            if (betas[j] == 0.0) continue;
            const double* v_r = &vr[(size_t)j * k];
            const double* v_i = &vi[(size_t)j * k];
            double sr, si;                                    // s = v^H y
            dot_conj(k - j - 1, v_r + j + 1, v_i + j + 1, yr.data() + j + 1, yi.data() + j + 1, sr, si);
            sr *= betas[j];
            si *= betas[j];
            for (int i = j + 1; i < k; ++i) {
                yr[i] -= v_r[i] * sr - v_i[i] * si;
                yi[i] -= v_r[i] * si + v_i[i] * sr;
            }
        }
        for (int i = 0; i < k; ++i) {
            Vout[2 * ((size_t)c * k + i)] = yr[i];
            Vout[2 * ((size_t)c * k + i) + 1] = yi[i];
        }
    }
    return converged;
}

namespace {

// Rayleigh-Ritz through the Cholesky factor of the diagonally scaled GB (unit
// diagonal): Bs = L L^H, M = L^{-1} As L^{-H}, C = D L^{-H} Y.  Declines (returns
// false) when a pivot falls below kMinPivot, i.e. when GB is too close to singular
// for the factor to be trusted; the caller then takes the SVQB route.
bool rr_cholesky(int k, const double* GA, const double* GB, const std::vector<double>& dsc, int nwant,
                 double* theta, double* C, int* nout, bool* qr_ok) {
    constexpr double kMinPivot = 1e-4;
    const size_t kk = (size_t)k * k;
    // L row-major (real and imaginary parts), lower triangle, row by row
    std::vector<double> Lr(kk, 0.0), Li(kk, 0.0), inv(k);
    for (int i = 0; i < k; ++i) {
        const double* ar = &Lr[(size_t)i * k];
        const double* ai = &Li[(size_t)i * k];
        for (int j = 0; j <= i; ++j) {
            const size_t o = 2 * ((size_t)j * k + i);               // GB(i, j), lower triangle as given
            const double sc = dsc[i] * dsc[j];
            double sr = GB[o] * sc, si = (i == j) ? 0.0 : GB[o + 1] * sc;
            double dr, di;                                           // - sum_t L(i,t) conj(L(j,t))
            dot_conj(j, &Lr[(size_t)j * k], &Li[(size_t)j * k], ar, ai, dr, di);
            sr -= dr;
            si -= di;
            if (i == j) {
                if (!(sr > kMinPivot)) return false;
                const double l = std::sqrt(sr);
                Lr[(size_t)i * k + i] = l;
                inv[i] = 1.0 / l;
            } else {
                Lr[(size_t)i * k + j] = sr * inv[j];
                Li[(size_t)i * k + j] = si * inv[j];
            }
        }
    }
    // forward substitution x = L^{-1} b in place on one column (real and imaginary parts)
    auto lsolve = [&](double* xr, double* xi) {
        for (int i = 0; i < k; ++i) {
            const double* ar = &Lr[(size_t)i * k];
            const double* ai = &Li[(size_t)i * k];
            double sr, si;
            dot_plain(i, ar, ai, xr, xi, sr, si);
            xr[i] = (xr[i] - sr) * inv[i];
            xi[i] = (xi[i] - si) * inv[i];
        }
    };
    // Y = L^{-1} As column by column (As Hermitian from its lower triangle), column-major
    std::vector<double> Yr(kk), Yi(kk);
    for (int c = 0; c < k; ++c) {
        double* yr = &Yr[(size_t)c * k];
        double* yi = &Yi[(size_t)c * k];
        for (int i = 0; i < k; ++i) {
            const double sc = dsc[i] * dsc[c];
            if (i >= c) {
                const size_t o = 2 * ((size_t)c * k + i);
                yr[i] = GA[o] * sc;
                yi[i] = (i == c) ? 0.0 : GA[o + 1] * sc;
            } else {
                const size_t o = 2 * ((size_t)i * k + c);
                yr[i] = GA[o] * sc;
                yi[i] = -GA[o + 1] * sc;
            }
        }
        lsolve(yr, yi);
    }
    // M = L^{-1} Y^H = L^{-1} As L^{-H}; column r from row r of Y, conjugated
    std::vector<double> M(2 * kk);
    std::vector<double> wr(k), wi(k);
    for (int r = 0; r < k; ++r) {
        for (int i = 0; i < k; ++i) {
            wr[i] = Yr[(size_t)i * k + r];
            wi[i] = -Yi[(size_t)i * k + r];
        }
        lsolve(wr.data(), wi.data());
        for (int i = 0; i < k; ++i) {
            M[2 * ((size_t)r * k + i)] = wr[i];
            M[2 * ((size_t)r * k + i) + 1] = wi[i];
        }
    }
    const int nv = std::min(nwant, k);
    std::vector<double> th(k), V(2 * (size_t)k * nv);
    *qr_ok = herm_eig_n(k, M.data(), th.data(), V.data(), nv);
    // C = D L^{-H} V (back substitution with L^H)
    for (int j = 0; j < nv; ++j) {
        theta[j] = th[j];
        for (int i = k - 1; i >= 0; --i) {
            double vr = V[2 * ((size_t)j * k + i)], vi = V[2 * ((size_t)j * k + i) + 1];
            for (int t = i + 1; t < k; ++t) {                        // - conj(L(t,i)) z_t
                const double lr = Lr[(size_t)t * k + i], li = Li[(size_t)t * k + i];
                const double zr = wr[t], zi = wi[t];
                vr -= lr * zr + li * zi;
                vi -= lr * zi - li * zr;
            }
            wr[i] = vr * inv[i];
            wi[i] = vi * inv[i];
        }
        for (int i = 0; i < k; ++i) {
            C[2 * ((size_t)j * k + i)] = wr[i] * dsc[i];
            C[2 * ((size_t)j * k + i) + 1] = wi[i] * dsc[i];
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
    bool qr_ok = true;
    if (try_cholesky && rr_cholesky(k, GA, GB, dsc, nwant, theta, C, &nout, &qr_ok))
        return qr_ok ? nout : kRRNoConv;
    std::vector<double> Bs(2 * (size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            const size_t o = 2 * ((size_t)j * k + i);
            Bs[o] = GB[o] * dsc[i] * dsc[j];
            Bs[o + 1] = GB[o + 1] * dsc[i] * dsc[j];
        }
    std::vector<double> mu(k), U(2 * (size_t)k * k);
    if (!herm_eig(k, Bs.data(), mu.data(), U.data())) return kRRNoConv;
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
    if (!herm_eig_n(kk, M.data(), th.data(), V.data(), nout)) return kRRNoConv;
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
