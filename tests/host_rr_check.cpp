// Standalone check of the host Rayleigh-Ritz solver (csrc/rr.cpp), built and run by
// test_host_rr.py with the host C++ compiler.  For a pencil with a known spectrum,
//   GB = C^H C,  GA = C^H U diag(lambda) U^H C   (C well conditioned, U unitary),
// GA c = theta GB c has exactly the eigenvalues lambda, so the solver's theta, its
// residuals and the GB-orthonormality of its vectors are checked against the
// mathematics rather than against another implementation.
//
// Usage: host_rr_check <spectrum> <k> <m> <cholesky 0|1> <seed> [total qr sweep limit]
// Prints: "theta_err <e> resid <r> orth <o> got <n>" (errors relative to max |lambda|;
// got = -2 when the implicit QR ran out of sweeps).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

int rayleigh_ritz(int k, const double* GA, const double* GB, int nwant, double drop, double* theta, double* C,
                  bool try_cholesky);
void rr_set_qr_sweep_limit(int total);

using cd = std::complex<double>;

int main(int argc, char** argv) {
    if (argc != 6 && argc != 7) return 2;
    if (argc == 7) rr_set_qr_sweep_limit(std::atoi(argv[6]));
    const char* spec = argv[1];
    const int k = std::atoi(argv[2]), m = std::atoi(argv[3]);
    const bool chol = std::atoi(argv[4]) != 0;
    std::mt19937_64 g(std::strtoull(argv[5], nullptr, 10));
    std::normal_distribution<double> N;
    std::vector<double> lam(k);
    for (int i = 0; i < k; ++i) {
        if (!std::strcmp(spec, "spread")) lam[i] = 1.0 + i + 0.3 * N(g);
        else if (!std::strcmp(spec, "triples")) lam[i] = (i < 2 * k / 3) ? 1.0 + i / 3 : 10.0 + i;
        else if (!std::strcmp(spec, "pairs9")) lam[i] = (i < 2 * k / 3) ? 1.0 + i / 2 + 1e-9 * (i % 2) : 100.0 + i;
        else if (!std::strcmp(spec, "pairs13")) lam[i] = (i < 2 * k / 3) ? 1.0 + i / 2 + 1e-13 * (i % 2) : 100.0 + i;
        else if (!std::strcmp(spec, "cluster")) lam[i] = (i < k / 2) ? 1.0 + 1e-6 * i : 1e4 + i;
        else if (!std::strcmp(spec, "flat")) lam[i] = 1.0 + 1e-8 * N(g);
        else if (!std::strcmp(spec, "graded")) lam[i] = (i % 5 == 0) ? 0.0 : std::pow(10.0, -6 + 0.3 * i);
        else return 2;
    }
    std::sort(lam.begin(), lam.end());
    // U: unitary from Gram-Schmidt of a Gaussian matrix; C = I + 0.3 G / sqrt(k)
    std::vector<cd> U((size_t)k * k), Cm((size_t)k * k);
    for (auto& x : U) x = cd(N(g), N(g));
    for (int j = 0; j < k; ++j) {
        for (int p = 0; p < j; ++p) {
            cd s = 0;
            for (int i = 0; i < k; ++i) s += std::conj(U[(size_t)p * k + i]) * U[(size_t)j * k + i];
            for (int i = 0; i < k; ++i) U[(size_t)j * k + i] -= s * U[(size_t)p * k + i];
        }
        double n = 0;
        for (int i = 0; i < k; ++i) n += std::norm(U[(size_t)j * k + i]);
        n = std::sqrt(n);
        for (int i = 0; i < k; ++i) U[(size_t)j * k + i] /= n;
    }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i)
            Cm[(size_t)j * k + i] = (i == j ? 1.0 : 0.0) + 0.3 * cd(N(g), N(g)) / std::sqrt(2.0 * k);
    // H = U diag(lam) U^H, T = H C, GA = C^H T, GB = C^H C (column-major, interleaved)
    std::vector<cd> H((size_t)k * k), T((size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            cd s = 0;
            for (int t = 0; t < k; ++t) s += U[(size_t)t * k + i] * lam[t] * std::conj(U[(size_t)t * k + j]);
            H[(size_t)j * k + i] = s;
        }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            cd s = 0;
            for (int t = 0; t < k; ++t) s += H[(size_t)t * k + i] * Cm[(size_t)j * k + t];
            T[(size_t)j * k + i] = s;
        }
    std::vector<double> GA(2 * (size_t)k * k), GB(2 * (size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            cd a = 0, b = 0;
            for (int t = 0; t < k; ++t) {
                a += std::conj(Cm[(size_t)i * k + t]) * T[(size_t)j * k + t];
                b += std::conj(Cm[(size_t)i * k + t]) * Cm[(size_t)j * k + t];
            }
            GA[2 * ((size_t)j * k + i)] = a.real();
            GA[2 * ((size_t)j * k + i) + 1] = a.imag();
            GB[2 * ((size_t)j * k + i)] = b.real();
            GB[2 * ((size_t)j * k + i) + 1] = b.imag();
        }
    std::vector<double> theta(m), C(2 * (size_t)k * m);
    const int got = rayleigh_ritz(k, GA.data(), GB.data(), m, 1e-14, theta.data(), C.data(), chol);
    double scale = 0;
    for (double x : lam) scale = std::max(scale, std::fabs(x));
    scale = std::max(scale, 1e-300);
    double terr = 0, res = 0, orth = 0;
    auto el = [&](const std::vector<double>& M, int i, int j) {
        return cd(M[2 * ((size_t)j * k + i)], M[2 * ((size_t)j * k + i) + 1]);
    };
    auto cv = [&](int j, int i) { return cd(C[2 * ((size_t)j * k + i)], C[2 * ((size_t)j * k + i) + 1]); };
    for (int j = 0; j < got; ++j) {
        terr = std::max(terr, std::fabs(theta[j] - lam[j]) / scale);
        double cn = 0;
        for (int i = 0; i < k; ++i) cn += std::norm(cv(j, i));
        cn = std::sqrt(cn);
        for (int i = 0; i < k; ++i) {
            cd ra = 0, rb = 0;
            for (int t = 0; t < k; ++t) {
                ra += el(GA, i, t) * cv(j, t);
                rb += el(GB, i, t) * cv(j, t);
            }
            res = std::max(res, std::abs(ra - theta[j] * rb) / (scale * cn));
        }
        for (int p = 0; p < got; ++p) {
            cd s = 0;
            for (int i = 0; i < k; ++i)
                for (int t = 0; t < k; ++t) s += std::conj(cv(p, i)) * el(GB, i, t) * cv(j, t);
            orth = std::max(orth, std::abs(s - (p == j ? 1.0 : 0.0)));
        }
    }
    std::printf("theta_err %.3e resid %.3e orth %.3e got %d\n", terr, res, orth, got);
    return 0;
}
