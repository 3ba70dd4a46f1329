// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fame.h"

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename R> struct cpx;
template <> struct cpx<float> { using T = float2; };
template <> struct cpx<double> { using T = double2; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
template <typename C>
__host__ __device__ __forceinline__ C cmulc(C a, C b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
template <typename C>
__host__ __device__ __forceinline__ C conjc(C a) { return mk(a.x, -a.y); }

// ---------------------------------------------------------------------------
// Lattice plan (Section 2.2)
// ---------------------------------------------------------------------------
struct LatticePlan {
    int n[3];
    int perm[3];
    int m[3];
    int rho[3];
    int s[3];
    double delta[3];
    double a[3][3];      // a[row][col]: column l is a_l of eq. (transvec)
    double kappa[3];
    double len[3];
    double cos_in[3];    // gamma', beta', alpha'
    double cos_c[3];     // corrected gamma, beta, alpha
};

// Returns an empty string on success, else the reason.
std::string build_lattice(const double* a1, const double* a2, const double* a3, int n1, int n2,
                          int n3, const double* bloch, LatticePlan* out);
void compute_kappa(const double* a1, const double* a2, const double* a3, const double* bloch,
                   LatticePlan* plan);
// radix list of a length (factors 8, 4, 2, 3, 5); empty if unsupported
std::vector<int> radix_list(int L);

// ---------------------------------------------------------------------------
// Per-axis FFT plan, passed to kernels by value.
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 12;
struct AxisPlan {
    int L;
    int nst;
    int radix[kMaxStages];
};

// Twist-fraction representation.  For complex64 kernels a fraction f in
// [0, 1) is split into hi (a multiple of 2^-13) and lo = f - hi so that
// products idx * hi with idx < 1024 are exact in float.
struct Frac32 { float hi, lo; };

template <typename R> struct FracT;
template <> struct FracT<float> { using T = Frac32; };
template <> struct FracT<double> { using T = double; };

// Everything a transform kernel needs about one (lattice, k).
template <typename R>
struct KParams {
    int n1, n2, n3;
    R inv_dx, inv_dy, inv_dz;
    typename FracT<R>::T f1;           // c1 / n1 mod 1
    const typename FracT<R>::T* f2;    // [n1]   c2(p) / n2 mod 1
    const typename FracT<R>::T* f3;    // [n2][n1] c3(p, q) / n3 mod 1
    const typename cpx<R>::T* tw[3];   // per-axis e^{-2 pi i t / L}
    AxisPlan ax[3];
    const R* invB;                     // [3][n] 1/B
    const uint32_t* alt;               // [ceil(n/32)] reference-vector decision bits
    R scale;                           // 1/n for a full apply
    // twist and Lambda_3 tables evaluated once per (lattice, k) in FP64
    const typename cpx<R>::T* tw3;     // [n3][n2][n1] e^{2 pi i c f3(p, q)}, c the z index
    const typename cpx<R>::T* lam3;    // [n3][n2][n1] Lambda_3 at frequency (p, q, r)
    const typename cpx<R>::T* tw2;     // [n2][n1] e^{2 pi i b f2(p)}, b the y index
    const typename cpx<R>::T* tw1;     // [n1] e^{2 pi i a f1}, a the x index
    // Z-in expands Lambda x (Pi_r y) / Lambda_q instead of Sigma_r Pi_r y: the left
    // singular vectors P_r y (eq. SVD) of the H field; the generic kernels only
    int curl;
};

// Device tables of one precision.
template <typename R>
struct DevTables {
    typename FracT<R>::T* f2 = nullptr;
    typename FracT<R>::T* f3 = nullptr;
    typename cpx<R>::T* tw[3] = {nullptr, nullptr, nullptr};
    R* invB = nullptr;
    R* tinv = nullptr;   // [n] preconditioner 1/(Lambda_q mean(1/B)), 0 where Lambda_q = 0
    typename cpx<R>::T* tw3 = nullptr;
    typename cpx<R>::T* lam3 = nullptr;
    typename cpx<R>::T* tw2 = nullptr;
    typename cpx<R>::T* tw1 = nullptr;
    typename FracT<R>::T f1;
};

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct GrowBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Launch choices of the A_r apply (0 = automatic): Z-pass kernel family (1 fixed-length,
// 2 two-level, 3 Stockham), XY kernel family (1 fixed-length, 2 two-level plane,
// 3 Stockham plane, 4 split y / x / y passes), vectors per Z-pass block.
struct ApplyPlan {
    int zfam = 0, xyfam = 0, vpc = 0;
};

struct fame_ctx {
    LatticePlan plan;
    double in_vec[3][3];           // the primitive vectors as given (for kappa)
    int device = 0;
    long long n = 0;
    DevTables<float> tf;
    DevTables<double> td;
    uint32_t* alt_mask = nullptr;  // reference-vector decision per frequency (FP64)
    bool eps_set = false;
    // complex128 applies of the current solve in double-float arithmetic (set per solve)
    bool df128 = false;
    double mean_invB = 0.0;
    double min_invB = 0.0, max_invB = 0.0;   // spectrum bounds of Q_r^* B^{-1} Q_r
    GrowBuf cheb;                  // Chebyshev preconditioner blocks (complex64)
    GrowBuf work;                  // transform workspace [m][3][n] complex
    ApplyPlan apply_plan[2];       // per dtype (FAME_C64, FAME_C128), set by fame_set_apply_plan / fame_autotune
    // solver state
    std::vector<double> lambda;    // last eigenvalues
    double* Y = nullptr;           // device [nev][2][n] complex128 eigenvectors
    int Y_nev = 0;
    GrowBuf solver;                // solver blocks
    GrowBuf solver2;               // complex128 blocks of the fallback phase (on demand)
    GrowBuf partial;               // Gram partial sums
    GrowBuf pinned;                // page-locked host mirror of the solver's small buffers
    GrowBuf tcerr;                 // device flag: a bounded wait of a tensor-core kernel gave up (sticky)
    fame_solve_stats stats{};
    double stats_rr_ms = 0.0;
    std::string err;
};

// error helpers
fame_status set_err(fame_ctx* c, fame_status s, const std::string& msg);
#define FAME_CUDA_TRY(ctx, call)                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_err((ctx), FAME_E_CUDA,                                               \
                           std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

fame_status grow(fame_ctx* c, GrowBuf& b, size_t bytes);
// raise a kernel's dynamic shared-memory limit to smem (never lowered; thread safe) and
// prefer the largest shared-memory carveout
fame_status kernel_smem(fame_ctx* c, const void* fn, size_t smem);
fame_status grow_pinned(fame_ctx* c, GrowBuf& b, size_t bytes);   // page-locked host memory
void count_launch(int k = 1);

// kernel kinds for the opt-in profiler (profile.cpp)
enum KernelKind { K_ZIN, K_XY, K_ZOUT, K_YPASS, K_XPASS, K_GRAM, K_GRAM_RED, K_COMBINE, K_RESID,
                  K_CONVERT, K_GRAD, K_SETUP, K_GRAM_HERM, K_ORTH, K_COMBINE_DF, K_PRECOND,
                  K_ZIN_DF, K_XY_DF, K_ZOUT_DF, K_COUNT };
// Brackets a launch with events on its stream when profiling is on; attaches the
// launch's algorithmic bytes and flops.
// NVTX range on the calling host thread (header-only NVTX 3: a no-op branch unless a
// profiler such as Nsight Systems or Nsight Compute is attached).  The solver marks
// its phases with these, and every ProfScope marks its kernel pass.
class NvtxRange {
  public:
    explicit NvtxRange(const char* name);
    ~NvtxRange();
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

class ProfScope {
  public:
    ProfScope(int kind, bool dbl, cudaStream_t st, double bytes, double flops = 0.0);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
  private:
    int id_;
    cudaStream_t st_;
    double bytes_, flops_;
    cudaEvent_t ev_;
};

// tables (plan.cpp / tables.cu)
fame_status build_tables(fame_ctx* c);      // twiddles, twist fractions, preconditioner
fame_status build_precond(fame_ctx* c, cudaStream_t st);
template <typename R> KParams<R> make_params(const fame_ctx* c);
template <> KParams<float> make_params<float>(const fame_ctx* c);
template <> KParams<double> make_params<double>(const fame_ctx* c);
// 1/B in float and double from a device [3][n] array; returns mean(1/B)
fame_status eps_from_device(fame_ctx* c, const double* B, cudaStream_t st, double* mean_invB);

// transforms (transforms.cu)
template <typename R>
fame_status run_apply(fame_ctx* c, const typename cpx<R>::T* y, typename cpx<R>::T* Ay, int m,
                      cudaStream_t st);
// the same apply with a caller-provided workspace of 3 m n complex entries
template <typename R>
fame_status run_apply_into(fame_ctx* c, const typename cpx<R>::T* y, typename cpx<R>::T* Ay, int m,
                           typename cpx<R>::T* W, cudaStream_t st);
template <typename R>
fame_status run_lift(fame_ctx* c, const typename cpx<R>::T* y, typename cpx<R>::T* x, int m,
                     cudaStream_t st);
// complex128 apply / lift; with df (and where the two-level passes cover the grid) in
// double-float arithmetic on the FP32 units, else in FP64
bool c128_df_available(const fame_ctx* c, int m);
fame_status run_apply_c128(fame_ctx* c, const double2* y, double2* Ay, int m, bool df, cudaStream_t st);
fame_status run_lift_c128(fame_ctx* c, const double2* y, double2* x, int m, bool df, cudaStream_t st);
// FP64 arithmetic forced for every complex128 step (environment FAME_FP64_NATIVE=1)
bool fp64_native();
// E = B^{-1} Q_r Sigma_r y and H = -i sqrt(lambda) P_r y for m eigenpairs (complex128)
fame_status run_fields(fame_ctx* c, const double2* y, const double* lambda, double2* E, double2* H, int m,
                       cudaStream_t st);
fame_status run_grad(fame_ctx* c, const double2* Y, const double* w, int nev, double* dB,
                     cudaStream_t st);
fame_status run_precond_table(fame_ctx* c, cudaStream_t st);

// apply plans: which kernel families exist for this context's grid (transforms.cu)
bool apply_zfam_available(const fame_ctx* c, int dtype, int zfam, int m);
bool apply_xyfam_available(const fame_ctx* c, int dtype, int xyfam);

// fixed-length passes (apply3.cu), complex64
bool z3_supported(int L);
bool xy3_supported(int n1, int n2);
template <typename R>
fame_status run_z3(fame_ctx* c, const KParams<R>& P, const typename cpx<R>::T* in,
                   typename cpx<R>::T* out, int m, bool zin, int vpc, bool prefetch, cudaStream_t st);
template <typename R>
fame_status run_xy3(fame_ctx* c, const KParams<R>& P, typename cpx<R>::T* W, int m, int mode,
                    R lift_scale, bool wide, cudaStream_t st);
bool xy3_wide_supported(int n1, int n2);
fame_status run_basis_mask(fame_ctx* c);
fame_status run_twist_tables(fame_ctx* c);

// error flag of the tensor-core kernels (tc_gram.cu): cleared by tc_reset_err, set by
// any CTA whose bounded wait gave up; tc_wait_failed reads it (synchronous)
fame_status tc_reset_err(fame_ctx* c, cudaStream_t st);
bool tc_wait_failed(fame_ctx* c);

// G = U^H V for device blocks of 2n complex rows (blockops.cu)
template <typename C>
fame_status block_gram(fame_ctx* c, const C* U, int ku, const C* V, int kv, size_t ld, double2* G,
                       cudaStream_t st);

// Preconditioner of the block eigensolver (precond.cu): W <- S P_K(M) S (W / (S^2/mean)),
// W given as tinv .* R, its ncols columns replaced by the Chebyshev inexact A_r^{-1} R
template <typename C>
fame_status precond_cheb(fame_ctx* c, C* W, int ncols, cudaStream_t st);
int cheb_degree();

// solver (solver.cu)
fame_status run_eigs_batched(fame_ctx* const* ctxs, int nprob, int nev, double tol, int max_iter,
                             int flags, double* lambda_out, int* iters_out, cudaStream_t st);
fame_status run_eigs(fame_ctx* c, int nev, double tol, int max_iter, int flags, double* lambda_out,
                     void* Y_out, int* iters_out, cudaStream_t st);
// the paper's solver: Lanczos on A_r^{-1} with inner CG on Q_r^* B^{-1} Q_r (lanczos.cu)
fame_status run_inv_lanczos(fame_ctx* c, int nev, double tol, int max_iter, double* lambda_out, void* Y_out,
                            int* iters_out, cudaStream_t st);

// small dense FP64 Rayleigh-Ritz (rr.cpp): solve GA c = theta GB c for the k x k
// Hermitian pair (column-major complex, interleaved), return the nwant smallest
// pairs.  drop: relative threshold on the scaled GB spectrum below which
// directions are discarded.  try_cholesky: reduce through the Cholesky factor of
// GB when it is well conditioned (else, and when false, through its
// eigen-decomposition).  Returns the number of pairs produced, or kRRNoConv if an
// implicit QR ran out of sweeps (the outputs are then not eigenpairs).
constexpr int kRRNoConv = -2;
int rayleigh_ritz(int k, const double* GA, const double* GB, int nwant, double drop,
                  double* theta, double* C, bool try_cholesky = true);
// Hermitian eigensolver (ascending), A column-major k x k complex; V may alias nothing.
// false if the implicit QR did not converge within its sweep limit.
bool herm_eig(int k, const double* A, double* w, double* V);
// total sweep limit of the implicit QR (0: the default of 60 per matrix order; for tests)
void rr_set_qr_sweep_limit(int total);
