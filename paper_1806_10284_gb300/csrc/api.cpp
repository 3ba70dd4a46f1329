#include <algorithm>
// C ABI entry points (declared in include/fame.h).
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bounds.cuh"
#include "fame_internal.h"

namespace {
std::atomic<unsigned long long> g_launches{0};
thread_local std::string g_create_err;

bool bad3(const double* v) {
    return !v || !std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2]);
}

template <typename T>
void free_dev(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_tables(fame_ctx* c) {
    for (int a = 0; a < 3; ++a) { free_dev(c->tf.tw[a]); free_dev(c->td.tw[a]); }
    free_dev(c->tf.f2); free_dev(c->td.f2);
    free_dev(c->tf.f3); free_dev(c->td.f3);
    free_dev(c->tf.invB); free_dev(c->td.invB);
    free_dev(c->tf.tinv); free_dev(c->td.tinv);
    free_dev(c->tf.tw3); free_dev(c->td.tw3);
    free_dev(c->tf.lam3); free_dev(c->td.lam3);
    free_dev(c->tf.tw2); free_dev(c->td.tw2);
    free_dev(c->tf.tw1); free_dev(c->td.tw1);
    free_dev(c->alt_mask);
}

fame_status check_ctx(fame_ctx* c) {
    if (!c) return FAME_E_ARG;
    c->err.clear();
    return FAME_OK;
}
}  // namespace

void count_launch(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

fame_status set_err(fame_ctx* c, fame_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return s;
}

fame_status grow(fame_ctx* c, GrowBuf& b, size_t bytes) {
    if (b.bytes >= bytes) return FAME_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, FAME_E_NOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return FAME_OK;
}

fame_status grow_pinned(fame_ctx* c, GrowBuf& b, size_t bytes) {
    if (b.bytes >= bytes) return FAME_OK;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaHostAlloc(&b.p, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, FAME_E_NOMEM, "cudaHostAlloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return FAME_OK;
}

extern "C" {

const char* fame_version(void) { return "fame-gb300 0.1 (sm_103a)"; }

int fame_bounds_violations(int* code, long long* index) {
#ifdef FAME_CHECK_BOUNDS
    const BoundsRec recs[] = {bounds_take_tc_gram(), bounds_take_apply3(), bounds_take_blockops(),
                              bounds_take_transforms()};
    long long total = 0;
    bool first = true;
    for (const BoundsRec& r : recs) {
        total += r.count;
        if (r.count && first) {
            if (code) *code = r.code;
            if (index) *index = r.index;
            first = false;
        }
    }
    if (first) {
        if (code) *code = 0;
        if (index) *index = 0;
    }
    return (int)std::min<long long>(total, 0x7fffffff);
#else
    if (code) *code = 0;
    if (index) *index = 0;
    return -1;
#endif
}

unsigned long long fame_launch_count(void) { return g_launches.load(); }

const char* fame_last_error(const fame_ctx* c) {
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

fame_status fame_create(fame_ctx** out, int lattice, const double a1[3], const double a2[3],
                        const double a3[3], int n1, int n2, int n3, const double bloch[3]) {
    g_create_err.clear();
    if (!out) return set_err(nullptr, FAME_E_ARG, "out is NULL");
    *out = nullptr;
    if (lattice < 0 || lattice > 14) return set_err(nullptr, FAME_E_ARG, "lattice id must be 0..14");
    if (bad3(a1) || bad3(a2) || bad3(a3) || bad3(bloch))
        return set_err(nullptr, FAME_E_ARG, "null or non-finite vector");
    const int ns[3] = {n1, n2, n3};
    for (int i = 0; i < 3; ++i)
        if (radix_list(ns[i]).empty())
            return set_err(nullptr, FAME_E_RADIX, "grid size " + std::to_string(ns[i]) +
                                                      " must be in [2, 1024] with prime factors 2, 3, 5");
    LatticePlan plan;
    std::string why = build_lattice(a1, a2, a3, n1, n2, n3, bloch, &plan);
    if (!why.empty()) return set_err(nullptr, FAME_E_LATTICE, why);
    fame_ctx* c = new (std::nothrow) fame_ctx();
    if (!c) return set_err(nullptr, FAME_E_NOMEM, "host allocation");
    c->plan = plan;
    c->n = (long long)n1 * n2 * n3;
    for (int i = 0; i < 3; ++i) {
        c->in_vec[0][i] = a1[i];
        c->in_vec[1][i] = a2[i];
        c->in_vec[2][i] = a3[i];
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return set_err(nullptr, FAME_E_CUDA, "no CUDA device");
    }
    fame_status s = build_tables(c);
    if (s != FAME_OK) {
        g_create_err = c->err;
        free_tables(c);
        delete c;
        return s;
    }
    *out = c;
    return FAME_OK;
}

static void plan_to_info(const LatticePlan& p, fame_plan_info* info) {
    for (int i = 0; i < 3; ++i) {
        info->n[i] = p.n[i];
        info->perm[i] = p.perm[i];
        info->m[i] = p.m[i];
        info->rho[i] = p.rho[i];
        info->s[i] = p.s[i];
        info->delta[i] = p.delta[i];
        info->kappa[i] = p.kappa[i];
        for (int r = 0; r < 3; ++r) info->a[3 * i + r] = p.a[r][i];
    }
}

fame_status fame_plan_lattice(const double a1[3], const double a2[3], const double a3[3], int n1,
                              int n2, int n3, const double bloch[3], fame_plan_info* info) {
    g_create_err.clear();
    if (!info || bad3(a1) || bad3(a2) || bad3(a3) || bad3(bloch))
        return set_err(nullptr, FAME_E_ARG, "null or non-finite argument");
    const int ns[3] = {n1, n2, n3};
    for (int i = 0; i < 3; ++i)
        if (radix_list(ns[i]).empty())
            return set_err(nullptr, FAME_E_RADIX, "grid size " + std::to_string(ns[i]) +
                                                      " must be in [2, 1024] with prime factors 2, 3, 5");
    LatticePlan plan;
    std::string why = build_lattice(a1, a2, a3, n1, n2, n3, bloch, &plan);
    if (!why.empty()) return set_err(nullptr, FAME_E_LATTICE, why);
    plan_to_info(plan, info);
    return FAME_OK;
}

fame_status fame_get_plan(const fame_ctx* c, fame_plan_info* info) {
    if (!c || !info) return FAME_E_ARG;
    plan_to_info(c->plan, info);
    return FAME_OK;
}

fame_status fame_set_k(fame_ctx* c, const double bloch[3]) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (bad3(bloch)) return set_err(c, FAME_E_ARG, "bloch vector null or non-finite");
    compute_kappa(c->in_vec[0], c->in_vec[1], c->in_vec[2], bloch, &c->plan);
    fame_status s = build_tables(c);
    if (s != FAME_OK) return s;
    if (c->eps_set) return run_precond_table(c, nullptr);
    return FAME_OK;
}

}  // extern "C"

extern "C" {

fame_status fame_set_eps_device(fame_ctx* c, const double* B, void* stream);

fame_status fame_set_eps(fame_ctx* c, const double* B1, const double* B2, const double* B3,
                         void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!B1 || !B2 || !B3) return set_err(c, FAME_E_ARG, "eps array is NULL");
    const size_t n = (size_t)c->n;
    std::vector<double> h(3 * n);
    std::memcpy(h.data(), B1, n * sizeof(double));
    std::memcpy(h.data() + n, B2, n * sizeof(double));
    std::memcpy(h.data() + 2 * n, B3, n * sizeof(double));
    for (size_t i = 0; i < 3 * n; ++i)
        if (!(h[i] > 0.0) || !std::isfinite(h[i]))
            return set_err(c, FAME_E_ARG, "eps must be finite and > 0 (index " + std::to_string(i) + ")");
    double* d = nullptr;
    if (cudaMalloc((void**)&d, 3 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, FAME_E_NOMEM, "cudaMalloc eps staging");
    }
    cudaError_t e = cudaMemcpy(d, h.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice);
    fame_status s = (e == cudaSuccess) ? fame_set_eps_device(c, d, stream)
                                       : set_err(c, FAME_E_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamSynchronize(st);
    cudaFree(d);
    return s;
}

}  // extern "C"

fame_status eps_from_device(fame_ctx* c, const double* B, cudaStream_t st, double* mean_invB);

extern "C" fame_status fame_set_eps_device(fame_ctx* c, const double* B, void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!B) return set_err(c, FAME_E_ARG, "eps array is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)c->n;
    if (!c->tf.invB && cudaMalloc((void**)&c->tf.invB, 3 * n * sizeof(float)) != cudaSuccess)
        return set_err(c, FAME_E_NOMEM, "cudaMalloc invB");
    if (!c->td.invB && cudaMalloc((void**)&c->td.invB, 3 * n * sizeof(double)) != cudaSuccess)
        return set_err(c, FAME_E_NOMEM, "cudaMalloc invB");
    if (!c->tf.tinv && cudaMalloc((void**)&c->tf.tinv, n * sizeof(float)) != cudaSuccess)
        return set_err(c, FAME_E_NOMEM, "cudaMalloc precond");
    if (!c->td.tinv && cudaMalloc((void**)&c->td.tinv, n * sizeof(double)) != cudaSuccess)
        return set_err(c, FAME_E_NOMEM, "cudaMalloc precond");
    double mean = 0.0;
    fame_status s = eps_from_device(c, B, st, &mean);
    if (s != FAME_OK) return s;
    c->mean_invB = mean;
    c->eps_set = true;
    return run_precond_table(c, st);
}

extern "C" {

fame_status fame_apply_Ar(fame_ctx* c, const void* y, void* Ay, int m, int dtype, void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!y || !Ay || m < 1 || m > 4096) return set_err(c, FAME_E_ARG, "bad y/Ay/m");
    if (y == Ay) return set_err(c, FAME_E_ARG, "y and Ay must not overlap");
    if (!c->eps_set) return set_err(c, FAME_E_STATE, "fame_set_eps has not been called");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == FAME_C64)
        return run_apply<float>(c, static_cast<const float2*>(y), static_cast<float2*>(Ay), m, st);
    if (dtype == FAME_C128 || dtype == FAME_C128_DF)
        return run_apply_c128(c, static_cast<const double2*>(y), static_cast<double2*>(Ay), m,
                              dtype == FAME_C128_DF, st);
    return set_err(c, FAME_E_ARG, "dtype must be FAME_C64, FAME_C128 or FAME_C128_DF");
}

fame_status fame_lift(fame_ctx* c, const void* y, void* x, int m, int dtype, void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!y || !x || m < 1 || m > 4096) return set_err(c, FAME_E_ARG, "bad y/x/m");
    if (!c->eps_set) return set_err(c, FAME_E_STATE, "fame_set_eps has not been called");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == FAME_C64)
        return run_lift<float>(c, static_cast<const float2*>(y), static_cast<float2*>(x), m, st);
    if (dtype == FAME_C128 || dtype == FAME_C128_DF)
        return run_lift_c128(c, static_cast<const double2*>(y), static_cast<double2*>(x), m,
                             dtype == FAME_C128_DF, st);
    return set_err(c, FAME_E_ARG, "dtype must be FAME_C64, FAME_C128 or FAME_C128_DF");
}

fame_status fame_eigs(fame_ctx* c, int nev, double tol, int max_iter, int flags, double* lambda_out,
                      void* Y_out, int* iters_out, void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (nev < 1 || nev > 64 || !(tol > 0.0) || max_iter < 1 || !lambda_out)
        return set_err(c, FAME_E_ARG, "bad nev/tol/max_iter/lambda_out");
    if (!(flags & (FAME_MIXED | FAME_FP64 | FAME_INV_LANCZOS)))
        return set_err(c, FAME_E_ARG, "flags need FAME_MIXED, FAME_FP64 or FAME_INV_LANCZOS");
    if (!c->eps_set) return set_err(c, FAME_E_STATE, "fame_set_eps has not been called");
    if (2LL * c->n < 3LL * (nev + 4)) return set_err(c, FAME_E_ARG, "grid too small for nev");
    if (flags & FAME_INV_LANCZOS) {
        fame_status s = tc_reset_err(c, static_cast<cudaStream_t>(stream));
        if (s != FAME_OK) return s;
        return run_inv_lanczos(c, nev, tol, max_iter, lambda_out, Y_out, iters_out, static_cast<cudaStream_t>(stream));
    }
    return run_eigs(c, nev, tol, max_iter, flags, lambda_out, Y_out, iters_out,
                    static_cast<cudaStream_t>(stream));
}

fame_status fame_get_stats(const fame_ctx* c, fame_solve_stats* stats) {
    if (!c || !stats) return FAME_E_ARG;
    *stats = c->stats;
    return FAME_OK;
}

fame_status fame_grad_eps(fame_ctx* c, int nev, const double* dobj, double rel_cluster,
                          double* dB_out, void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!dobj || !dB_out || nev < 1 || !(rel_cluster >= 0.0)) return set_err(c, FAME_E_ARG, "bad arguments");
    if (!c->Y || (int)c->lambda.size() < nev) return set_err(c, FAME_E_STATE, "no eigenpairs: call fame_eigs first");
    // weights: every band gets the cluster mean of dobj/dlambda over its degenerate cluster
    std::vector<double> w(nev);
    int j = 0;
    while (j < nev) {
        int e = j + 1;
        while (e < nev && std::fabs(c->lambda[e] - c->lambda[e - 1]) <= rel_cluster * std::fabs(c->lambda[e - 1])) ++e;
        double sum = 0.0;
        for (int i = j; i < e; ++i) sum += dobj[i];
        for (int i = j; i < e; ++i) w[i] = sum / (e - j);
        j = e;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fame_status s = run_grad(c, reinterpret_cast<const double2*>(c->Y), w.data(), nev, dB_out, st);
    if (s != FAME_OK) return s;
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    return FAME_OK;
}

fame_status fame_eigs_batched(fame_ctx* const* ctxs, int nprob, int nev, double tol, int max_iter,
                              int flags, double* lambda_out, int* iters_out, void* stream) {
    if (!ctxs || nprob < 1 || !lambda_out) return set_err(nullptr, FAME_E_ARG, "bad batch arguments");
    for (int i = 0; i < nprob; ++i) {
        if (!ctxs[i]) return set_err(nullptr, FAME_E_ARG, "null context in batch");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return set_err(nullptr, FAME_E_ARG, "context repeated in batch");
    }
    return run_eigs_batched(ctxs, nprob, nev, tol, max_iter, flags, lambda_out, iters_out,
                            static_cast<cudaStream_t>(stream));
}

fame_status fame_fields(fame_ctx* c, const void* y, const double* lambda, void* E, void* H, int m, int dtype,
                        void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!y || (!E && !H) || m < 1 || m > 4096) return set_err(c, FAME_E_ARG, "bad y/E/H/m");
    if (H && !lambda) return set_err(c, FAME_E_ARG, "H needs the eigenvalues");
    if (dtype != FAME_C128) return set_err(c, FAME_E_ARG, "fields are computed in complex128 (FAME_C128)");
    if (!c->eps_set) return set_err(c, FAME_E_STATE, "fame_set_eps has not been called");
    if (H && y == H) return set_err(c, FAME_E_ARG, "y and H must not overlap");
    return run_fields(c, static_cast<const double2*>(y), lambda, static_cast<double2*>(E), static_cast<double2*>(H), m,
                      static_cast<cudaStream_t>(stream));
}

fame_status fame_block_gram(fame_ctx* c, const void* U, int ku, const void* V, int kv, int dtype, void* G,
                            void* stream) {
    if (check_ctx(c)) return FAME_E_ARG;
    if (!U || !V || !G || ku < 1 || kv < 1 || ku > 4096 || kv > 4096)
        return set_err(c, FAME_E_ARG, "bad U/V/G/ku/kv");
    const size_t ld = 2 * (size_t)c->n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fame_status s = tc_reset_err(c, st);
    if (s != FAME_OK) return s;
    if (dtype == FAME_C64)
        return block_gram<float2>(c, static_cast<const float2*>(U), ku, static_cast<const float2*>(V), kv, ld,
                                  static_cast<double2*>(G), st);
    if (dtype == FAME_C128)
        return block_gram<double2>(c, static_cast<const double2*>(U), ku, static_cast<const double2*>(V), kv, ld,
                                   static_cast<double2*>(G), st);
    return set_err(c, FAME_E_ARG, "dtype must be FAME_C64 or FAME_C128");
}

void fame_destroy(fame_ctx* c) {
    if (!c) return;
    free_tables(c);
    if (c->work.p) cudaFree(c->work.p);
    if (c->solver.p) cudaFree(c->solver.p);
    if (c->solver2.p) cudaFree(c->solver2.p);
    if (c->partial.p) cudaFree(c->partial.p);
    if (c->pinned.p) cudaFreeHost(c->pinned.p);
    if (c->tcerr.p) cudaFree(c->tcerr.p);
    if (c->cheb.p) cudaFree(c->cheb.p);
    if (c->Y) cudaFree(c->Y);
    delete c;
}

}  // extern "C"
