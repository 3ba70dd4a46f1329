// Apply plans: the launch choices of the A_r apply (Z-pass and XY kernel family,
// vectors per Z-pass block), set explicitly or picked by timing every available
// choice on this context's grid.
#include <string>
#include <vector>

#include "fame_internal.h"

namespace {

constexpr int kZFamilies = 4, kXYFamilies = 5;

fame_status check_plan(fame_ctx* c, int dtype, const fame_apply_plan& p) {
    if (p.z_kernel < 0 || p.z_kernel > kZFamilies || p.xy_kernel < 0 || p.xy_kernel > kXYFamilies ||
        p.vectors_per_block < 0 ||
        p.vectors_per_block > 4096)
        return set_err(c, FAME_E_ARG, "apply plan field out of range");
    if (p.z_kernel && !apply_zfam_available(c, dtype, p.z_kernel, 1))
        return set_err(c, FAME_E_ARG, "Z-pass kernel family " + std::to_string(p.z_kernel) +
                                          " not available for this grid and precision");
    if (p.xy_kernel && !apply_xyfam_available(c, dtype, p.xy_kernel))
        return set_err(c, FAME_E_ARG, "XY kernel family " + std::to_string(p.xy_kernel) +
                                          " not available for this grid and precision");
    return FAME_OK;
}

// mean milliseconds of one apply of m vectors under the context's current plan
fame_status time_apply(fame_ctx* c, int dtype, const void* y, void* Ay, int m, cudaStream_t st,
                       cudaEvent_t e0, cudaEvent_t e1, double* ms) {
    constexpr int kReps = 3;
    auto once = [&]() {
        return dtype == FAME_C64
                   ? run_apply<float>(c, static_cast<const float2*>(y), static_cast<float2*>(Ay), m, st)
                   : run_apply<double>(c, static_cast<const double2*>(y), static_cast<double2*>(Ay), m, st);
    };
    fame_status s = once();          // warm-up (workspace growth, attributes)
    if (s != FAME_OK) return s;
    FAME_CUDA_TRY(c, cudaEventRecord(e0, st));
    for (int r = 0; r < kReps; ++r)
        if ((s = once()) != FAME_OK) return s;
    FAME_CUDA_TRY(c, cudaEventRecord(e1, st));
    FAME_CUDA_TRY(c, cudaEventSynchronize(e1));
    float t = 0.f;
    FAME_CUDA_TRY(c, cudaEventElapsedTime(&t, e0, e1));
    *ms = t / kReps;
    return FAME_OK;
}

}  // namespace

extern "C" {

fame_status fame_set_apply_plan(fame_ctx* c, int dtype, const fame_apply_plan* plan) {
    if (!c) return FAME_E_ARG;
    c->err.clear();
    if (!plan || (dtype != FAME_C64 && dtype != FAME_C128)) return set_err(c, FAME_E_ARG, "bad plan or dtype");
    fame_status s = check_plan(c, dtype, *plan);
    if (s != FAME_OK) return s;
    c->apply_plan[dtype] = ApplyPlan{plan->z_kernel, plan->xy_kernel, plan->vectors_per_block};
    return FAME_OK;
}

fame_status fame_get_apply_plan(const fame_ctx* c, int dtype, fame_apply_plan* plan) {
    if (!c || !plan || (dtype != FAME_C64 && dtype != FAME_C128)) return FAME_E_ARG;
    const ApplyPlan& a = c->apply_plan[dtype];
    plan->z_kernel = a.zfam;
    plan->xy_kernel = a.xyfam;
    plan->vectors_per_block = a.vpc;
    return FAME_OK;
}

fame_status fame_autotune(fame_ctx* c, int m, int dtype, double* best_ms, void* stream) {
    if (!c) return FAME_E_ARG;
    c->err.clear();
    if (m < 1 || m > 4096 || (dtype != FAME_C64 && dtype != FAME_C128)) return set_err(c, FAME_E_ARG, "bad m or dtype");
    if (!c->eps_set) return set_err(c, FAME_E_STATE, "fame_set_eps has not been called");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)m * 2 * (size_t)c->n * (dtype == FAME_C64 ? sizeof(float2) : sizeof(double2));
    void* buf = nullptr;
    if (cudaMalloc(&buf, 2 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, FAME_E_NOMEM, "autotune scratch");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fame_status s = FAME_OK;
    const ApplyPlan saved = c->apply_plan[dtype];
    ApplyPlan best{};
    double best_t = 1e300;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, 2 * bytes, st) != cudaSuccess) {
        cudaGetLastError();
        s = set_err(c, FAME_E_CUDA, "autotune setup");
    }
    void* y = buf;
    void* Ay = static_cast<char*>(buf) + bytes;
    // Z family and vectors per block first (XY automatic), then the XY family
    for (int zf = 1; s == FAME_OK && zf <= kZFamilies; ++zf) {
        if (!apply_zfam_available(c, dtype, zf, m)) continue;
        for (int vpc : {1, 2, 4, 8, 16}) {
            if (vpc > m && vpc > 1) break;
            c->apply_plan[dtype] = ApplyPlan{zf, 0, vpc};
            double t = 0.0;
            if ((s = time_apply(c, dtype, y, Ay, m, st, e0, e1, &t)) != FAME_OK) break;
            if (t < best_t) { best_t = t; best = c->apply_plan[dtype]; }
        }
    }
    for (int xf = 1; s == FAME_OK && xf <= kXYFamilies; ++xf) {
        if (!apply_xyfam_available(c, dtype, xf)) continue;
        c->apply_plan[dtype] = ApplyPlan{best.zfam, xf, best.vpc};
        double t = 0.0;
        if ((s = time_apply(c, dtype, y, Ay, m, st, e0, e1, &t)) != FAME_OK) break;
        if (t < best_t) { best_t = t; best = c->apply_plan[dtype]; }
    }
    if (best.xyfam == 0 && s == FAME_OK) {
        // automatic XY kept: record the family it resolves to
        for (int xf = 1; xf <= kXYFamilies; ++xf)
            if (apply_xyfam_available(c, dtype, xf)) { best.xyfam = xf; break; }
    }
    c->apply_plan[dtype] = (s == FAME_OK) ? best : saved;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (s == FAME_OK && best_ms) *best_ms = best_t;
    return s;
}

}  // extern "C"
