// Opt-in per-kernel timing with CUDA events on the launching stream, and NVTX
// ranges named for each kernel pass ("zin_c64", ...) that are always on.
#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "fame_internal.h"

namespace {

struct Rec {
    int id;
    cudaEvent_t a, b;
    double bytes, flops;
};

struct Prof {
    std::mutex mu;
    bool on = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
};

Prof& prof() {
    static Prof p;
    return p;
}

const char* kNames[K_COUNT] = {"zin", "xy", "zout", "ypass", "xpass", "gram", "gram_reduce",
                               "combine", "resid", "convert", "grad_accum", "setup", "gram_herm",
                               "orth", "combine_df", "precond", "zin_df", "xy_df", "zout_df"};

// "zin_c64", "zin_c128", ... in the order of the profiler's ids
struct RangeNames {
    char s[2 * K_COUNT][32];
    RangeNames() {
        for (int i = 0; i < 2 * K_COUNT; ++i)
            std::snprintf(s[i], sizeof(s[i]), "%s_%s", kNames[i / 2], (i & 1) ? "c128" : "c64");
    }
};

const RangeNames& range_names() {
    static const RangeNames r;
    return r;
}

}  // namespace

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

ProfScope::ProfScope(int kind, bool dbl, cudaStream_t st, double bytes, double flops)
    : id_(-1), st_(st), bytes_(bytes), flops_(flops), ev_(nullptr) {
    nvtxRangePushA(range_names().s[kind * 2 + (dbl ? 1 : 0)]);
    Prof& p = prof();
    if (!p.on) return;
    std::lock_guard<std::mutex> g(p.mu);
    ev_ = p.get();
    if (!ev_) return;
    id_ = kind * 2 + (dbl ? 1 : 0);
    cudaEventRecord(ev_, st_);
}

ProfScope::~ProfScope() {
    nvtxRangePop();
    if (id_ < 0) return;
    Prof& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    cudaEvent_t e2 = p.get();
    if (!e2) return;
    cudaEventRecord(e2, st_);
    p.recs.push_back(Rec{id_, ev_, e2, bytes_, flops_});
}

extern "C" {

fame_status fame_profile(int enable) {
    Prof& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (enable) {
        cudaDeviceSynchronize();
        for (auto& r : p.recs) {
            p.pool.push_back(r.a);
            p.pool.push_back(r.b);
        }
        p.recs.clear();
    }
    p.on = enable != 0;
    return FAME_OK;
}

int fame_profile_read(fame_kernel_stat* out, int max) {
    Prof& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    cudaDeviceSynchronize();
    std::vector<fame_kernel_stat> agg(2 * K_COUNT);
    for (int i = 0; i < 2 * K_COUNT; ++i) {
        std::memset(&agg[i], 0, sizeof(fame_kernel_stat));
        std::snprintf(agg[i].name, sizeof(agg[i].name), "%s_%s", kNames[i / 2], (i & 1) ? "c128" : "c64");
    }
    for (auto& r : p.recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        agg[r.id].launches += 1;
        agg[r.id].total_ms += ms;
        agg[r.id].bytes += r.bytes;
        agg[r.id].flops += r.flops;
    }
    int k = 0;
    for (auto& a : agg)
        if (a.launches > 0 && k < max && out) out[k++] = a;
    return k;
}

}  // extern "C"
