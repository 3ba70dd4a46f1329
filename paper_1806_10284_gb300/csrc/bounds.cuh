// Bounds checks of the debug build (compiled with -DFAME_CHECK_BOUNDS).
//
// In that build the kernels test the index arithmetic they rely on -- TMA
// coordinates, global offsets of the FFT passes, the rows of the staged copies --
// before the access: a failed check skips the access (a load reads nothing, a
// store or copy is not issued) and is recorded on the device, so a wrong index is
// reported instead of faulting.  fame_bounds_violations() returns and clears the
// records.  In the normal build bounds_ok() is the constant true and the checks
// compile away.
//
// Each translation unit that checks keeps its own record (a file-local device
// variable: no relocatable device code needed) and defines its reader with
// FAME_BOUNDS_READER(name); api.cpp sums the readers.
#pragma once

#include <cuda_runtime.h>

struct BoundsRec {
    unsigned int count;      // failed checks since the last read
    int code;                // kBnd* of the first one
    long long index;         // the offending index or coordinate of the first one
};

// what failed (the code of the first failed check)
enum BoundsCode {
    kBndTmaX = 1,            // tensor-core Gram: TMA x coordinate not 16-byte aligned
    kBndTcOut = 2,           // tensor-core Gram: partial entry outside [MA][NB]
    kBndZLoad = 3,           // fixed-length Z pass: global load outside its array
    kBndZStore = 4,          // fixed-length Z pass: global store outside its array
    kBndRing = 5,            // ring-staged block kernels: a 16-byte copy past the column's end
    kBndXRows = 6,           // refinement update: staged complex128 row outside the column
    kBndZ2Store = 7,         // two-level Z passes: workspace store outside [m][3][n]
};

#ifdef FAME_CHECK_BOUNDS
namespace {
__device__ BoundsRec g_bounds;
}
__device__ __forceinline__ bool bounds_ok(bool ok, int code, long long index) {
    if (!ok && atomicAdd(&g_bounds.count, 1u) == 0u) {
        g_bounds.code = code;
        g_bounds.index = index;
    }
    return ok;
}
#define FAME_BOUNDS_READER(name)                                                  \
    BoundsRec bounds_take_##name() {                                              \
        BoundsRec r{0u, 0, 0};                                                    \
        if (cudaMemcpyFromSymbol(&r, g_bounds, sizeof(r)) != cudaSuccess) {        \
            cudaGetLastError();                                                   \
            return BoundsRec{0u, 0, 0};                                           \
        }                                                                         \
        const BoundsRec z{0u, 0, 0};                                              \
        if (cudaMemcpyToSymbol(g_bounds, &z, sizeof(z)) != cudaSuccess) cudaGetLastError(); \
        return r;                                                                 \
    }
#else
__device__ __forceinline__ constexpr bool bounds_ok(bool, int, long long) { return true; }
#define FAME_BOUNDS_READER(name) \
    BoundsRec bounds_take_##name() { return BoundsRec{0u, 0, 0}; }
#endif

// the readers (one per checking translation unit)
BoundsRec bounds_take_tc_gram();
BoundsRec bounds_take_apply3();
BoundsRec bounds_take_blockops();
BoundsRec bounds_take_transforms();
