// Tall-skinny Gram matrices P = A^H B of complex64 column blocks on the tensor
// cores (tcgen05, kind::tf32), for the Rayleigh-Ritz and orthogonalisation steps
// of the block eigensolver.
//
// Arithmetic.  A column is a float array with real and imaginary parts interleaved;
// taking that interleaved index as the contraction index K,
//   Re P_ij = sum_K a_i[K] b_j[K],   Im P_ij = sum_K a_i[K] b'_j[K],
// with b' = (Im b, -Re b) interleaved (i.e. -i b).  Each real operand x is the
// sum of its TF32 high part (x with the low 13 mantissa bits dropped: what the
// tensor core reads from a 32-bit operand) and its remainder rounded to the
// nearest TF32 value, so x = high + low to about 2^-22 relative with unbiased
// rounding; every product is formed from all four terms high*high + high*low +
// low*high + low*low (the split-operand idea of Ootomo and Yokota, 2022).  Products
// are summed in FP32 in tensor memory over one CTA's rows (about two thousand) and
// the CTA partials in FP64 by a reduction kernel in a fixed order (deterministic).
//
// Data flow per CTA (a contiguous range of rows, 16 complex rows per chunk, NS stages):
//   warp 0      TMA: one 2D box per column block into the stage's raw tile with the
//               128-byte swizzle -- exactly the K-major operand layout of the MMA, so
//               the raw tile is the high part of A and B as it stands;
//   warps 2-9   write the low parts of every staged row, and the B operand tile
//               [b high; b' high; b low; b' low] (4 NP rows, same layout), so that
//               one MMA of N = 4 NP covers real and imaginary parts and both halves
//               of the split (N = 2 NP and two MMAs when 4 NP > 256);
//   warp 1      one thread issues the 8 (or 16) MMAs of a chunk and commits them to the
//               stage's "empty" barrier (the producer then reloads it); after the
//               last chunk, to the accumulator barrier;
//   warps 2-9   read the accumulators from tensor memory and write the CTA partial.
// Every wait is bounded (FAME_WAIT_TIMEOUT_MS, default 1000 ms): on expiry the CTA
// sets an error flag, lets its copies and MMAs in flight finish, frees its tensor
// memory and returns; the reduction then writes NaN, and the solver reports
// FAME_E_TIMEOUT.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "blockops.h"
#include "bounds.cuh"
#include "tc.cuh"

namespace {

constexpr int KC = 16;                 // complex rows per chunk (32 floats = 128 bytes per column)
constexpr int kConvWarps = 8;
constexpr int kThreads = 64 + 32 * kConvWarps;
constexpr int kMaxBlocks = 6;          // column blocks per side

struct TcMaps {
    CUtensorMap m[2 * kMaxBlocks];     // A blocks, then B blocks
};

struct TcGramArgs {
    int nA, nB;                        // tensor maps of A, of B (B: 0 when it aliases A's first columns)
    int cols[2 * kMaxBlocks];          // columns of each map's block
    int rawoff[2 * kMaxBlocks];        // first raw row of each map's block (multiples of 8)
    int MA, NB;                        // columns of A, of B
    int nraw;                          // staged rows (columns of A and B, each block padded to 8)
    int bstart, nbraw, NP;             // first staged row of B, its staged rows, N of the MMA (multiple of 16)
    int NS;                            // stages
    uint32_t raw_bytes;                // bytes delivered per stage
    size_t ld, rows_per_cta;
    double2* partial;                  // [grid][NB][MA]
    int* err;
    unsigned long long timeout_ns;
    int skip_chunk;                    // test hook: this chunk is never loaded (-1: none)
    int plant;                         // bounds-checked build, test hook: the first CTA's chunk 0 fails its TMA check
};

struct SmemLayout {
    uint32_t stage, raw, lo, rot, bars, misc, total;
};

// Per stage: raw rows (the high parts), their low parts, and the B operand tile of
// 4 NP rows; all 1024-aligned.  The 128-row A operand may read past a stage's rows
// into whatever follows (those rows only feed accumulator rows that are never read):
// the layout keeps 16 KB of shared memory after the last stage's low tile.
__host__ __device__ inline SmemLayout gram_layout(int nraw, int NP, int NS) {
    SmemLayout L;
    L.raw = 0;
    L.lo = (uint32_t)nraw * 128;
    L.rot = L.lo + (uint32_t)nraw * 128;
    L.stage = L.rot + 4u * NP * 128;
    uint32_t end = (uint32_t)NS * L.stage;
    const uint32_t need = (uint32_t)(NS - 1) * L.stage + L.lo + 16384;   // last stage's low tile + 128 rows
    if (end < need) end = need;
    L.bars = end;
    L.misc = L.bars + 8 * (3 * 8 + 1);                                  // up to 8 stages x 3 barriers, acc
    L.total = L.misc + 16 + 4 * 128 + 4 * 256;                           // slots; A row map; B row map
    return L;
}

__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(const __grid_constant__ TcMaps maps, const TcGramArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzled tiles want 1024-byte alignment (the launch reserves the slack)
    unsigned char* sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int NS = a.NS, NP = a.NP;
    const SmemLayout L = gram_layout(a.nraw, NP, NS);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bars);
    uint64_t* conv = full + 8;
    uint64_t* empty = conv + 8;
    uint64_t* acc_full = empty + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + L.misc);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L.misc + 4);
    volatile int* never = reinterpret_cast<volatile int*>(sm + L.misc + 8);   // stays 0: waits that must not be cut short
    int* amap = reinterpret_cast<int*>(sm + L.misc + 16);                      // [128] staged row -> A column
    int* bmap = amap + 128;                                                    // [256] B row offset -> B column
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // N of the MMA: 4 NP (B high and low stacked) when it fits the 256-column limit, else 2 NP
    const bool wide = 4 * NP <= 256;
    const int NN = wide ? 4 * NP : 2 * NP;
    const uint32_t ncols_tmem = (NN <= 32) ? 32 : (NN <= 64) ? 64 : (NN <= 128) ? 128 : 256;

    const size_t row0 = (size_t)blockIdx.x * a.rows_per_cta;
    const size_t row1 = min(a.ld, row0 + a.rows_per_cta);
    const int nchunk = (int)((row1 - row0 + KC - 1) / KC);

    // set-up: barriers, row maps, zeroed stages (padding rows stay zero), tensor memory
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&conv[s], kConvWarps);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(acc_full, 1);
        *abort = 0;
        *never = 0;
        tc::mbar_fence_init();
    }
    for (int r = tid; r < 128; r += kThreads) amap[r] = -1;
    for (int r = tid; r < 256; r += kThreads) bmap[r] = -1;
    {
        uint4* z = reinterpret_cast<uint4*>(sm);
        const int n16 = (int)(L.bars / 16);
        for (int e = tid; e < n16; e += kThreads) z[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (int b = tid; b < a.nA + a.nB; b += kThreads) {
        int first = 0;                                   // column index of the block's first column
        for (int q = (b < a.nA ? 0 : a.nA); q < b; ++q) first += a.cols[q];
        for (int y = 0; y < a.cols[b]; ++y) {
            const int r = a.rawoff[b] + y;
            if (b < a.nA) {
                amap[r] = first + y;
                if (r - a.bstart >= 0 && r - a.bstart < a.nbraw && first + y < a.NB) bmap[r - a.bstart] = first + y;
            } else {
                bmap[r - a.bstart] = first + y;
            }
        }
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, ncols_tmem);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    tc::fence_proxy_async();                              // the zeroed tiles, for the tensor core
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const unsigned long long tmo = a.timeout_ns;
    auto fail = [&]() {
        *abort = 1;
        atomicExch(a.err, 1);
    };

    if (warp == 0) {
        // ---------------- producer: TMA boxes into the stages ----------------
        if (lane == 0)
            for (int b = 0; b < a.nA + a.nB; ++b) tc::prefetch_tmap(&maps.m[b]);
        int issued = 0;
        bool skipped0 = false;                                 // chunk 0 failed its bounds check
        for (int ch = 0; ch < nchunk; ++ch) {
            const int s = ch % NS;
            // lane 0 waits, the warp follows its verdict (no divergence around __syncwarp)
            bool go = lane == 0 ? tc::mbar_wait(&empty[s], ((ch / NS) & 1) ^ 1, tc::global_ns() + tmo, abort) : true;
            go = __shfl_sync(0xffffffffu, go ? 1 : 0, 0) != 0;
            if (!go) {
                if (lane == 0) fail();
                break;
            }
            if (ch == a.skip_chunk) continue;                  // test hook: never delivered
#ifdef FAME_CHECK_BOUNDS
            {
                // the box's x coordinate (floats) must start on a 16-byte boundary
                const long long x = 2 * (long long)(row0 + (size_t)ch * KC);
                const bool okx = lane == 0 ? bounds_ok((x & 3) == 0 && !(a.plant && ch == 0 && blockIdx.x == 0), kBndTmaX, x) : true;
                if (__shfl_sync(0xffffffffu, okx ? 1 : 0, 0) == 0) {
                    skipped0 = skipped0 || ch == 0;
                    continue;                                  // not issued: the waits on it give up
                }
            }
#endif
            if (lane == 0) tc::mbar_arrive_expect_tx(&full[s], a.raw_bytes);
            __syncwarp();
            if (lane < a.nA + a.nB) {
                unsigned char* dst = sm + (size_t)s * L.stage + L.raw + (size_t)a.rawoff[lane] * 128;
                tc::tma_load_2d(dst, &maps.m[lane], &full[s], (int)(2 * (row0 + (size_t)ch * KC)), 0);
            }
            issued = ch + 1;
        }
        // copies in flight must land before the CTA leaves
        if (lane == 0)
            for (int ch = std::max(0, issued - NS); ch < issued; ++ch) {
                if (ch == a.skip_chunk || (ch == 0 && skipped0)) continue;
                tc::mbar_wait(&full[ch % NS], (ch / NS) & 1, tc::global_ns() + tmo, never);
            }
    } else if (warp == 1) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, NN);
            bool started = false;
            for (int ch = 0; ch < nchunk; ++ch) {
                const int s = ch % NS;
                if (!tc::mbar_wait(&conv[s], (ch / NS) & 1, tc::global_ns() + tmo, abort)) {
                    fail();
                    break;
                }
                tc::fence_after_sync();
                const uint32_t base = tc::smem_u32(sm + (size_t)s * L.stage);
                const uint32_t Ah = base + L.raw, Al = base + L.lo;
                const uint32_t Bh = base + L.rot, Bl = Bh + 2u * NP * 128;   // [b; b'] high, then low
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t o = (uint32_t)k * 32;       // 8 TF32 of K per MMA
                    const uint64_t ah = tc::desc_kmajor_sw128(Ah + o), al = tc::desc_kmajor_sw128(Al + o);
                    const uint64_t bh = tc::desc_kmajor_sw128(Bh + o), bl = tc::desc_kmajor_sw128(Bl + o);
                    if (wide) {
                        // D = [Re hh | Im hh | Re hl | Im hl] + the same with A low
                        tc::mma_tf32(tmem, al, bh, idesc, started);
                        tc::mma_tf32(tmem, ah, bh, idesc, true);
                    } else {
                        tc::mma_tf32(tmem, al, bl, idesc, started);
                        tc::mma_tf32(tmem, al, bh, idesc, true);
                        tc::mma_tf32(tmem, ah, bl, idesc, true);
                        tc::mma_tf32(tmem, ah, bh, idesc, true);
                    }
                    started = true;
                }
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(acc_full);                         // every MMA issued above
        }
        __syncwarp();
    } else {
        // ---------------- low parts and rotated B rows (warps 2-9), then the epilogue ----------------
        const int ct = tid - 64;                               // 0..255
        bool ok = true;
        for (int ch = 0; ch < nchunk && ok; ++ch) {
            const int s = ch % NS;
            bool go = lane == 0 ? tc::mbar_wait(&full[s], (ch / NS) & 1, tc::global_ns() + tmo, abort) : true;
            go = __shfl_sync(0xffffffffu, go ? 1 : 0, 0) != 0;
            if (!go) {
                if (lane == 0) fail();
                ok = false;
                break;
            }
            unsigned char* st = sm + (size_t)s * L.stage;
            for (int e = ct; e < a.nraw * 8; e += 32 * kConvWarps) {
                const int c = e >> 3, q = e & 7;
                const int off = c * 128 + ((q ^ (c & 7)) << 4);   // swizzled position of logical chunk q
                const float4 v = *reinterpret_cast<const float4*>(st + L.raw + off);
                const float4 l = make_float4(tc::tf32_low(v.x), tc::tf32_low(v.y), tc::tf32_low(v.z),
                                             tc::tf32_low(v.w));
                *reinterpret_cast<float4*>(st + L.lo + off) = l;
                const int rb = c - a.bstart;
                if (rb >= 0 && rb < a.nbraw) {
                    // B tile rows: b high, b' = -i b high (re, im) -> (im, -re), b low, b' low; rows rb and
                    // c share (r & 7) since bstart and NP are multiples of 8
                    const int roff = rb * 128 + ((q ^ (c & 7)) << 4);
                    unsigned char* bt = st + L.rot + roff;
                    *reinterpret_cast<float4*>(bt) = v;
                    *reinterpret_cast<float4*>(bt + (size_t)NP * 128) = make_float4(v.y, -v.x, v.w, -v.z);
                    *reinterpret_cast<float4*>(bt + (size_t)2 * NP * 128) = l;
                    *reinterpret_cast<float4*>(bt + (size_t)3 * NP * 128) = make_float4(l.y, -l.x, l.w, -l.z);
                }
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&conv[s]);
        }
        // epilogue: wait for every MMA, then tensor memory -> FP64 partial
        bool done = lane == 0 ? tc::mbar_wait(acc_full, 0, tc::global_ns() + tmo, abort) : true;
        done = __shfl_sync(0xffffffffu, done ? 1 : 0, 0) != 0;
        if (!done) {
            if (lane == 0) fail();
            ok = false;
        }
        ok = __shfl_sync(0xffffffffu, (ok && !*abort) ? 1 : 0, 0) != 0;
        tc::fence_after_sync();
        if (ok) {
            // two warps per TMEM lane quarter, each taking every other group of 16 columns
            const int q = warp & 3, half = (warp - 2) >> 2, i = 32 * q + lane;
            const int acol = amap[i];
            double2* out = a.partial + (size_t)blockIdx.x * a.MA * a.NB;
            const uint32_t lanes = (uint32_t)(32 * q) << 16;
            for (int j0 = 16 * half; j0 < NP; j0 += 32) {
                float re[16], im[16];
                tc::tmem_ld16(tmem + lanes + (uint32_t)j0, re);
                tc::tmem_ld16(tmem + lanes + (uint32_t)(NP + j0), im);
                if (wide) {
                    float re2[16], im2[16];
                    tc::tmem_ld16(tmem + lanes + (uint32_t)(2 * NP + j0), re2);
                    tc::tmem_ld16(tmem + lanes + (uint32_t)(3 * NP + j0), im2);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        re[jj] += re2[jj];
                        im[jj] += im2[jj];
                    }
                }
                if (acol >= 0) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int bcol = bmap[j0 + jj];
                        if (bcol >= 0 && bounds_ok(bcol < a.NB && acol < a.MA, kBndTcOut, (long long)bcol * a.MA + acol))
                            out[(size_t)bcol * a.MA + acol] = make_double2((double)re[jj], (double)im[jj]);
                    }
                }
            }
        }
        tc::fence_before_sync();
    }
    __syncthreads();
    if (warp == 1) {
        // every MMA has completed once acc_full has (the MMA thread commits it last)
        if (lane == 0) tc::mbar_wait(acc_full, 0, tc::global_ns() + tmo, never);
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols_tmem);
    }
}

// G from the partials in a fixed order; one warp per entry.  mode 0: G (MA x NB) = P;
// mode 1: G (NB x MA) = P^H; mode 2: G (k x 2k, k = NB) = [P[:k, :] | P[k:, :]^H].
// A set error flag turns every entry into NaN (the caller's check reports it).
__global__ void k_gram_tc_reduce(const double2* __restrict__ partial, int nblk, int MA, int NB, int mode,
                                 double2* __restrict__ G, const int* __restrict__ err) {
    const int total = MA * NB;
    const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (e >= total) return;
    int src, dst;
    bool conj = false;
    if (mode == 0) {
        src = dst = e;
    } else if (mode == 1) {
        const int i = e % NB, j = e / NB;                  // G[i][j], NB rows
        src = i * MA + j;
        dst = e;
        conj = true;
    } else {
        const int k = NB, i = e % k, j = e / k;           // G[i][j], j < 2k
        if (j < k) {
            src = j * MA + i;
        } else {
            src = i * MA + j;                              // P[j][i] with j in [k, 2k)
            conj = true;
        }
        dst = e;
    }
    double sr = 0.0, si = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = partial[(size_t)b * total + src];
        sr += v.x;
        si += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
        if (*err) sr = si = __longlong_as_double(0x7ff8000000000000LL);
        G[dst] = make_double2(sr, conj ? -si : si);
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2D map of one column block: dim 0 = 2 ld floats (a column, re/im interleaved),
// dim 1 = its columns (stride ld complex); box = 16 complex rows x all columns,
// 128-byte swizzle.
bool encode_block(CUtensorMap* m, const float2* base, size_t ld, int cols) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * ld), (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(float2))};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * KC), (cuuint32_t)cols};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the non-empty blocks of L, in order
BlockList<float2> compact(const BlockList<float2>& L) {
    BlockList<float2> out;
    int k = 0;
    for (int b = 0; b < BlockList<float2>::kMax; ++b) {
        out.ptr[b] = nullptr;
        out.cols[b] = 0;
    }
    for (int b = 0; b < BlockList<float2>::kMax; ++b)
        if (L.cols[b] > 0) {
            out.ptr[k] = L.ptr[b];
            out.cols[k] = L.cols[b];
            ++k;
        }
    out.total = L.total;
    return out;
}

int blocks_of(const BlockList<float2>& L) {
    int nb = 0;
    while (nb < BlockList<float2>::kMax && L.cols[nb] > 0) ++nb;
    return nb;
}

// true if S's blocks are the leading blocks of L (same pointers and widths)
bool is_prefix(const BlockList<float2>& S, const BlockList<float2>& L) {
    const int ns = blocks_of(S);
    if (ns > blocks_of(L)) return false;
    for (int b = 0; b < ns; ++b)
        if (S.ptr[b] != L.ptr[b] || S.cols[b] != L.cols[b]) return false;
    return true;
}

unsigned long long wait_timeout_ns() {
    const char* v = std::getenv("FAME_WAIT_TIMEOUT_MS");
    const double ms = v ? std::atof(v) : 1000.0;
    return (unsigned long long)(std::max(1.0, ms) * 1e6);
}

int skip_chunk_hook() {
    const char* v = std::getenv("FAME_TEST_TC_SKIP_CHUNK");
    return v ? std::atoi(v) : -1;
}

int plant_hook() {
    const char* v = std::getenv("FAME_TEST_BOUNDS_PLANT");
    return v && v[0] == '1' ? 1 : 0;
}

}  // namespace

FAME_BOUNDS_READER(tc_gram)

fame_status tc_reset_err(fame_ctx* c, cudaStream_t st) {
    fame_status s = grow(c, c->tcerr, 256);
    if (s != FAME_OK) return s;
    FAME_CUDA_TRY(c, cudaMemsetAsync(c->tcerr.p, 0, sizeof(int), st));
    return FAME_OK;
}

bool tc_wait_failed(fame_ctx* c) {
    if (!c->tcerr.p) return false;
    int v = 0;
    if (cudaMemcpy(&v, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return v != 0;
}

bool tensor_cores_enabled() {
    const char* v = std::getenv("FAME_NO_TC");
    return !(v && v[0] == '1');
}

// P = A^H B on the tensor cores, G written in the layout of mode (see k_gram_tc_reduce).
// Returns FAME_E_ARG (nothing launched) when the shapes do not fit this kernel.
fame_status gram_tc(fame_ctx* c, const BlockList<float2>& Ain, const BlockList<float2>& Bin, size_t ld, int mode,
                    double2* G, cudaStream_t st) {
    const BlockList<float2> A = compact(Ain), B = compact(Bin);
    const int MA = A.total, NB = B.total;
    const int nA = blocks_of(A);
    const bool alias = is_prefix(B, A);
    const int nB = alias ? 0 : blocks_of(B);
    if (MA < 1 || NB < 1 || (ld & 1) || nA + nB > 2 * kMaxBlocks || !encode_fn()) return FAME_E_ARG;
    TcMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    TcGramArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nA = nA;
    a.nB = nB;
    int raw = 0, araw = 0, braw_alias = 0;
    for (int b = 0; b < nA + nB; ++b) {
        const float2* p = b < nA ? A.ptr[b] : B.ptr[b - nA];
        const int cols = b < nA ? A.cols[b] : B.cols[b - nA];
        if (cols > 256 || (reinterpret_cast<uintptr_t>(p) & 15) || !encode_block(&maps.m[b], p, ld, cols))
            return FAME_E_ARG;
        a.cols[b] = cols;
        a.rawoff[b] = raw;
        raw += (cols + 7) & ~7;
        if (b < nA) araw = raw;
        if (alias && b < blocks_of(B)) braw_alias = raw;
    }
    a.MA = MA;
    a.NB = NB;
    a.nraw = raw;
    a.bstart = alias ? 0 : araw;
    a.nbraw = alias ? braw_alias : raw - araw;
    a.NP = (a.nbraw + 15) & ~15;
    if (araw > 128 || a.NP > 128) return FAME_E_ARG;    // one 128-row MMA operand; TMEM for two CTAs per SM
    a.raw_bytes = 0;
    for (int b = 0; b < nA + nB; ++b) a.raw_bytes += (uint32_t)a.cols[b] * 2 * KC * 4;
    a.ld = ld;
    // stages: as many as fit (2..4), preferring two CTAs per SM
    int per_sm = 2, NS = 0;
    size_t smem = 0;
    for (int want = 2; want >= 1 && NS == 0; --want)
        for (int ns = 4; ns >= 2; --ns) {
            const size_t b = gram_layout(a.nraw, a.NP, ns).total + 1024;
            if (b * want <= 226u * 1024u && b <= 227u * 1024u) {
                NS = ns;
                per_sm = want;
                smem = b;
                break;
            }
        }
    if (NS == 0) return FAME_E_ARG;
    a.NS = NS;
    // CTAs: a contiguous multiple of 16 rows each, one wave
    const size_t chunks = (ld + KC - 1) / KC;
    const size_t grid0 = std::min<size_t>((size_t)152 * per_sm, chunks);
    a.rows_per_cta = ((ld + grid0 - 1) / grid0 + KC - 1) / KC * KC;
    const int grid = (int)((ld + a.rows_per_cta - 1) / a.rows_per_cta);
    fame_status s;
    if (!c->tcerr.p && (s = tc_reset_err(c, st)) != FAME_OK) return s;
    if ((s = grow(c, c->partial, (size_t)grid * MA * NB * sizeof(double2))) != FAME_OK) return s;
    a.partial = reinterpret_cast<double2*>(c->partial.p);
    a.err = reinterpret_cast<int*>(c->tcerr.p);
    a.timeout_ns = wait_timeout_ns();
    a.skip_chunk = skip_chunk_hook();
    a.plant = plant_hook();
    if ((s = kernel_smem(c, (const void*)k_gram_tc, smem)) != FAME_OK) return s;
    {
        // algorithmic bytes: every distinct column read once; 8 flops per complex MAC
        const int ncol = MA + (alias ? 0 : NB);
        ProfScope ps(mode == 2 ? K_GRAM_HERM : K_GRAM, false, st, (double)ld * ncol * sizeof(float2),
                     8.0 * (double)MA * NB * ld);
        k_gram_tc<<<grid, kThreads, smem, st>>>(maps, a);
    }
    {
        const int kk = MA * NB;
        ProfScope ps(K_GRAM_RED, false, st, (double)grid * kk * sizeof(double2), 2.0 * grid * kk);
        k_gram_tc_reduce<<<(kk + 7) / 8, 256, 0, st>>>(a.partial, grid, MA, NB, mode, G, a.err);
    }
    count_launch(2);
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}
