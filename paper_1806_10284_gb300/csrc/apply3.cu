// Fixed-length fused passes of the A_r apply (eq. NFSEP) for the common grid
// lengths.  The same three passes as the generic kernels in transforms.cu
// (Z-in, XY, Z-out; Algorithms 5.2 and 5.1 with the Pi_r / Sigma_r and B^{-1}
// stages fused in), rearranged so that each pass touches HBM once per element
// and shared memory once per radix step:
//
//  * the lengths and their radix split L = R1 * R2 are template constants, so
//    every index is compile-time arithmetic and every small DFT stays in
//    registers;
//  * the first radix step of each transform reads its inputs straight from
//    global memory (Z passes: the frequency expansion Sigma_r Pi_r is applied
//    on the fly) and the last radix step writes straight to global memory
//    (Z-in: with the D_a3 twist; Z-out: with the Pi_r^H contraction), so a Z
//    pass does a single shared-memory exchange per vector; a Z block that takes
//    several vectors can request the next vector's inputs into registers while
//    it transforms the current one, so its loads overlap its arithmetic;
//  * in the XY pass every radix step writes its outputs to the slots it read
//    its inputs from, so one plane buffer serves all seven steps with one
//    barrier between steps; the B^{-1} plane is copied to shared memory
//    asynchronously (cp.async) while the y and x inverse transforms run.  The
//    plane is taken by 256 threads, or for the larger planes by 512 threads
//    with a register budget of three blocks per SM.
//
// Radix steps follow the four-step split of fft2.cuh: for L = A * B and input
// index t + B t1 (t < B, t1 < A), an A-point DFT over t1, the twiddle
// w_L^{t k1}, then a B-point DFT over t giving output k1 + A k2.
#include <algorithm>
#include <cmath>

#include "bounds.cuh"
#include "fame_internal.h"
#include "fft2.cuh"
#include "phases.cuh"

namespace {

using fft2::Dft;

template <int L> struct Sp {
    static constexpr int R1 = fft2::split_of(L).R1;
    static constexpr int R2 = fft2::split_of(L).R2;
    static constexpr int RMAX = R1 > R2 ? R1 : R2;
};
// Z-pass blocks per SM asked of the register allocator: about 640 resident threads
// where that fits without spills, else about 512 (the prefetching forms hold a second
// vector's inputs in registers)
template <int L, int NT, bool OUT, bool PF = false> struct ZOcc {
    static constexpr int threads = ((L == 64 && !OUT && !PF) || (L <= 32 && !(OUT && PF))) ? 640 : 512;
    static constexpr int value = threads / NT > 0 ? threads / NT : 1;
};

// x * w_L^{t k}, w_L = e^{-2 pi i/L}, conjugated for an inverse transform; tw holds w_L^j.
// k is a compile-time index in the callers' unrolled loops (k = 0: no factor); t = 0
// multiplies by tw[0] = 1 exactly.
template <bool INV, typename C>
__device__ __forceinline__ C twid(C x, const C* tw, int t, int k) {
    if (k == 0) return x;
    C w = tw[t * k];
    if (INV) w.y = -w.y;
    return cmul(x, w);
}

__device__ __forceinline__ void cp_async(float* dst, const float* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Basis-switch bits of TP consecutive x-frequencies starting at flat index f0.
template <int TP>
__device__ __forceinline__ uint32_t tile_bits(const uint32_t* mask, size_t f0, size_t n) {
    const size_t last = min(f0 + TP - 1, n - 1);
    unsigned long long w = mask[f0 >> 5];
    if ((last >> 5) != (f0 >> 5)) w |= (unsigned long long)mask[last >> 5] << 32;
    return (uint32_t)(w >> (f0 & 31)) & (uint32_t)((1ull << TP) - 1);
}

// Per-tile tables of the Z passes: Lambda_1, Lambda_2 and the z-twist fraction of
// each x-frequency, Lambda_3 and the D_a3 twist of each (z, x) pair, the
// basis-switch bits and the z twiddles.
template <typename R, int L, int TP>
struct ZTile {
    using C = typename cpx<R>::T;
    using F = typename FracT<R>::T;
    C tw[L];
    C tws[L][TP];
    C L2[L][TP];
    PencilBasis<R> PB[TP];
    F F3[TP];
    uint32_t bits[L];
};

template <typename R, int L, int TP>
__device__ __forceinline__ void ztile_setup(ZTile<R, L, TP>& T, const KParams<R>& P, int q, int p0) {
    constexpr int NT = TP * Sp<L>::RMAX;
    const int tid = threadIdx.x, n1 = P.n1, n2 = P.n2;
    const size_t n = (size_t)n1 * n2 * L;
    for (int i = tid; i < L; i += NT) {
        T.tw[i] = P.tw[2][i];
        T.bits[i] = tile_bits<TP>(P.alt, ((size_t)i * n2 + q) * n1 + p0, n);
    }
    for (int pp = tid; pp < TP; pp += NT) {
        const int p = min(p0 + pp, n1 - 1);
        const typename cpx<R>::T L0 = lambda_of(p, n1, P.f1, P.inv_dx), L1 = lambda_of(q, n2, P.f2[p], P.inv_dy);
        T.PB[pp] = PencilBasis<R>{L0, L1, L0 + L1, L0 - L1, L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y};
        T.F3[pp] = P.f3[(size_t)q * n1 + p];
    }
    __syncthreads();
    for (int e = tid; e < L * TP; e += NT) {
        const int pp = e % TP, c = e / TP;
        T.tws[c][pp] = cis(frac_mul(c, T.F3[pp]));
        T.L2[c][pp] = lambda_of(c, L, T.F3[pp], P.inv_dz);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Z-in: y (2 per frequency) -> Sigma_r Pi_r -> inverse z-DFT -> D_a3 twist.
// Block: TP consecutive x-frequencies at one y-frequency q, vectors
// [z vpc, (z+1) vpc).  Thread (pp, t): first radix step of pencil pp for the
// three components; thread (pp, k1): second radix step.
// ---------------------------------------------------------------------------
template <typename R, int L, int TP, bool PF>
__global__ void __launch_bounds__(TP * Sp<L>::RMAX, (ZOcc<L, TP * Sp<L>::RMAX, false, PF>::value))
k_zin3(KParams<R> P, const typename cpx<R>::T* __restrict__ y, typename cpx<R>::T* __restrict__ W,
       int m, int vpc) {
    using C = typename cpx<R>::T;
    constexpr int R1 = Sp<L>::R1, R2 = Sp<L>::R2;
    __shared__ ZTile<R, L, TP> T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Y = reinterpret_cast<C*>(smem_raw);   // [3][L][TP]
    const int n1 = P.n1, n2 = P.n2;
    const size_t n = (size_t)n1 * n2 * L, plane = (size_t)n1 * n2;
    const int q = blockIdx.y, p0 = blockIdx.x * TP;
    const int pp = threadIdx.x % TP, t = threadIdx.x / TP, p = p0 + pp;
    const bool valid = p < n1;
    const size_t base = (size_t)q * n1 + p;
    const int v1 = min(m, (int)(blockIdx.z + 1) * vpc);
    // this thread's inputs of vector v (rows t + R2 t1 of pencil pp, both components);
    // with PF the next vector's are requested as soon as these are consumed
    C a1[R1], a2[R1];
    auto load = [&](int v) {
        const C* yv = y + (size_t)v * 2 * n + base;
#pragma unroll
        for (int t1 = 0; t1 < R1; ++t1) {
            const size_t off = (size_t)(t + R2 * t1) * plane;
            const bool ld_ok = valid && bounds_ok(base + off < n, kBndZLoad, (long long)(base + off));
            a1[t1] = ld_ok ? yv[off] : mk((R)0, (R)0);
            a2[t1] = ld_ok ? yv[n + off] : mk((R)0, (R)0);
        }
    };
    // with PF the first vector's loads are in flight while the tile tables are built
    if (PF && t < R2 && blockIdx.z * vpc < v1) load(blockIdx.z * vpc);
    ztile_setup<R, L, TP>(T, P, q, p0);
    for (int v = blockIdx.z * vpc; v < v1; ++v) {
        if (t < R2) {
            if (!PF) load(v);
            // expansion; components 1 and 2 wait in this thread's own slots of Y
            // (rows t + R2 j of pencil pp), which its radix step overwrites in turn
            C x0[R1];
#pragma unroll
            for (int t1 = 0; t1 < R1; ++t1) {
                const int r = t + R2 * t1;
                C o1, o2;
                expand<R>(T.PB[pp], T.L2[r][pp], (T.bits[r] >> pp) & 1u, a1[t1], a2[t1], x0[t1], o1, o2);
                Y[(L + r) * TP + pp] = o1;
                Y[(2 * L + r) * TP + pp] = o2;
            }
            if (PF && v + 1 < v1) load(v + 1);
            Dft<R1, true, C>::run(x0);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) Y[(k1 * R2 + t) * TP + pp] = twid<true>(x0[k1], T.tw, t, k1);
#pragma unroll
            for (int l = 1; l < 3; ++l) {
#pragma unroll
                for (int t1 = 0; t1 < R1; ++t1) x0[t1] = Y[(l * L + t + R2 * t1) * TP + pp];
                Dft<R1, true, C>::run(x0);
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1)
                    Y[(l * L + k1 * R2 + t) * TP + pp] = twid<true>(x0[k1], T.tw, t, k1);
            }
        }
        __syncthreads();
        if (t < R1) {
            const int k1 = t;
            C* Wv = W + (size_t)v * 3 * n + base;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                C u[R2];
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) u[k2] = Y[(l * L + k1 * R2 + k2) * TP + pp];
                Dft<R2, true, C>::run(u);
                if (valid) {
#pragma unroll
                    for (int k2 = 0; k2 < R2; ++k2) {
                        const int c = k1 + R1 * k2;
                        if (bounds_ok(base + (size_t)c * plane < n, kBndZStore, (long long)(base + (size_t)c * plane)))
                            Wv[(size_t)l * n + (size_t)c * plane] = cmul(u[k2], T.tws[c][pp]);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Z-out: conj D_a3 twist -> forward z-DFT -> Pi_r^H contraction, Sigma_r.
// ---------------------------------------------------------------------------
template <typename R, int L, int TP, bool PF>
__global__ void __launch_bounds__(TP * Sp<L>::RMAX, (ZOcc<L, TP * Sp<L>::RMAX, true, PF>::value))
k_zout3(KParams<R> P, const typename cpx<R>::T* __restrict__ W, typename cpx<R>::T* __restrict__ out,
        int m, int vpc) {
    using C = typename cpx<R>::T;
    constexpr int R1 = Sp<L>::R1, R2 = Sp<L>::R2;
    __shared__ ZTile<R, L, TP> T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Y = reinterpret_cast<C*>(smem_raw);   // [3][L][TP]
    const int n1 = P.n1, n2 = P.n2;
    const size_t n = (size_t)n1 * n2 * L, plane = (size_t)n1 * n2;
    const int q = blockIdx.y, p0 = blockIdx.x * TP;
    const int pp = threadIdx.x % TP, t = threadIdx.x / TP, p = p0 + pp;
    const bool valid = p < n1;
    const size_t base = (size_t)q * n1 + p;
    const int v1 = min(m, (int)(blockIdx.z + 1) * vpc);
    // this thread's inputs of vector v; with PF the next vector's are requested
    // once these have gone through the first radix step
    C g[3][R1];
    auto load = [&](int v) {
        const C* Wv = W + (size_t)v * 3 * n + base;
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int t1 = 0; t1 < R1; ++t1)
                g[l][t1] = (valid && bounds_ok(base + (size_t)(t + R2 * t1) * plane < n, kBndZLoad,
                                               (long long)(base + (size_t)(t + R2 * t1) * plane)))
                               ? Wv[(size_t)l * n + (size_t)(t + R2 * t1) * plane]
                               : mk((R)0, (R)0);
    };
    // with PF the first vector's loads are in flight while the tile tables are built
    if (PF && t < R2 && blockIdx.z * vpc < v1) load(blockIdx.z * vpc);
    ztile_setup<R, L, TP>(T, P, q, p0);
    for (int v = blockIdx.z * vpc; v < v1; ++v) {
        if (t < R2) {
            if (!PF) load(v);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
#pragma unroll
                for (int t1 = 0; t1 < R1; ++t1) g[l][t1] = cmulc(T.tws[t + R2 * t1][pp], g[l][t1]);
                Dft<R1, false, C>::run(g[l]);
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1)
                    Y[(l * L + k1 * R2 + t) * TP + pp] = twid<false>(g[l][k1], T.tw, t, k1);
            }
            if (PF && v + 1 < v1) load(v + 1);
        }
        __syncthreads();
        if (t < R1) {
            const int k1 = t;
            C u[3][R2];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) u[l][k2] = Y[(l * L + k1 * R2 + k2) * TP + pp];
                Dft<R2, false, C>::run(u[l]);
            }
            if (valid) {
                C* ov = out + (size_t)v * 2 * n + base;
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) {
                    const int r = k1 + R1 * k2;
                    C z1, z2;
                    contract<R>(T.PB[pp], T.L2[r][pp], (T.bits[r] >> pp) & 1u, u[0][k2], u[1][k2], u[2][k2], z1, z2);
                    if (bounds_ok(base + (size_t)r * plane < n, kBndZStore, (long long)(base + (size_t)r * plane))) {
                        ov[(size_t)r * plane] = z1;
                        ov[n + (size_t)r * plane] = z2;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// XY: one (vector, component, z) plane of LY rows (y) by LX columns (x) per block.
// After the inverse y transform, logical row b sits in physical row
// rho(b) = (b mod RY1) RY2 + floor(b / RY1); rows are walked in physical order
// so that consecutive lanes hit consecutive rows (odd row stride LX + 1).
// mode 0: full apply; mode 1: lift x = B^{-1} T (...) (stops after the
// inverse x transform, applies the D_a1 twist and lift_scale).
// ---------------------------------------------------------------------------
constexpr int kXYThreads = 256, kXYThreadsWide = 512;

template <typename R, int LX, int LY>
struct XYLayout {
    using C = typename cpx<R>::T;
    using F = typename FracT<R>::T;
    static constexpr int S = LX + 1;
    static constexpr size_t x_off = 0;
    static constexpr size_t ib_off = x_off + (size_t)LY * S * sizeof(C);
    static constexpr size_t twx_off = (ib_off + (size_t)LY * S * sizeof(R) + 15) / 16 * 16;
    static constexpr size_t twy_off = twx_off + LX * sizeof(C);
    static constexpr size_t f2_off = twy_off + LY * sizeof(C);
    static constexpr size_t bytes = f2_off + LX * sizeof(F);
};

template <typename R, int LX, int LY, int NT>
__device__ __forceinline__ void xy3_plane(const KParams<R>& P, typename cpx<R>::T* __restrict__ W, int mode,
                                          R lift_scale) {
    using C = typename cpx<R>::T;
    using F = typename FracT<R>::T;
    using Lay = XYLayout<R, LX, LY>;
    constexpr int RX1 = Sp<LX>::R1, RX2 = Sp<LX>::R2, RY1 = Sp<LY>::R1, RY2 = Sp<LY>::R2;
    constexpr int S = Lay::S, NP = LX * LY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* X = reinterpret_cast<C*>(smem_raw + Lay::x_off);
    R* ibs = reinterpret_cast<R*>(smem_raw + Lay::ib_off);
    C* twx = reinterpret_cast<C*>(smem_raw + Lay::twx_off);
    C* twy = reinterpret_cast<C*>(smem_raw + Lay::twy_off);
    F* F2s = reinterpret_cast<F*>(smem_raw + Lay::f2_off);
    const int tid = threadIdx.x;
    const int n3 = P.n3;
    const int plane = blockIdx.x, c = plane % n3, l = (plane / n3) % 3;
    C* g = W + (size_t)plane * NP;
    const R* ib = P.invB + ((size_t)l * n3 + c) * NP;

    // B^{-1} plane into shared memory (row rho(b), column a), in flight during the inverse transforms
    for (int e = tid; e < NP; e += NT) {
        const int b = e / LX, a = e - b * LX;
        cp_async(&ibs[((b % RY1) * RY2 + b / RY1) * S + a], ib + e);
    }
    for (int i = tid; i < LX; i += NT) { twx[i] = P.tw[0][i]; F2s[i] = P.f2[i]; }
    for (int i = tid; i < LY; i += NT) twy[i] = P.tw[1][i];

    // A: inverse y, first radix step, inputs from global memory (thread: column p, offset ty)
    {
        constexpr int IA = (LX * RY2 + NT - 1) / NT;
        C v[IA][RY1];
#pragma unroll
        for (int i = 0; i < IA; ++i) {
            const int w = tid + i * NT;
            if (w < LX * RY2) {
                const int p = w % LX, ty = w / LX;
#pragma unroll
                for (int t1 = 0; t1 < RY1; ++t1) v[i][t1] = g[(ty + RY2 * t1) * LX + p];
            }
        }
        __syncthreads();   // tables
#pragma unroll
        for (int i = 0; i < IA; ++i) {
            const int w = tid + i * NT;
            if (w < LX * RY2) {
                const int p = w % LX, ty = w / LX;
                Dft<RY1, true, C>::run(v[i]);
#pragma unroll
                for (int k1 = 0; k1 < RY1; ++k1) X[(k1 * RY2 + ty) * S + p] = twid<true>(v[i][k1], twy, ty, k1);
            }
        }
    }
    __syncthreads();
    // B: inverse y, second radix step, then the D_a2 twist e^{2 pi i b f2(p)}, b = k1 + RY1 k2
    for (int w = tid; w < LX * RY1; w += NT) {
        const int p = w % LX, k1 = w / LX;
        C u[RY2];
#pragma unroll
        for (int k2 = 0; k2 < RY2; ++k2) u[k2] = X[(k1 * RY2 + k2) * S + p];
        Dft<RY2, true, C>::run(u);
        C cur = cis(frac_mul(k1, F2s[p]));
        const C stp = cis(frac_mul(RY1, F2s[p]));
#pragma unroll
        for (int k2 = 0; k2 < RY2; ++k2) {
            X[(k1 * RY2 + k2) * S + p] = cmul(u[k2], cur);
            cur = cmul(cur, stp);
        }
    }
    __syncthreads();
    // C: inverse x, first radix step (thread: physical row rho, offset tx)
    for (int w = tid; w < LY * RX2; w += NT) {
        const int rho = w % LY, tx = w / LY;
        C x[RX1];
#pragma unroll
        for (int t1 = 0; t1 < RX1; ++t1) x[t1] = X[rho * S + tx + RX2 * t1];
        Dft<RX1, true, C>::run(x);
#pragma unroll
        for (int k1 = 0; k1 < RX1; ++k1) X[rho * S + tx + RX2 * k1] = twid<true>(x[k1], twx, tx, k1);
    }
    cp_async_wait();
    __syncthreads();
    if (mode == 0) {
        // D: inverse x second step -> B^{-1}/n -> forward x first step (inputs a = k1 + RX1 j)
        for (int w = tid; w < LY * RX1; w += NT) {
            const int rho = w % LY, k1 = w / LY;
            C u[RX2];
#pragma unroll
            for (int k2 = 0; k2 < RX2; ++k2) u[k2] = X[rho * S + RX2 * k1 + k2];
            Dft<RX2, true, C>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < RX2; ++k2) u[k2] = (ibs[rho * S + k1 + RX1 * k2] * P.scale) * u[k2];
            Dft<RX2, false, C>::run(u);
#pragma unroll
            for (int k = 0; k < RX2; ++k) X[rho * S + RX2 * k1 + k] = twid<false>(u[k], twx, k1, k);
        }
        __syncthreads();
        // E: forward x second step; output a = k + RX2 k2 lands in column a
        for (int w = tid; w < LY * RX2; w += NT) {
            const int rho = w % LY, k = w / LY;
            C u[RX1];
#pragma unroll
            for (int t = 0; t < RX1; ++t) u[t] = X[rho * S + RX2 * t + k];
            Dft<RX1, false, C>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < RX1; ++k2) X[rho * S + RX2 * k2 + k] = u[k2];
        }
        __syncthreads();
        // F: conj D_a2 twist, forward y first step over b = k1 + RY1 j (physical rows k1 RY2 + j)
        for (int w = tid; w < LX * RY1; w += NT) {
            const int p = w % LX, k1 = w / LX;
            C u[RY2];
            C cur = conjc(cis(frac_mul(k1, F2s[p])));
            const C stp = conjc(cis(frac_mul(RY1, F2s[p])));
#pragma unroll
            for (int j = 0; j < RY2; ++j) {
                u[j] = cmul(X[(k1 * RY2 + j) * S + p], cur);
                cur = cmul(cur, stp);
            }
            Dft<RY2, false, C>::run(u);
#pragma unroll
            for (int k = 0; k < RY2; ++k) X[(k1 * RY2 + k) * S + p] = twid<false>(u[k], twy, k1, k);
        }
        __syncthreads();
        // G: forward y second step, output row k + RY2 k2 to global memory
        for (int w = tid; w < LX * RY2; w += NT) {
            const int p = w % LX, k = w / LX;
            C u[RY1];
#pragma unroll
            for (int t = 0; t < RY1; ++t) u[t] = X[(t * RY2 + k) * S + p];
            Dft<RY1, false, C>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < RY1; ++k2) g[(k + RY2 * k2) * LX + p] = u[k2];
        }
    } else {
        // D': inverse x second step, D_a1 twist, B^{-1} lift_scale; a = k1 + RX1 k2 stays in column RX2 k1 + k2
        for (int w = tid; w < LY * RX1; w += NT) {
            const int rho = w % LY, k1 = w / LY;
            C u[RX2];
#pragma unroll
            for (int k2 = 0; k2 < RX2; ++k2) u[k2] = X[rho * S + RX2 * k1 + k2];
            Dft<RX2, true, C>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < RX2; ++k2) {
                const int a = k1 + RX1 * k2;
                X[rho * S + RX2 * k1 + k2] =
                    (ibs[rho * S + a] * lift_scale) * cmul(u[k2], cis(frac_mul(a, P.f1)));
            }
        }
        __syncthreads();
        for (int e = tid; e < NP; e += NT) {
            const int b = e / LX, a = e - b * LX;
            g[e] = X[((b % RY1) * RY2 + b / RY1) * S + (a % RX1) * RX2 + a / RX1];
        }
    }
}

// 256 threads: the register allocator's own choice; 512 threads: as many blocks per SM
// as shared memory allows, at most 3
template <typename R, int LX, int LY, int NT> struct XYOcc {
    static constexpr int by_smem = (int)((227u * 1024u) / XYLayout<R, LX, LY>::bytes);
    static constexpr int value = by_smem < 1 ? 1 : (by_smem > 3 ? 3 : by_smem);
};

template <typename R, int LX, int LY>
__global__ void __launch_bounds__(kXYThreads)
k_xy3(KParams<R> P, typename cpx<R>::T* __restrict__ W, int mode, R lift_scale) {
    xy3_plane<R, LX, LY, kXYThreads>(P, W, mode, lift_scale);
}

template <typename R, int LX, int LY>
__global__ void __launch_bounds__(kXYThreadsWide, (XYOcc<R, LX, LY, kXYThreadsWide>::value))
k_xy3w(KParams<R> P, typename cpx<R>::T* __restrict__ W, int mode, R lift_scale) {
    xy3_plane<R, LX, LY, kXYThreadsWide>(P, W, mode, lift_scale);
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
constexpr int kZTP = 16;

template <typename R, int L>
size_t z3_dyn_smem() { return (size_t)3 * L * kZTP * sizeof(typename cpx<R>::T); }

template <typename R, int L, bool PF>
fame_status launch_z3(fame_ctx* c, const KParams<R>& P, const typename cpx<R>::T* in,
                      typename cpx<R>::T* out, int m, bool zin, int vpc_req, cudaStream_t st) {
    const int n1 = c->plan.n[0], n2 = c->plan.n[1];
    constexpr int NT = kZTP * Sp<L>::RMAX;
    const size_t smem = z3_dyn_smem<R, L>();
    const void* fn = zin ? (const void*)k_zin3<R, L, kZTP, PF> : (const void*)k_zout3<R, L, kZTP, PF>;
    if (smem + sizeof(ZTile<R, L, kZTP>) > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long tiles = (long long)((n1 + kZTP - 1) / kZTP) * n2;
    // enough blocks for several waves over 152 SMs; the rest of the vectors loop in a block
    int vpc = 1;
    while (vpc < m && tiles * ((m + 2 * vpc - 1) / (2 * vpc)) >= 152 * 8) vpc *= 2;
    if (vpc_req > 0) vpc = std::min(vpc_req, m);
    dim3 grid((n1 + kZTP - 1) / kZTP, n2, (m + vpc - 1) / vpc);
    const double nm = (double)c->n * m;
    ProfScope ps(zin ? K_ZIN : K_ZOUT, sizeof(R) == 8, st, 5.0 * nm * sizeof(typename cpx<R>::T),
                 3 * nm * 5.0 * std::log2((double)L) + 60.0 * nm);
    if (zin)
        k_zin3<R, L, kZTP, PF><<<grid, NT, smem, st>>>(P, in, out, m, vpc);
    else
        k_zout3<R, L, kZTP, PF><<<grid, NT, smem, st>>>(P, in, out, m, vpc);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename R, int LX, int LY, int NT>
fame_status launch_xy3(fame_ctx* c, const KParams<R>& P, typename cpx<R>::T* W, int m, int mode,
                       R lift_scale, cudaStream_t st) {
    using C = typename cpx<R>::T;
    const size_t smem = XYLayout<R, LX, LY>::bytes;
    const void* fn;
    if constexpr (NT == kXYThreads)
        fn = (const void*)k_xy3<R, LX, LY>;
    else
        fn = (const void*)k_xy3w<R, LX, LY>;
    if (smem > 48 * 1024)
        FAME_CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const double nm = (double)c->n * m;
    const double lg = std::log2((double)LX) + std::log2((double)LY);
    ProfScope ps(K_XY, sizeof(R) == 8, st, 2.0 * 3 * nm * sizeof(C) + 3.0 * c->n * sizeof(R),
                 3 * nm * 5.0 * (mode == 0 ? 2.0 : 1.0) * lg);
    const unsigned blocks = (unsigned)(3LL * m * c->plan.n[2]);
    if constexpr (NT == kXYThreads)
        k_xy3<R, LX, LY><<<blocks, NT, smem, st>>>(P, W, mode, lift_scale);
    else
        k_xy3w<R, LX, LY><<<blocks, NT, smem, st>>>(P, W, mode, lift_scale);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

}  // namespace

FAME_BOUNDS_READER(apply3)

// Lengths with a fixed-length Z pass, and (n1, n2) pairs with a fixed-length XY pass.
bool z3_supported(int L) { return L == 16 || L == 32 || L == 48 || L == 64 || L == 80 || L == 96; }
bool xy3_supported(int n1, int n2) {
    return (n1 == n2 && (n1 == 16 || n1 == 32 || n1 == 48 || n1 == 64 || n1 == 96)) ||
           (n1 == 80 && n2 == 96);
}

template <typename R, bool PF>
fame_status run_z3_len(fame_ctx* c, const KParams<R>& P, const typename cpx<R>::T* in,
                       typename cpx<R>::T* out, int m, bool zin, int vpc, cudaStream_t st) {
    switch (c->plan.n[2]) {
        case 16: return launch_z3<R, 16, PF>(c, P, in, out, m, zin, vpc, st);
        case 32: return launch_z3<R, 32, PF>(c, P, in, out, m, zin, vpc, st);
        case 48: return launch_z3<R, 48, PF>(c, P, in, out, m, zin, vpc, st);
        case 64: return launch_z3<R, 64, PF>(c, P, in, out, m, zin, vpc, st);
        case 80: return launch_z3<R, 80, PF>(c, P, in, out, m, zin, vpc, st);
        case 96: return launch_z3<R, 96, PF>(c, P, in, out, m, zin, vpc, st);
        default: return set_err(c, FAME_E_ARG, "fixed-length Z pass: unsupported n3");
    }
}

template <typename R>
fame_status run_z3(fame_ctx* c, const KParams<R>& P, const typename cpx<R>::T* in,
                   typename cpx<R>::T* out, int m, bool zin, int vpc, bool prefetch, cudaStream_t st) {
    return prefetch ? run_z3_len<R, true>(c, P, in, out, m, zin, vpc, st)
                    : run_z3_len<R, false>(c, P, in, out, m, zin, vpc, st);
}

// planes with at least 512 work items per radix step also have a 512-thread form
bool xy3_wide_supported(int n1, int n2) { return xy3_supported(n1, n2) && n1 * n2 >= 4096; }

template <typename R>
fame_status run_xy3(fame_ctx* c, const KParams<R>& P, typename cpx<R>::T* W, int m, int mode,
                    R lift_scale, bool wide, cudaStream_t st) {
    const int n1 = c->plan.n[0], n2 = c->plan.n[1];
    if (wide) {
        if (n1 == 80 && n2 == 96) return launch_xy3<R, 80, 96, kXYThreadsWide>(c, P, W, m, mode, lift_scale, st);
        if (n1 == 64 && n2 == 64) return launch_xy3<R, 64, 64, kXYThreadsWide>(c, P, W, m, mode, lift_scale, st);
        if (n1 == 96 && n2 == 96) return launch_xy3<R, 96, 96, kXYThreadsWide>(c, P, W, m, mode, lift_scale, st);
        return set_err(c, FAME_E_ARG, "fixed-length XY pass, 512 threads: unsupported (n1, n2)");
    }
    if (n1 == 80 && n2 == 96) return launch_xy3<R, 80, 96, kXYThreads>(c, P, W, m, mode, lift_scale, st);
    if (n1 == n2) {
        switch (n1) {
            case 16: return launch_xy3<R, 16, 16, kXYThreads>(c, P, W, m, mode, lift_scale, st);
            case 32: return launch_xy3<R, 32, 32, kXYThreads>(c, P, W, m, mode, lift_scale, st);
            case 48: return launch_xy3<R, 48, 48, kXYThreads>(c, P, W, m, mode, lift_scale, st);
            case 64: return launch_xy3<R, 64, 64, kXYThreads>(c, P, W, m, mode, lift_scale, st);
            case 96: return launch_xy3<R, 96, 96, kXYThreads>(c, P, W, m, mode, lift_scale, st);
            default: break;
        }
    }
    return set_err(c, FAME_E_ARG, "fixed-length XY pass: unsupported (n1, n2)");
}

template fame_status run_z3<float>(fame_ctx*, const KParams<float>&, const float2*, float2*, int, bool, int,
                                   bool, cudaStream_t);
template fame_status run_xy3<float>(fame_ctx*, const KParams<float>&, float2*, int, int, float, bool,
                                    cudaStream_t);
