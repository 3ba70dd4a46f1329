// Register-resident DFT building blocks and the two-level pencil transform.
//
// A length-L pencil with L = R1 * R2 (R1, R2 <= 16) is transformed by R2
// threads each doing an R1-point DFT on elements t + R2 t1 (t1 < R1), one
// twiddle e^{-+2 pi i t k1 / L}, an exchange through shared memory, and R1
// threads each doing an R2-point DFT (the four-step factorisation
// X[k1 + R1 k2] = sum_t2 w_R2^{t2 k2} w_L^{t2 k1} sum_t1 x[t2 + R2 t1] w_R1^{t1 k1}).
// The small DFTs are compile-time: radix 2, 3, 4, 5, 8 written out, and
// 6, 10, 12, 16 composed from them the same way with constant twiddles.
#pragma once

#include "fame_internal.h"

namespace fft2 {

// Butterfly sums: one paired single-precision instruction for both components
// where the target has it, componentwise arithmetic otherwise (same rounding).
__host__ __device__ __forceinline__ float2 badd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 bsub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);   // a - b, rounded once
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ double2 badd(double2 a, double2 b) { return a + b; }
__host__ __device__ __forceinline__ double2 bsub(double2 a, double2 b) { return a - b; }

// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C>
__host__ __device__ __forceinline__ C rot(C a) { return INV ? mk(-a.y, a.x) : mk(a.y, -a.x); }

// cos and sin of 2 pi j / R for the composite radices (exact where rational)
struct Tw {
    static constexpr double s3 = 0.86602540378443864676;   // sqrt(3)/2
    static constexpr double c5 = 0.80901699437494742410;   // cos(pi/5)
    static constexpr double s5 = 0.58778525229247312917;   // sin(pi/5)
    static constexpr double c10 = 0.30901699437494742410;  // cos(2 pi/5)
    static constexpr double s10 = 0.95105651629515357212;  // sin(2 pi/5)
    static constexpr double r2 = 0.70710678118654752440;   // 1/sqrt(2)
    static constexpr double c8 = 0.92387953251128675613;   // cos(pi/8)
    static constexpr double s8 = 0.38268343236508977173;   // sin(pi/8)
};

// cos and sin of 2 pi j / R, evaluated at compile time: the angle is reduced by
// exact integer arithmetic to a quarter turn q (0..3) plus y = (pi/2) r / R with
// 0 <= y <= pi/4 (using the complementary angle above pi/4), where Taylor series
// of 14 terms are accurate to double rounding.
__host__ __device__ constexpr double ct_sin_q(double y) {
    double term = y, sum = y;
    for (int k = 1; k < 14; ++k) {
        term *= -y * y / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos_q(double y) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -y * y / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
// returns cos (want_sin = false) or sin of 2 pi j / R
__host__ __device__ constexpr double ct_trig(int j, int R, bool want_sin) {
    constexpr double half_pi = 1.57079632679489661923132169163975;
    const long long jj = ((long long)j % R + R) % R;
    const long long q4 = 4 * jj;                 // angle = (pi/2) q4 / R
    const int quad = (int)(q4 / R);
    const long long r = q4 - (long long)quad * R;   // 0 <= r < R
    double c = 0.0, sn = 0.0;
    if (2 * r <= R) {
        const double y = half_pi * (double)r / (double)R;
        c = ct_cos_q(y);
        sn = ct_sin_q(y);
    } else {
        const double y = half_pi * (double)(R - r) / (double)R;
        c = ct_sin_q(y);
        sn = ct_cos_q(y);
    }
    // rotate by quad quarter turns
    const double cq = quad == 0 ? c : quad == 1 ? -sn : quad == 2 ? -c : sn;
    const double sq = quad == 0 ? sn : quad == 1 ? c : quad == 2 ? -sn : -c;
    return want_sin ? sq : cq;
}

template <int R>
__host__ __device__ constexpr double cosr(int j) { return ct_trig(j, R, false); }
template <int R>
__host__ __device__ constexpr double sinr(int j) { return ct_trig(j, R, true); }

template <> __host__ __device__ constexpr double cosr<6>(int j) {
    return (j % 6 == 0) ? 1.0 : (j % 6 == 1 || j % 6 == 5) ? 0.5 : (j % 6 == 3) ? -1.0 : -0.5;
}
template <> __host__ __device__ constexpr double sinr<6>(int j) {
    return (j % 3 == 0) ? 0.0 : (j % 6 == 1 || j % 6 == 2) ? Tw::s3 : -Tw::s3;
}
template <> __host__ __device__ constexpr double cosr<10>(int j) {
    return (j % 10 == 0) ? 1.0 : (j % 10 == 1 || j % 10 == 9) ? Tw::c5
         : (j % 10 == 2 || j % 10 == 8) ? Tw::c10 : (j % 10 == 3 || j % 10 == 7) ? -Tw::c10
         : (j % 10 == 4 || j % 10 == 6) ? -Tw::c5 : -1.0;
}
template <> __host__ __device__ constexpr double sinr<10>(int j) {
    return (j % 5 == 0) ? 0.0 : (j % 10 == 1 || j % 10 == 4) ? Tw::s5
         : (j % 10 == 2 || j % 10 == 3) ? Tw::s10 : (j % 10 == 6 || j % 10 == 9) ? -Tw::s5 : -Tw::s10;
}
template <> __host__ __device__ constexpr double cosr<12>(int j) {
    return (j % 12 == 0) ? 1.0 : (j % 12 == 1 || j % 12 == 11) ? Tw::s3
         : (j % 12 == 2 || j % 12 == 10) ? 0.5 : (j % 12 == 3 || j % 12 == 9) ? 0.0
         : (j % 12 == 4 || j % 12 == 8) ? -0.5 : (j % 12 == 5 || j % 12 == 7) ? -Tw::s3 : -1.0;
}
template <> __host__ __device__ constexpr double sinr<12>(int j) {
    return (j % 6 == 0) ? 0.0 : (j % 12 == 1 || j % 12 == 5) ? 0.5
         : (j % 12 == 2 || j % 12 == 4) ? Tw::s3 : (j % 12 == 3) ? 1.0
         : (j % 12 == 7 || j % 12 == 11) ? -0.5 : (j % 12 == 8 || j % 12 == 10) ? -Tw::s3 : -1.0;
}
template <> __host__ __device__ constexpr double cosr<16>(int j) {
    return (j % 16 == 0) ? 1.0 : (j % 16 == 1 || j % 16 == 15) ? Tw::c8
         : (j % 16 == 2 || j % 16 == 14) ? Tw::r2 : (j % 16 == 3 || j % 16 == 13) ? Tw::s8
         : (j % 16 == 4 || j % 16 == 12) ? 0.0 : (j % 16 == 5 || j % 16 == 11) ? -Tw::s8
         : (j % 16 == 6 || j % 16 == 10) ? -Tw::r2 : (j % 16 == 7 || j % 16 == 9) ? -Tw::c8 : -1.0;
}
template <> __host__ __device__ constexpr double sinr<16>(int j) {
    return (j % 8 == 0) ? 0.0 : (j % 16 == 1 || j % 16 == 7) ? Tw::s8
         : (j % 16 == 2 || j % 16 == 6) ? Tw::r2 : (j % 16 == 3 || j % 16 == 5) ? Tw::c8
         : (j % 16 == 4) ? 1.0 : (j % 16 == 9 || j % 16 == 15) ? -Tw::s8
         : (j % 16 == 10 || j % 16 == 14) ? -Tw::r2 : (j % 16 == 11 || j % 16 == 13) ? -Tw::c8 : -1.0;
}

// Small DFT: v[k] <- sum_t v[t] w_R^{t k}, w_R = e^{-2 pi i / R} (forward) or e^{+2 pi i / R}.
template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<1, INV, C> {
    __host__ __device__ __forceinline__ static void run(C*) {}
};
template <bool INV, typename C> struct Dft<2, INV, C> {
    __host__ __device__ __forceinline__ static void run(C* v) {
        const C t = bsub(v[0], v[1]);
        v[0] = badd(v[0], v[1]);
        v[1] = t;
    }
};
template <bool INV, typename C> struct Dft<4, INV, C> {
    __host__ __device__ __forceinline__ static void run(C* v) {
        const C t0 = badd(v[0], v[2]), t1 = bsub(v[0], v[2]), t2 = badd(v[1], v[3]);
        const C t3 = rot<INV>(bsub(v[1], v[3]));
        v[0] = badd(t0, t2);
        v[2] = bsub(t0, t2);
        v[1] = badd(t1, t3);
        v[3] = bsub(t1, t3);
    }
};
template <bool INV, typename C> struct Dft<3, INV, C> {
    __host__ __device__ __forceinline__ static void run(C* v) {
        using R = decltype(v[0].x);
        const R h = (R)Tw::s3;
        const C s = badd(v[1], v[2]);
        const C d = rot<INV>(bsub(v[1], v[2]));
        const C m = v[0] - (R)0.5 * s;   // componentwise, so products fuse into FMAs
        v[0] = badd(v[0], s);
        v[1] = m + h * d;
        v[2] = m - h * d;
    }
};
template <bool INV, typename C> struct Dft<5, INV, C> {
    __host__ __device__ __forceinline__ static void run(C* v) {
        using R = decltype(v[0].x);
        const R c1 = (R)Tw::c10, c2 = (R)(-Tw::c5), s1 = (R)Tw::s10, s2 = (R)Tw::s5;
        const C a14 = badd(v[1], v[4]), b14 = bsub(v[1], v[4]);
        const C a23 = badd(v[2], v[3]), b23 = bsub(v[2], v[3]);
        const C x0 = badd(badd(v[0], a14), a23);
        const C m1 = v[0] + c1 * a14 + c2 * a23;   // componentwise, fused into FMAs
        const C m2 = v[0] + c2 * a14 + c1 * a23;
        const C n1 = rot<INV>(s1 * b14 + s2 * b23);
        const C n2 = rot<INV>(s2 * b14 - s1 * b23);
        v[0] = x0;
        v[1] = badd(m1, n1);
        v[4] = bsub(m1, n1);
        v[2] = badd(m2, n2);
        v[3] = bsub(m2, n2);
    }
};
template <bool INV, typename C> struct Dft<8, INV, C> {
    __host__ __device__ __forceinline__ static void run(C* v) {
        using R = decltype(v[0].x);
        const R h = (R)Tw::r2;
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV, C>::run(e);
        Dft<4, INV, C>::run(o);
        const C t1 = INV ? mk(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                         : mk(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        const C t2 = rot<INV>(o[2]);
        const C t3 = INV ? mk(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                         : mk(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        v[0] = badd(e[0], o[0]); v[4] = bsub(e[0], o[0]);
        v[1] = badd(e[1], t1);   v[5] = bsub(e[1], t1);
        v[2] = badd(e[2], t2);   v[6] = bsub(e[2], t2);
        v[3] = badd(e[3], t3);   v[7] = bsub(e[3], t3);
    }
};

// Composite R = A * B (t = t2 + B t1, k = k1 + A k2) with constant twiddles w_R^{t2 k1}.
template <int R, int A, int B, bool INV, typename C>
struct DftComposite {
    __host__ __device__ __forceinline__ static void run(C* v) {
        using Re = decltype(v[0].x);
        C y[B][A];
#pragma unroll
        for (int t2 = 0; t2 < B; ++t2) {
#pragma unroll
            for (int t1 = 0; t1 < A; ++t1) y[t2][t1] = v[t2 + B * t1];
            Dft<A, INV, C>::run(y[t2]);
#pragma unroll
            for (int k1 = 1; k1 < A; ++k1) {
                if (t2 > 0) {
                    const Re cr = (Re)cosr<R>(t2 * k1);
                    const Re si = (Re)(INV ? sinr<R>(t2 * k1) : -sinr<R>(t2 * k1));
                    const C x = y[t2][k1];
                    y[t2][k1] = mk(x.x * cr - x.y * si, x.x * si + x.y * cr);
                }
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            C u[B];
#pragma unroll
            for (int t2 = 0; t2 < B; ++t2) u[t2] = y[t2][k1];
            Dft<B, INV, C>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = u[k2];
        }
    }
};
template <bool INV, typename C> struct Dft<6, INV, C> : DftComposite<6, 3, 2, INV, C> {};
template <bool INV, typename C> struct Dft<10, INV, C> : DftComposite<10, 5, 2, INV, C> {};
template <bool INV, typename C> struct Dft<12, INV, C> : DftComposite<12, 4, 3, INV, C> {};
template <bool INV, typename C> struct Dft<16, INV, C> : DftComposite<16, 4, 4, INV, C> {};

// Factorisation L = R1 * R2 used for each supported pencil length.
struct Split { int R1, R2; };
__host__ __device__ constexpr Split split_of(int L) {
    return L == 8 ? Split{4, 2} : L == 12 ? Split{4, 3} : L == 16 ? Split{4, 4} :
           L == 20 ? Split{5, 4} : L == 24 ? Split{6, 4} : L == 32 ? Split{8, 4} :
           L == 40 ? Split{8, 5} : L == 48 ? Split{8, 6} : L == 60 ? Split{10, 6} :
           L == 64 ? Split{8, 8} : L == 80 ? Split{10, 8} : L == 96 ? Split{12, 8} :
           L == 120 ? Split{12, 10} : L == 128 ? Split{16, 8} : L == 160 ? Split{16, 10} :
           L == 192 ? Split{16, 12} : L == 256 ? Split{16, 16} : Split{0, 0};
}
inline bool supported(int L) { return split_of(L).R1 > 0; }
__host__ __device__ constexpr int threads_per_pencil(int L) {
    return split_of(L).R1 > split_of(L).R2 ? split_of(L).R1 : split_of(L).R2;
}

}  // namespace fft2

namespace fft2 {

// Cooperative transform of npen pencils of length L = R1 * R2 by the whole block.
// ld(pc, e) returns element e of pencil pc; st(pc, e, v) stores output element e.
// Y is shared scratch of L * npen entries (layout [element][pencil], conflict-free
// for consecutive pencils); tw is the shared table e^{-2 pi i j / L}, j < L.
// Ends with __syncthreads().
template <int R1, int R2, bool INV, typename C, typename Load, typename Store>
__device__ __forceinline__ void pencils(int npen, const C* __restrict__ tw, C* __restrict__ Y,
                                        Load ld, Store st) {
    constexpr int L = R1 * R2;
    // w / npen through a float reciprocal: exact for w < 2^20 and npen <= 1024
    const float inv = 1.0f / (float)npen;
    // step 1: R2 threads per pencil, R1-point DFTs on elements t + R2 t1
    for (int w = threadIdx.x; w < npen * R2; w += blockDim.x) {
        const int t = __float2int_rz(((float)w + 0.5f) * inv), pc = w - t * npen;
        C v[R1];
#pragma unroll
        for (int t1 = 0; t1 < R1; ++t1) v[t1] = ld(pc, t + R2 * t1);
        Dft<R1, INV, C>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            C x = v[k1];
            if (k1 > 0 && t > 0) {
                C q = tw[t * k1];
                if (INV) q.y = -q.y;
                x = cmul(x, q);
            }
            Y[(k1 * R2 + t) * npen + pc] = x;
        }
    }
    __syncthreads();
    // step 2: R1 threads per pencil, R2-point DFTs
    for (int w = threadIdx.x; w < npen * R1; w += blockDim.x) {
        const int k1 = __float2int_rz(((float)w + 0.5f) * inv), pc = w - k1 * npen;
        C u[R2];
#pragma unroll
        for (int t2 = 0; t2 < R2; ++t2) u[t2] = Y[(k1 * R2 + t2) * npen + pc];
        Dft<R2, INV, C>::run(u);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) st(pc, k1 + R1 * k2, u[k2]);
    }
    __syncthreads();
    (void)L;
}

// Runtime dispatch over the supported lengths.
template <bool INV, typename C, typename Load, typename Store>
__device__ __forceinline__ void pencils_any(int L, int npen, const C* tw, C* Y, Load ld, Store st) {
    switch (L) {
        case 8:   pencils<4, 2, INV>(npen, tw, Y, ld, st); break;
        case 12:  pencils<4, 3, INV>(npen, tw, Y, ld, st); break;
        case 16:  pencils<4, 4, INV>(npen, tw, Y, ld, st); break;
        case 20:  pencils<5, 4, INV>(npen, tw, Y, ld, st); break;
        case 24:  pencils<6, 4, INV>(npen, tw, Y, ld, st); break;
        case 32:  pencils<8, 4, INV>(npen, tw, Y, ld, st); break;
        case 40:  pencils<8, 5, INV>(npen, tw, Y, ld, st); break;
        case 48:  pencils<8, 6, INV>(npen, tw, Y, ld, st); break;
        case 60:  pencils<10, 6, INV>(npen, tw, Y, ld, st); break;
        case 64:  pencils<8, 8, INV>(npen, tw, Y, ld, st); break;
        case 80:  pencils<10, 8, INV>(npen, tw, Y, ld, st); break;
        case 96:  pencils<12, 8, INV>(npen, tw, Y, ld, st); break;
        case 120: pencils<12, 10, INV>(npen, tw, Y, ld, st); break;
        case 128: pencils<16, 8, INV>(npen, tw, Y, ld, st); break;
        case 160: pencils<16, 10, INV>(npen, tw, Y, ld, st); break;
        case 192: pencils<16, 12, INV>(npen, tw, Y, ld, st); break;
        default:  pencils<16, 16, INV>(npen, tw, Y, ld, st); break;   // 256
    }
}

}  // namespace fft2
