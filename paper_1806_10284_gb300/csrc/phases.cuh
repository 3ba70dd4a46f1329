// Phase, Lambda and range-basis evaluation shared by the transform kernels.
//
// Lambda_l follows eqs. (ewK1), (ewK2), (acute_ewK3) of Section 4 with the
// twist fractions of the index-shift lattice; the unit range basis Pi_1, Pi_2
// is eqs. (range_basis1), (range_basis2) and Sigma_r = Lambda_q^{1/2} is eq. (SVD)
// of Section 5.1.
#pragma once

#include "fame_internal.h"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
// Reference vector switch: the paper's e = (1,1,1) unless 3 Lq - |Ls|^2 < G_TOL * 3 Lq.
constexpr double kGTol = 1.0 / 16.0;

// ---------------------------------------------------------------------------
// phases
// ---------------------------------------------------------------------------
// idx * f mod 1, in [-1/2, 1/2]
__device__ __forceinline__ float frac_mul(int idx, Frac32 f) {
    float t = (float)idx * f.hi;  // exact: idx < 1024, hi a multiple of 2^-13
    t -= rintf(t);
    t = fmaf((float)idx, f.lo, t);
    return t - rintf(t);
}
__device__ __forceinline__ double frac_mul(int idx, double f) {
    double t = (double)idx * f;
    return t - rint(t);
}
// e^{+2 pi i phi}, |phi| <= 1/2
__device__ __forceinline__ float2 cis(float phi) {
    float s, c;
    __sincosf((float)kTwoPi * phi, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ double2 cis(double phi) {
    double s, c;
    sincospi(2.0 * phi, &s, &c);
    return make_double2(c, s);
}
// Lambda = (e^{2 pi i (idx + L f)/L} - 1) * inv_delta, evaluated as
// 2 i sin(pi x) e^{i pi x} * inv_delta with x = (idx + L f)/L reduced to [-1/2, 1/2)
// in exact arithmetic first, so small |x| keeps full relative precision.
__device__ __forceinline__ float2 lambda_of(int idx, int L, Frac32 f, float inv_delta) {
    const float Lf = (float)L;
    float u = Lf * f.hi;                 // exact
    float t = (float)idx + u;            // exact (< 2048, 13 fractional bits)
    if (t >= 0.5f * Lf) t -= Lf;
    if (t >= 0.5f * Lf) t -= Lf;
    t = fmaf(Lf, f.lo, t);
    float x = t / Lf;
    if (x >= 0.5f) x -= 1.0f;
    if (x < -0.5f) x += 1.0f;
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(-2.0f * s * s * inv_delta, 2.0f * s * c * inv_delta);
}
__device__ __forceinline__ double2 lambda_of(int idx, int L, double f, double inv_delta) {
    double t = (double)idx + (double)L * f;
    double x = t / (double)L;
    x -= rint(x);
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(-2.0 * s * s * inv_delta, 2.0 * s * c * inv_delta);
}

__device__ __forceinline__ bool alt_bit(const uint32_t* mask, size_t f) {
    return (mask[f >> 5] >> (f & 31)) & 1u;
}

// 1/sqrt and sqrt.  Single precision: the hardware approximation (a few ulp, far
// below the complex64 path's tolerance).  Double precision: the single-precision
// estimate refined by two Newton-Raphson steps y <- y (3 - x y^2) / 2 (each doubles
// the correct digits: about 2^-22 -> 2^-44 -> below double rounding), which costs a
// handful of FP64 operations instead of a division and a square root; arguments
// outside the single-precision range take the division.
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) {
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
    y = y * (1.5 - hx * y * y);
    y = y * (1.5 - hx * y * y);
    return y;
}
__device__ __forceinline__ float root(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double root(double x) { return x * rsq(x); }

template <typename R>
struct Basis {
    typename cpx<R>::T p1[3], p2[3];
    R sig;
};

// Pi_1, Pi_2 of eqs. (range_basis1), (range_basis2) with unit columns, and
// Sigma_r = Lq^{1/2} (eq. SVD); reference vector e = (1,1,1), or (1,-1,0)
// where Lambda is close to parallel to (1,1,1) (alt, read from the FP64 mask).
template <typename R>
__device__ __forceinline__ Basis<R> make_basis(typename cpx<R>::T L0, typename cpx<R>::T L1,
                                                typename cpx<R>::T L2, bool alt) {
    using C = typename cpx<R>::T;
    Basis<R> b;
    const R Lq = L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y + L2.x * L2.x + L2.y * L2.y;
    if (!(Lq > (R)0)) {
        b.sig = (R)0;
        for (int l = 0; l < 3; ++l) { b.p1[l] = mk((R)0, (R)0); b.p2[l] = mk((R)0, (R)0); }
        return b;
    }
    const R e0 = (R)1, e1 = alt ? (R)-1 : (R)1, e2 = alt ? (R)0 : (R)1;
    const C ed = mk(e0 * L0.x + e1 * L1.x + e2 * L2.x, e0 * L0.y + e1 * L1.y + e2 * L2.y);
    const R een = alt ? (R)2 : (R)3;
    const R g = een * Lq - (ed.x * ed.x + ed.y * ed.y);
    const R r1 = rsq(Lq * g);
    const R r2 = rsq(g);
    // Pi_1 = (Lq e - Lambda conj(e.Lambda)) / sqrt(Lq g)
    const C edc = conjc(ed);
    const C m0 = cmul(L0, edc), m1 = cmul(L1, edc), m2 = cmul(L2, edc);
    b.p1[0] = mk((Lq * e0 - m0.x) * r1, -m0.y * r1);
    b.p1[1] = mk((Lq * e1 - m1.x) * r1, -m1.y * r1);
    b.p1[2] = mk((Lq * e2 - m2.x) * r1, -m2.y * r1);
    // Pi_2 = conj(e x Lambda) / sqrt(g)
    const C x0 = e1 * L2 - e2 * L1;
    const C x1 = e2 * L0 - e0 * L2;
    const C x2 = e0 * L1 - e1 * L0;
    b.p2[0] = mk(x0.x * r2, -x0.y * r2);
    b.p2[1] = mk(x1.x * r2, -x1.y * r2);
    b.p2[2] = mk(x2.x * r2, -x2.y * r2);
    b.sig = root(Lq);
    return b;
}

// Per-pencil parts of the range basis (one x-frequency p at one y-frequency q):
// Lambda_1, Lambda_2, |Lambda_1|^2 + |Lambda_2|^2, and the partial sums
// Lambda_1 + Lambda_2, Lambda_1 - Lambda_2 of e.Lambda for the two reference
// vectors e = (1,1,1) and e = (1,-1,0).
template <typename R>
struct PencilBasis {
    typename cpx<R>::T L0, L1, S01, D01;
    R P01;
};

// (o_0, o_1, o_2) = Sigma_r [Pi_1 Pi_2] (y1, y2) at one frequency, eqs. (range_basis1),
// (range_basis2), (SVD) written out: with g = |e|^2 Lq - |e.Lambda|^2 and x = e x Lambda,
//   o_l = g^{-1/2} [ (Lq e_l - Lambda_l conj(e.Lambda)) y1 + Lq^{1/2} conj(x_l) y2 ].
template <typename R>
__device__ __forceinline__ void expand(const PencilBasis<R>& b, typename cpx<R>::T L2, bool alt,
                                       typename cpx<R>::T y1, typename cpx<R>::T y2,
                                       typename cpx<R>::T& o0, typename cpx<R>::T& o1,
                                       typename cpx<R>::T& o2) {
    using C = typename cpx<R>::T;
    const R Lq = b.P01 + L2.x * L2.x + L2.y * L2.y;
    if (!(Lq > (R)0)) {
        o0 = o1 = o2 = mk((R)0, (R)0);
        return;
    }
    C ed, x0, x1, x2;
    R een, e1, e2;
    if (!alt) {
        ed = b.S01 + L2; x0 = L2 - b.L1; x1 = b.L0 - L2; x2 = b.L1 - b.L0; een = 3; e1 = 1; e2 = 1;
    } else {
        ed = b.D01; x0 = mk(-L2.x, -L2.y); x1 = x0; x2 = b.S01; een = 2; e1 = -1; e2 = 0;
    }
    const R r2 = rsq(een * Lq - (ed.x * ed.x + ed.y * ed.y));
    const R sr = root(Lq) * r2;
    const C u = r2 * y1, v = sr * y2;
    const C d = cmulc(ed, u);                        // conj(e.Lambda) u
    const C w = Lq * u;
    o0 = w - cmul(b.L0, d) + cmulc(x0, v);
    o1 = e1 * w - cmul(b.L1, d) + cmulc(x1, v);
    o2 = e2 * w - cmul(L2, d) + cmulc(x2, v);
}

// The adjoint: (z1, z2) = Sigma_r [Pi_1 Pi_2]^H (W_0, W_1, W_2) at one frequency,
//   z1 = g^{-1/2} [ Lq e.W - (e.Lambda) conj(Lambda).W ],  z2 = g^{-1/2} Lq^{1/2} x.W.
template <typename R>
__device__ __forceinline__ void contract(const PencilBasis<R>& b, typename cpx<R>::T L2, bool alt,
                                         typename cpx<R>::T W0, typename cpx<R>::T W1,
                                         typename cpx<R>::T W2, typename cpx<R>::T& z1,
                                         typename cpx<R>::T& z2) {
    using C = typename cpx<R>::T;
    const R Lq = b.P01 + L2.x * L2.x + L2.y * L2.y;
    if (!(Lq > (R)0)) {
        z1 = z2 = mk((R)0, (R)0);
        return;
    }
    C ed, eW, xW;
    R een;
    if (!alt) {
        ed = b.S01 + L2;
        eW = W0 + W1 + W2;
        xW = cmul(L2 - b.L1, W0) + cmul(b.L0 - L2, W1) + cmul(b.L1 - b.L0, W2);
        een = 3;
    } else {
        ed = b.D01;
        eW = W0 - W1;
        xW = cmul(b.S01, W2) - cmul(L2, W0 + W1);
        een = 2;
    }
    const R r2 = rsq(een * Lq - (ed.x * ed.x + ed.y * ed.y));
    const C lw = cmulc(b.L0, W0) + cmulc(b.L1, W1) + cmulc(L2, W2);     // conj(Lambda).W
    z1 = r2 * (Lq * eW - cmul(ed, lw));
    z2 = (root(Lq) * r2) * xW;
}

// (o_0, o_1, o_2) <- Lambda x (o_0, o_1, o_2) / Lambda_q: applied to Sigma_r Pi_r y this
// gives the frequency-side curl C^ Pi_r y / Sigma_r, C^ the 3 x 3 curl symbol with
// C_l T = T Lambda_l (Section 4), i.e. the left singular vectors P_r y of eq. (SVD).
template <typename C>
__device__ __forceinline__ void curl_of(C L0, C L1, C L2, C& o0, C& o1, C& o2) {
    using R = decltype(C().x);
    const R Lq = L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y + L2.x * L2.x + L2.y * L2.y;
    if (!(Lq > (R)0)) {
        o0 = o1 = o2 = mk((R)0, (R)0);
        return;
    }
    const R inv = (R)1 / Lq;
    const C c0 = cmul(L1, o2) - cmul(L2, o1), c1 = cmul(L2, o0) - cmul(L0, o2), c2 = cmul(L0, o1) - cmul(L1, o0);
    o0 = inv * c0;
    o1 = inv * c1;
    o2 = inv * c2;
}

template <typename C>
__device__ __forceinline__ void load_table(C* dst, const C* src, int L) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = src[i];
}

}  // namespace
