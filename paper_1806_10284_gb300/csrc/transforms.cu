// Twisted 3D DFT kernels for A_r = Sigma_r Q_r^* B^{-1} Q_r Sigma_r (eq. NFSEP).
//
// Q_r = (I_3 (x) T)[Pi_1 Pi_2] with T the lattice-twisted inverse DFT of
// eq. (T); T q is Algorithm 5.2 (z transform then the D_a3 twist, y transform
// then the D_a2 twist, x transform then the D_a1 twist) and T^* p is
// Algorithm 5.1 in reverse order with conjugate twists.  One apply is three
// fused passes over HBM:
//
//   Z-in  : y (2 coords/frequency) -> Sigma_r, Pi_r expansion to 3 components
//           -> inverse z-DFT -> D_a3 twist                      (per x-tile, y)
//   XY    : per z-plane: inverse y-DFT -> D_a2 -> inverse x-DFT -> B^{-1}/n
//           -> forward x-DFT -> conj D_a2 -> forward y-DFT    (D_a1 cancels)
//   Z-out : conj D_a3 -> forward z-DFT -> Pi_r^H contraction, Sigma_r
//
// When an x-y plane does not fit in shared memory the XY pass is split into
// a y pass, an x pass and a y pass.  All DFTs are shared-memory Stockham
// passes (radix 2, 3, 4, 5, 8) with precomputed twiddle tables; twist phases
// and Lambda_l are evaluated in the kernels from exact fractions.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "bounds.cuh"
#include "fame_internal.h"
#include "dfloat.cuh"
#include "fft2.cuh"
#include "phases.cuh"

// double-float complex arithmetic over complex128 storage (dfloat.cuh)
template <> struct cpx<dfr> { using T = dfc; };

namespace {
// The two-level kernels below take the arithmetic complex type A as a template
// argument: the storage type itself (float2, double2), or dfc over complex128
// storage, converted at every global load and store.
template <typename A, typename C>
__device__ __forceinline__ A as_arith(const C& v) {
    if constexpr (std::is_same<A, C>::value) return v;
    else return to_df(v);
}
template <typename C, typename A>
__device__ __forceinline__ C as_store(const A& v) {
    if constexpr (std::is_same<A, C>::value) return v;
    else return to_double(v);
}
template <typename Ar, typename R>
__device__ __forceinline__ Ar as_arith_r(R v) {
    if constexpr (std::is_same<Ar, R>::value) return v;
    else return to_df(v);
}
}  // namespace

namespace {
// ---------------------------------------------------------------------------
// Stockham radix butterflies
// ---------------------------------------------------------------------------
// multiply by -i (forward) or +i (inverse)
template <typename C>
__device__ __forceinline__ C rot_i(C a, bool inv) { return inv ? mk(-a.y, a.x) : mk(a.y, -a.x); }

template <typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a - b;
    a = a + b;
    b = t;
}
template <typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3, bool inv) {
    C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = rot_i(a1 - a3, inv);
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + t3;
    a3 = t1 - t3;
}

template <typename C, int R> struct Dft;
template <typename C> struct Dft<C, 2> {
    __device__ __forceinline__ static void run(C* v, bool) { dft2(v[0], v[1]); }
};
template <typename C> struct Dft<C, 4> {
    __device__ __forceinline__ static void run(C* v, bool inv) { dft4(v[0], v[1], v[2], v[3], inv); }
};
template <typename C> struct Dft<C, 8> {
    __device__ __forceinline__ static void run(C* v, bool inv) {
        using R = decltype(v[0].x);
        const R h = (R)0.70710678118654752440084436210485;  // 1/sqrt(2)
        C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4(e0, e1, e2, e3, inv);
        dft4(o0, o1, o2, o3, inv);
        // o1 *= w8, o2 *= w8^2, o3 *= w8^3 with w8 = e^{-+ i pi/4}
        C t1 = inv ? mk(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mk(h * (o1.x + o1.y), h * (o1.y - o1.x));
        C t2 = rot_i(o2, inv);
        C t3 = inv ? mk(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mk(h * (o3.y - o3.x), -h * (o3.x + o3.y));
        v[0] = e0 + o0; v[4] = e0 - o0;
        v[1] = e1 + t1; v[5] = e1 - t1;
        v[2] = e2 + t2; v[6] = e2 - t2;
        v[3] = e3 + t3; v[7] = e3 - t3;
    }
};
template <typename C> struct Dft<C, 3> {
    __device__ __forceinline__ static void run(C* v, bool inv) {
        using R = decltype(v[0].x);
        const R h = (R)0.86602540378443864676372317075294;  // sqrt(3)/2
        C s = v[1] + v[2];
        C d = rot_i(v[1] - v[2], inv);
        C m = v[0] - (R)0.5 * s;
        v[0] = v[0] + s;
        v[1] = m + h * d;
        v[2] = m - h * d;
    }
};
template <typename C> struct Dft<C, 5> {
    __device__ __forceinline__ static void run(C* v, bool inv) {
        using R = decltype(v[0].x);
        const R c1 = (R)0.30901699437494742410229341718282;   // cos(2 pi/5)
        const R c2 = (R)-0.80901699437494742410229341718282;  // cos(4 pi/5)
        const R s1 = (R)0.95105651629515357211643933337938;   // sin(2 pi/5)
        const R s2 = (R)0.58778525229247312916870595463907;   // sin(4 pi/5)
        C a14 = v[1] + v[4], b14 = v[1] - v[4];
        C a23 = v[2] + v[3], b23 = v[2] - v[3];
        C x0 = v[0] + a14 + a23;
        C m1 = v[0] + c1 * a14 + c2 * a23;
        C m2 = v[0] + c2 * a14 + c1 * a23;
        C n1 = rot_i(s1 * b14 + s2 * b23, inv);
        C n2 = rot_i(s2 * b14 - s1 * b23, inv);
        v[0] = x0;
        v[1] = m1 + n1;
        v[4] = m1 - n1;
        v[2] = m2 + n2;
        v[3] = m2 - n2;
    }
};

// Pencils held in shared memory: element e of pencil j sits at
// buf[(j / inner) * outer + (j % inner) * istride + e * es].
struct Pencils {
    int count, inner, istride, outer, es;
    bool pencil_fast;   // thread mapping: consecutive threads -> consecutive pencils
};

// One Stockham stage (radix R, Ns points already combined) over all pencils,
// out of place: src -> dst (same layout).  Each thread holds one radix-R
// butterfly at a time.
template <typename C, int R>
__device__ __forceinline__ void fft_stage(const C* __restrict__ src, C* __restrict__ dst,
                                          const Pencils& P, int L, int Ns, const C* tw, bool inv) {
    const int nb = L / R;
    const int total = P.count * nb;
    const int tstep = L / (Ns * R);
#pragma unroll 1
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int pen, j;
        if (P.pencil_fast) { pen = w % P.count; j = w / P.count; }
        else { pen = w / nb; j = w - pen * nb; }
        const int base = (pen / P.inner) * P.outer + (pen % P.inner) * P.istride;
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C x = src[base + (j + r * nb) * P.es];
            if (r > 0 && k > 0) {
                C t = tw[r * k * tstep];
                if (inv) t.y = -t.y;
                x = cmul(x, t);
            }
            v[r] = x;
        }
        Dft<C, R>::run(v, inv);
        const int ob = base + ((j / Ns) * Ns * R + k) * P.es;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[ob + r * Ns * P.es] = v[r];
    }
    __syncthreads();
}

// Full transform along one axis; a holds the input, b is scratch of the same
// size.  Returns the buffer holding the result.
template <typename C>
__device__ C* fft_axis(C* a, C* b, const Pencils& P, const AxisPlan& A, const C* tw, bool inv) {
    int Ns = 1;
    for (int s = 0; s < A.nst; ++s) {
        const int R = A.radix[s];
        switch (R) {
            case 8: fft_stage<C, 8>(a, b, P, A.L, Ns, tw, inv); break;
            case 4: fft_stage<C, 4>(a, b, P, A.L, Ns, tw, inv); break;
            case 2: fft_stage<C, 2>(a, b, P, A.L, Ns, tw, inv); break;
            case 3: fft_stage<C, 3>(a, b, P, A.L, Ns, tw, inv); break;
            default: fft_stage<C, 5>(a, b, P, A.L, Ns, tw, inv); break;
        }
        Ns *= R;
        C* t = a;
        a = b;
        b = t;
    }
    return a;
}

// ---------------------------------------------------------------------------
// Z-in: Sigma_r and Pi_r expansion, inverse z-DFT, D_a3 twist.
// grid (ceil(n1/TP), n2, ceil(m/vpc)); smem: tw_z[n3], L01[2][TP], two bufs [3][n3][TP]
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(512) k_zin(KParams<R> P, const typename cpx<R>::T* __restrict__ y,
                      typename cpx<R>::T* __restrict__ W, int m, int TP, int vpc) {
    using C = typename cpx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const size_t n = (size_t)n1 * n2 * n3;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* L0s = tw + n3;
    C* L1s = L0s + TP;
    C* buf = L1s + TP;
    C* buf2 = buf + 3 * n3 * TP;
    const int q = blockIdx.y, p0 = blockIdx.x * TP;
    load_table(tw, P.tw[2], n3);
    for (int pp = threadIdx.x; pp < TP; pp += blockDim.x) {
        const int p = min(p0 + pp, n1 - 1);
        L0s[pp] = lambda_of(p, n1, P.f1, P.inv_dx);
        L1s[pp] = lambda_of(q, n2, P.f2[p], P.inv_dy);
    }
    __syncthreads();
    const Pencils pen{3 * TP, TP, 1, n3 * TP, TP, true};
    const int tile = n3 * TP;
    const int v1 = min(m, (int)(blockIdx.z + 1) * vpc);
    for (int v = blockIdx.z * vpc; v < v1; ++v) {
        const C* yv = y + (size_t)v * 2 * n;
        for (int e = threadIdx.x; e < tile; e += blockDim.x) {
            const int r = e / TP, pp = e - r * TP, p = p0 + pp;
            C o0 = mk((R)0, (R)0), o1 = o0, o2 = o0;
            if (p < n1) {
                const size_t f = ((size_t)r * n2 + q) * n1 + p;
                const C y1 = yv[f], y2 = yv[n + f];
                const C L2 = P.lam3[f];
                const Basis<R> b = make_basis<R>(L0s[pp], L1s[pp], L2, alt_bit(P.alt, f));
                const C s1 = b.sig * y1, s2 = b.sig * y2;
                o0 = cmul(b.p1[0], s1) + cmul(b.p2[0], s2);
                o1 = cmul(b.p1[1], s1) + cmul(b.p2[1], s2);
                o2 = cmul(b.p1[2], s1) + cmul(b.p2[2], s2);
                if (P.curl) curl_of(L0s[pp], L1s[pp], L2, o0, o1, o2);
            }
            buf[e] = o0;
            buf[tile + e] = o1;
            buf[2 * tile + e] = o2;
        }
        __syncthreads();
        const C* res = fft_axis(buf, buf2, pen, P.ax[2], tw, true);
        C* Wv = W + (size_t)v * 3 * n;
        for (int e = threadIdx.x; e < 3 * tile; e += blockDim.x) {
            const int l = e / tile, rem = e - l * tile, c = rem / TP, pp = rem - c * TP;
            const int p = p0 + pp;
            if (p < n1) {
                const C x = cmul(res[e], P.tw3[((size_t)c * n2 + q) * n1 + p]);
                Wv[(size_t)l * n + ((size_t)c * n2 + q) * n1 + p] = x;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Z-out: conj D_a3 twist, forward z-DFT, Pi_r^H contraction and Sigma_r.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(512) k_zout(KParams<R> P, const typename cpx<R>::T* __restrict__ W,
                       typename cpx<R>::T* __restrict__ out, int m, int TP, int vpc) {
    using C = typename cpx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const size_t n = (size_t)n1 * n2 * n3;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* L0s = tw + n3;
    C* L1s = L0s + TP;
    C* buf = L1s + TP;
    C* buf2 = buf + 3 * n3 * TP;
    const int q = blockIdx.y, p0 = blockIdx.x * TP;
    load_table(tw, P.tw[2], n3);
    for (int pp = threadIdx.x; pp < TP; pp += blockDim.x) {
        const int p = min(p0 + pp, n1 - 1);
        L0s[pp] = lambda_of(p, n1, P.f1, P.inv_dx);
        L1s[pp] = lambda_of(q, n2, P.f2[p], P.inv_dy);
    }
    __syncthreads();
    const Pencils pen{3 * TP, TP, 1, n3 * TP, TP, true};
    const int tile = n3 * TP;
    const int v1 = min(m, (int)(blockIdx.z + 1) * vpc);
    for (int v = blockIdx.z * vpc; v < v1; ++v) {
        const C* Wv = W + (size_t)v * 3 * n;
        for (int e = threadIdx.x; e < 3 * tile; e += blockDim.x) {
            const int l = e / tile, rem = e - l * tile, c = rem / TP, pp = rem - c * TP;
            const int p = p0 + pp;
            C x = mk((R)0, (R)0);
            if (p < n1) {
                x = Wv[(size_t)l * n + ((size_t)c * n2 + q) * n1 + p];
                x = cmulc(P.tw3[((size_t)c * n2 + q) * n1 + p], x);
            }
            buf[e] = x;
        }
        __syncthreads();
        const C* res = fft_axis(buf, buf2, pen, P.ax[2], tw, false);
        C* ov = out + (size_t)v * 2 * n;
        for (int e = threadIdx.x; e < tile; e += blockDim.x) {
            const int r = e / TP, pp = e - r * TP, p = p0 + pp;
            if (p < n1) {
                const size_t f = ((size_t)r * n2 + q) * n1 + p;
                const C L2 = P.lam3[f];
                const Basis<R> b = make_basis<R>(L0s[pp], L1s[pp], L2, alt_bit(P.alt, f));
                const C w0 = res[e], w1 = res[tile + e], w2 = res[2 * tile + e];
                const C z1 = cmulc(b.p1[0], w0) + cmulc(b.p1[1], w1) + cmulc(b.p1[2], w2);
                const C z2 = cmulc(b.p2[0], w0) + cmulc(b.p2[1], w1) + cmulc(b.p2[2], w2);
                ov[f] = b.sig * z1;
                ov[n + f] = b.sig * z2;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// XY: one z-plane (vector v, component l, z index c) per block, in shared memory.
//   mode 0 (apply): y-inv, D_a2, x-inv, *B^{-1}/n, x-fwd, conj D_a2, y-fwd
//   mode 1 (lift) : y-inv, D_a2, x-inv, D_a1, *B^{-1}/sqrt(n)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(512) k_xy(KParams<R> P, typename cpx<R>::T* __restrict__ W,
                                            int mode, R lift_scale) {
    using C = typename cpx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const int np = n1 * n2;
    C* twx = reinterpret_cast<C*>(smem_raw);
    C* twy = twx + n1;
    C* A = twy + n2;
    C* B = A + np;
    const int plane = blockIdx.x;
    const int c = plane % n3;
    const int l = (plane / n3) % 3;
    C* g = W + (size_t)plane * np;
    load_table(twx, P.tw[0], n1);
    load_table(twy, P.tw[1], n2);
    for (int e = threadIdx.x; e < np; e += blockDim.x) A[e] = g[e];
    __syncthreads();
    const Pencils cols{n1, n1, 1, 0, n1, true};
    const Pencils rows{n2, 1, 0, n1, 1, false};
    C* cur = fft_axis(A, B, cols, P.ax[1], twy, true);
    C* oth = (cur == A) ? B : A;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int b = e / n1, p = e - b * n1;
        cur[e] = cmul(cur[e], P.tw2[e]);
    }
    __syncthreads();
    cur = fft_axis(cur, oth, rows, P.ax[0], twx, true);
    oth = (cur == A) ? B : A;
    const R* ib = P.invB + (size_t)l * n3 * np + (size_t)c * np;
    if (mode == 0) {
        for (int e = threadIdx.x; e < np; e += blockDim.x) cur[e] = (ib[e] * P.scale) * cur[e];
        __syncthreads();
        cur = fft_axis(cur, oth, rows, P.ax[0], twx, false);
        oth = (cur == A) ? B : A;
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            const int b = e / n1, p = e - b * n1;
            cur[e] = cmulc(P.tw2[e], cur[e]);
        }
        __syncthreads();
        cur = fft_axis(cur, oth, cols, P.ax[1], twy, false);
        for (int e = threadIdx.x; e < np; e += blockDim.x) g[e] = cur[e];
    } else {
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            const int a = e % n1;
            g[e] = (mode == 2 ? lift_scale : ib[e] * lift_scale) * cmul(cur[e], P.tw1[a]);
        }
    }
}

// ---------------------------------------------------------------------------
// Split XY for planes that do not fit: y pass over x-tiles, x pass over rows.
// y pass: grid (ceil(n1/TP), n3, 3m); dir 0 = inverse then D_a2, 1 = conj D_a2 then forward
// ---------------------------------------------------------------------------
template <typename R, typename A = typename cpx<R>::T>
__global__ void __launch_bounds__(256) k_ypass(KParams<R> P, A* __restrict__ W, int TP, int dir) {
    using Ar = decltype(A().x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const size_t np = (size_t)n1 * n2;
    A* tw = reinterpret_cast<A*>(smem_raw);
    A* buf = tw + n2;
    A* buf2 = buf + n2 * TP;
    const int p0 = blockIdx.x * TP, c = blockIdx.y;
    A* g = W + ((size_t)blockIdx.z * n3 + c) * np;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw[i] = as_arith<A>(P.tw[1][i]);
    const int tile = n2 * TP;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
        const int b = e / TP, pp = e - b * TP, p = p0 + pp;
        A x = mk((Ar)0, (Ar)0);
        if (p < n1) {
            x = g[(size_t)b * n1 + p];
            if (dir == 1) x = cmulc(as_arith<A>(P.tw2[(size_t)b * n1 + p]), x);
        }
        buf[e] = x;
    }
    __syncthreads();
    const Pencils pen{TP, TP, 1, 0, TP, true};
    const A* res = fft_axis(buf, buf2, pen, P.ax[1], tw, dir == 0);
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
        const int b = e / TP, pp = e - b * TP, p = p0 + pp;
        if (p < n1) {
            A x = res[e];
            if (dir == 0) x = cmul(x, as_arith<A>(P.tw2[(size_t)b * n1 + p]));
            g[(size_t)b * n1 + p] = x;
        }
    }
}

// x pass: RPB rows per block, grid ceil(3 m n3 n2 / RPB); mode 0 apply (inv, *B^{-1}/n, fwd),
// mode 1 lift (inv, D_a1, *B^{-1} lift_scale)
// With A the double-float type, W holds double-float values on entry; mode 0 leaves
// double-float values, modes 1 and 2 (the lift's last pass) write complex128.
template <typename R, typename A = typename cpx<R>::T>
__global__ void __launch_bounds__(256) k_xpass(KParams<R> P, A* __restrict__ W, long long nrows, int RPB,
                                               int mode, R lift_scale) {
    using C = typename cpx<R>::T;
    using Ar = decltype(A().x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    A* tw = reinterpret_cast<A*>(smem_raw);
    A* buf = tw + n1;
    A* buf2 = buf + RPB * n1;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw[i] = as_arith<A>(P.tw[0][i]);
    const long long r0 = (long long)blockIdx.x * RPB;
    const int nr = (int)min((long long)RPB, nrows - r0);
    A* g = W + r0 * n1;
    for (int e = threadIdx.x; e < RPB * n1; e += blockDim.x)
        buf[e] = (e < nr * n1) ? g[e] : mk((Ar)0, (Ar)0);
    __syncthreads();
    const Pencils rows{RPB, 1, 0, n1, 1, false};
    A* cur = fft_axis(buf, buf2, rows, P.ax[0], tw, true);
    A* oth = (cur == buf) ? buf2 : buf;
    const size_t nsp = (size_t)n1 * n2 * n3;
    const Ar sc = as_arith_r<Ar>(P.scale), ls = as_arith_r<Ar>(lift_scale);
    for (int e = threadIdx.x; e < nr * n1; e += blockDim.x) {
        const long long row = r0 + e / n1;          // row = ((v*3 + l)*n3 + c)*n2 + b
        const int a = e % n1;
        const long long rb = row % ((long long)n3 * n2);
        const int l = (int)((row / ((long long)n3 * n2)) % 3);
        const Ar ib = as_arith_r<Ar>(P.invB[(size_t)l * nsp + (size_t)rb * n1 + a]);
        if (mode == 0) cur[e] = (ib * sc) * cur[e];
        else cur[e] = (mode == 2 ? ls : ib * ls) * cmul(cur[e], as_arith<A>(P.tw1[a]));
    }
    __syncthreads();
    if (mode == 0) {
        cur = fft_axis(cur, oth, rows, P.ax[0], tw, false);
        for (int e = threadIdx.x; e < nr * n1; e += blockDim.x) g[e] = cur[e];
    } else {
        // the complex128 result goes over the double-float input in place (same size)
        C* gc = reinterpret_cast<C*>(g);
        for (int e = threadIdx.x; e < nr * n1; e += blockDim.x) gc[e] = as_store<C>(cur[e]);
    }
}

// weights of up to kGradChunk lifted bands
constexpr int kGradChunk = 16;
struct GradWeights { double w[kGradChunk]; };

// dB[i] -= sum_j w_j |x_j[i]|^2 over mc lifted vectors x_j ([mc][3][n], N = 3n)
__global__ void k_grad_accum(const double2* __restrict__ x, GradWeights w, int mc,
                             double* __restrict__ dB, size_t N) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < mc; ++j) {
            const double2 v = x[(size_t)j * N + i];
            acc += w.w[j] * (v.x * v.x + v.y * v.y);
        }
        dB[i] -= acc;
    }
}

// Reference-vector decision per frequency, taken once in FP64 for both precisions:
// bit f set where 3 Lq - |Ls|^2 < G_TOL * 3 Lq (Lambda close to parallel to (1,1,1)).
__global__ void k_basis_mask(KParams<double> P, uint32_t* __restrict__ mask) {
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const size_t n = (size_t)n1 * n2 * n3;
    const size_t nw = (n + 31) / 32;
    for (size_t wd = blockIdx.x * (size_t)blockDim.x + threadIdx.x; wd < nw;
         wd += (size_t)gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const size_t f = wd * 32 + b;
            if (f >= n) break;
            const int p = (int)(f % n1);
            const int q = (int)((f / n1) % n2);
            const int r = (int)(f / ((size_t)n1 * n2));
            const double2 L0 = lambda_of(p, n1, P.f1, P.inv_dx);
            const double2 L1 = lambda_of(q, n2, P.f2[p], P.inv_dy);
            const double2 L2 = lambda_of(r, n3, P.f3[(size_t)q * n1 + p], P.inv_dz);
            const double Lq = L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y + L2.x * L2.x + L2.y * L2.y;
            const double sx = L0.x + L1.x + L2.x, sy = L0.y + L1.y + L2.y;
            const double g1 = 3.0 * Lq - (sx * sx + sy * sy);
            if (Lq > 0.0 && g1 < kGTol * 3.0 * Lq) bits |= 1u << b;
        }
        mask[wd] = bits;
    }
}

// Twist and Lambda_3 tables of one (lattice, k): D_a3 twist e^{2 pi i c f3(p,q)} and
// Lambda_3 at every (p, q, c/r) in [n3][n2][n1] order, D_a2 twist e^{2 pi i b f2(p)}
// in [n2][n1], D_a1 twist e^{2 pi i a f1} in [n1]; evaluated in FP64, stored in
// both precisions.
__global__ void k_twist_tables(KParams<double> P, float2* __restrict__ tw3f, double2* __restrict__ tw3d,
                               float2* __restrict__ lam3f, double2* __restrict__ lam3d,
                               float2* __restrict__ tw2f, double2* __restrict__ tw2d,
                               float2* __restrict__ tw1f, double2* __restrict__ tw1d) {
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const size_t plane = (size_t)n1 * n2, n = plane * n3;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t f = blockIdx.x * (size_t)blockDim.x + threadIdx.x; f < n; f += stride) {
        const size_t pq = f % plane;
        const int c = (int)(f / plane);
        const double F3 = P.f3[pq];
        const double2 t = cis(frac_mul(c, F3));
        const double2 l = lambda_of(c, n3, F3, P.inv_dz);
        tw3d[f] = t;
        tw3f[f] = make_float2((float)t.x, (float)t.y);
        lam3d[f] = l;
        lam3f[f] = make_float2((float)l.x, (float)l.y);
    }
    for (size_t f = blockIdx.x * (size_t)blockDim.x + threadIdx.x; f < plane; f += stride) {
        const int p = (int)(f % n1), b = (int)(f / n1);
        const double2 t = cis(frac_mul(b, P.f2[p]));
        tw2d[f] = t;
        tw2f[f] = make_float2((float)t.x, (float)t.y);
    }
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < (size_t)n1; a += stride) {
        const double2 t = cis(frac_mul((int)a, P.f1));
        tw1d[a] = t;
        tw1f[a] = make_float2((float)t.x, (float)t.y);
    }
}

// preconditioner table: 1/(Lambda_q mean(1/B)) per frequency, 0 where Lambda_q = 0
template <typename R>
__global__ void k_precond(KParams<R> P, R* __restrict__ tinv, R mean_invB) {
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const size_t n = (size_t)n1 * n2 * n3;
    for (size_t f = blockIdx.x * (size_t)blockDim.x + threadIdx.x; f < n;
         f += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(f % n1);
        const int q = (int)((f / n1) % n2);
        const int r = (int)(f / ((size_t)n1 * n2));
        const auto L0 = lambda_of(p, n1, P.f1, P.inv_dx);
        const auto L1 = lambda_of(q, n2, P.f2[p], P.inv_dy);
        const auto L2 = lambda_of(r, n3, P.f3[(size_t)q * n1 + p], P.inv_dz);
        const R Lq = L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y + L2.x * L2.x + L2.y * L2.y;
        tinv[f] = (Lq > (R)0) ? (R)1 / (Lq * mean_invB) : (R)0;
    }
}

// ---------------------------------------------------------------------------
// Two-level kernels for the lengths fft2::supported accepts: the same passes
// as k_zin / k_xy / k_zout, with register-resident radix-R1 and radix-R2 DFTs,
// one twiddled shared-memory exchange per transform, pencils mapped to
// consecutive lanes, and planes stored with an odd row stride.
// ---------------------------------------------------------------------------
// q / d for 0 <= q < 2^20, d <= 1024, via a float reciprocal (exact in that range)
__device__ __forceinline__ int fdiv(int q, float inv_d) { return __float2int_rz(((float)q + 0.5f) * inv_d); }

template <typename R, typename A = typename cpx<R>::T>
__global__ void __launch_bounds__(512) k_zin2(KParams<R> P, const typename cpx<R>::T* __restrict__ y,
                                              A* __restrict__ W, int m, int lgTP, int vpc) {
    using C = typename cpx<R>::T;
    using Ar = decltype(A().x);
    using F = typename FracT<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const int TP = 1 << lgTP, NP = 3 * TP;
    const size_t n = (size_t)n1 * n2 * n3;
    A* tw = reinterpret_cast<A*>(smem_raw);
    A* L0s = tw + n3;
    A* L1s = L0s + TP;
    F* F3s = reinterpret_cast<F*>(L1s + TP);
    A* X = L1s + 2 * TP;                 // F3s occupies TP entries of A size
    A* Y = X + (size_t)n3 * NP;
    const int q = blockIdx.y, p0 = blockIdx.x * TP;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = as_arith<A>(P.tw[2][i]);
    for (int pp = threadIdx.x; pp < TP; pp += blockDim.x) {
        const int p = min(p0 + pp, n1 - 1);
        L0s[pp] = as_arith<A>(lambda_of(p, n1, P.f1, P.inv_dx));
        L1s[pp] = as_arith<A>(lambda_of(q, n2, P.f2[p], P.inv_dy));
        F3s[pp] = P.f3[(size_t)q * n1 + p];
    }
    __syncthreads();
    const int tile = n3 * TP;
    const int v1 = min(m, (int)(blockIdx.z + 1) * vpc);
    for (int v = blockIdx.z * vpc; v < v1; ++v) {
        const C* yv = y + (size_t)v * 2 * n;
        for (int e = threadIdx.x; e < tile; e += blockDim.x) {
            const int r = e >> lgTP, pp = e & (TP - 1), p = p0 + pp;
            A o0 = mk((Ar)0, (Ar)0), o1 = o0, o2 = o0;
            if (p < n1) {
                const size_t f = ((size_t)r * n2 + q) * n1 + p;
                const A y1 = as_arith<A>(yv[f]), y2 = as_arith<A>(yv[n + f]);
                const A L0 = L0s[pp], L1 = L1s[pp];
                const PencilBasis<Ar> pb{L0, L1, L0 + L1, L0 - L1,
                                         L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y};
                expand<Ar>(pb, as_arith<A>(P.lam3[f]), alt_bit(P.alt, f), y1, y2, o0, o1, o2);
                if constexpr (std::is_same<A, C>::value) {
                    if (P.curl) curl_of(L0, L1, P.lam3[f], o0, o1, o2);
                }
            }
            X[r * NP + pp] = o0;
            X[r * NP + TP + pp] = o1;
            X[r * NP + 2 * TP + pp] = o2;
        }
        __syncthreads();
        A* Wv = W + (size_t)v * 3 * n;
        fft2::pencils_any<true>(
            n3, NP, tw, Y, [&](int pc, int e) { return X[e * NP + pc]; },
            [&](int pc, int c, A val) {
                const int l = pc >> lgTP, pp = pc & (TP - 1), p = p0 + pp;
                const size_t o = (size_t)l * n + ((size_t)c * n2 + q) * n1 + p;
                if (p < n1 && bounds_ok(o < 3 * n, kBndZ2Store, (long long)o))
                    Wv[o] = cmul(val, as_arith<A>(P.tw3[((size_t)c * n2 + q) * n1 + p]));
            });
    }
}

template <typename R, typename A = typename cpx<R>::T>
__global__ void __launch_bounds__(512) k_zout2(KParams<R> P, const A* __restrict__ W,
                                               typename cpx<R>::T* __restrict__ out, int m, int lgTP,
                                               int vpc) {
    using C = typename cpx<R>::T;
    using Ar = decltype(A().x);
    using F = typename FracT<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const int TP = 1 << lgTP, NP = 3 * TP;
    const size_t n = (size_t)n1 * n2 * n3;
    A* tw = reinterpret_cast<A*>(smem_raw);
    A* L0s = tw + n3;
    A* L1s = L0s + TP;
    F* F3s = reinterpret_cast<F*>(L1s + TP);
    A* X = L1s + 2 * TP;
    A* Y = X + (size_t)n3 * NP;
    const int q = blockIdx.y, p0 = blockIdx.x * TP;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = as_arith<A>(P.tw[2][i]);
    for (int pp = threadIdx.x; pp < TP; pp += blockDim.x) {
        const int p = min(p0 + pp, n1 - 1);
        L0s[pp] = as_arith<A>(lambda_of(p, n1, P.f1, P.inv_dx));
        L1s[pp] = as_arith<A>(lambda_of(q, n2, P.f2[p], P.inv_dy));
        F3s[pp] = P.f3[(size_t)q * n1 + p];
    }
    __syncthreads();
    const int tile = n3 * TP;
    const int v1 = min(m, (int)(blockIdx.z + 1) * vpc);
    for (int v = blockIdx.z * vpc; v < v1; ++v) {
        const A* Wv = W + (size_t)v * 3 * n;
        fft2::pencils_any<false>(
            n3, NP, tw, Y,
            [&](int pc, int c) {
                const int l = pc >> lgTP, pp = pc & (TP - 1), p = p0 + pp;
                if (p >= n1) return mk((Ar)0, (Ar)0);
                const A x = Wv[(size_t)l * n + ((size_t)c * n2 + q) * n1 + p];
                return cmulc(as_arith<A>(P.tw3[((size_t)c * n2 + q) * n1 + p]), x);
            },
            [&](int pc, int r, A val) { X[r * NP + pc] = val; });
        C* ov = out + (size_t)v * 2 * n;
        for (int e = threadIdx.x; e < tile; e += blockDim.x) {
            const int r = e >> lgTP, pp = e & (TP - 1), p = p0 + pp;
            if (p < n1) {
                const size_t f = ((size_t)r * n2 + q) * n1 + p;
                const A L0 = L0s[pp], L1 = L1s[pp];
                const PencilBasis<Ar> pb{L0, L1, L0 + L1, L0 - L1,
                                         L0.x * L0.x + L0.y * L0.y + L1.x * L1.x + L1.y * L1.y};
                A z1, z2;
                contract<Ar>(pb, as_arith<A>(P.lam3[f]), alt_bit(P.alt, f), X[r * NP + pp], X[r * NP + TP + pp],
                             X[r * NP + 2 * TP + pp], z1, z2);
                ov[f] = as_store<C>(z1);
                ov[n + f] = as_store<C>(z2);
            }
        }
        __syncthreads();
    }
}

// One z-plane per block; plane kept with row stride n1 + 1.
// With A the double-float type, W holds double-float values on entry; mode 0 leaves
// double-float values, modes 1 and 2 (the lift's last pass) write complex128.
template <typename R, typename A = typename cpx<R>::T>
__global__ void __launch_bounds__(512) k_xy2(KParams<R> P, A* __restrict__ W, int mode, R lift_scale) {
    using C = typename cpx<R>::T;
    using Ar = decltype(A().x);
    using F = typename FracT<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.n1, n2 = P.n2, n3 = P.n3;
    const int np = n1 * n2, S = n1 + 1;
    A* twx = reinterpret_cast<A*>(smem_raw);
    A* twy = twx + n1;
    F* F2s = reinterpret_cast<F*>(twy + n2);
    A* X = twy + n2 + n1;                // F2s occupies n1 entries of A size
    A* Y = X + (size_t)n2 * S;
    const int plane = blockIdx.x;
    const int c = plane % n3;
    const int l = (plane / n3) % 3;
    A* g = W + (size_t)plane * np;
    const float inv_n1 = 1.0f / (float)n1;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) twx[i] = as_arith<A>(P.tw[0][i]);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) twy[i] = as_arith<A>(P.tw[1][i]);
    for (int p = threadIdx.x; p < n1; p += blockDim.x) F2s[p] = P.f2[p];
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int b = fdiv(e, inv_n1), a = e - b * n1;
        X[b * S + a] = g[e];
    }
    __syncthreads();
    // inverse y-DFT over columns, then D_a2
    fft2::pencils_any<true>(
        n2, n1, twy, Y, [&](int p, int b) { return X[b * S + p]; },
        [&](int p, int b, A v) { X[b * S + p] = cmul(v, as_arith<A>(P.tw2[b * n1 + p])); });
    // inverse x-DFT over rows
    fft2::pencils_any<true>(
        n1, n2, twx, Y, [&](int b, int a) { return X[b * S + a]; },
        [&](int b, int a, A v) { X[b * S + a] = v; });
    const R* ib = P.invB + (size_t)l * n3 * np + (size_t)c * np;
    if (mode == 0) {
        const Ar sc = as_arith_r<Ar>(P.scale);
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            const int b = fdiv(e, inv_n1), a = e - b * n1;
            X[b * S + a] = (as_arith_r<Ar>(ib[e]) * sc) * X[b * S + a];
        }
        __syncthreads();
        fft2::pencils_any<false>(
            n1, n2, twx, Y, [&](int b, int a) { return X[b * S + a]; },
            [&](int b, int a, A v) { X[b * S + a] = v; });
        fft2::pencils_any<false>(
            n2, n1, twy, Y,
            [&](int p, int b) { return cmulc(as_arith<A>(P.tw2[b * n1 + p]), X[b * S + p]); },
            [&](int p, int b, A v) { X[b * S + p] = v; });
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            const int b = fdiv(e, inv_n1), a = e - b * n1;
            g[e] = X[b * S + a];
        }
    } else {
        // the complex128 result goes over the double-float input in place (same size)
        C* gc = reinterpret_cast<C*>(g);
        const Ar ls = as_arith_r<Ar>(lift_scale);
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            const int b = fdiv(e, inv_n1), a = e - b * n1;
            const Ar s = mode == 2 ? ls : as_arith_r<Ar>(ib[e]) * ls;
            gc[e] = as_store<C>(s * cmul(X[b * S + a], as_arith<A>(P.tw1[a])));
        }
    }
}

// ---------------------------------------------------------------------------
// launch configuration
// ---------------------------------------------------------------------------
constexpr size_t kSmemCap = 200 * 1024;

// The dynamic shared-memory limit is one value per kernel for the whole process, and
// contexts on other host threads (the batched solver's workers) launch the same
// kernels with other sizes: the limit is only ever raised, under a lock, and the
// largest value set so far is kept per kernel.
template <typename R>
fame_status set_smem(fame_ctx* c, const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> limit;
    if (bytes <= 48 * 1024) return FAME_OK;
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit.find(fn);
    if (it != limit.end() && it->second >= bytes) return FAME_OK;
    FAME_CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    limit[fn] = bytes;
    return FAME_OK;
}

struct ZCfg { int TP, vpc, threads; size_t smem; };

// Z-pass tiles: TP consecutive x-frequencies by the whole z axis, three components,
// two ping-pong buffers.
template <typename R>
ZCfg z_config(const fame_ctx* c, int m) {
    using C = typename cpx<R>::T;
    const int n1 = c->plan.n[0], n2 = c->plan.n[1], n3 = c->plan.n[2];
    ZCfg z;
    z.TP = 16;
    while (z.TP > 1 && (size_t)(n3 + 2 * z.TP + 6 * z.TP * n3) * sizeof(C) > kSmemCap) z.TP /= 2;
    if (z.TP > n1) {
        int t = 1;
        while (t * 2 <= n1) t *= 2;
        z.TP = t;
    }
    z.threads = (3 * z.TP * n3 >= 4096) ? 512 : 256;
    z.smem = (size_t)(n3 + 2 * z.TP + 6 * z.TP * n3) * sizeof(C);
    // enough blocks to fill 152 SMs several times over, amortising the per-tile tables
    const long long tiles = (long long)((n1 + z.TP - 1) / z.TP) * n2;
    z.vpc = 1;
    while (z.vpc < m && tiles * ((m + z.vpc * 2 - 1) / (z.vpc * 2)) >= 152 * 6) z.vpc *= 2;
    return z;
}

// Two-level Z-pass configuration (TP a power of two).
struct Z2Cfg { int lgTP, vpc, threads; size_t smem; bool ok; };

template <typename R>
Z2Cfg z2_config(const fame_ctx* c, int m) {
    using C = typename cpx<R>::T;
    const int n1 = c->plan.n[0], n2 = c->plan.n[1], n3 = c->plan.n[2];
    Z2Cfg z;
    z.ok = fft2::supported(n3);
    int TP = 16;
    while (TP > 1 && (size_t)(n3 + 3 * TP + 6 * (size_t)TP * n3) * sizeof(C) > kSmemCap) TP /= 2;
    while (TP > 1 && TP > n1) TP /= 2;
    z.lgTP = 0;
    while ((1 << z.lgTP) < TP) ++z.lgTP;
    z.smem = (size_t)(n3 + 3 * TP + 6 * (size_t)TP * n3) * sizeof(C);
    const fft2::Split sp = fft2::split_of(n3);
    const int work = 3 * TP * std::max(sp.R1, sp.R2);
    z.threads = std::min(512, std::max(128, ((work + 31) / 32) * 32));
    const long long tiles = (long long)((n1 + TP - 1) / TP) * n2;
    z.vpc = 1;
    while (z.vpc < m && tiles * ((m + z.vpc * 2 - 1) / (z.vpc * 2)) >= 152 * 6) z.vpc *= 2;
    if (z.smem > kSmemCap) z.ok = false;
    return z;
}

template <typename R>
size_t xy2_smem(int n1, int n2) {
    using C = typename cpx<R>::T;
    return (size_t)(2 * n1 + n2 + (size_t)n2 * (n1 + 1) + (size_t)n1 * n2) * sizeof(C);
}

}  // namespace

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
// log2 of a grid length, for flop counts (5 N log2 N per complex DFT of length N)
static double lg2(int L) { return std::log2((double)L); }

bool apply_zfam_available(const fame_ctx* c, int dtype, int zfam, int m) {
    const int n3 = c->plan.n[2];
    switch (zfam) {
        case 1: return dtype == FAME_C64 && z3_supported(n3);
        case 2: return dtype == FAME_C64 ? z2_config<float>(c, m).ok : z2_config<double>(c, m).ok;
        case 3: return true;
        case 4: return dtype == FAME_C64 && z3_supported(n3);
        default: return false;
    }
}

bool apply_xyfam_available(const fame_ctx* c, int dtype, int xyfam) {
    const int n1 = c->plan.n[0], n2 = c->plan.n[1];
    const size_t esz = dtype == FAME_C64 ? sizeof(float2) : sizeof(double2);
    switch (xyfam) {
        case 1: return dtype == FAME_C64 && xy3_supported(n1, n2);
        case 2: return fft2::supported(n1) && fft2::supported(n2) &&
                       (dtype == FAME_C64 ? xy2_smem<float>(n1, n2) : xy2_smem<double>(n1, n2)) <= kSmemCap;
        case 3: return (size_t)(n1 + n2 + 2 * n1 * n2) * esz <= kSmemCap;
        case 4: return true;
        case 5: return dtype == FAME_C64 && xy3_wide_supported(n1, n2);
        default: return false;
    }
}

template <typename R>
static fame_status xy_stage(fame_ctx* c, const KParams<R>& P, typename cpx<R>::T* W, int m,
                            int mode, R lift_scale, cudaStream_t st) {
    using C = typename cpx<R>::T;
    const bool dbl = sizeof(R) == 8;
    const int n1 = c->plan.n[0], n2 = c->plan.n[1], n3 = c->plan.n[2];
    const double nm = (double)c->n * m;
    const size_t plane_smem = (size_t)(n1 + n2 + 2 * n1 * n2) * sizeof(C);
    fame_status s;
    const int dtype = dbl ? FAME_C128 : FAME_C64;
    int fam = c->apply_plan[dtype].xyfam;
    if (fam == 0 || !apply_xyfam_available(c, dtype, fam))
        for (fam = 1; !apply_xyfam_available(c, dtype, fam); ++fam) {}
    if constexpr (std::is_same<R, float>::value) {
        if (fam == 1 || fam == 5) return run_xy3<R>(c, P, W, m, mode, lift_scale, fam == 5, st);
    }
    const size_t smem2 = xy2_smem<R>(n1, n2);
    if (fam == 2) {
        if ((s = set_smem<R>(c, (const void*)k_xy2<R>, smem2)) != FAME_OK) return s;
        const fft2::Split sx = fft2::split_of(n1), sy = fft2::split_of(n2);
        const int work = std::max(n1 * std::max(sy.R1, sy.R2), n2 * std::max(sx.R1, sx.R2));
        const int th = std::min(512, std::max(128, ((work + 31) / 32) * 32));
        const double bytes = 2.0 * 3 * nm * sizeof(C) + 3.0 * c->n * sizeof(R);
        const double flops = 3 * nm * 5.0 * (mode == 0 ? 2.0 : 1.0) * (lg2(n1) + lg2(n2));
        ProfScope ps(K_XY, dbl, st, bytes, flops);
        k_xy2<R><<<(unsigned)(3LL * m * n3), th, smem2, st>>>(P, W, mode, lift_scale);
        count_launch();
        FAME_CUDA_TRY(c, cudaGetLastError());
        return FAME_OK;
    }
    if (fam == 3) {
        if ((s = set_smem<R>(c, (const void*)k_xy<R>, plane_smem)) != FAME_OK) return s;
        const int th = (n1 * n2 >= 2048) ? 512 : 256;
        // reads and writes the 3 m n workspace once, reads B^{-1} (3n) once
        const double bytes = 2.0 * 3 * nm * sizeof(C) + 3.0 * c->n * sizeof(R);
        const double flops = 3 * nm * 5.0 * (mode == 0 ? 2.0 : 1.0) * (lg2(n1) + lg2(n2));
        ProfScope ps(K_XY, dbl, st, bytes, flops);
        k_xy<R><<<(unsigned)(3LL * m * n3), th, plane_smem, st>>>(P, W, mode, lift_scale);
        count_launch();
        FAME_CUDA_TRY(c, cudaGetLastError());
        return FAME_OK;
    }
    // split path: y pass, x pass, y pass
    int TPy = 16;
    while (TPy > 1 && (size_t)(n2 + 2 * TPy * n2) * sizeof(C) > kSmemCap) TPy /= 2;
    const size_t ysm = (size_t)(n2 + 2 * TPy * n2) * sizeof(C);
    if ((s = set_smem<R>(c, (const void*)k_ypass<R>, ysm)) != FAME_OK) return s;
    int RPB = 16;
    while (RPB > 1 && (size_t)(n1 + 2 * RPB * n1) * sizeof(C) > kSmemCap) RPB /= 2;
    const size_t xsm = (size_t)(n1 + 2 * RPB * n1) * sizeof(C);
    if ((s = set_smem<R>(c, (const void*)k_xpass<R>, xsm)) != FAME_OK) return s;
    const long long nrows = 3LL * m * n3 * n2;
    dim3 yg((n1 + TPy - 1) / TPy, n3, 3 * m);
    const double ybytes = 2.0 * 3 * nm * sizeof(C), yflops = 3 * nm * 5.0 * lg2(n2);
    {
        ProfScope ps(K_YPASS, dbl, st, ybytes, yflops);
        k_ypass<R><<<yg, 256, ysm, st>>>(P, W, TPy, 0);
    }
    {
        ProfScope ps(K_XPASS, dbl, st, ybytes + 3.0 * c->n * sizeof(R),
                     3 * nm * 5.0 * lg2(n1) * (mode == 0 ? 2.0 : 1.0));
        k_xpass<R><<<(unsigned)((nrows + RPB - 1) / RPB), 256, xsm, st>>>(P, W, nrows, RPB, mode, lift_scale);
    }
    count_launch(2);
    if (mode == 0) {
        ProfScope ps(K_YPASS, dbl, st, ybytes, yflops);
        k_ypass<R><<<yg, 256, ysm, st>>>(P, W, TPy, 1);
        count_launch();
    }
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename R>
fame_status run_apply(fame_ctx* c, const typename cpx<R>::T* y, typename cpx<R>::T* Ay, int m,
                      cudaStream_t st) {
    using C = typename cpx<R>::T;
    if (m <= 0) return FAME_OK;
    const size_t need = (size_t)m * 3 * (size_t)c->n * sizeof(C);
    fame_status s = grow(c, c->work, need);
    if (s != FAME_OK) return s;
    return run_apply_into<R>(c, y, Ay, m, reinterpret_cast<C*>(c->work.p), st);
}

// One Z pass (zin: Z-in from y into the workspace; else Z-out from the workspace),
// kernel family and vectors per block from the context's apply plan.
template <typename R>
static fame_status z_pass(fame_ctx* c, const KParams<R>& P, const typename cpx<R>::T* in,
                          typename cpx<R>::T* out, int m, bool zin, cudaStream_t st) {
    using C = typename cpx<R>::T;
    const bool dbl = sizeof(R) == 8;
    const int dtype = dbl ? FAME_C128 : FAME_C64;
    const int n1 = c->plan.n[0], n2 = c->plan.n[1], n3 = c->plan.n[2];
    const double nm = (double)c->n * m;
    const ApplyPlan& ap = c->apply_plan[dtype];
    int fam = ap.zfam;
    if (fam == 0 || !apply_zfam_available(c, dtype, fam, m))
        for (fam = 1; !apply_zfam_available(c, dtype, fam, m); ++fam) {}
    const int vpc_req = ap.vpc > 0 ? std::min(ap.vpc, m) : 0;
    fame_status s;
    if constexpr (std::is_same<R, float>::value) {
        if (fam == 1 || fam == 4) return run_z3<R>(c, P, in, out, m, zin, vpc_req, fam == 1, st);
    }
    const int kind = zin ? K_ZIN : K_ZOUT;
    const double bytes = 5.0 * nm * sizeof(C), flops = 3 * nm * 5.0 * lg2(n3) + 60.0 * nm;
    if (fam == 2) {
        Z2Cfg z2 = z2_config<R>(c, m);
        if (vpc_req) z2.vpc = vpc_req;
        const void* fn = zin ? (const void*)k_zin2<R> : (const void*)k_zout2<R>;
        if ((s = set_smem<R>(c, fn, z2.smem)) != FAME_OK) return s;
        const int TP = 1 << z2.lgTP;
        dim3 grid((n1 + TP - 1) / TP, n2, (m + z2.vpc - 1) / z2.vpc);
        {
            ProfScope ps(kind, dbl, st, bytes, flops);
            if (zin)
                k_zin2<R><<<grid, z2.threads, z2.smem, st>>>(P, in, out, m, z2.lgTP, z2.vpc);
            else
                k_zout2<R><<<grid, z2.threads, z2.smem, st>>>(P, in, out, m, z2.lgTP, z2.vpc);
        }
    } else {
        ZCfg z = z_config<R>(c, m);
        if (vpc_req) z.vpc = vpc_req;
        const void* fn = zin ? (const void*)k_zin<R> : (const void*)k_zout<R>;
        if ((s = set_smem<R>(c, fn, z.smem)) != FAME_OK) return s;
        dim3 grid((n1 + z.TP - 1) / z.TP, n2, (m + z.vpc - 1) / z.vpc);
        {
            ProfScope ps(kind, dbl, st, bytes, flops);
            if (zin)
                k_zin<R><<<grid, z.threads, z.smem, st>>>(P, in, out, m, z.TP, z.vpc);
            else
                k_zout<R><<<grid, z.threads, z.smem, st>>>(P, in, out, m, z.TP, z.vpc);
        }
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template <typename R>
fame_status run_apply_into(fame_ctx* c, const typename cpx<R>::T* y, typename cpx<R>::T* Ay, int m,
                           typename cpx<R>::T* W, cudaStream_t st) {
    if (m <= 0) return FAME_OK;
    const KParams<R> P = make_params<R>(c);
    fame_status s;
    if ((s = z_pass<R>(c, P, y, W, m, true, st)) != FAME_OK) return s;
    if ((s = xy_stage<R>(c, P, W, m, 0, (R)0, st)) != FAME_OK) return s;
    return z_pass<R>(c, P, W, Ay, m, false, st);
}

template <typename R>
fame_status run_lift(fame_ctx* c, const typename cpx<R>::T* y, typename cpx<R>::T* x, int m,
                     cudaStream_t st) {
    if (m <= 0) return FAME_OK;
    const KParams<R> P = make_params<R>(c);
    fame_status s;
    if ((s = z_pass<R>(c, P, y, x, m, true, st)) != FAME_OK) return s;
    return xy_stage<R>(c, P, x, m, 1, (R)(1.0 / std::sqrt((double)c->n)), st);
}

FAME_BOUNDS_READER(transforms)

// ---------------------------------------------------------------------------
// Complex128 apply and lift in double-float arithmetic: the two-level passes with
// A = dfc.  y, Ay and the lift's output are complex128; the workspace between the
// passes holds double-float values (the same 16 bytes per complex entry).
// ---------------------------------------------------------------------------
bool c128_df_available(const fame_ctx* c, int m) {
    // the two-level Z passes; the XY stage as one plane kernel or as y / x / y passes
    return z2_config<double>(c, m).ok;
}

static fame_status z_pass_df(fame_ctx* c, const KParams<double>& P, const double2* y, dfc* W,
                             const dfc* Wz, double2* out, int m, bool zin, cudaStream_t st) {
    const Z2Cfg z2 = z2_config<double>(c, m);
    const void* fn = zin ? (const void*)k_zin2<double, dfc> : (const void*)k_zout2<double, dfc>;
    fame_status s = set_smem<double>(c, fn, z2.smem);
    if (s != FAME_OK) return s;
    const int n1 = c->plan.n[0], n2 = c->plan.n[1], n3 = c->plan.n[2], TP = 1 << z2.lgTP;
    const double nm = (double)c->n * m;
    dim3 grid((n1 + TP - 1) / TP, n2, (m + z2.vpc - 1) / z2.vpc);
    {
        ProfScope ps(zin ? K_ZIN_DF : K_ZOUT_DF, true, st, 5.0 * nm * sizeof(double2),
                     3 * nm * 5.0 * lg2(n3) + 60.0 * nm);
        if (zin)
            k_zin2<double, dfc><<<grid, z2.threads, z2.smem, st>>>(P, y, W, m, z2.lgTP, z2.vpc);
        else
            k_zout2<double, dfc><<<grid, z2.threads, z2.smem, st>>>(P, Wz, out, m, z2.lgTP, z2.vpc);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

static fame_status xy_df(fame_ctx* c, const KParams<double>& P, dfc* W, int m, int mode, double lift_scale,
                         cudaStream_t st) {
    const int n1 = c->plan.n[0], n2 = c->plan.n[1], n3 = c->plan.n[2];
    const size_t smem2 = xy2_smem<double>(n1, n2);
    if (!(fft2::supported(n1) && fft2::supported(n2) && smem2 <= kSmemCap)) {
        // the plane does not fit: y pass, x pass (B^{-1} or the lift), y pass
        int TPy = 16;
        while (TPy > 1 && (size_t)(n2 + 2 * TPy * n2) * sizeof(dfc) > kSmemCap) TPy /= 2;
        const size_t ysm = (size_t)(n2 + 2 * TPy * n2) * sizeof(dfc);
        fame_status s = set_smem<double>(c, (const void*)k_ypass<double, dfc>, ysm);
        if (s != FAME_OK) return s;
        int RPB = 16;
        while (RPB > 1 && (size_t)(n1 + 2 * RPB * n1) * sizeof(dfc) > kSmemCap) RPB /= 2;
        const size_t xsm = (size_t)(n1 + 2 * RPB * n1) * sizeof(dfc);
        if ((s = set_smem<double>(c, (const void*)k_xpass<double, dfc>, xsm)) != FAME_OK) return s;
        const long long nrows = 3LL * m * n3 * n2;
        const double nm = (double)c->n * m;
        dim3 yg((n1 + TPy - 1) / TPy, n3, 3 * m);
        const double ybytes = 2.0 * 3 * nm * sizeof(double2);
        {
            ProfScope ps(K_XY_DF, true, st, ybytes, 3 * nm * 5.0 * lg2(n2));
            k_ypass<double, dfc><<<yg, 256, ysm, st>>>(P, W, TPy, 0);
        }
        {
            ProfScope ps(K_XY_DF, true, st, ybytes + 3.0 * c->n * sizeof(double),
                         3 * nm * 5.0 * lg2(n1) * (mode == 0 ? 2.0 : 1.0));
            k_xpass<double, dfc><<<(unsigned)((nrows + RPB - 1) / RPB), 256, xsm, st>>>(P, W, nrows, RPB, mode,
                                                                                      lift_scale);
        }
        count_launch(2);
        if (mode == 0) {
            ProfScope ps(K_XY_DF, true, st, ybytes, 3 * nm * 5.0 * lg2(n2));
            k_ypass<double, dfc><<<yg, 256, ysm, st>>>(P, W, TPy, 1);
            count_launch();
        }
        FAME_CUDA_TRY(c, cudaGetLastError());
        return FAME_OK;
    }
    fame_status s = set_smem<double>(c, (const void*)k_xy2<double, dfc>, smem2);
    if (s != FAME_OK) return s;
    const fft2::Split sx = fft2::split_of(n1), sy = fft2::split_of(n2);
    const int work = std::max(n1 * std::max(sy.R1, sy.R2), n2 * std::max(sx.R1, sx.R2));
    const int th = std::min(512, std::max(128, ((work + 31) / 32) * 32));
    const double nm = (double)c->n * m;
    {
        ProfScope ps(K_XY_DF, true, st, 2.0 * 3 * nm * sizeof(double2) + 3.0 * c->n * sizeof(double),
                     3 * nm * 5.0 * (mode == 0 ? 2.0 : 1.0) * (lg2(n1) + lg2(n2)));
        k_xy2<double, dfc><<<(unsigned)(3LL * m * n3), th, smem2, st>>>(P, W, mode, lift_scale);
    }
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

fame_status run_apply_c128(fame_ctx* c, const double2* y, double2* Ay, int m, bool df, cudaStream_t st) {
    if (m <= 0) return FAME_OK;
    if (!df || !c128_df_available(c, m)) return run_apply<double>(c, y, Ay, m, st);
    fame_status s = grow(c, c->work, (size_t)m * 3 * (size_t)c->n * sizeof(dfc));
    if (s != FAME_OK) return s;
    const KParams<double> P = make_params<double>(c);
    dfc* W = reinterpret_cast<dfc*>(c->work.p);
    if ((s = z_pass_df(c, P, y, W, nullptr, nullptr, m, true, st)) != FAME_OK) return s;
    if ((s = xy_df(c, P, W, m, 0, 0.0, st)) != FAME_OK) return s;
    return z_pass_df(c, P, nullptr, nullptr, W, Ay, m, false, st);
}

fame_status run_lift_c128(fame_ctx* c, const double2* y, double2* x, int m, bool df, cudaStream_t st) {
    if (m <= 0) return FAME_OK;
    if (!df || !c128_df_available(c, m)) return run_lift<double>(c, y, x, m, st);
    const KParams<double> P = make_params<double>(c);
    dfc* W = reinterpret_cast<dfc*>(x);
    fame_status s;
    if ((s = z_pass_df(c, P, y, W, nullptr, nullptr, m, true, st)) != FAME_OK) return s;
    return xy_df(c, P, W, m, 1, 1.0 / std::sqrt((double)c->n), st);
}

namespace {
// H_j <- -i sqrt(lambda_j) H_j for the m fields [m][3n]
__global__ void k_h_scale(double2* __restrict__ H, const double* __restrict__ w, int m, size_t N3) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)m * N3;
         i += (size_t)gridDim.x * blockDim.x) {
        const double s = w[i / N3];
        const double2 h = H[i];
        H[i] = make_double2(s * h.y, -s * h.x);
    }
}
}  // namespace

// E = B^{-1} Q_r Sigma_r y (the lift) and H = C E / (i omega) = -i omega P_r y,
// omega = sqrt(lambda) (mu_0 = 1): since C = P_r Sigma_r Q_r^* on the range (eq. SVD)
// and Sigma_r Q_r^* E = A_r y = lambda y for an eigenpair.  P_r y is the inverse
// twisted DFT of the per-frequency curl symbol applied to Pi_r y (divided by Sigma_r).
fame_status run_fields(fame_ctx* c, const double2* y, const double* lambda, double2* E, double2* H, int m,
                       cudaStream_t st) {
    if (m <= 0) return FAME_OK;
    fame_status s;
    if (E && (s = run_lift<double>(c, y, E, m, st)) != FAME_OK) return s;
    if (!H) return FAME_OK;
    KParams<double> P = make_params<double>(c);
    P.curl = 1;
    // the generic (two-level / Stockham) Z-in kernels implement the curl expansion
    const ApplyPlan saved = c->apply_plan[FAME_C128];
    if (!(saved.zfam == 2 || saved.zfam == 3)) c->apply_plan[FAME_C128].zfam = apply_zfam_available(c, FAME_C128, 2, m) ? 2 : 3;
    s = z_pass<double>(c, P, y, H, m, true, st);
    c->apply_plan[FAME_C128] = saved;
    if (s != FAME_OK) return s;
    if ((s = xy_stage<double>(c, P, H, m, 2, 1.0 / std::sqrt((double)c->n), st)) != FAME_OK) return s;
    std::vector<double> w(m);
    for (int j = 0; j < m; ++j) w[j] = std::sqrt(std::max(lambda[j], 0.0));
    if ((s = grow(c, c->partial, (size_t)m * sizeof(double))) != FAME_OK) return s;
    double* wd = static_cast<double*>(c->partial.p);
    FAME_CUDA_TRY(c, cudaMemcpyAsync(wd, w.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    k_h_scale<<<1216, 256, 0, st>>>(H, wd, m, 3 * (size_t)c->n);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    FAME_CUDA_TRY(c, cudaStreamSynchronize(st));
    return FAME_OK;
}

fame_status run_grad(fame_ctx* c, const double2* Y, const double* w, int nev, double* dB,
                     cudaStream_t st) {
    const size_t N = 3 * (size_t)c->n;
    // bands lifted together, the workspace kept near 1 GiB at most
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(kGradChunk, ((size_t)1 << 30) / (N * sizeof(double2))));
    fame_status s = grow(c, c->work, (size_t)chunk * N * sizeof(double2));
    if (s != FAME_OK) return s;
    double2* x = reinterpret_cast<double2*>(c->work.p);   // lifted bands, [chunk][3][n]
    FAME_CUDA_TRY(c, cudaMemsetAsync(dB, 0, N * sizeof(double), st));
    for (int j0 = 0; j0 < nev; j0 += chunk) {
        const int mc = std::min(chunk, nev - j0);
        GradWeights gw{};
        bool any = false;
        for (int j = 0; j < mc; ++j) {
            gw.w[j] = w[j0 + j];
            any = any || w[j0 + j] != 0.0;
        }
        if (!any) continue;
        if ((s = run_lift_c128(c, Y + (size_t)j0 * 2 * c->n, x, mc, !fp64_native(), st)) != FAME_OK) return s;
        {
            ProfScope ps(K_GRAD, true, st, (double)N * (mc * sizeof(double2) + 2 * sizeof(double)), 4.0 * N * mc);
            k_grad_accum<<<1216, 256, 0, st>>>(x, gw, mc, dB, N);
        }
        count_launch();
        FAME_CUDA_TRY(c, cudaGetLastError());
    }
    return FAME_OK;
}

fame_status run_basis_mask(fame_ctx* c) {
    const size_t nw = ((size_t)c->n + 31) / 32;
    if (!c->alt_mask && cudaMalloc((void**)&c->alt_mask, nw * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, FAME_E_NOMEM, "cudaMalloc basis mask");
    }
    const KParams<double> Pd = make_params<double>(c);
    k_basis_mask<<<608, 128>>>(Pd, c->alt_mask);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    FAME_CUDA_TRY(c, cudaDeviceSynchronize());
    return FAME_OK;
}

fame_status run_twist_tables(fame_ctx* c) {
    const size_t n = (size_t)c->n, plane = (size_t)c->plan.n[0] * c->plan.n[1], n1 = (size_t)c->plan.n[0];
    struct { void** p; size_t bytes; } bufs[] = {
        {(void**)&c->tf.tw3, n * sizeof(float2)},   {(void**)&c->td.tw3, n * sizeof(double2)},
        {(void**)&c->tf.lam3, n * sizeof(float2)},  {(void**)&c->td.lam3, n * sizeof(double2)},
        {(void**)&c->tf.tw2, plane * sizeof(float2)}, {(void**)&c->td.tw2, plane * sizeof(double2)},
        {(void**)&c->tf.tw1, n1 * sizeof(float2)},  {(void**)&c->td.tw1, n1 * sizeof(double2)}};
    for (auto& b : bufs)
        if (!*b.p && cudaMalloc(b.p, b.bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, FAME_E_NOMEM, "cudaMalloc twist tables");
        }
    const KParams<double> Pd = make_params<double>(c);
    k_twist_tables<<<1216, 256>>>(Pd, c->tf.tw3, c->td.tw3, c->tf.lam3, c->td.lam3, c->tf.tw2, c->td.tw2,
                                  c->tf.tw1, c->td.tw1);
    count_launch();
    FAME_CUDA_TRY(c, cudaGetLastError());
    FAME_CUDA_TRY(c, cudaDeviceSynchronize());
    return FAME_OK;
}

fame_status run_precond_table(fame_ctx* c, cudaStream_t st) {
    const KParams<float> Pf = make_params<float>(c);
    const KParams<double> Pd = make_params<double>(c);
    k_precond<float><<<1216, 256, 0, st>>>(Pf, c->tf.tinv, (float)c->mean_invB);
    k_precond<double><<<1216, 256, 0, st>>>(Pd, c->td.tinv, c->mean_invB);
    count_launch(2);
    FAME_CUDA_TRY(c, cudaGetLastError());
    return FAME_OK;
}

template fame_status run_apply<float>(fame_ctx*, const float2*, float2*, int, cudaStream_t);
template fame_status run_apply<double>(fame_ctx*, const double2*, double2*, int, cudaStream_t);
template fame_status run_apply_into<float>(fame_ctx*, const float2*, float2*, int, float2*, cudaStream_t);
template fame_status run_apply_into<double>(fame_ctx*, const double2*, double2*, int, double2*,
                                            cudaStream_t);
template fame_status run_lift<float>(fame_ctx*, const float2*, float2*, int, cudaStream_t);
template fame_status run_lift<double>(fame_ctx*, const double2*, double2*, int, cudaStream_t);
