// Host-side plan: the lattice of Section 2.2 and the per-axis tables used by
// the transform kernels (twiddles and twist fractions of Section 4.2).
#include <cmath>
#include <cstring>

#include "fame_internal.h"

namespace {

double dot3(const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }
double norm3(const double* u) { return std::sqrt(dot3(u, u)); }

// Section 2.2 rounding: floor when the fractional part is below 1/2, else ceiling.
int round_half_up(double x) {
    double f = std::floor(x);
    return (x - f < 0.5) ? (int)f : (int)f + 1;
}

const int kOrders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

}  // namespace

std::vector<int> radix_list(int L) {
    std::vector<int> r;
    if (L < 2 || L > 1024) return {};
    int x = L;
    while (x % 8 == 0) { r.push_back(8); x /= 8; }
    if (x % 4 == 0) { r.push_back(4); x /= 4; }
    if (x % 2 == 0) { r.push_back(2); x /= 2; }
    while (x % 3 == 0) { r.push_back(3); x /= 3; }
    while (x % 5 == 0) { r.push_back(5); x /= 5; }
    if (x != 1 || (int)r.size() > kMaxStages) return {};
    return r;
}

void compute_kappa(const double* a1, const double* a2, const double* a3, const double* bloch,
                   LatticePlan* p) {
    const double* v[3] = {a1, a2, a3};
    // kappa_l = k . a_l with 2 pi k = bloch; the corrected lattice keeps the reduced
    // coordinates of k (the map Omega of Section 2.3), so the input vectors are used.
    for (int l = 0; l < 3; ++l) p->kappa[l] = dot3(bloch, v[p->perm[l]]) / (2.0 * M_PI);
}

std::string build_lattice(const double* a1, const double* a2, const double* a3, int n1, int n2,
                          int n3, const double* bloch, LatticePlan* out) {
    const double* in[3] = {a1, a2, a3};
    LatticePlan p;
    std::memset(&p, 0, sizeof(p));
    p.n[0] = n1; p.n[1] = n2; p.n[2] = n3;
    // linear independence
    double cr[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2],
                    a2[0] * a3[1] - a2[1] * a3[0]};
    double vol = std::fabs(dot3(a1, cr));
    if (!(vol > 1e-12 * norm3(a1) * norm3(a2) * norm3(a3)))
        return "lattice vectors are linearly dependent";
    // choose the order: a1 longest, and |a2| sin g > |a3| |cos a - cos g cos b| / sin g
    int ord = -1;
    double L[3], cg = 0, cb = 0, ca = 0;
    for (int o = 0; o < 6 && ord < 0; ++o) {
        const double* v[3] = {in[kOrders[o][0]], in[kOrders[o][1]], in[kOrders[o][2]]};
        for (int l = 0; l < 3; ++l) L[l] = norm3(v[l]);
        if (L[0] < L[1] * (1 - 1e-12) || L[0] < L[2] * (1 - 1e-12)) continue;
        cg = dot3(v[0], v[1]) / (L[0] * L[1]);
        cb = dot3(v[0], v[2]) / (L[0] * L[2]);
        ca = dot3(v[1], v[2]) / (L[1] * L[2]);
        double sg = std::sqrt(std::fmax(0.0, 1.0 - cg * cg));
        if (sg > 0.0 && L[1] * sg > L[2] * std::fabs(ca - cg * cb) / sg) ord = o;
    }
    if (ord < 0) return "no ordering of the lattice vectors meets the conditions of Section 2.2";
    for (int l = 0; l < 3; ++l) p.perm[l] = kOrders[ord][l];
    p.len[0] = L[0]; p.len[1] = L[1]; p.len[2] = L[2];
    p.cos_in[0] = cg; p.cos_in[1] = cb; p.cos_in[2] = ca;

    const double dx = L[0] / n1;
    double cosg, cosb, cosa;
    // m1: case I (theta_gamma' <= pi/2) and case II
    if (cg >= 0.0) {
        p.m[0] = round_half_up(L[1] * cg / dx);
        cosg = p.m[0] * dx / L[1];
        p.rho[0] = 0;
    } else {
        p.m[0] = round_half_up((L[0] + L[1] * cg) / dx);
        cosg = (p.m[0] * dx - L[0]) / L[1];
        p.rho[0] = 1;
    }
    double sing = std::sqrt(L[1] * L[1] - (L[1] * cosg) * (L[1] * cosg)) / L[1];
    if (!(sing > 0.0)) return "corrected gamma angle is degenerate";
    const double l2 = L[1] * sing;
    const double dy = l2 / n2;
    // m2: cases on theta_beta'
    if (cb >= 0.0) {
        p.m[1] = round_half_up(L[2] * cb / dx);
        cosb = p.m[1] * dx / L[2];
        p.rho[1] = 0;
    } else {
        p.m[1] = round_half_up((L[0] + L[2] * cb) / dx);
        cosb = (p.m[1] * dx - L[0]) / L[2];
        p.rho[1] = 1;
    }
    // m3: cases on cos(alpha') - cos(gamma) cos(beta), corrected gamma and beta
    const double d = ca - cosg * cosb;
    if (d >= 0.0) {
        p.m[2] = round_half_up(L[2] / dy * d / sing);
        cosa = p.m[2] * dy / L[2] * sing + cosg * cosb;
        p.rho[2] = 0;
    } else {
        p.m[2] = round_half_up((L[1] * sing * sing + L[2] * d) / (dy * sing));
        cosa = (p.m[2] * dy * sing - L[1] * sing * sing) / L[2] + cosg * cosb;
        p.rho[2] = 1;
    }
    const double zz = 1.0 - cosg * cosg - cosb * cosb - cosa * cosa + 2.0 * cosg * cosb * cosa;
    if (!(zz > 0.0)) return "corrected lattice is degenerate";
    p.cos_c[0] = cosg; p.cos_c[1] = cosb; p.cos_c[2] = cosa;
    // eq. (transvec), stored row-major a[row][col]
    p.a[0][0] = L[0];  p.a[0][1] = L[1] * cosg; p.a[0][2] = L[2] * cosb;
    p.a[1][0] = 0.0;   p.a[1][1] = L[1] * sing; p.a[1][2] = L[2] * (cosa - cosg * cosb) / sing;
    p.a[2][0] = 0.0;   p.a[2][1] = 0.0;         p.a[2][2] = L[2] * std::sqrt(zz) / sing;
    p.delta[0] = dx;
    p.delta[1] = dy;
    p.delta[2] = p.a[2][2] / n3;
    // index shifts of a2 and a3 on the grid
    p.s[0] = p.m[0] - p.rho[0] * n1;
    p.s[1] = p.m[1] - p.rho[1] * n1;
    p.s[2] = p.m[2] - p.rho[2] * n2;
    compute_kappa(a1, a2, a3, bloch, &p);
    *out = p;
    return "";
}

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------
namespace {

// fraction x reduced to [0, 1)
double frac01(double x) {
    double f = x - std::floor(x);
    return (f >= 1.0) ? 0.0 : f;
}

Frac32 split32(double f) {
    // hi: multiple of 2^-13 nearest to f; lo: remainder (|lo| <= 2^-14)
    double hi = std::nearbyint(f * 8192.0) / 8192.0;
    Frac32 r;
    r.hi = (float)hi;
    r.lo = (float)(f - hi);
    return r;
}

template <typename T>
fame_status upload(fame_ctx* c, T** dst, const std::vector<T>& src) {
    if (*dst == nullptr) {
        cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
        if (e != cudaSuccess) return set_err(c, FAME_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    FAME_CUDA_TRY(c, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FAME_OK;
}

}  // namespace

fame_status build_tables(fame_ctx* c) {
    const LatticePlan& p = c->plan;
    const int n1 = p.n[0], n2 = p.n[1], n3 = p.n[2];
    // twiddles e^{-2 pi i t / L} per axis, computed in double
    for (int ax = 0; ax < 3; ++ax) {
        const int L = p.n[ax];
        std::vector<float2> tf(L);
        std::vector<double2> td(L);
        for (int t = 0; t < L; ++t) {
            // exact-angle evaluation through the reduced fraction t/L
            double s = std::sin(2.0 * M_PI * t / L), co = std::cos(2.0 * M_PI * t / L);
            if (4 * t == L) { s = 1.0; co = 0.0; }
            if (2 * t == L) { s = 0.0; co = -1.0; }
            if (4 * t == 3 * L) { s = -1.0; co = 0.0; }
            td[t] = make_double2(co, -s);
            tf[t] = make_float2((float)co, (float)-s);
        }
        fame_status st = upload(c, &c->tf.tw[ax], tf);
        if (st != FAME_OK) return st;
        st = upload(c, &c->td.tw[ax], td);
        if (st != FAME_OK) return st;
    }
    // twist fractions of Section 4 on the index-shift lattice:
    //   c1 = kappa1, c2(p) = kappa2 - s1 (p + c1)/n1,
    //   c3(p,q) = kappa3 - s2 (p + c1)/n1 - s3 (q + c2(p))/n2
    const double k1 = p.kappa[0], k2 = p.kappa[1], k3 = p.kappa[2];
    const double c1 = k1;
    std::vector<double> c2(n1);
    std::vector<double> f2d(n1), f3d((size_t)n1 * n2);
    std::vector<Frac32> f2f(n1), f3f((size_t)n1 * n2);
    for (int pp = 0; pp < n1; ++pp) {
        c2[pp] = k2 - (double)p.s[0] * (pp + c1) / n1;
        f2d[pp] = frac01(c2[pp] / n2);
        f2f[pp] = split32(f2d[pp]);
    }
    for (int q = 0; q < n2; ++q)
        for (int pp = 0; pp < n1; ++pp) {
            double c3 = k3 - (double)p.s[1] * (pp + c1) / n1 - (double)p.s[2] * (q + c2[pp]) / n2;
            double f = frac01(c3 / n3);
            f3d[(size_t)q * n1 + pp] = f;
            f3f[(size_t)q * n1 + pp] = split32(f);
        }
    c->td.f1 = frac01(c1 / n1);
    c->tf.f1 = split32(c->td.f1);
    fame_status st;
    if ((st = upload(c, &c->td.f2, f2d)) != FAME_OK) return st;
    if ((st = upload(c, &c->tf.f2, f2f)) != FAME_OK) return st;
    if ((st = upload(c, &c->td.f3, f3d)) != FAME_OK) return st;
    if ((st = upload(c, &c->tf.f3, f3f)) != FAME_OK) return st;
    if ((st = run_basis_mask(c)) != FAME_OK) return st;
    return run_twist_tables(c);
}

template <typename R>
static void fill_common(const fame_ctx* c, KParams<R>& k, const DevTables<R>& t) {
    const LatticePlan& p = c->plan;
    k.n1 = p.n[0]; k.n2 = p.n[1]; k.n3 = p.n[2];
    k.inv_dx = (R)(1.0 / p.delta[0]);
    k.inv_dy = (R)(1.0 / p.delta[1]);
    k.inv_dz = (R)(1.0 / p.delta[2]);
    k.f1 = t.f1;
    k.f2 = t.f2;
    k.f3 = t.f3;
    for (int ax = 0; ax < 3; ++ax) {
        k.tw[ax] = t.tw[ax];
        std::vector<int> r = radix_list(p.n[ax]);
        k.ax[ax].L = p.n[ax];
        k.ax[ax].nst = (int)r.size();
        for (int s = 0; s < (int)r.size(); ++s) k.ax[ax].radix[s] = r[s];
    }
    k.invB = t.invB;
    k.alt = c->alt_mask;
    k.tw3 = t.tw3;
    k.lam3 = t.lam3;
    k.tw2 = t.tw2;
    k.tw1 = t.tw1;
    k.scale = (R)(1.0 / (double)c->n);
    k.curl = 0;
}

template <>
KParams<float> make_params<float>(const fame_ctx* c) {
    KParams<float> k;
    fill_common<float>(c, k, c->tf);
    return k;
}
template <>
KParams<double> make_params<double>(const fame_ctx* c) {
    KParams<double> k;
    fill_common<double>(c, k, c->td);
    return k;
}
