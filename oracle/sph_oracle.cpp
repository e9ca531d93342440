/*
 * WCSPH oracle: a plain, slow, obviously-correct CPU implementation of the
 * per-timestep particle loop of weakly-compressible SPH described in the PySPH
 * paper (Sec. 2): uniform-grid neighbour search, summation density or
 * continuity, Tait equation of state, momentum with pressure, laminar viscosity
 * and Monaghan artificial viscosity, XSPH, and the predictor-corrector
 * integrator with periodic wrap and static wall particles.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library. The CUDA path never calls
 * it and shares no code, header, table or constant with it.
 *
 * Arithmetic is FP64 throughout. The one place where another precision enters is
 * the neighbour predicate, which is evaluated in the precision of the mode being
 * checked (FP64 or FP32), because that predicate defines the neighbour set.
 * Compile with -ffp-contract=off so no multiply-add is fused.
 *
 * Every function is templated on the scalar type T: T = double for the plain
 * run, T = Dual for forward-mode derivatives (exact derivative of the discrete
 * map with the neighbour set of each step held fixed).
 *
 * Readings of points the paper leaves open (each one is listed in the design notes):
 *  - quintic spline: Morris form, support 3h, sigma_2D = 7/(478 pi), sigma_3D = 1/(120 pi);
 *  - Wendland C2: (1-q/2)^4 (2q+1), support 2h, sigma_2D = 7/(4 pi), sigma_3D = 21/(16 pi);
 *  - cubic spline: 1 - 3q^2/2 + 3q^3/4 on [0,1), (2-q)^3/4 on [1,2), sigma_2D = 10/(7 pi),
 *    sigma_3D = 1/pi;
 *  - neighbour predicate: i != j and r^2 < (k h)^2 with r^2 = ((dx dx) + dy dy) + dz dz,
 *    minimum image dx -= L if dx > L/2, dx += L if dx < -L/2, in the mode's precision;
 *  - cell grid: n_d = floor(ext_d / (k h / R * 1.00001)) with R = 1 in 2D and 2 in 3D,
 *    cs_d = ext_d / n_d, c_d = floor(((double)x_mode - lo_d) / cs_d) clamped to
 *    [0, n_d - 1], a stencil of (2R + 1)^d cells;
 *  - eta = 0.01 in the laminar viscosity, Monaghan AV with beta = 0 and 0.01 h^2;
 *  - XSPH over fluid sources, entering the drift only;
 *  - predictor-corrector as kick-drift-kick for u and x; the density advanced like the
 *    positions with the continuity rate at (x^{n+1}, u^{n+1/2}) before the momentum
 *    evaluation at (x^{n+1}, u^{n+1/2}, rho^{n+1});
 *  - (option) the two-evaluation midpoint predict-evaluate-correct form of the same
 *    integrator (Monaghan 2005): a half step with the rates at t^n, the rates at the
 *    midpoint, a full step from t^n with those, then the rates at t^{n+1};
 *  - walls static (x and u fixed), wall density from continuity with fluid sources, or
 *    (option) the wall pressure of Adami et al. (2012) with the density from the EOS.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int KERNEL_QUINTIC = 0;
constexpr int KERNEL_WENDLAND_C2 = 1;
constexpr int KERNEL_CUBIC_SPLINE = 2;
constexpr int ROLE_FLUID = 0;
constexpr int PREC_FP32 = 1;
constexpr int DENSITY_CONTINUITY = 0;
constexpr int DENSITY_SUMMATION = 1;
constexpr int DENSITY_EDAC = 2;
constexpr int WALL_ADAMI = 1;
constexpr int INTEGRATOR_PEC = 1;
constexpr double PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- dual numbers */
struct Dual {
    double v;  // value
    double d;  // derivative along the seeded direction
    Dual() : v(0.0), d(0.0) {}
    Dual(double value) : v(value), d(0.0) {}
    Dual(double value, double deriv) : v(value), d(deriv) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt_(Dual a) {
    double s = std::sqrt(a.v);
    return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline double sqrt_(double a) { return std::sqrt(a); }
inline Dual pow_(Dual a, double e) {
    double p = std::pow(a.v, e);
    return Dual(p, e * std::pow(a.v, e - 1.0) * a.d);
}
inline double pow_(double a, double e) { return std::pow(a, e); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

template <class T> T ipow(T a, int e) {
    T r = T(1.0);
    for (int i = 0; i < e; ++i) r = r * a;
    return r;
}

}  // namespace

extern "C" {

/* Parameters of one problem. Layout mirrored by the Python wrapper (ctypes). */
typedef struct {
    int32_t dim;          // 2 or 3
    int32_t kernel;       // 0 quintic spline, 1 Wendland C2
    int32_t precision;    // precision of the neighbour predicate: 0 FP64, 1 FP32
    int32_t density;      // 0 continuity equation, 1 summation density, 2 EDAC pressure equation
    int32_t periodic[3];  // per axis
    int32_t brute;        // 1: neighbour search by all-pairs loop instead of cells
    int32_t wall_bc;      // 0: wall density from continuity, 1: wall pressure of Adami et al.
    int32_t integrator;   // 0: kick-drift-kick, 1: midpoint predict-evaluate-correct
    double h;             // smoothing length
    double lo[3], hi[3];  // cell box (periodic box on periodic axes)
    double rho0, c0, gamma;
    double nu;            // kinematic viscosity of the laminar term
    double eta;           // regulariser of the laminar term (eta h^2)
    double alpha;         // Monaghan artificial viscosity coefficient
    double xsph_eps;      // XSPH coefficient
    double g[3];          // body acceleration
    double edac_alpha;    // EDAC: pressure diffusivity nu_e = edac_alpha h c0 / 8
} ora_params;

}  // extern "C"

namespace {

double support_factor(int kernel) { return kernel == KERNEL_QUINTIC ? 3.0 : 2.0; }

/* ------------------------------------------------------------------ kernels
 * Sec. 2, Eq. (sph:interpolation:sum): W(r, h) = sigma / h^d * w(q), q = r / h.
 * dW/dr = sigma / h^(d+1) * w'(q).
 */
template <class T>
void kernel_eval(int kernel, int dim, double h, T r, T* W, T* dWdr) {
    T q = r / h;
    T w = T(0.0), dw = T(0.0);
    double sigma;
    if (kernel == KERNEL_QUINTIC) {
        sigma = dim == 2 ? 7.0 / (478.0 * PI) : 1.0 / (120.0 * PI);
        double qv = val(q);
        if (qv < 3.0) { T t = 3.0 - q; w += ipow(t, 5); dw -= 5.0 * ipow(t, 4); }
        if (qv < 2.0) { T t = 2.0 - q; w -= 6.0 * ipow(t, 5); dw += 30.0 * ipow(t, 4); }
        if (qv < 1.0) { T t = 1.0 - q; w += 15.0 * ipow(t, 5); dw -= 75.0 * ipow(t, 4); }
    } else if (kernel == KERNEL_CUBIC_SPLINE) {
        /* M4 cubic B-spline (Monaghan and Lattanzio 1985), support 2h, piecewise form */
        sigma = dim == 2 ? 10.0 / (7.0 * PI) : 1.0 / PI;
        double qv = val(q);
        if (qv < 1.0) {
            w = 1.0 - 1.5 * q * q + 0.75 * q * q * q;
            dw = -3.0 * q + 2.25 * q * q;
        } else if (qv < 2.0) {
            T t = 2.0 - q;
            w = 0.25 * ipow(t, 3);
            dw = -0.75 * t * t;
        }
    } else {
        sigma = dim == 2 ? 7.0 / (4.0 * PI) : 21.0 / (16.0 * PI);
        if (val(q) < 2.0) {
            T t = 1.0 - 0.5 * q;
            w = ipow(t, 4) * (2.0 * q + 1.0);
            dw = -5.0 * q * ipow(t, 3);
        }
    }
    double hd = std::pow(h, dim);
    *W = (sigma / hd) * w;
    *dWdr = (sigma / (hd * h)) * dw;
}

/* ------------------------------------------------------------------- grid
 * Sec. 2.2: a uniform cell grid searched with a stencil of (2R + 1)^d cells: R = 1 in 2D
 * (cells no smaller than the support radius kh, 3 x 3), R = 2 in 3D (cells no smaller than
 * kh / 2, 5 x 5 x 5). Any pair inside the support lies at most R cells apart per axis.
 */
int reach_of(int dim) { return dim == 3 ? 2 : 1; }

struct Grid {
    int dim;
    int n[3];
    double cs[3];
    double lo[3];
    int64_t ncells;
};

int make_grid(const ora_params* P, Grid* G) {
    if (P->dim != 2 && P->dim != 3) return -1;
    double kh = support_factor(P->kernel) * P->h;
    G->dim = P->dim;
    G->ncells = 1;
    for (int d = 0; d < 3; ++d) {
        if (d < P->dim) {
            double ext = P->hi[d] - P->lo[d];
            if (!(ext > 0.0) || !(kh > 0.0)) return -1;
            const int R = reach_of(P->dim);
            double nd = std::floor(ext / (kh / R * 1.00001));
            if (nd < 1.0) nd = 1.0;
            if (nd > 1e7) return -1;
            G->n[d] = (int)nd;
            if (P->periodic[d] && G->n[d] < 2 * R + 1) return -2;
            G->cs[d] = ext / (double)G->n[d];
            G->lo[d] = P->lo[d];
        } else {
            G->n[d] = 1;
            G->cs[d] = 1.0;
            G->lo[d] = 0.0;
        }
        G->ncells *= G->n[d];
    }
    return 0;
}

/* Position as seen by the predicate and the binning: rounded once to the mode's precision. */
double mode_value(const ora_params* P, double x) {
    return P->precision == PREC_FP32 ? (double)(float)x : x;
}

int cell_coord(const Grid& G, const ora_params* P, int d, double x) {
    double v = (mode_value(P, x) - G.lo[d]) / G.cs[d];
    double c = std::floor(v);
    if (!(c >= 0.0)) return 0;  // also catches NaN
    if (c > (double)(G.n[d] - 1)) return G.n[d] - 1;
    return (int)c;
}

/* ------------------------------------------------------------ the predicate */
template <class P_>
bool within_support_t(const ora_params* P, const double* xi, const double* xj) {
    P_ r2 = (P_)0;
    for (int d = 0; d < P->dim; ++d) {
        P_ dx = (P_)xi[d] - (P_)xj[d];
        if (P->periodic[d]) {
            P_ L = (P_)(P->hi[d] - P->lo[d]);
            P_ half = L * (P_)0.5;
            if (dx > half) dx = dx - L;
            else if (dx < -half) dx = dx + L;
        }
        r2 = r2 + dx * dx;
    }
    P_ kh = (P_)support_factor(P->kernel) * (P_)P->h;
    return r2 < kh * kh;
}

bool within_support(const ora_params* P, const double* xi, const double* xj) {
    if (P->precision == PREC_FP32) return within_support_t<float>(P, xi, xj);
    return within_support_t<double>(P, xi, xj);
}

/* ----------------------------------------------------------- neighbour sets */
struct Neighbours {
    const ora_params* P;
    Grid G;
    int64_t n;
    std::vector<double> pos;        // n x 3, primal positions
    std::vector<int32_t> cell3;     // n x 3 cell coordinates
    std::vector<int64_t> start;     // ncells + 1
    std::vector<int64_t> members;   // particle ids grouped by cell, ascending inside a cell

    void build(const ora_params* prm, int64_t n_, const double* const* x) {
        P = prm;
        n = n_;
        make_grid(P, &G);
        pos.assign((size_t)n * 3, 0.0);
        cell3.assign((size_t)n * 3, 0);
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < P->dim; ++d) {
                pos[i * 3 + d] = x[d][i];
                cell3[i * 3 + d] = cell_coord(G, P, d, x[d][i]);
            }
        start.assign((size_t)G.ncells + 1, 0);
        std::vector<int64_t> lin(n);
        for (int64_t i = 0; i < n; ++i) {
            lin[i] = linear(&cell3[i * 3]);
            start[lin[i] + 1]++;
        }
        for (int64_t c = 0; c < G.ncells; ++c) start[c + 1] += start[c];
        members.assign(n, 0);
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < n; ++i) members[fill[lin[i]]++] = i;
    }

    int64_t linear(const int32_t* c) const {
        return (int64_t)c[0] + (int64_t)G.n[0] * ((int64_t)c[1] + (int64_t)G.n[1] * (int64_t)c[2]);
    }

    /* Neighbours of i (j != i, predicate true), ascending id; returns the candidates examined. */
    int64_t of(int64_t i, std::vector<int64_t>& out) const {
        out.clear();
        int64_t cand = 0;
        if (P->brute) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                ++cand;
                if (within_support(P, &pos[i * 3], &pos[j * 3])) out.push_back(j);
            }
            return cand;
        }
        const int32_t* ci = &cell3[i * 3];
        int lo3[3], hi3[3];
        const int R = reach_of(P->dim);
        for (int d = 0; d < 3; ++d) {
            if (d < P->dim) { lo3[d] = -R; hi3[d] = R; } else { lo3[d] = 0; hi3[d] = 0; }
        }
        for (int oz = lo3[2]; oz <= hi3[2]; ++oz)
            for (int oy = lo3[1]; oy <= hi3[1]; ++oy)
                for (int ox = lo3[0]; ox <= hi3[0]; ++ox) {
                    int off[3] = {ox, oy, oz};
                    int32_t c[3];
                    bool skip = false;
                    for (int d = 0; d < 3; ++d) {
                        int v = ci[d] + off[d];
                        if (v < 0 || v >= G.n[d]) {
                            if (d < P->dim && P->periodic[d]) v = (v + G.n[d]) % G.n[d];
                            else skip = true;
                        }
                        c[d] = v;
                    }
                    if (skip) continue;
                    int64_t lc = linear(c);
                    for (int64_t k = start[lc]; k < start[lc + 1]; ++k) {
                        int64_t j = members[k];
                        if (j == i) continue;
                        ++cand;
                        if (within_support(P, &pos[i * 3], &pos[j * 3])) out.push_back(j);
                    }
                }
        std::sort(out.begin(), out.end());
        return cand;
    }
};

/* ----------------------------------------------------------------- state */
template <class T>
struct State {
    std::vector<T> x[3], u[3], rho;
    std::vector<T> p;  // EDAC: the pressure, a state variable (else unused)
};

template <class T>
struct Rates {
    std::vector<T> arho, a[3], xs[3], p;
};

/* Periodic wrap into [lo, hi) (Sec. 3 update_domain). */
double wrap1(double x, double lo, double hi) {
    double L = hi - lo;
    if (x >= lo && x < hi) return x;
    double k = std::floor((x - lo) / L);
    x = x - k * L;
    if (x >= hi) x = x - L;
    if (x < lo) x = lo;
    return x;
}

template <class T>
T wrap_t(T x, double lo, double hi);
template <>
double wrap_t<double>(double x, double lo, double hi) { return wrap1(x, lo, hi); }
template <>
Dual wrap_t<Dual>(Dual x, double lo, double hi) { return Dual(wrap1(x.v, lo, hi), x.d); }

/* EOS, Eq. (eos): p = c0^2 rho0 / gamma * ((rho / rho0)^gamma - 1), evaluated as
 * B expm1(gamma log1p(delta)) with delta = (rho - rho0) / rho0: the same quantity
 * without the cancellation of (rho/rho0)^gamma - 1 near rho0 (condition ~ 1/delta). */
inline double tait_ratio(double delta, double gamma) {
    return std::expm1(gamma * std::log1p(delta));
}
inline Dual tait_ratio(Dual delta, double gamma) {
    double l = std::log1p(delta.v);
    double e = std::expm1(gamma * l);
    // d/ddelta expm1(gamma log1p(delta)) = gamma (1 + delta)^(gamma - 1)
    return Dual(e, gamma * std::exp((gamma - 1.0) * l) * delta.d);
}
template <class T>
T tait(const ora_params* P, T rho) {
    double B = P->c0 * P->c0 * P->rho0 / P->gamma;
    T delta = (rho - P->rho0) / P->rho0;
    return B * tait_ratio(delta, P->gamma);
}

struct Counts {
    int64_t pairs = 0;       // ordered interacting pairs i != j
    int64_t candidates = 0;  // ordered (i, j) pairs examined in the (2R + 1)^d stencil, j != i
};

/* ------------------------------------------------------------- the RHS
 * One evaluation of the right-hand sides at state S, in the group order of
 * Sec. 3.2: the density group (summation density, Eq. 2, or the continuity rate,
 * Eq. continuity:sph, with the density advanced by dt_rho times that rate), the EOS
 * on all particles, then momentum (with XSPH) on every fluid destination. Sources
 * are visited in ascending particle id. dt_rho = 0 leaves the density unchanged
 * (an evaluation without a step).
 */
template <class T>
void rhs(const ora_params* P, T nu, T alpha, int64_t n, State<T>& S, const double* m,
         const uint8_t* role, Rates<T>& R, Counts* counts, double dt_rho) {
    const int dim = P->dim;
    std::vector<double> px[3];
    const double* xp[3] = {nullptr, nullptr, nullptr};
    for (int d = 0; d < dim; ++d) {
        px[d].resize(n);
        for (int64_t i = 0; i < n; ++i) px[d][i] = val(S.x[d][i]);
        xp[d] = px[d].data();
    }
    Neighbours NB;
    NB.build(P, n, xp);

    std::vector<std::vector<int64_t>> nbr(n);
    std::vector<int64_t> cand(n, 0);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) cand[i] = NB.of(i, nbr[i]);

    auto diff = [&](int64_t i, int64_t j, T* r) {
        for (int d = 0; d < 3; ++d) r[d] = T(0.0);
        for (int d = 0; d < dim; ++d) {
            T dx = S.x[d][i] - S.x[d][j];
            if (P->periodic[d]) {
                double L = P->hi[d] - P->lo[d];
                if (val(dx) > 0.5 * L) dx = dx - L;
                else if (val(dx) < -0.5 * L) dx = dx + L;
            }
            r[d] = dx;
        }
    };
    auto kern = [&](const T* r, T* W, T* gW) {
        T r2 = T(0.0);
        for (int d = 0; d < dim; ++d) r2 = r2 + r[d] * r[d];
        T rr = val(r2) > 0.0 ? sqrt_(r2) : T(0.0);
        T dWdr;
        kernel_eval(P->kernel, dim, P->h, rr, W, &dWdr);
        for (int d = 0; d < 3; ++d) gW[d] = T(0.0);
        if (val(rr) > 0.0)
            for (int d = 0; d < dim; ++d) gW[d] = dWdr * r[d] / rr;
        return r2;
    };

    /* Eq. (2), summation density (self term included). */
    if (P->density == DENSITY_SUMMATION) {
        std::vector<T> rho_new(n);
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            T W0, dW0;
            kernel_eval(P->kernel, dim, P->h, T(0.0), &W0, &dW0);
            T s = m[i] * W0;
            for (int64_t j : nbr[i]) {
                T r[3], W, gW[3];
                diff(i, j, r);
                kern(r, &W, gW);
                s = s + m[j] * W;
            }
            rho_new[i] = s;
        }
        S.rho = rho_new;
    }

    /* Eq. (continuity:sph); wall destinations take fluid sources only. The density
     * is then advanced with the rate, like the positions (Sec. 2.1 reading). */
    R.arho.assign(n, T(0.0));
    if (P->density == DENSITY_CONTINUITY) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            const bool fluid_i = role[i] == ROLE_FLUID;
            T arho = T(0.0);
            for (int64_t j : nbr[i]) {
                if (!fluid_i && role[j] != ROLE_FLUID) continue;
                T r[3], W, gW[3];
                diff(i, j, r);
                kern(r, &W, gW);
                T vdotg = T(0.0);
                for (int d = 0; d < dim; ++d) vdotg = vdotg + (S.u[d][i] - S.u[d][j]) * gW[d];
                arho = arho + m[j] * vdotg;
            }
            R.arho[i] = arho;
        }
        if (dt_rho != 0.0)
            for (int64_t i = 0; i < n; ++i) S.rho[i] = S.rho[i] + dt_rho * R.arho[i];
    }

    /* The EDAC scheme (Sec. 2.3 lists it; Sec. 4.1 solves the Taylor-Green vortex with it):
     * the pressure is a particle variable evolved by
     *   dp/dt = -rho0 c0^2 div u + nu_e lap p,   nu_e = edac_alpha h c0 / 8,
     * with the density held at rho0 (particle volumes m / rho0). The SPH forms: the
     * divergence as in the continuity equation, the Laplacian in the form of the laminar
     * viscosity term (Eq. mom:sph:visc) with the 0.01 h^2 regulariser,
     *   dp_i/dt = c0^2 sum_j m_j u_ij . grad_i W_ij
     *           + (2 nu_e / rho0) sum_j m_j (p_i - p_j) (r_ij . grad_i W_ij) / (r_ij^2 + 0.01 h^2).
     * The rate sits in the density-rate slot (arho); the pressure is advanced with it like
     * the density of the continuity form, before the momentum equation reads it. */
    if (P->density == DENSITY_EDAC) {
        const double nu_e = P->edac_alpha * P->h * P->c0 / 8.0;
        const double c2 = P->c0 * P->c0;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            T ap = T(0.0);
            for (int64_t j : nbr[i]) {
                T r[3], W, gW[3];
                diff(i, j, r);
                T r2 = kern(r, &W, gW);
                T vdotg = T(0.0), rdotg = T(0.0);
                for (int d = 0; d < dim; ++d) {
                    vdotg = vdotg + (S.u[d][i] - S.u[d][j]) * gW[d];
                    rdotg = rdotg + r[d] * gW[d];
                }
                ap = ap + c2 * m[j] * vdotg;
                ap = ap + 2.0 * nu_e / P->rho0 * m[j] * (S.p[i] - S.p[j]) * rdotg /
                              (r2 + 0.01 * P->h * P->h);
            }
            R.arho[i] = ap;
        }
        if (dt_rho != 0.0)
            for (int64_t i = 0; i < n; ++i) S.p[i] = S.p[i] + dt_rho * R.arho[i];
    }

    R.p.assign(n, T(0.0));
    for (int64_t i = 0; i < n; ++i) R.p[i] = P->density == DENSITY_EDAC ? S.p[i] : tait(P, S.rho[i]);

    /* Solid-wall pressure of Adami, Hu and Adams (2012), the wall boundary condition listed
     * among the schemes of Sec. 2.3 (formula from that reference): a wall particle w takes the kernel-weighted mean of its fluid
     * neighbours' pressure plus the hydrostatic part of the body force (static walls, no
     * wall acceleration),
     *   p_w = (sum_f p_f W_wf + g . sum_f rho_f r_wf W_wf) / sum_f W_wf,  r_wf = x_w - x_f,
     * and the density the Tait EOS maps to p_w, rho_w = rho0 (1 + p_w / B)^(1 / gamma).
     * A wall with no fluid neighbour takes p_w = 0 and rho_w = rho0. The fluid values are
     * those of this evaluation (after the density update above). */
    if (P->wall_bc == WALL_ADAMI) {
        const double B = P->c0 * P->c0 * P->rho0 / P->gamma;
        std::vector<T> pw(n, T(0.0)), rw(n, T(0.0));
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            if (role[i] == ROLE_FLUID) continue;
            T sw = T(0.0), sp = T(0.0), sg = T(0.0);
            for (int64_t j : nbr[i]) {
                if (role[j] != ROLE_FLUID) continue;
                T r[3], W, gW[3];
                diff(i, j, r);
                kern(r, &W, gW);
                T gr = T(0.0);
                for (int d = 0; d < dim; ++d) gr = gr + P->g[d] * r[d];
                sw = sw + W;
                sp = sp + R.p[j] * W;
                sg = sg + S.rho[j] * gr * W;
            }
            if (val(sw) > 0.0) {
                pw[i] = (sp + sg) / sw;
                rw[i] = P->rho0 * pow_(1.0 + pw[i] / B, 1.0 / P->gamma);
            } else {
                pw[i] = T(0.0);
                rw[i] = T(P->rho0);
            }
        }
        for (int64_t i = 0; i < n; ++i)
            if (role[i] != ROLE_FLUID) {
                R.p[i] = pw[i];
                S.rho[i] = rw[i];
            }
    }

    for (int d = 0; d < 3; ++d) {
        R.a[d].assign(n, T(0.0));
        R.xs[d].assign(n, T(0.0));
    }
    std::vector<int64_t> npairs(n, 0);
    const double h = P->h;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        const bool fluid_i = role[i] == ROLE_FLUID;
        T a[3] = {T(0.0), T(0.0), T(0.0)}, xs[3] = {T(0.0), T(0.0), T(0.0)};
        const T Pr_i = R.p[i] / (S.rho[i] * S.rho[i]);
        for (int64_t j : nbr[i]) {
            const bool fluid_j = role[j] == ROLE_FLUID;
            if (!fluid_i && !fluid_j) continue;  // wall-wall: no equation couples them
            ++npairs[i];
            T r[3], W, gW[3];
            diff(i, j, r);
            T r2 = kern(r, &W, gW);
            if (!fluid_i) continue;
            T vij[3], vdotr = T(0.0), rdotg = T(0.0);
            for (int d = 0; d < 3; ++d) vij[d] = S.u[d][i] - S.u[d][j];
            for (int d = 0; d < dim; ++d) {
                vdotr = vdotr + vij[d] * r[d];
                rdotg = rdotg + r[d] * gW[d];
            }
            /* Eq. (mom:sph:press). */
            T Pr_j = R.p[j] / (S.rho[j] * S.rho[j]);
            T pf = Pr_i + Pr_j;
            for (int d = 0; d < dim; ++d) a[d] = a[d] - m[j] * pf * gW[d];
            T rhobar = 0.5 * (S.rho[i] + S.rho[j]);
            /* Eq. (mom:sph:visc), laminar viscosity. */
            if (val(nu) != 0.0) {
                T f = m[j] * 4.0 * nu / (S.rho[i] + S.rho[j]) * rdotg / (r2 + P->eta * h * h);
                for (int d = 0; d < dim; ++d) a[d] = a[d] + f * vij[d];
            }
            /* Monaghan artificial viscosity (classic WCSPH scheme), beta = 0. */
            if (val(alpha) != 0.0 && val(vdotr) < 0.0) {
                T mu = h * vdotr / (r2 + 0.01 * h * h);
                T Pi = -alpha * P->c0 * mu / rhobar;
                for (int d = 0; d < dim; ++d) a[d] = a[d] - m[j] * Pi * gW[d];
            }
            /* XSPH velocity correction over fluid sources. */
            if (P->xsph_eps != 0.0 && fluid_j) {
                T f = P->xsph_eps * m[j] / rhobar * W;
                for (int d = 0; d < dim; ++d) xs[d] = xs[d] - f * vij[d];
            }
        }
        if (fluid_i)
            for (int d = 0; d < dim; ++d) a[d] = a[d] + P->g[d];  // body force, Eq. (mom:sph)
        for (int d = 0; d < 3; ++d) { R.a[d][i] = a[d]; R.xs[d][i] = xs[d]; }
    }
    if (counts) {
        counts->pairs = 0;
        counts->candidates = 0;
        for (int64_t i = 0; i < n; ++i) {
            counts->pairs += npairs[i];
            counts->candidates += cand[i];
        }
    }
}

/* Diagnostics record: t, dt, KE, max|u|, Px, Py, Pz, max|a|, pairs, candidates. */
constexpr int HIST = 10;

template <class T>
void diagnostics(const ora_params* P, int64_t n, const State<T>& S, const Rates<T>& R,
                 const double* m, const uint8_t* role, double t, double dt, const Counts& c,
                 double* rec) {
    double ke = 0.0, umax = 0.0, amax = 0.0, mom[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        if (role[i] != ROLE_FLUID) continue;
        double u2 = 0.0, a2 = 0.0;
        for (int d = 0; d < P->dim; ++d) {
            double ud = val(S.u[d][i]);
            double ad = val(R.a[d][i]);
            u2 += ud * ud;
            a2 += ad * ad;
            mom[d] += m[i] * ud;
        }
        ke += 0.5 * m[i] * u2;
        umax = std::max(umax, std::sqrt(u2));
        amax = std::max(amax, std::sqrt(a2));
    }
    rec[0] = t; rec[1] = dt; rec[2] = ke; rec[3] = umax;
    rec[4] = mom[0]; rec[5] = mom[1]; rec[6] = mom[2]; rec[7] = amax;
    rec[8] = (double)c.pairs; rec[9] = (double)c.candidates;
}

/* Time step from the CFL-type criteria (reading of Sec. 2.1): acoustic, force, viscous. */
double cfl_dt(const ora_params* P, double umax, double amax) {
    double dt = 0.25 * P->h / (P->c0 + umax);
    if (amax > 0.0) dt = std::min(dt, 0.25 * std::sqrt(P->h / amax));
    if (P->nu > 0.0) dt = std::min(dt, 0.125 * P->h * P->h / P->nu);
    return dt;
}

/* ------------------------------------------------------- the integrator
 * Sec. 2.1 predictor-corrector, read as kick-drift-kick for u and x, with the
 * density advanced like the positions (it is a function of the configuration):
 *   u^{n+1/2} = u^n + dt/2 a^n,
 *   x^{n+1} = wrap(x^n + dt (u^{n+1/2} + xsph^n)),
 *   arho^{n+1} = D(x^{n+1}, u^{n+1/2}),  rho^{n+1} = rho^n + dt arho^{n+1},
 *   (a, xsph)^{n+1} = momentum(x^{n+1}, u^{n+1/2}, rho^{n+1}),
 *   u^{n+1} = u^{n+1/2} + dt/2 a^{n+1}.
 * (Kicking the density like the velocity instead makes the half-step sequence a
 * forward-Euler map of the acoustic pair (u, rho) and diverges.) Walls keep x and
 * u; their density is advanced. With summation density the RHS replaces rho.
 */
/* The midpoint predict-evaluate-correct form (Monaghan 2005), two evaluations per step.
 * R holds the rates at t^n on entry and at t^{n+1} on return:
 *   u* = u^n + dt/2 a^n,  x* = wrap(x^n + dt/2 (u^n + xsph^n)),  rho* = rho^n + dt/2 arho^n,
 *   (arho, a, xsph)* = RHS(x*, u*, rho*),
 *   u^{n+1} = u^n + dt a*,  x^{n+1} = wrap(x^n + dt (u^n + dt/2 a* + xsph*)),
 *   rho^{n+1} = rho^n + dt arho*,
 *   (arho, a, xsph)^{n+1} = RHS(x^{n+1}, u^{n+1}, rho^{n+1}).
 * x^n + dt (u^n + dt/2 a*) is the corrected midpoint velocity carried over the full
 * step. Walls keep x and u and have their density advanced like the fluid's; with
 * summation density every RHS replaces rho and the density is not integrated. */
template <class T>
void pec_step(const ora_params* P, T nu, T alpha, int64_t n, State<T>& S, const double* m,
              const uint8_t* role, Rates<T>& R, Counts& c, double dt) {
    const int dim = P->dim;
    const bool cont = P->density == DENSITY_CONTINUITY;
    State<T> S0 = S;
    for (int64_t i = 0; i < n; ++i) {
        if (role[i] == ROLE_FLUID)
            for (int d = 0; d < dim; ++d) {
                S.u[d][i] = S0.u[d][i] + 0.5 * dt * R.a[d][i];
                T xh = S0.x[d][i] + 0.5 * dt * (S0.u[d][i] + R.xs[d][i]);
                S.x[d][i] = P->periodic[d] ? wrap_t(xh, P->lo[d], P->hi[d]) : xh;
            }
        if (cont) S.rho[i] = S0.rho[i] + 0.5 * dt * R.arho[i];
    }
    rhs(P, nu, alpha, n, S, m, role, R, &c, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        if (role[i] == ROLE_FLUID)
            for (int d = 0; d < dim; ++d) {
                T ubar = S0.u[d][i] + 0.5 * dt * R.a[d][i];
                T xn = S0.x[d][i] + dt * (ubar + R.xs[d][i]);
                S.x[d][i] = P->periodic[d] ? wrap_t(xn, P->lo[d], P->hi[d]) : xn;
                S.u[d][i] = S0.u[d][i] + dt * R.a[d][i];
            }
        if (cont) S.rho[i] = S0.rho[i] + dt * R.arho[i];
    }
    rhs(P, nu, alpha, n, S, m, role, R, &c, 0.0);
}

template <class T>
double run(const ora_params* P, T nu, T alpha, int64_t n, State<T>& S, const double* m,
           const uint8_t* role, double dt_fixed, int nsteps, double* hist, Rates<T>* R_out) {
    const int dim = P->dim;
    for (int d = 0; d < dim; ++d)
        if (P->periodic[d])
            for (int64_t i = 0; i < n; ++i) S.x[d][i] = wrap_t(S.x[d][i], P->lo[d], P->hi[d]);
    Rates<T> R;
    Counts c;
    rhs(P, nu, alpha, n, S, m, role, R, &c, 0.0);
    double t = 0.0;
    std::vector<double> rec(HIST);
    diagnostics(P, n, S, R, m, role, t, 0.0, c, rec.data());
    if (hist) std::memcpy(hist, rec.data(), sizeof(double) * HIST);
    for (int step = 0; step < nsteps; ++step) {
        double dt = dt_fixed > 0.0 ? dt_fixed : cfl_dt(P, rec[3], rec[7]);
        if (P->integrator == INTEGRATOR_PEC) {
            pec_step(P, nu, alpha, n, S, m, role, R, c, dt);
            t += dt;
            diagnostics(P, n, S, R, m, role, t, dt, c, rec.data());
            if (hist) std::memcpy(hist + (size_t)(step + 1) * HIST, rec.data(), sizeof(double) * HIST);
            continue;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (role[i] == ROLE_FLUID) {
                for (int d = 0; d < dim; ++d) {
                    S.u[d][i] = S.u[d][i] + 0.5 * dt * R.a[d][i];
                    T xn = S.x[d][i] + dt * (S.u[d][i] + R.xs[d][i]);
                    S.x[d][i] = P->periodic[d] ? wrap_t(xn, P->lo[d], P->hi[d]) : xn;
                }
            }
        }
        rhs(P, nu, alpha, n, S, m, role, R, &c, dt);
        for (int64_t i = 0; i < n; ++i)
            if (role[i] == ROLE_FLUID)
                for (int d = 0; d < dim; ++d) S.u[d][i] = S.u[d][i] + 0.5 * dt * R.a[d][i];
        t += dt;
        diagnostics(P, n, S, R, m, role, t, dt, c, rec.data());
        if (hist) std::memcpy(hist + (size_t)(step + 1) * HIST, rec.data(), sizeof(double) * HIST);
    }
    if (R_out) *R_out = R;
    return t;
}

template <class T>
void load_state(const ora_params* P, int64_t n, const double* const* x, const double* const* u,
                const double* rho, State<T>& S, const double* p = nullptr) {
    for (int d = 0; d < 3; ++d) {
        S.x[d].assign(n, T(0.0));
        S.u[d].assign(n, T(0.0));
    }
    S.rho.assign(n, T(0.0));
    S.p.assign(n, T(0.0));
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < P->dim; ++d) {
            S.x[d][i] = T(x[d][i]);
            S.u[d][i] = T(u[d][i]);
        }
        S.rho[i] = T(rho[i]);
        if (p) S.p[i] = T(p[i]);
    }
}

/* The EDAC form is built for fluid-only problems with the kick-drift-kick integrator:
 * -5 for walls or the midpoint integrator with it, else 0. */
int check_edac(const ora_params* P, int64_t n, const uint8_t* role) {
    if (P->density != DENSITY_EDAC) return 0;
    if (P->integrator != 0) return -5;
    for (int64_t i = 0; i < n; ++i)
        if (role[i] != ROLE_FLUID) return -5;
    return 0;
}

}  // namespace

extern "C" {

/* Kernel value and radial derivative at distance r (pins and plots). */
int ora_kernel(int32_t kernel, int32_t dim, double h, double r, double* W, double* dWdr) {
    if ((kernel != KERNEL_QUINTIC && kernel != KERNEL_WENDLAND_C2 && kernel != KERNEL_CUBIC_SPLINE) ||
        (dim != 2 && dim != 3))
        return -1;
    kernel_eval<double>(kernel, dim, h, r, W, dWdr);
    return 0;
}

/* Cell grid of a problem: cells per axis, cell sizes, total cells. */
int ora_grid(const ora_params* P, int32_t* n_out, double* cs_out, int64_t* ncells) {
    Grid G;
    int rc = make_grid(P, &G);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d) { n_out[d] = G.n[d]; cs_out[d] = G.cs[d]; }
    *ncells = G.ncells;
    return 0;
}

/* Cell table: linear cell of every particle, offsets[c] = number of particles in cells < c
 * (ncells + 1 entries), and the particle ids in cell order (stable: ascending id in a cell). */
int ora_cells(const ora_params* P, int64_t n, const double* x, const double* y, const double* z,
              uint32_t* cell_of, uint32_t* offsets, int64_t* order) {
    const double* xs[3] = {x, y, z};
    Neighbours NB;
    Grid G;
    int rc = make_grid(P, &G);
    if (rc) return rc;
    NB.build(P, n, xs);
    for (int64_t i = 0; i < n; ++i) cell_of[i] = (uint32_t)NB.linear(&NB.cell3[i * 3]);
    if (offsets)
        for (int64_t c = 0; c <= G.ncells; ++c) offsets[c] = (uint32_t)NB.start[c];
    if (order)
        for (int64_t k = 0; k < n; ++k) order[k] = NB.members[k];
    return 0;
}

/* Neighbour lists in CSR form, ascending ids. With idx == NULL only offsets are filled.
 * Returns nnz (>= 0) or a negative error. candidates receives the pairs examined. */
int64_t ora_neighbors(const ora_params* P, int64_t n, const double* x, const double* y,
                      const double* z, int64_t* offsets, int32_t* idx, int64_t* candidates) {
    const double* xs[3] = {x, y, z};
    Grid G;
    int rc = make_grid(P, &G);
    if (rc) return rc;
    Neighbours NB;
    NB.build(P, n, xs);
    std::vector<int64_t> out;
    int64_t nnz = 0, cand = 0;
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        cand += NB.of(i, out);
        if (idx)
            for (size_t k = 0; k < out.size(); ++k) idx[nnz + (int64_t)k] = (int32_t)out[k];
        nnz += (int64_t)out.size();
        offsets[i + 1] = nnz;
    }
    if (candidates) *candidates = cand;
    return nnz;
}

/* One RHS evaluation (the SPHEvaluator use of Sec. 3.4). Outputs per particle:
 * arho (the pressure rate with EDAC), a (3 arrays), xsph (3 arrays), the density used
 * (summation or input) and p. p_in: the pressure of the EDAC form (NULL otherwise). */
int ora_rhs(const ora_params* P, int64_t n, const double* x, const double* y, const double* z,
            const double* u, const double* v, const double* w, const double* rho,
            const double* m, const uint8_t* role, double* arho, double* ax, double* ay,
            double* az, double* xsx, double* xsy, double* xsz, double* rho_out, double* p_out,
            int64_t* pairs, int64_t* candidates, const double* p_in) {
    Grid G;
    int rc = make_grid(P, &G);
    if (rc) return rc;
    if ((rc = check_edac(P, n, role))) return rc;
    const double* xs[3] = {x, y, z};
    const double* us[3] = {u, v, w};
    State<double> S;
    load_state(P, n, xs, us, rho, S, p_in);
    Rates<double> R;
    Counts c;
    rhs<double>(P, P->nu, P->alpha, n, S, m, role, R, &c, 0.0);
    double* outs_a[3] = {ax, ay, az};
    double* outs_x[3] = {xsx, xsy, xsz};
    for (int64_t i = 0; i < n; ++i) {
        arho[i] = R.arho[i];
        for (int d = 0; d < 3; ++d) {
            if (outs_a[d]) outs_a[d][i] = R.a[d][i];
            if (outs_x[d]) outs_x[d][i] = R.xs[d][i];
        }
        if (rho_out) rho_out[i] = S.rho[i];
        if (p_out) p_out[i] = R.p[i];
    }
    if (pairs) *pairs = c.pairs;
    if (candidates) *candidates = c.candidates;
    return 0;
}

/* nsteps predictor-corrector steps in place on x, y, z, u, v, w, rho (and p, the EDAC
 * pressure; NULL otherwise). hist (optional) receives (nsteps + 1) records of 10 doubles.
 * dt <= 0 selects the CFL-type time step. Returns 0 or a negative error. */
int ora_run(const ora_params* P, int64_t n, double* x, double* y, double* z, double* u,
            double* v, double* w, double* rho, const double* m, const uint8_t* role, double dt,
            int32_t nsteps, double* hist, double* p) {
    Grid G;
    int rc = make_grid(P, &G);
    if (rc) return rc;
    if ((rc = check_edac(P, n, role))) return rc;
    double* xs[3] = {x, y, z};
    double* us[3] = {u, v, w};
    const double* cx[3] = {x, y, z};
    const double* cu[3] = {u, v, w};
    State<double> S;
    load_state(P, n, cx, cu, rho, S, p);
    run<double>(P, P->nu, P->alpha, n, S, m, role, dt, nsteps, hist, nullptr);
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < P->dim; ++d) {
            xs[d][i] = S.x[d][i];
            us[d][i] = S.u[d][i];
        }
        rho[i] = S.rho[i];
        if (p) p[i] = S.p[i];
    }
    return 0;
}

/* Forward-mode derivative of the final kinetic energy KE = 1/2 sum_fluid m |u^K|^2 after
 * K steps with fixed dt, along the direction (du0 on the initial fluid velocities,
 * dnu on the laminar viscosity, dalpha on the artificial viscosity). du0 holds dim
 * arrays of n (NULL for zero). Neighbour sets of each step are those of the primal run. */
int ora_grad(const ora_params* P, int64_t n, const double* x, const double* y, const double* z,
             const double* u, const double* v, const double* w, const double* rho,
             const double* m, const uint8_t* role, double dt, int32_t K, const double* du,
             const double* dv, const double* dw, double dnu, double dalpha, double* ke,
             double* dke) {
    Grid G;
    int rc = make_grid(P, &G);
    if (rc) return rc;
    if (!(dt > 0.0)) return -3;
    if (P->integrator != 0) return -4;  // derivative of the kick-drift-kick map only
    if (P->density == DENSITY_EDAC) return -5;  // the adjoint covers the density forms
    const double* cx[3] = {x, y, z};
    const double* cu[3] = {u, v, w};
    const double* dirs[3] = {du, dv, dw};
    State<Dual> S;
    load_state(P, n, cx, cu, rho, S);
    for (int d = 0; d < P->dim; ++d)
        if (dirs[d])
            for (int64_t i = 0; i < n; ++i)
                if (role[i] == ROLE_FLUID) S.u[d][i].d = dirs[d][i];
    Dual nu(P->nu, dnu), alpha(P->alpha, dalpha);
    run<Dual>(P, nu, alpha, n, S, m, role, dt, K, nullptr, nullptr);
    Dual e(0.0);
    for (int64_t i = 0; i < n; ++i) {
        if (role[i] != ROLE_FLUID) continue;
        for (int d = 0; d < P->dim; ++d) e = e + 0.5 * m[i] * S.u[d][i] * S.u[d][i];
    }
    *ke = e.v;
    *dke = e.d;
    return 0;
}

/* ------------------------------------------------ variable smoothing length
 * Sec. 2.2: with a support radius that varies from particle to particle a uniform grid
 * needs cells of the largest radius, so the paper searches such particle sets with an
 * octree. What the search computes has a plain definition (reading C-VH): particle i
 * carries its own h_i, and j != i is a neighbour of i when
 *   |x_i - x_j|^2 < (k max(h_i, h_j))^2,
 * a symmetric relation (each pair seen from both ends), with k the kernel's support
 * factor, r^2 = ((dx dx) + dy dy) + dz dz and R = k max(h_i, h_j) formed in the precision
 * of the mode from the positions and h rounded to it; no periodic axes. The oracle
 * examines every pair (the octree only decides which pairs need examining). */
}  // extern "C"

namespace {

template <class P_>
bool vh_within(int dim, double k, const double* xi, const double* xj, double hi, double hj) {
    P_ r2 = (P_)0;
    for (int d = 0; d < dim; ++d) {
        P_ dx = (P_)xi[d] - (P_)xj[d];
        r2 = r2 + dx * dx;
    }
    const P_ hm = (P_)hi > (P_)hj ? (P_)hi : (P_)hj;
    const P_ R = (P_)k * hm;
    return r2 < R * R;
}

}  // namespace

extern "C" {

/* Neighbour lists in CSR form (ascending ids); idx == NULL: offsets only. Returns nnz or
 * a negative error. */
int64_t ora_vh_neighbors(int32_t dim, int32_t kernel, int32_t precision, int64_t n,
                         const double* x, const double* y, const double* z, const double* h,
                         int64_t* offsets, int32_t* idx) {
    if ((dim != 2 && dim != 3) || n < 0 || (kernel < 0 || kernel > 2)) return -1;
    const double k = support_factor(kernel);
    const double* xs[3] = {x, y, z};
    std::vector<double> pos((size_t)n * 3, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < dim; ++d) pos[(size_t)i * 3 + d] = xs[d][i];
    std::vector<int64_t> cnt((size_t)n, 0);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const bool in = precision == PREC_FP32
                                ? vh_within<float>(dim, k, &pos[(size_t)i * 3], &pos[(size_t)j * 3], h[i], h[j])
                                : vh_within<double>(dim, k, &pos[(size_t)i * 3], &pos[(size_t)j * 3], h[i], h[j]);
            c += in ? 1 : 0;
        }
        cnt[(size_t)i] = c;
    }
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + cnt[(size_t)i];
    if (idx) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int64_t w = offsets[i];
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                const bool in = precision == PREC_FP32
                                    ? vh_within<float>(dim, k, &pos[(size_t)i * 3], &pos[(size_t)j * 3], h[i], h[j])
                                    : vh_within<double>(dim, k, &pos[(size_t)i * 3], &pos[(size_t)j * 3], h[i], h[j]);
                if (in) idx[w++] = (int32_t)j;
            }
        }
    }
    return offsets[n];
}

/* The same relation and density for selected particles only (rows[0..nrows)): their
 * neighbour counts, their neighbours (ascending ids, CSR over the selection) and their
 * densities, every pair of a selected particle examined. For particle sets too large for
 * the all-pairs lists. */
int64_t ora_vh_rows(int32_t dim, int32_t kernel, int32_t precision, int64_t n, const double* x,
                    const double* y, const double* z, const double* h, const double* m,
                    const int64_t* rows, int64_t nrows, int64_t* offsets, int32_t* idx,
                    double* rho) {
    if ((dim != 2 && dim != 3) || n < 0 || nrows < 0 || (kernel < 0 || kernel > 2)) return -1;
    const double k = support_factor(kernel);
    const double* xs[3] = {x, y, z};
    std::vector<std::vector<int32_t>> lists((size_t)nrows);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        double xi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) xi[d] = xs[d][i];
        double W, dW;
        kernel_eval<double>(kernel, dim, h[i], 0.0, &W, &dW);
        double s = m[i] * W;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double xj[3] = {0, 0, 0};
            for (int d = 0; d < dim; ++d) xj[d] = xs[d][j];
            const bool in = precision == PREC_FP32 ? vh_within<float>(dim, k, xi, xj, h[i], h[j])
                                                   : vh_within<double>(dim, k, xi, xj, h[i], h[j]);
            if (!in) continue;
            lists[(size_t)r].push_back((int32_t)j);
            double r2 = 0.0;
            for (int d = 0; d < dim; ++d) {
                const double dx = xi[d] - xj[d];
                r2 = r2 + dx * dx;
            }
            kernel_eval<double>(kernel, dim, 0.5 * (h[i] + h[j]), std::sqrt(r2), &W, &dW);
            s += m[j] * W;
        }
        if (rho) rho[r] = s;
    }
    offsets[0] = 0;
    for (int64_t r = 0; r < nrows; ++r) offsets[r + 1] = offsets[r] + (int64_t)lists[(size_t)r].size();
    if (idx)
        for (int64_t r = 0; r < nrows; ++r)
            std::copy(lists[(size_t)r].begin(), lists[(size_t)r].end(), idx + offsets[r]);
    return offsets[nrows];
}

/* Summation density with variable smoothing length (Eq. 2 with the pair smoothing length
 * h_ij = (h_i + h_j) / 2, the symmetrised kernel of variable-h SPH, reading C-VH):
 *   rho_i = m_i W(0, h_i) + sum_{j in N(i)} m_j W(|x_i - x_j|, h_ij)
 * over the neighbour set of the mode, in FP64 (k h_ij <= k max(h_i, h_j), so every pair
 * the kernel reaches is in the set). */
int ora_vh_density(int32_t dim, int32_t kernel, int32_t precision, int64_t n, const double* x,
                   const double* y, const double* z, const double* h, const double* m,
                   double* rho) {
    if ((dim != 2 && dim != 3) || n < 0 || (kernel < 0 || kernel > 2)) return -1;
    const double k = support_factor(kernel);
    const double* xs[3] = {x, y, z};
    std::vector<double> pos((size_t)n * 3, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < dim; ++d) pos[(size_t)i * 3 + d] = xs[d][i];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double W, dW;
        kernel_eval<double>(kernel, dim, h[i], 0.0, &W, &dW);
        double s = m[i] * W;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const bool in = precision == PREC_FP32
                                ? vh_within<float>(dim, k, &pos[(size_t)i * 3], &pos[(size_t)j * 3], h[i], h[j])
                                : vh_within<double>(dim, k, &pos[(size_t)i * 3], &pos[(size_t)j * 3], h[i], h[j]);
            if (!in) continue;
            double r2 = 0.0;
            for (int d = 0; d < dim; ++d) {
                const double dx = pos[(size_t)i * 3 + d] - pos[(size_t)j * 3 + d];
                r2 = r2 + dx * dx;
            }
            kernel_eval<double>(kernel, dim, 0.5 * (h[i] + h[j]), std::sqrt(r2), &W, &dW);
            s += m[j] * W;
        }
        rho[i] = s;
    }
    return 0;
}

/* Threads the oracle's parallel loops use (1 without OpenMP). */
int ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
