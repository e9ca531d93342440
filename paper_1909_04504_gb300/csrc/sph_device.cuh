// Device-side definitions shared by the CUDA translation units of the WCSPH library:
// the particle-set layout in HBM, the launch argument blocks, the neighbour predicate,
// the smoothing kernels and the compensated accumulator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

constexpr int QUINTIC = 0;
constexpr int WENDLAND_C2 = 1;
constexpr int CUBIC_SPLINE = 2;
constexpr uint32_t WALL_BIT = 0x80000000u;  // tag = global id | WALL_BIT for wall particles
constexpr uint32_t ID_MASK = 0x7fffffffu;

// Status bits raised on the device (host maps them to sph_status).
constexpr unsigned ST_NONFINITE = 1u;
constexpr unsigned ST_TIMEOUT = 2u;
constexpr unsigned ST_CAPACITY = 4u;

// Equation switches of one right-hand-side evaluation.
constexpr int F_CONTINUITY = 1;   // Eq. continuity:sph (else summation density, Eq. 2)
constexpr int F_LAMINAR = 2;      // Eq. mom:sph:visc
constexpr int F_AV = 4;           // Monaghan artificial viscosity
constexpr int F_XSPH = 8;         // XSPH correction
constexpr int F_WALLP = 16;       // solid-wall pressure of Adami et al. (Sec. 2.3 wall condition)
constexpr int F_EDAC = 32;        // EDAC pressure equation (Sec. 2.3 scheme list, Sec. 4.1)

constexpr int DIAG_N = 13;
constexpr int HIST_CAP = 65536;

// 16- and 32-byte vectors: one vector load per particle record.
struct __align__(16) F4 { float x, y, z, w; };
struct __align__(32) D4 { double x, y, z, w; };
template <class Real> struct V4;
template <> struct V4<float> { using T = F4; };
template <> struct V4<double> { using T = D4; };

// One copy of the FP64 particle state, struct of arrays, in the device's internal
// (cell-sorted) order. Two copies exist; a rebuild gathers one into the other.
struct ParticleSet {
    double* x[3];
    double* u[3];
    double* rho;
    double* m;
    double* arho;   // rates of the last evaluation
    double* a[3];
    double* xs[3];  // XSPH velocity correction
    double* p;      // EDAC: the pressure (a state variable there; else unused)
    uint32_t* tag;  // global id | WALL_BIT
};

// Device control block: time, step size, diagnostics, status.
struct Control {
    double dt;            // step used by the next drift / kick
    double t;
    double rec[DIAG_N];   // diagnostics record of the last evaluation
    unsigned long long step;
    unsigned int status;
    unsigned int ticket;  // last-block counter of the reduction
    unsigned int outside; // particles clamped into an edge cell at the last key build
    unsigned int hist_count;
    unsigned long long stamp[8];  // persistent step: global timer (ns) at each phase end
    // grid barrier of the persistent step: arrivals and generation, each on its own
    // 128-byte line so that the pollers of one do not contend with the atomics on the other
    alignas(128) unsigned int bar_count;
    alignas(128) unsigned int bar_gen;
    // momentum pass, one lane per destination: the next chunk of 32 destinations a warp
    // takes, and the blocks done (the last block resets both for the next launch)
    alignas(128) unsigned int mom_next;
    unsigned int mom_done;
    // density pass, one lane per destination: the same for its chunks
    alignas(128) unsigned int dens_next;
    unsigned int dens_done;
};

// Grid of cells (Sec. 2.2): cells no smaller than the support radius.
struct Grid {
    int dim;
    int nc[3];
    int periodic[3];
    int ncells;
    int run_shift;  // every periodic axis has >= 5 cells: the minimum image is a per-run shift
    float lo_f[3], inv_cs_f[3];  // lo and 1 / cs rounded to FP32 (screened cell coordinate)
    double lo[3], cs[3], L[3], hi[3];
};

// Constants of the pair loops in the precision of the mode.
template <class Real>
struct PairConst {
    Real L[3], halfL[3];
    Real kh2;       // (k h)^2, computed as (k * h) * (k * h) in Real
    Real inv_h;
    Real h;
    Real wfac;      // sigma / h^d
    Real gfac;      // sigma / h^(d+2)
    Real eta_h2;    // eta h^2
    Real av_h2;     // 0.01 h^2
    Real nu4;       // 4 nu
    Real alpha_c0;  // alpha c0
    Real c0;
    Real xsph;
    Real inv_rho0;  // EDAC: 1 / rho0 (the density is held at rho0)
    Real edac_d;    // EDAC: 2 nu_e / rho0, nu_e = h c0 / 16
    Real c02;       // EDAC: c0^2
    int flags;
};

// Constants of the FP64 per-particle stages.
struct StepConst {
    double rho0, inv_rho0, B, gamma;  // Tait: p = B ((rho/rho0)^gamma - 1)
    double g[3];
    double h, c0, nu;
    double dt_fixed;                  // > 0 fixed step, else CFL-type step
    int continuity;
    int gamma7;                       // gamma == 7: power by multiplications
    int precision;                    // 1: positions rounded to float for binning
};

// --------------------------------------------------------------- rounding helpers
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

// Separation of the neighbour test: difference with the minimum image on periodic
// axes. Every operation is rounded on its own (no fused multiply-add), so the result
// is the same IEEE value on any machine.
template <class Real>
__device__ __forceinline__ Real min_image(Real d, int periodic, Real L, Real halfL) {
    const Real up = rn_sub(d, L), dn = rn_add(d, L);  // selected, not branched on
    Real r = (periodic && d > halfL) ? up : d;
    r = (periodic && d < -halfL) ? dn : r;
    return r;
}

// r^2 = ((dx dx) + dy dy) + dz dz, each operation rounded separately.
template <class Real, int DIM>
__device__ __forceinline__ Real dist2(Real dx, Real dy, Real dz) {
    Real r2 = rn_add(rn_mul(dx, dx), rn_mul(dy, dy));
    if (DIM == 3) r2 = rn_add(r2, rn_mul(dz, dz));
    return r2;
}

// Cell coordinate of a position on one axis: floor((x_mode - lo) / cs) in FP64, clamped.
__device__ __forceinline__ int cell_coord(double xm, double lo, double cs, int n, int* clamped) {
    double v = __ddiv_rn(__dsub_rn(xm, lo), cs);
    double c = floor(v);
    if (!(c >= 0.0)) { *clamped = 1; return 0; }
    if (c > (double)(n - 1)) { *clamped = 1; return n - 1; }
    return (int)c;
}

// The same cell coordinate, screened in FP32: q = (x_f - lo_f) * inv_cs_f differs from the
// FP64 quotient by at most 8 u ((|x_f| + |lo_f|) inv_cs_f + |q| + 1), u = 2^-24 (each of the
// five FP32 roundings contributes at most u times its operand). When no integer lies
// within that bound of q, floor(q) is the FP64 result; otherwise (about one coordinate in
// a few thousand) the FP64 quotient decides. The FP64 pipe of this part runs at 1/64 of
// FP32 and its divide costs many instructions, so the screen keeps it off the common path.
// x is the FP64 position and xf = x rounded to float; the binned position is xf widened
// (to_float: FP32 pair loops) or x itself, formed only on the rare FP64 path.
__device__ __forceinline__ int cell_coord_screened(double x, float xf, int to_float, double lo,
                                                   double cs, float lo_f, float inv_cs_f, int n,
                                                   int* clamped) {
    const float q = (xf - lo_f) * inv_cs_f;
    const float m = 4.7683716e-7f * ((fabsf(xf) + fabsf(lo_f)) * inv_cs_f + fabsf(q) + 1.0f);
    const float lo_q = floorf(q - m), hi_q = floorf(q + m);
    if (!(lo_q == hi_q))  // near a cell edge, NaN
        return cell_coord(to_float ? (double)xf : x, lo, cs, n, clamped);
    if (!(lo_q >= 0.0f)) { *clamped = 1; return 0; }
    if (lo_q > (float)(n - 1)) { *clamped = 1; return n - 1; }
    return (int)lo_q;
}

// Fused multiply-add with one rounding, written out where an expression adds two
// products: left to the compiler, which product is fused could differ between two
// instantiations of the same arithmetic (the single-problem and the batch kernels), and
// their results would then differ in the last bit.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// a . b in DIM dimensions as a chain of fused multiply-adds.
template <class Real, int DIM>
__device__ __forceinline__ Real dot_rn(Real ax, Real ay, Real az, Real bx, Real by, Real bz) {
    return DIM == 3 ? fma_rn(ax, bx, fma_rn(ay, by, az * bz)) : fma_rn(ax, bx, ay * by);
}

// Square root, reciprocal and quotient of the pair arithmetic: in FP32 the hardware
// approximations (relative error of a few 2^-23, far inside the FP32 mode's tolerance and
// with no slow path), in FP64 the correctly rounded operations.
template <class Real>
struct PairMath;

template <>
struct PairMath<float> {
    static __device__ __forceinline__ float sqrt(float x) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float rcp(float x) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
};

template <>
struct PairMath<double> {
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
};

// ------------------------------------------------------------------- kernels
// Unnormalised smoothing function w(q) and f(q) = w'(q) / q, so that
// W = wfac w(q) and grad_i W = gfac f(q) (x_i - x_j) with no division by r.
//  quintic (support 3): w = (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5 with terms where positive;
//    f = -50 q^3 + 120 q^2 - 120 on [0,1), (-5 (3-q)^4 + 30 (2-q)^4) / q on [1,2),
//    -5 (3-q)^4 / q on [2,3).
//  Wendland C2 (support 2): w = (1 - q/2)^4 (2q + 1), f = -5 (1 - q/2)^3.
//  cubic spline (support 2, four times the M4 B-spline): w = (2-q)^3 - 4 (1-q)^3 with
//    terms where positive; f = 9 q - 12 on [0,1), -3 (2-q)^2 / q on [1,2).
template <class Real, int KERNEL>
__device__ __forceinline__ Real kernel_f(Real q) {
    if (KERNEL == QUINTIC) {
        if (sizeof(Real) == 8) {  // FP64: the divide is costly, keep it off the inner branch
            if (q < Real(1)) return fma_rn(fma_rn(Real(-50), q, Real(120)) * q, q, Real(-120));
            Real t3 = Real(3) - q;
            Real t3s = t3 * t3;
            Real p = Real(-5) * t3s * t3s;
            Real t2 = q < Real(2) ? Real(2) - q : Real(0);
            Real t2s = t2 * t2;
            p = fma_rn(Real(30) * t2s, t2s, p);
            return PairMath<Real>::div(p, q);
        }
        // FP32: both branches evaluated and one selected (neighbours of a warp spread over q)
        const Real inner = fma_rn(fma_rn(Real(-50), q, Real(120)) * q, q, Real(-120));
        Real t3 = Real(3) - q;
        Real t3s = t3 * t3;
        Real p = Real(-5) * t3s * t3s;
        Real t2 = q < Real(2) ? Real(2) - q : Real(0);
        Real t2s = t2 * t2;
        p = fma_rn(Real(30) * t2s, t2s, p);
        const Real outer = PairMath<Real>::div(p, q);
        return q < Real(1) ? inner : outer;
    } else if (KERNEL == CUBIC_SPLINE) {
        const Real inner = fma_rn(Real(9), q, Real(-12));
        if (sizeof(Real) == 8 && q < Real(1)) return inner;
        const Real t2 = q < Real(2) ? Real(2) - q : Real(0);
        const Real outer = PairMath<Real>::div(Real(-3) * t2 * t2, q);
        return q < Real(1) ? inner : outer;
    } else {
        Real t = fma_rn(Real(-0.5), q, Real(1));
        return Real(-5) * t * t * t;
    }
}

template <class Real, int KERNEL>
__device__ __forceinline__ Real kernel_w(Real q) {
    if (KERNEL == QUINTIC) {
        // the terms (2 - q)^5 and (1 - q)^5 vanish outside their intervals: clamped, not
        // branched on
        Real t3 = Real(3) - q;
        Real t3s = t3 * t3;
        Real w = t3s * t3s * t3;
        Real t2 = q < Real(2) ? Real(2) - q : Real(0);
        Real t2s = t2 * t2;
        w = fma_rn(-(Real(6) * t2s * t2s), t2, w);
        Real t1 = q < Real(1) ? Real(1) - q : Real(0);
        Real t1s = t1 * t1;
        w = fma_rn(Real(15) * t1s * t1s, t1, w);
        return w;
    } else if (KERNEL == CUBIC_SPLINE) {
        const Real t2 = q < Real(2) ? Real(2) - q : Real(0);
        const Real t1 = q < Real(1) ? Real(1) - q : Real(0);
        return fma_rn(Real(-4), t1 * t1 * t1, t2 * t2 * t2);
    } else {
        Real t = fma_rn(Real(-0.5), q, Real(1));
        Real t2 = t * t;
        return t2 * t2 * fma_rn(Real(2), q, Real(1));
    }
}

// Tait EOS (Eq. eos) in FP64: p = B ((rho/rho0)^gamma - 1), evaluated through
// delta = (rho - rho0) / rho0 without the cancellation of the difference near rho0:
// for gamma = 7 the exact binomial polynomial delta (7 + 21 delta + 35 delta^2 + ...),
// otherwise expm1(gamma log1p(delta)).
__device__ __forceinline__ double tait_pressure(double rho, const StepConst& C) {
    const double d = (rho - C.rho0) * C.inv_rho0;
    double e;
    if (C.gamma7) {
        e = d * fma_rn(d, fma_rn(d, fma_rn(d, fma_rn(d, fma_rn(d, 7.0 + d, 21.0), 35.0), 35.0), 21.0), 7.0);
    } else {
        e = expm1(C.gamma * log1p(d));
    }
    return C.B * e;
}

// The pair-loop shadow p / rho^2 in the pair-loop precision: FP64 mode from the FP64 EOS;
// FP32 mode with delta formed in FP64 (no cancellation) and the polynomial (or
// expm1(gamma log1p(delta))) and the quotient in FP32, the precision the pair loop reads.
template <class Real>
__device__ __forceinline__ Real pressure_over_rho2(double rho, const StepConst& C);

template <>
__device__ __forceinline__ double pressure_over_rho2<double>(double rho, const StepConst& C) {
    return tait_pressure(rho, C) / (rho * rho);
}

template <>
__device__ __forceinline__ float pressure_over_rho2<float>(double rho, const StepConst& C) {
    const float d = (float)((rho - C.rho0) * C.inv_rho0);
    float e;
    if (C.gamma7) {
        e = d * fma_rn(d, fma_rn(d, fma_rn(d, fma_rn(d, fma_rn(d, 7.f + d, 21.f), 35.f), 35.f), 21.f), 7.f);
    } else {
        e = expm1f((float)C.gamma * log1pf(d));
    }
    const float r = (float)rho;
    return (float)C.B * e / (r * r);
}

// --------------------------------------------------------- compensated sums
// Neumaier's improved Kahan-Babuska summation for FP32 per-particle sums; a plain sum
// in FP64 mode. The value is read out in FP64 as s + c.
template <class Real>
struct Acc {
    Real s, c;
    __device__ __forceinline__ void zero() { s = Real(0); c = Real(0); }
    __device__ __forceinline__ void add(Real v) {
        if (sizeof(Real) == 4) {
            // each operation rounded on its own (no product of the caller fused into them)
            const Real t = rn_add(s, v);
            const Real e = (fabs(s) >= fabs(v)) ? rn_add(rn_sub(s, t), v) : rn_add(rn_sub(v, t), s);
            c = rn_add(c, e);
            s = t;
        } else {
            s += v;
        }
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace sph
