// wb_sweep.cuh -- characteristic WENO5 flux sweeps (Donnert et al. 2018,
// Sec. 2.1 eq. FWENO; Sec. 2.2 dimension-by-dimension sweeps).  Included by
// wb_sweep_f32.cu (compiled with fast single-precision division and square
// root) and wb_sweep_f64.cu, which instantiate it for float and double.
//
// One thread computes the numerical flux through one interface.  A block
// owns a 2-D slab of interfaces: TA along the sweep axis times TP pencils.
// The TA+5 cells each pencil needs (3 below, 2 above the slab) are staged
// once in shared memory with everything the interface step reads per cell:
// the rotated conserved 7-vector, its physical flux, the seven |lambda| and
// the primitives used by the interface average.  The sweep never moves the
// grid ("rotation" of Sec. 2.2 is an index mapping): for the x sweep the
// thread's x index walks the axis, for y and z the thread's x index walks
// the pencils, so every global load and store is x-contiguous.
//
// Per interface (cells i-2..i+3 of the stencil):
//   1. interface state = mean of the primitives of cells i, i+1;
//   2. closed-form 7-wave eigensystem (Roe-Balsara normalisation) at it;
//   3. projection of U_k, F_k on the left eigenvectors, done as
//      (dW/dU) x followed by the sparse left vectors, in two groups of
//      characteristic fields (fast+slow, then Alfven+entropy) so that the
//      projected stencil fits in registers in FP64 too;
//   4. local Lax-Friedrichs splitting, alpha_s = max |lambda_s| over the
//      stencil and the interface state;
//   5. WENO5-JS weights and phi_N for both split fluxes;
//   6. back-projection (dU/dW applied to the primitive right vectors) plus
//      the fourth-order central flux (-F_{i-1} + 7F_i + 7F_{i+1} - F_{i+2})/12.
// The flux is written in global component order (rho, mx, my, mz, E,
// B_t1, B_t2) to the face array of the lower face of cell i+1.
#pragma once
#include "../../include/wombat_gb300.h"
#include "wb_internal.h"

// Characteristic fields are projected two groups at a time (fast+slow,
// then Alfven+entropy) by default; 4 processes one field pair at a time.
#ifndef WB_SWEEP_PARK
#define WB_SWEEP_PARK 1                // 1: project each stencil vector once, park the second group
#endif
#ifndef WB_SWEEP_GROUPS
#define WB_SWEEP_GROUPS 2
#endif

namespace wb {
namespace {

// ---- shared-memory slots per staged cell ----------------------------------
enum : int {
    SU = 0,      // U7: rho, m_n, m_t1, m_t2, B_t1, B_t2, E        (0..6)
    SF = 7,      // F7 in the same order                           (7..13)
    SL = 14,     // |lambda_s|, s = 0..6                           (14..20)
    SP_U = 21, SP_V1, SP_V2, SP_BN, SP_P,   // primitives for the mean
    kNSlot = 26
};

template <class T> __device__ __forceinline__ T sq_root(T x);
template <> __device__ __forceinline__ float sq_root<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double sq_root<double>(double x) { return sqrt(x); }

template <class T> __device__ __forceinline__ T rsq_root(T x);
template <> __device__ __forceinline__ float rsq_root<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq_root<double>(double x) { return rsqrt(x); }

template <class T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
// |a| by clearing the sign bit (no floating-point compare on the FP64 pipe)
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
// max of two values >= 0: for non-negative IEEE values the bit patterns
// order like the values, so FP64 takes an integer max, off the FP64 pipe
__device__ __forceinline__ float tmax_nonneg(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax_nonneg(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}

__device__ __forceinline__ int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Sec. 2.1: phi_N(a,b,c,d) = 1/3 w0 (a-2b+c) + 1/6 (w2-1/2)(b-2c+d) with
// IS_0..2 as printed, alpha_k = d_k/(eps+IS_k)^2, d = (1, 6, 3), eps = 1e-6.
// The weights depend only on the ratios of the eps + IS_k, so each is formed
// divided by three, (13/3) t^2 + t'^2 + eps/3: one multiply and two fused
// multiply-adds, the eps folded in.
// eps3 = eps / 3; phi_N(s a, s b, s c, s d) with s^2 eps3 is s phi_N(a, b, c, d).
constexpr double kEps3 = 1e-6 / 3.0;
__device__ __forceinline__ double phi_n(double a, double b, double c, double d, double eps3 = kEps3) {
    const double k13 = 13.0 / 3.0;
    const double t0 = a - b, t1 = a - 3.0 * b;
    const double t2 = b - c, t3 = b + c;
    const double t4 = c - d, t5 = 3.0 * c - d;
    double e0 = fma(k13 * t0, t0, fma(t1, t1, eps3));
    double e1 = fma(k13 * t2, t2, fma(t3, t3, eps3));
    double e2 = fma(k13 * t4, t4, fma(t5, t5, eps3));
    e0 *= e0; e1 *= e1; e2 *= e2;
    // omega_k = (d_k / e_k) / sum_j (d_j / e_j): one division in FP64
    double n0 = e1 * e2, n2 = 3.0 * e0 * e1;
    double r = 1.0 / (n0 + 6.0 * e0 * e2 + n2);
    double w0 = n0 * r, w2 = n2 * r;
    return w0 * (a - 2.0 * b + c) * (1.0 / 3.0) + (w2 - 0.5) * (b - 2.0 * c + d) * (1.0 / 6.0);
}

constexpr float kEps3f = 1e-6f / 3.0f;
// phi_N(am, bm, cm, dm) - phi_N(ap, bp, cp, dp) in FP64 with one division
// for both: each side's weights are n_k / den, and the two denominators
// share the reciprocal of their product (falling back to one division each
// where that product would leave the FP64 range).
__device__ __forceinline__ void phi_n_parts(double a, double b, double c, double d, double eps3, double& n0,
                                            double& n2, double& den) {
    const double k13 = 13.0 / 3.0;
    const double t0 = a - b, t1 = a - 3.0 * b;
    const double t2 = b - c, t3 = b + c;
    const double t4 = c - d, t5 = 3.0 * c - d;
    double e0 = fma(k13 * t0, t0, fma(t1, t1, eps3));
    double e1 = fma(k13 * t2, t2, fma(t3, t3, eps3));
    double e2 = fma(k13 * t4, t4, fma(t5, t5, eps3));
    e0 *= e0; e1 *= e1; e2 *= e2;
    n0 = e1 * e2;
    n2 = 3.0 * e0 * e1;
    den = n0 + 6.0 * e0 * e2 + n2;
}
__device__ __forceinline__ double phi_n_diff(double am, double bm, double cm, double dm, double ap, double bp,
                                             double cp, double dp, double eps3) {
    double n0m, n2m, denm, n0p, n2p, denp;
    phi_n_parts(am, bm, cm, dm, eps3, n0m, n2m, denm);
    phi_n_parts(ap, bp, cp, dp, eps3, n0p, n2p, denp);
    const double prod = denm * denp;
    double rm, rp;
    if (prod < 1e300) {
        const double R = 1.0 / prod;
        rm = denp * R;
        rp = denm * R;
    } else {
        rm = 1.0 / denm;
        rp = 1.0 / denp;
    }
    const double phm = n0m * rm * (am - 2.0 * bm + cm) * (1.0 / 3.0) + (n2m * rm - 0.5) * (bm - 2.0 * cm + dm) * (1.0 / 6.0);
    const double php = n0p * rp * (ap - 2.0 * bp + cp) * (1.0 / 3.0) + (n2p * rp - 0.5) * (bp - 2.0 * cp + dp) * (1.0 / 6.0);
    return phm - php;
}

__device__ __forceinline__ float phi_n(float a, float b, float c, float d, float eps3 = kEps3f) {
    const float k13 = 13.0f / 3.0f;
    const float t0 = a - b, t1 = a - 3.0f * b;
    const float t2 = b - c, t3 = b + c;
    const float t4 = c - d, t5 = 3.0f * c - d;
    const float e0 = fmaf(k13 * t0, t0, fmaf(t1, t1, eps3));
    const float e1 = fmaf(k13 * t2, t2, fmaf(t3, t3, eps3));
    const float e2 = fmaf(k13 * t4, t4, fmaf(t5, t5, eps3));
    // reciprocals keep the FP32 range: (eps+IS)^2 products could overflow
    float a0 = 1.0f / (e0 * e0), a1 = 6.0f / (e1 * e1), a2 = 3.0f / (e2 * e2);
    float r = 1.0f / (a0 + a1 + a2);
    float w0 = a0 * r, w2 = a2 * r;
    return w0 * (a - 2.0f * b + c) * (1.0f / 3.0f) + (w2 - 0.5f) * (b - 2.0f * c + d) * (1.0f / 6.0f);
}

// phi_N of the minus side (lane x) and the plus side (lane y) of one field
// at once, in packed FP32 pairs (one instruction for both lanes); each lane
// computes what phi_n(float) does, with the products and sums spelled as
// fused multiply-adds.
#ifndef WB_SWEEP_PACKED
#define WB_SWEEP_PACKED 1
#endif
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 phi_n2(float2 a, float2 b, float2 c, float2 d, float eps3f = kEps3f) {
    // (eps + IS_k) / 3 as in phi_n
    const float2 k13 = splat2(13.0f / 3.0f), eps3 = splat2(eps3f);
    const float2 t0 = __ffma2_rn(b, splat2(-1.0f), a), t1 = __ffma2_rn(b, splat2(-3.0f), a);
    const float2 t2 = __ffma2_rn(c, splat2(-1.0f), b), t3 = __fadd2_rn(b, c);
    // t5 enters squared: d - 3c serves for 3c - d
    const float2 t4 = __ffma2_rn(d, splat2(-1.0f), c), t5 = __ffma2_rn(c, splat2(-3.0f), d);
    float2 e0 = __ffma2_rn(__fmul2_rn(t0, k13), t0, __ffma2_rn(t1, t1, eps3));
    float2 e1 = __ffma2_rn(__fmul2_rn(t2, k13), t2, __ffma2_rn(t3, t3, eps3));
    float2 e2 = __ffma2_rn(__fmul2_rn(t4, k13), t4, __ffma2_rn(t5, t5, eps3));
    e0 = __fmul2_rn(e0, e0);
    e1 = __fmul2_rn(e1, e1);
    e2 = __fmul2_rn(e2, e2);
    const float2 a0 = make_float2(1.0f / e0.x, 1.0f / e0.y);
    const float2 a1 = __fmul2_rn(make_float2(1.0f / e1.x, 1.0f / e1.y), splat2(6.0f));
    const float2 a2 = __fmul2_rn(make_float2(1.0f / e2.x, 1.0f / e2.y), splat2(3.0f));
    const float2 sum = __fadd2_rn(__fadd2_rn(a0, a1), a2);
    const float2 r = make_float2(1.0f / sum.x, 1.0f / sum.y);
    const float2 w0 = __fmul2_rn(a0, r);
    const float2 h2 = __ffma2_rn(a2, r, splat2(-0.5f));
    const float2 p = __ffma2_rn(b, splat2(-2.0f), __fadd2_rn(a, c));
    const float2 q = __ffma2_rn(c, splat2(-2.0f), __fadd2_rn(b, d));
    return __ffma2_rn(__fmul2_rn(w0, splat2(1.0f / 3.0f)), p, __fmul2_rn(__fmul2_rn(h2, splat2(1.0f / 6.0f)), q));
}

// WENO-Z interpolant (the alternative Sec. 2.1 names): same IS_k, weights
// alpha_k = d_k (1 + tau5 / (eps + IS_k)), tau5 = |IS_0 - IS_2|.
template <class T>
__device__ __forceinline__ T phi_n_z(T a, T b, T c, T d) {
    const T eps = T(1e-6);
    const T t0 = a - b, t1 = a - T(3) * b;
    const T is0 = T(13) * t0 * t0 + T(3) * t1 * t1;
    const T t2 = b - c, t3 = b + c;
    const T is1 = T(13) * t2 * t2 + T(3) * t3 * t3;
    const T t4 = c - d, t5 = T(3) * c - d;
    const T is2 = T(13) * t4 * t4 + T(3) * t5 * t5;
    const T tau = is0 > is2 ? is0 - is2 : is2 - is0;
    const T a0 = T(1) + tau / (eps + is0);
    const T a1 = T(6) * (T(1) + tau / (eps + is1));
    const T a2 = T(3) * (T(1) + tau / (eps + is2));
    const T r = T(1) / (a0 + a1 + a2);
    return a0 * r * (a - T(2) * b + c) * T(1.0 / 3.0) + (a2 * r - T(0.5)) * (b - T(2) * c + d) * T(1.0 / 6.0);
}

// phi_n_z on the (minus, plus) pair of one field, as phi_n2 does for
// phi_n; tau5 and the three weights per lane as in phi_n_z.
__device__ __forceinline__ float2 phi_n_z2(float2 a, float2 b, float2 c, float2 d) {
    const float2 t0 = __ffma2_rn(b, splat2(-1.0f), a), t1 = __ffma2_rn(b, splat2(-3.0f), a);
    const float2 is0 = __ffma2_rn(__fmul2_rn(t0, splat2(13.0f)), t0, __fmul2_rn(__fmul2_rn(t1, splat2(3.0f)), t1));
    const float2 t2 = __ffma2_rn(c, splat2(-1.0f), b), t3 = __fadd2_rn(b, c);
    const float2 is1 = __ffma2_rn(__fmul2_rn(t2, splat2(13.0f)), t2, __fmul2_rn(__fmul2_rn(t3, splat2(3.0f)), t3));
    const float2 t4 = __ffma2_rn(d, splat2(-1.0f), c), t5 = __ffma2_rn(c, splat2(3.0f), __fmul2_rn(d, splat2(-1.0f)));
    const float2 is2 = __ffma2_rn(__fmul2_rn(t4, splat2(13.0f)), t4, __fmul2_rn(__fmul2_rn(t5, splat2(3.0f)), t5));
    const float2 dt = __ffma2_rn(is2, splat2(-1.0f), is0);
    const float2 tau = make_float2(fabsf(dt.x), fabsf(dt.y));
    const float2 e0 = __fadd2_rn(is0, splat2(1e-6f)), e1 = __fadd2_rn(is1, splat2(1e-6f)),
                 e2 = __fadd2_rn(is2, splat2(1e-6f));
    const float2 a0 = __ffma2_rn(tau, make_float2(1.0f / e0.x, 1.0f / e0.y), splat2(1.0f));
    const float2 a1 = __fmul2_rn(__ffma2_rn(tau, make_float2(1.0f / e1.x, 1.0f / e1.y), splat2(1.0f)), splat2(6.0f));
    const float2 a2 = __fmul2_rn(__ffma2_rn(tau, make_float2(1.0f / e2.x, 1.0f / e2.y), splat2(1.0f)), splat2(3.0f));
    const float2 sum = __fadd2_rn(__fadd2_rn(a0, a1), a2);
    const float2 r = make_float2(1.0f / sum.x, 1.0f / sum.y);
    const float2 w0 = __fmul2_rn(a0, r);
    const float2 h2 = __ffma2_rn(a2, r, splat2(-0.5f));
    const float2 p = __ffma2_rn(b, splat2(-2.0f), __fadd2_rn(a, c));
    const float2 q = __ffma2_rn(c, splat2(-2.0f), __fadd2_rn(b, d));
    return __ffma2_rn(__fmul2_rn(w0, splat2(1.0f / 3.0f)), p, __fmul2_rn(__fmul2_rn(h2, splat2(1.0f / 6.0f)), q));
}

// Correction of eq. FWENO for one characteristic field:
// -phi_N(D+_{i-3/2}, D+_{i-1/2}, D+_{i+1/2}, D+_{i+3/2})
// +phi_N(D-_{i+5/2}, D-_{i+3/2}, D-_{i+1/2}, D-_{i-1/2}),
// D+-_{k+1/2} = g+-_{k+1} - g+-_k, g+- = (g +- alpha w)/2.
template <class T, bool Z = false>
__device__ __forceinline__ T weno_corr(const T (&w)[6], const T (&g)[6], T alpha) {
    const T ha = T(0.5) * alpha;
    T gp[5], gm[5];
#pragma unroll
    for (int k = 0; k < 5; k++) gp[k] = T(0.5) * g[k] + ha * w[k];
#pragma unroll
    for (int k = 0; k < 5; k++) gm[k] = T(0.5) * g[k + 1] - ha * w[k + 1];
    // gm[k] holds g-_{k+1}
    T dp0 = gp[1] - gp[0], dp1 = gp[2] - gp[1], dp2 = gp[3] - gp[2], dp3 = gp[4] - gp[3];
    T dm1 = gm[1] - gm[0], dm2 = gm[2] - gm[1], dm3 = gm[3] - gm[2], dm4 = gm[4] - gm[3];
    if constexpr (Z && WB_SWEEP_PACKED && sizeof(T) == 4) {
        const float2 ph = phi_n_z2(make_float2(dm4, dp0), make_float2(dm3, dp1), make_float2(dm2, dp2),
                                   make_float2(dm1, dp3));
        return ph.x - ph.y;
    } else if constexpr (Z) {
        return phi_n_z(dm4, dm3, dm2, dm1) - phi_n_z(dp0, dp1, dp2, dp3);
    } else if constexpr (WB_SWEEP_PACKED && sizeof(T) == 4) {
        const float2 ph = phi_n2(make_float2(dm4, dp0), make_float2(dm3, dp1), make_float2(dm2, dp2),
                                 make_float2(dm1, dp3));
        return ph.x - ph.y;
    } else {
        return phi_n(dm4, dm3, dm2, dm1) - phi_n(dp0, dp1, dp2, dp3);
    }
}

// The same correction from the projected differences of the stencil,
// dw_m = l_s (U_{m+1} - U_m), dg_m = l_s (F_{m+1} - F_m), m = 0..4 (the
// projection is linear, so D+-_{m+1/2} = (dg_m +- alpha dw_m) / 2).
template <class T> constexpr T eps3_of() { return sizeof(T) == 4 ? T(kEps3f) : T(kEps3); }
template <class T, bool Z = false>
__device__ __forceinline__ T weno_corr_d(const T (&dw)[5], const T (&dg)[5], T alpha) {
    if constexpr (!Z) {
        // phi_N taken on 2 D+- = dg_m +- alpha dw_m with 4 eps and halved:
        // scaling by two is exact, so the value is the same, and the halving
        // of the eight differences becomes one multiply
        const T dp0 = dg[0] + alpha * dw[0], dp1 = dg[1] + alpha * dw[1], dp2 = dg[2] + alpha * dw[2],
                dp3 = dg[3] + alpha * dw[3];
        const T dm1 = dg[1] - alpha * dw[1], dm2 = dg[2] - alpha * dw[2], dm3 = dg[3] - alpha * dw[3],
                dm4 = dg[4] - alpha * dw[4];
        constexpr T eps3 = T(4) * eps3_of<T>();
        if constexpr (WB_SWEEP_PACKED && sizeof(T) == 4) {
            const float2 ph = phi_n2(make_float2(dm4, dp0), make_float2(dm3, dp1), make_float2(dm2, dp2),
                                     make_float2(dm1, dp3), eps3);
            return T(0.5) * (ph.x - ph.y);
        } else if constexpr (sizeof(T) == 8) {
            return T(0.5) * phi_n_diff(dm4, dm3, dm2, dm1, dp0, dp1, dp2, dp3, eps3);
        } else {
            return T(0.5) * (phi_n(dm4, dm3, dm2, dm1, eps3) - phi_n(dp0, dp1, dp2, dp3, eps3));
        }
    } else {
        const T ha = T(0.5) * alpha;
        T hg[5];
#pragma unroll
        for (int m = 0; m < 5; m++) hg[m] = T(0.5) * dg[m];
        const T dp0 = hg[0] + ha * dw[0], dp1 = hg[1] + ha * dw[1], dp2 = hg[2] + ha * dw[2],
                dp3 = hg[3] + ha * dw[3];
        const T dm1 = hg[1] - ha * dw[1], dm2 = hg[2] - ha * dw[2], dm3 = hg[3] - ha * dw[3],
                dm4 = hg[4] - ha * dw[4];
        if constexpr (WB_SWEEP_PACKED && sizeof(T) == 4) {
            const float2 ph = phi_n_z2(make_float2(dm4, dp0), make_float2(dm3, dp1), make_float2(dm2, dp2),
                                       make_float2(dm1, dp3));
            return ph.x - ph.y;
        } else {
            return phi_n_z(dm4, dm3, dm2, dm1) - phi_n_z(dp0, dp1, dp2, dp3);
        }
    }
}

// Weight policy of the classic scheme: Jiang-Shu weights for every field,
// or the WENO-Z weights when Z is set (a separate kernel instance).
template <class T, bool Z = false>
struct JsWeights {
    static constexpr bool kDiff = true;      // works on projected differences
    __device__ __forceinline__ T corr(int, const T (&w)[6], const T (&g)[6], T alpha) {
        return weno_corr<T, Z>(w, g, alpha);
    }
    __device__ __forceinline__ T corr_d(int, const T (&dw)[5], const T (&dg)[5], T alpha) {
        return weno_corr_d<T, Z>(dw, dg, alpha);
    }
};

// Interface eigen-structure: everything the projection and back-projection
// need, with 1/rho and (gamma-1) folded into the left coefficients.
template <class T>
struct Eig {
    T rho, u, v1, v2, b1, b2, hv2;
    T be1, be2;
    T cf, cs, ca;
    T Af, Bf, Cf, Df, As, Bs, Cs, Ds, Aa, Ba, Ee;
};

// Coefficients only the back-projection needs; parked in shared memory (one
// slot per thread) while the WENO step runs, to keep registers for it.
enum : int { BP_ALF = 0, BP_ALS, BP_AFCF, BP_ASCS, BP_ASR, BP_SSR, BP_RA2, BP_IGM1, kNBack = 8 };
// Per-thread slots after the back-projection ones where the Alfven/entropy
// projections (3 fields x (w, g) x 6 cells, or x 5 differences) wait while
// the fast/slow group is reconstructed, when each stencil vector is
// projected only once.
#ifndef WB_SWEEP_DELTA
#define WB_SWEEP_DELTA 1               // 1: project the stencil's differences (PARK path)
#endif
constexpr int kNPark = 36;
constexpr int kNThreadSlots = kNBack + (WB_SWEEP_PARK ? kNPark : 0);

// |lambda_s| of the interface state, s = 0..6 (u-cf, u-ca, u-cs, u, u+cs,
// u+ca, u+cf)
template <class T>
__device__ __forceinline__ T lam_avg(const Eig<T>& e, int s) {
    const T c = (s == 0 || s == 6) ? e.cf : (s == 1 || s == 5) ? e.ca : (s == 2 || s == 4) ? e.cs : T(0);
    return tabs(s < 3 ? e.u - c : e.u + c);
}

// beta and (alpha_f, alpha_s) with the degeneracy rules; FP64 throughout.
__device__ __forceinline__ void degenerate_rules(double rho, double bn, double b1, double b2,
                                                 double p, double gamma,
                                                 double& be1, double& be2,
                                                 double& alf, double& als,
                                                 double& cf2o, double& cs2o) {
    double bp2 = b1 * b1 + b2 * b2;
    double bt2 = bn * bn + bp2;
    if (bp2 > 1e-24 * (bt2 > 1.0 ? bt2 : 1.0)) {
        const double ibp = rsqrt(bp2);
        be1 = b1 * ibp;
        be2 = b2 * ibp;
    } else {
        be1 = be2 = 0.70710678118654752440;
    }
    double a2 = gamma * p / rho;
    double ca2 = bn * bn / rho;
    double b2r = bt2 / rho;
    // D = cf^2 - cs^2 from a sum of non-negative terms (t = B_perp^2 / rho),
    // cf^2 from the sum of the roots, cs^2 from their product a^2 ca^2: no
    // cancellation near B_perp -> 0 or the triple point.  alpha_f^2 = x / D,
    // alpha_s^2 = y / D with x = a^2 - cs^2, y = cf^2 - a^2: the larger of
    // x, y from x + y = D and the smaller from x y = a^2 t, so the vanishing
    // weight goes to zero with B_perp
    const double t = bp2 / rho;
    // D and 1/D from one reciprocal square root (D = 0 kept exact)
    const double D2 = (a2 - ca2) * (a2 - ca2) + t * (2.0 * (a2 + ca2) + t);
    const double iD = D2 > 0.0 ? rsqrt(D2) : 0.0;
    const double D = D2 * iD;
    const double cf2 = 0.5 * ((a2 + ca2 + t) + D);
    const double cs2 = cf2 > 0.0 ? a2 * ca2 / cf2 : 0.0;
    if (D <= 1e-12 * (a2 + b2r)) {
        if (a2 >= ca2) { alf = 1.0; als = 0.0; } else { alf = 0.0; als = 1.0; }
    } else {
        double x = 0.5 * (D + (a2 - ca2) - t);
        double y = 0.5 * (D - (a2 - ca2) + t);
        if (x >= y) y = a2 * t / x;
        else x = a2 * t / y;
        alf = sqrt(x > 0.0 ? x * iD : 0.0);
        als = sqrt(y > 0.0 ? y * iD : 0.0);
    }
    cf2o = cf2;
    cs2o = cs2;
}

template <class T>
__device__ __forceinline__ void eigen(T rho, T u, T v1, T v2, T bn, T b1, T b2, T p, T gamma,
                                      Eig<T>& e, T* __restrict__ bp, int bstride) {
    const T isr = rsq_root(rho), rinv = isr * isr;     // 1/sqrt(rho), 1/rho
    const T a2 = gamma * p * rinv;
    const T ca2 = bn * bn * rinv;
    T cf2, be1, be2, alf, als;
    if constexpr (sizeof(T) == 8) {
        double dbe1, dbe2, dalf, dals, dcf2, dcs2;
        degenerate_rules(rho, bn, b1, b2, p, gamma, dbe1, dbe2, dalf, dals, dcf2, dcs2);
        be1 = T(dbe1); be2 = T(dbe2); alf = T(dalf); als = T(dals);
        cf2 = T(dcf2);
    } else {
        // FP32 bulk; the normalisation near B_perp -> 0 and near cf = cs
        // (fast/slow/Alfven coincidence) is taken in FP64.
        const T bp2 = b1 * b1 + b2 * b2;
        const T bt2 = bn * bn + bp2;
        const T b2r = bt2 * rinv;
        const T t = bp2 * rinv;
        const T D2 = (a2 - ca2) * (a2 - ca2) + t * (T(2) * (a2 + ca2) + t);
        const T iD = D2 > T(0) ? rsq_root(D2) : T(0);
        const T D = D2 * iD;
        cf2 = T(0.5) * ((a2 + ca2 + t) + D);
        const bool near_bperp = !(bp2 > T(1e-6) * bt2);
        const bool near_triple = !(D > T(1e-3) * (a2 + b2r));
        if (near_bperp || near_triple) {
            double dbe1, dbe2, dalf, dals, dcf2, dcs2;
            degenerate_rules(rho, bn, b1, b2, p, gamma, dbe1, dbe2, dalf, dals, dcf2, dcs2);
            be1 = T(dbe1); be2 = T(dbe2); alf = T(dalf); als = T(dals);
            cf2 = T(dcf2);
        } else {
            const T ibp = rsq_root(bp2);
            be1 = b1 * ibp;
            be2 = b2 * ibp;
            T x = T(0.5) * (D + (a2 - ca2) - t), y = T(0.5) * (D - (a2 - ca2) + t);
            if (x >= y) y = a2 * t / x;
            else x = a2 * t / y;
            alf = sq_root(tmax(x * iD, T(0)));
            als = sq_root(tmax(y * iD, T(0)));
        }
    }
    // sqrt(rho), sqrt(a^2), cf and their reciprocals from one reciprocal
    // square root each (isr above); ca = |B_n| / sqrt(rho) and, from the
    // product of the roots cf^2 cs^2 = a^2 ca^2, cs = a ca / cf
    const T ia = rsq_root(a2);
    const T sr = rho * isr, a = a2 * ia;
    const T icf = cf2 > T(0) ? rsq_root(cf2) : T(0);
    const T cf = cf2 * icf, ca = tabs(bn) * isr;
    const T cs = a * ca * icf, cs2 = cs * cs;
    const T S = bn >= T(0) ? T(1) : T(-1);
    const T gm1 = gamma - T(1);
    const T X = alf * alf * cf2 + als * als * cs2;
    const T hXr = T(0.5) / X * rinv;
    const T hia = T(0.5) * ia * isr;         // 1 / (2 a sqrt(rho))
    const T Ee = gm1 * ia * ia;              // (gamma-1) / a^2
    const T hgp = T(0.5) * Ee * rinv;        // (gamma-1) / (2 rho a^2)
    e.rho = rho; e.u = u; e.v1 = v1; e.v2 = v2; e.b1 = b1; e.b2 = b2;
    e.hv2 = T(0.5) * (u * u + v1 * v1 + v2 * v2);
    e.be1 = be1; e.be2 = be2;
    e.cf = cf; e.cs = cs; e.ca = ca;
    bp[BP_ALF * bstride] = alf;
    bp[BP_ALS * bstride] = als;
    bp[BP_AFCF * bstride] = alf * cf;
    bp[BP_ASCS * bstride] = als * cs;
    bp[BP_ASR * bstride] = a * sr;
    bp[BP_SSR * bstride] = S * sr;
    bp[BP_RA2 * bstride] = rho * a2;
    bp[BP_IGM1 * bstride] = T(1) / gm1;
    e.Af = alf * cf * hXr;
    e.Bf = -als * cs * S * hXr;
    e.Cf = als * hia;
    e.Df = alf * hgp;
    e.As = als * cs * hXr;
    e.Bs = alf * cf * S * hXr;
    e.Cs = -alf * hia;
    e.Ds = als * hgp;
    e.Aa = T(0.5) * rinv;
    e.Ba = T(0.5) * S * isr;
    e.Ee = Ee;
}

// ---- staging ---------------------------------------------------------------
// Per cell: cell B from the faces, rotation into the (n, t1, t2) frame,
// primitives, the physical flux along n, the seven |lambda| and, in the x
// sweep, the cell value of -v x B for the constrained-transport EMFs.  The
// loads of all cells a thread stages are issued first (load_cell), the
// derived quantities computed afterwards (derive_cell), so one global-load
// latency covers a thread's whole share of the tile.
template <class T>
struct RawCell {
    T rho, mx, my, mz, E, bx0, bx1, by0, by1, bz0, bz1;
};

// Loads of one staged cell: the cell values and its three upper faces.
template <class T>
__device__ __forceinline__ void load_cell_at(const SweepArgs<T>& A, long long c, long long cxp,
                                             long long cyp, long long czp, RawCell<T>& r) {
    const long long N = A.ncells;
    const T* __restrict__ q = A.src;
    c = chk(c, N, A.flag);
    cxp = chk(cxp, N, A.flag);
    cyp = chk(cyp, N, A.flag);
    czp = chk(czp, N, A.flag);
    r.rho = q[c]; r.mx = q[N + c]; r.my = q[2 * N + c]; r.mz = q[3 * N + c]; r.E = q[4 * N + c];
    r.bx0 = q[5 * N + c]; r.bx1 = q[5 * N + cxp];
    r.by0 = q[6 * N + c]; r.by1 = q[6 * N + cyp];
    r.bz0 = q[7 * N + c]; r.bz1 = q[7 * N + czp];
}

// Cell (i, j, k) of a periodic patch P, all three indices inside it.
template <class T>
__device__ __forceinline__ void load_cell(const SweepArgs<T>& A, const PatchDev& P, int i, int j,
                                          int k, RawCell<T>& r, long long& c) {
    c = P.off + ((long long)k * P.ny + j) * P.nx + i;
    const int ip = (i + 1 == P.nx) ? 0 : i + 1;
    const int jp = (j + 1 == P.ny) ? 0 : j + 1;
    const int kp = (k + 1 == P.nz) ? 0 : k + 1;
    load_cell_at(A, c, c + (ip - i), c + (long long)(jp - j) * P.nx,
                 c + (long long)(kp - k) * P.nx * P.ny, r);
}

// (i, j, k) are coordinates of patch p of a linked grid and may lie outside
// it (the stencil reaching into a neighbour).
template <class T>
__device__ __forceinline__ void load_cell_linked(const SweepArgs<T>& A, int p, const PatchDev& P,
                                                 int i, int j, int k, RawCell<T>& r, long long& c) {
    c = locate(A.patches, A.links, p, P, i, j, k);
    load_cell_at(A, c, locate(A.patches, A.links, p, P, i + 1, j, k),
                 locate(A.patches, A.links, p, P, i, j + 1, k),
                 locate(A.patches, A.links, p, P, i, j, k + 1), r);
}


template <class T, int AXIS>
__device__ __forceinline__ void derive_cell(const SweepArgs<T>& A, const RawCell<T>& r, long long c,
                                            T* __restrict__ sm, int nc, int idx, bool write_er) {
    const long long N = A.ncells;
    idx = (int)chk(idx, nc, A.flag);
    const T rho = r.rho, E = r.E;
    const T Bx = T(0.5) * (r.bx0 + r.bx1);
    const T By = T(0.5) * (r.by0 + r.by1);
    const T Bz = T(0.5) * (r.bz0 + r.bz1);
    const T mx = r.mx, my = r.my, mz = r.mz;
    T mn, m1, m2, bn, b1, b2;
    if (AXIS == 0) { mn = mx; m1 = my; m2 = mz; bn = Bx; b1 = By; b2 = Bz; }
    else if (AXIS == 1) { mn = my; m1 = mz; m2 = mx; bn = By; b1 = Bz; b2 = Bx; }
    else { mn = mz; m1 = mx; m2 = my; bn = Bz; b1 = Bx; b2 = By; }
    const T g = T(A.gamma);
    const T isr = rsq_root(rho), rinv = isr * isr;
    const T u = mn * rinv, v1 = m1 * rinv, v2 = m2 * rinv;
    const T bb = bn * bn + b1 * b1 + b2 * b2;
    const T kin = T(0.5) * (mn * u + m1 * v1 + m2 * v2);
    const T p = (g - T(1)) * (E - kin - T(0.5) * bb);
    const T pt = p + T(0.5) * bb;
    const T vb = u * bn + v1 * b1 + v2 * b2;
    sm[(SU + 0) * nc + idx] = rho;
    sm[(SU + 1) * nc + idx] = mn;
    sm[(SU + 2) * nc + idx] = m1;
    sm[(SU + 3) * nc + idx] = m2;
    sm[(SU + 4) * nc + idx] = b1;
    sm[(SU + 5) * nc + idx] = b2;
    sm[(SU + 6) * nc + idx] = E;
    sm[(SF + 0) * nc + idx] = mn;
    sm[(SF + 1) * nc + idx] = mn * u + pt - bn * bn;
    sm[(SF + 2) * nc + idx] = m1 * u - bn * b1;
    sm[(SF + 3) * nc + idx] = m2 * u - bn * b2;
    sm[(SF + 4) * nc + idx] = u * b1 - v1 * bn;
    sm[(SF + 5) * nc + idx] = u * b2 - v2 * bn;
    sm[(SF + 6) * nc + idx] = (E + pt) * u - bn * vb;
    const T a2 = g * p * rinv;
    const T ca2 = bn * bn * rinv;
    // fast and slow speeds without cancellation: D = cf^2 - cs^2 from a sum
    // of non-negative terms (t = B_perp^2 / rho), cf^2 from the sum of the
    // roots and cs^2 = a^2 ca^2 / cf^2 from their product
    const T t = (b1 * b1 + b2 * b2) * rinv;
    const T D = sq_root((a2 - ca2) * (a2 - ca2) + t * (T(2) * (a2 + ca2) + t));
    const T cf2 = T(0.5) * ((a2 + ca2 + t) + D);
    const T icf = cf2 > T(0) ? rsq_root(cf2) : T(0);
    const T cf = cf2 * icf;
    const T ca = tabs(bn) * isr;
    const T cs = sq_root(a2) * ca * icf;       // sqrt(a^2 ca^2 / cf^2)
    sm[(SL + 0) * nc + idx] = tabs(u - cf);
    sm[(SL + 1) * nc + idx] = tabs(u - ca);
    sm[(SL + 2) * nc + idx] = tabs(u - cs);
    sm[(SL + 3) * nc + idx] = tabs(u);
    sm[(SL + 4) * nc + idx] = tabs(u + cs);
    sm[(SL + 5) * nc + idx] = tabs(u + ca);
    sm[(SL + 6) * nc + idx] = tabs(u + cf);
    sm[SP_U * nc + idx] = u;
    sm[SP_V1 * nc + idx] = v1;
    sm[SP_V2 * nc + idx] = v2;
    sm[SP_BN * nc + idx] = bn;
    sm[SP_P * nc + idx] = p;
    if (AXIS == 0 && write_er) {
        // -v x B in the global frame (x sweep: u = vx, v1 = vy, v2 = vz)
        c = chk(c, N, A.flag);
        A.er[c] = v2 * b1 - v1 * b2;
        A.er[N + c] = u * b2 - v2 * bn;
        A.er[2 * N + c] = v1 * bn - u * b1;
    }
}

// ---- one interface ----------------------------------------------------------
template <class T>
__device__ __forceinline__ void load7(const T* __restrict__ sm, int nc, int base, int idx, T (&x)[7]) {
#pragma unroll
    for (int f = 0; f < 7; f++) x[f] = sm[(base + f) * nc + idx];
}

// first projection group: fast-, slow-, slow+, fast+ (s = 0, 2, 4, 6)
template <class T>
__device__ __forceinline__ void project_fs(const Eig<T>& e, const T (&x)[7], T (&o)[4]) {
    const T du = x[1] - e.u * x[0];
    const T dv1 = x[2] - e.v1 * x[0];
    const T dv2 = x[3] - e.v2 * x[0];
    const T P = x[6] + e.hv2 * x[0] - e.u * x[1] - e.v1 * x[2] - e.v2 * x[3]
              - e.b1 * x[4] - e.b2 * x[5];
    const T vpar = e.be1 * dv1 + e.be2 * dv2;
    const T bpar = e.be1 * x[4] + e.be2 * x[5];
    const T tf1 = e.Af * du + e.Bf * vpar, tf2 = e.Cf * bpar + e.Df * P;
    const T ts1 = e.As * du + e.Bs * vpar, ts2 = e.Cs * bpar + e.Ds * P;
    o[0] = tf2 - tf1;
    o[1] = ts2 - ts1;
    o[2] = ts2 + ts1;
    o[3] = tf2 + tf1;
}

// second projection group: Alfven-, entropy, Alfven+ (s = 1, 3, 5)
template <class T>
__device__ __forceinline__ void project_ae(const Eig<T>& e, const T (&x)[7], T (&o)[3]) {
    const T dv1 = x[2] - e.v1 * x[0];
    const T dv2 = x[3] - e.v2 * x[0];
    const T P = x[6] + e.hv2 * x[0] - e.u * x[1] - e.v1 * x[2] - e.v2 * x[3]
              - e.b1 * x[4] - e.b2 * x[5];
    const T vperp = e.be1 * dv2 - e.be2 * dv1;
    const T bperp = e.be1 * x[5] - e.be2 * x[4];
    const T t1 = e.Aa * vperp, t2 = e.Ba * bperp;
    o[0] = t1 + t2;
    o[1] = x[0] - e.Ee * P;
    o[2] = t1 - t2;
}

// all seven fields at once: the fast/slow group into o4, Alfven/entropy into
// o3 (the shared terms dv1, dv2, P formed once)
template <class T>
__device__ __forceinline__ void project_all(const Eig<T>& e, const T (&x)[7], T (&o4)[4], T (&o3)[3]) {
    const T du = x[1] - e.u * x[0];
    const T dv1 = x[2] - e.v1 * x[0];
    const T dv2 = x[3] - e.v2 * x[0];
    const T P = x[6] + e.hv2 * x[0] - e.u * x[1] - e.v1 * x[2] - e.v2 * x[3]
              - e.b1 * x[4] - e.b2 * x[5];
    const T vpar = e.be1 * dv1 + e.be2 * dv2;
    const T bpar = e.be1 * x[4] + e.be2 * x[5];
    const T tf1 = e.Af * du + e.Bf * vpar, tf2 = e.Cf * bpar + e.Df * P;
    const T ts1 = e.As * du + e.Bs * vpar, ts2 = e.Cs * bpar + e.Ds * P;
    o4[0] = tf2 - tf1;
    o4[1] = ts2 - ts1;
    o4[2] = ts2 + ts1;
    o4[3] = tf2 + tf1;
    const T vperp = e.be1 * dv2 - e.be2 * dv1;
    const T bperp = e.be1 * x[5] - e.be2 * x[4];
    const T t1 = e.Aa * vperp, t2 = e.Ba * bperp;
    o3[0] = t1 + t2;
    o3[1] = x[0] - e.Ee * P;
    o3[2] = t1 - t2;
}

// project_all on a (U difference, F difference) pair in packed FP32 lanes:
// the same coefficients act on both, one instruction for the two.
#ifndef WB_SWEEP_PAIRPROJ
#define WB_SWEEP_PAIRPROJ 1
#endif
__device__ __forceinline__ void project_all2(const Eig<float>& e, const float2 (&x)[7], float2 (&o4)[4],
                                             float2 (&o3)[3]) {
    const float2 du = __ffma2_rn(splat2(-e.u), x[0], x[1]);
    const float2 dv1 = __ffma2_rn(splat2(-e.v1), x[0], x[2]);
    const float2 dv2 = __ffma2_rn(splat2(-e.v2), x[0], x[3]);
    float2 P = __ffma2_rn(splat2(e.hv2), x[0], x[6]);
    P = __ffma2_rn(splat2(-e.u), x[1], P);
    P = __ffma2_rn(splat2(-e.v1), x[2], P);
    P = __ffma2_rn(splat2(-e.v2), x[3], P);
    P = __ffma2_rn(splat2(-e.b1), x[4], P);
    P = __ffma2_rn(splat2(-e.b2), x[5], P);
    const float2 vpar = __ffma2_rn(splat2(e.be1), dv1, __fmul2_rn(splat2(e.be2), dv2));
    const float2 bpar = __ffma2_rn(splat2(e.be1), x[4], __fmul2_rn(splat2(e.be2), x[5]));
    const float2 tf1 = __ffma2_rn(splat2(e.Af), du, __fmul2_rn(splat2(e.Bf), vpar));
    const float2 tf2 = __ffma2_rn(splat2(e.Cf), bpar, __fmul2_rn(splat2(e.Df), P));
    const float2 ts1 = __ffma2_rn(splat2(e.As), du, __fmul2_rn(splat2(e.Bs), vpar));
    const float2 ts2 = __ffma2_rn(splat2(e.Cs), bpar, __fmul2_rn(splat2(e.Ds), P));
    o4[0] = __ffma2_rn(tf1, splat2(-1.0f), tf2);
    o4[1] = __ffma2_rn(ts1, splat2(-1.0f), ts2);
    o4[2] = __fadd2_rn(ts2, ts1);
    o4[3] = __fadd2_rn(tf2, tf1);
    const float2 vperp = __ffma2_rn(splat2(e.be1), dv2, __fmul2_rn(splat2(-e.be2), dv1));
    const float2 bperp = __ffma2_rn(splat2(e.be1), x[5], __fmul2_rn(splat2(-e.be2), x[4]));
    const float2 t1 = __fmul2_rn(splat2(e.Aa), vperp), t2 = __fmul2_rn(splat2(e.Ba), bperp);
    o3[0] = __fadd2_rn(t1, t2);
    o3[1] = __ffma2_rn(splat2(-e.Ee), P, x[0]);
    o3[2] = __ffma2_rn(t2, splat2(-1.0f), t1);
}

// single field pair projections (fields processed two at a time keep the
// projected stencil small): G = 0 fast-/fast+ (s = 0, 6), 1 slow-/slow+
// (s = 2, 4), 2 Alfven-/Alfven+ (s = 1, 5), 3 entropy (s = 3).
template <int G, class T>
__device__ __forceinline__ void project_pair(const Eig<T>& e, const T (&x)[7], T (&o)[2]) {
    const T dv1 = x[2] - e.v1 * x[0];
    const T dv2 = x[3] - e.v2 * x[0];
    if constexpr (G == 2) {
        const T t1 = e.Aa * (e.be1 * dv2 - e.be2 * dv1);
        const T t2 = e.Ba * (e.be1 * x[5] - e.be2 * x[4]);
        o[0] = t1 + t2;
        o[1] = t1 - t2;
    } else {
        const T P = x[6] + e.hv2 * x[0] - e.u * x[1] - e.v1 * x[2] - e.v2 * x[3]
                  - e.b1 * x[4] - e.b2 * x[5];
        if constexpr (G == 3) {
            o[0] = x[0] - e.Ee * P;
            o[1] = o[0];
        } else {
            const T du = x[1] - e.u * x[0];
            const T vpar = e.be1 * dv1 + e.be2 * dv2;
            const T bpar = e.be1 * x[4] + e.be2 * x[5];
            const T t1 = G == 0 ? e.Af * du + e.Bf * vpar : e.As * du + e.Bs * vpar;
            const T t2 = G == 0 ? e.Cf * bpar + e.Df * P : e.Cs * bpar + e.Ds * P;
            o[0] = t2 - t1;
            o[1] = t2 + t1;
        }
    }
}

template <class T>
__device__ __forceinline__ T lf_speed(const T* __restrict__ sm, int nc, const int (&id)[6],
                                      int s, T lam_avg) {
    T al = lam_avg;
#pragma unroll
    for (int m = 0; m < 6; m++) al = tmax_nonneg(al, sm[(SL + s) * nc + id[m]]);
    return al;
}

template <class T, class Wt, bool PARK = false>
__device__ __forceinline__ void interface_flux(const T* __restrict__ sm, int nc, const int (&id)[6],
                                               T gamma, T* __restrict__ bp, int bstride, Wt& wt,
                                               T (&out)[7]) {
    // 1-2. interface state and eigen-structure
    Eig<T> e;
    {
        const int l = id[2], r = id[3];
        const T h = T(0.5);
        eigen<T>(h * (sm[SU * nc + l] + sm[SU * nc + r]),
                 h * (sm[SP_U * nc + l] + sm[SP_U * nc + r]),
                 h * (sm[SP_V1 * nc + l] + sm[SP_V1 * nc + r]),
                 h * (sm[SP_V2 * nc + l] + sm[SP_V2 * nc + r]),
                 h * (sm[SP_BN * nc + l] + sm[SP_BN * nc + r]),
                 h * (sm[(SU + 4) * nc + l] + sm[(SU + 4) * nc + r]),
                 h * (sm[(SU + 5) * nc + l] + sm[(SU + 5) * nc + r]),
                 h * (sm[SP_P * nc + l] + sm[SP_P * nc + r]), gamma, e, bp, bstride);
    }
    T corr[7];
#if WB_SWEEP_GROUPS == 4
    // 3-5. one field pair at a time
    {
        constexpr int NP = 4;
        constexpr int s0[NP] = {0, 2, 1, 3};
        constexpr int s1[NP] = {6, 4, 5, 3};
#pragma unroll
        for (int G = 0; G < NP; G++) {
            T w[2][6], g[2][6];
#pragma unroll
            for (int m = 0; m < 6; m++) {
                T x[7], o[2];
                load7(sm, nc, SU, id[m], x);
                if (G == 0) project_pair<0>(e, x, o);
                else if (G == 1) project_pair<1>(e, x, o);
                else if (G == 2) project_pair<2>(e, x, o);
                else project_pair<3>(e, x, o);
                w[0][m] = o[0]; w[1][m] = o[1];
                load7(sm, nc, SF, id[m], x);
                if (G == 0) project_pair<0>(e, x, o);
                else if (G == 1) project_pair<1>(e, x, o);
                else if (G == 2) project_pair<2>(e, x, o);
                else project_pair<3>(e, x, o);
                g[0][m] = o[0]; g[1][m] = o[1];
            }
            corr[s0[G]] = wt.corr(s0[G], w[0], g[0], lf_speed(sm, nc, id, s0[G], lam_avg(e, s0[G])));
            if (G != 3)
                corr[s1[G]] = wt.corr(s1[G], w[1], g[1], lf_speed(sm, nc, id, s1[G], lam_avg(e, s1[G])));
        }
    }
#else
    if constexpr (PARK && WB_SWEEP_DELTA && Wt::kDiff) {
        // 3. the five differences of the stencil's U and F, each projected
        // once onto all seven fields; the Alfven/entropy values wait in
        // this thread's shared-memory slots
        T* park = bp + kNBack * bstride;
        T dw[4][5], dg[4][5];
        if constexpr (sizeof(T) == 4 && WB_SWEEP_PAIRPROJ) {
            // U and F differences of a stencil step as one packed pair
            float2 p0[7];
#pragma unroll
            for (int f = 0; f < 7; f++) p0[f] = make_float2(sm[(SU + f) * nc + id[0]], sm[(SF + f) * nc + id[0]]);
#pragma unroll
            for (int m = 0; m < 5; m++) {
                float2 p1[7], x[7], o4[4], o3[3];
#pragma unroll
                for (int f = 0; f < 7; f++) {
                    p1[f] = make_float2(sm[(SU + f) * nc + id[m + 1]], sm[(SF + f) * nc + id[m + 1]]);
                    x[f] = __ffma2_rn(p0[f], splat2(-1.0f), p1[f]);
                }
                project_all2(e, x, o4, o3);
#pragma unroll
                for (int f = 0; f < 4; f++) { dw[f][m] = o4[f].x; dg[f][m] = o4[f].y; }
#pragma unroll
                for (int f = 0; f < 3; f++) {
                    park[(f * 5 + m) * bstride] = o3[f].x;
                    park[((3 + f) * 5 + m) * bstride] = o3[f].y;
                }
#pragma unroll
                for (int f = 0; f < 7; f++) p0[f] = p1[f];
            }
        } else {
        T u0[7], f0[7];
        load7(sm, nc, SU, id[0], u0);
        load7(sm, nc, SF, id[0], f0);
#pragma unroll
        for (int m = 0; m < 5; m++) {
            T u1[7], f1[7], x[7], o4[4], o3[3];
            load7(sm, nc, SU, id[m + 1], u1);
#pragma unroll
            for (int f = 0; f < 7; f++) x[f] = u1[f] - u0[f];
            project_all(e, x, o4, o3);
#pragma unroll
            for (int f = 0; f < 4; f++) dw[f][m] = o4[f];
#pragma unroll
            for (int f = 0; f < 3; f++) park[(f * 5 + m) * bstride] = o3[f];
            load7(sm, nc, SF, id[m + 1], f1);
#pragma unroll
            for (int f = 0; f < 7; f++) x[f] = f1[f] - f0[f];
            project_all(e, x, o4, o3);
#pragma unroll
            for (int f = 0; f < 4; f++) dg[f][m] = o4[f];
#pragma unroll
            for (int f = 0; f < 3; f++) park[((3 + f) * 5 + m) * bstride] = o3[f];
#pragma unroll
            for (int f = 0; f < 7; f++) { u0[f] = u1[f]; f0[f] = f1[f]; }
        }
        }
        // 4-5. fast and slow fields
#pragma unroll
        for (int f = 0; f < 4; f++) {
            const int s = 2 * f;
            corr[s] = wt.corr_d(s, dw[f], dg[f], lf_speed(sm, nc, id, s, lam_avg(e, s)));
        }
        // 4-5. Alfven and entropy fields
#pragma unroll
        for (int f = 0; f < 3; f++) {
            T wa[5], ga[5];
#pragma unroll
            for (int m = 0; m < 5; m++) {
                wa[m] = park[(f * 5 + m) * bstride];
                ga[m] = park[((3 + f) * 5 + m) * bstride];
            }
            const int s = 2 * f + 1;
            corr[s] = wt.corr_d(s, wa, ga, lf_speed(sm, nc, id, s, lam_avg(e, s)));
        }
    } else if constexpr (PARK) {
        // 3. each stencil vector projected once onto all seven fields; the
        // Alfven/entropy values wait in this thread's shared-memory slots
        T* park = bp + kNBack * bstride;
        T w[4][6], g[4][6];
#pragma unroll
        for (int m = 0; m < 6; m++) {
            T x[7], o4[4], o3[3];
            load7(sm, nc, SU, id[m], x);
            project_all(e, x, o4, o3);
#pragma unroll
            for (int f = 0; f < 4; f++) w[f][m] = o4[f];
#pragma unroll
            for (int f = 0; f < 3; f++) park[(f * 6 + m) * bstride] = o3[f];
            load7(sm, nc, SF, id[m], x);
            project_all(e, x, o4, o3);
#pragma unroll
            for (int f = 0; f < 4; f++) g[f][m] = o4[f];
#pragma unroll
            for (int f = 0; f < 3; f++) park[((3 + f) * 6 + m) * bstride] = o3[f];
        }
        // 4-5. fast and slow fields
#pragma unroll
        for (int f = 0; f < 4; f++) {
            const int s = 2 * f;
            corr[s] = wt.corr(s, w[f], g[f], lf_speed(sm, nc, id, s, lam_avg(e, s)));
        }
        // 4-5. Alfven and entropy fields
#pragma unroll
        for (int f = 0; f < 3; f++) {
            T wa[6], ga[6];
#pragma unroll
            for (int m = 0; m < 6; m++) {
                wa[m] = park[(f * 6 + m) * bstride];
                ga[m] = park[((3 + f) * 6 + m) * bstride];
            }
            const int s = 2 * f + 1;
            corr[s] = wt.corr(s, wa, ga, lf_speed(sm, nc, id, s, lam_avg(e, s)));
        }
    } else {
    // 3-5. fast and slow fields
    {
        T w[4][6], g[4][6];
#pragma unroll
        for (int m = 0; m < 6; m++) {
            T x[7], o[4];
            load7(sm, nc, SU, id[m], x);
            project_fs(e, x, o);
#pragma unroll
            for (int f = 0; f < 4; f++) w[f][m] = o[f];
            load7(sm, nc, SF, id[m], x);
            project_fs(e, x, o);
#pragma unroll
            for (int f = 0; f < 4; f++) g[f][m] = o[f];
        }
#pragma unroll
        for (int f = 0; f < 4; f++) {
            const int s = 2 * f;
            corr[s] = wt.corr(s, w[f], g[f], lf_speed(sm, nc, id, s, lam_avg(e, s)));
        }
    }
    // 3-5. Alfven and entropy fields
    {
        T w[3][6], g[3][6];
#pragma unroll
        for (int m = 0; m < 6; m++) {
            T x[7], o[3];
            load7(sm, nc, SU, id[m], x);
            project_ae(e, x, o);
#pragma unroll
            for (int f = 0; f < 3; f++) w[f][m] = o[f];
            load7(sm, nc, SF, id[m], x);
            project_ae(e, x, o);
#pragma unroll
            for (int f = 0; f < 3; f++) g[f][m] = o[f];
        }
#pragma unroll
        for (int f = 0; f < 3; f++) {
            const int s = 2 * f + 1;
            corr[s] = wt.corr(s, w[f], g[f], lf_speed(sm, nc, id, s, lam_avg(e, s)));
        }
    }
    }
#endif
    // 6. back-projection: sum_s r_s corr_s in primitive variables, then dU/dW,
    // added to the central flux (-F_{i-1} + 7F_i + 7F_{i+1} - F_{i+2}) / 12
    const T alf = bp[BP_ALF * bstride], als = bp[BP_ALS * bstride];
    const T afcf = bp[BP_AFCF * bstride], ascs = bp[BP_ASCS * bstride];
    const T Fp = corr[6] + corr[0], Fm = corr[6] - corr[0];
    const T Sp = corr[4] + corr[2], Sm = corr[4] - corr[2];
    const T Ap = corr[5] + corr[1], Am = corr[5] - corr[1];
    const T fs = alf * Fp + als * Sp;
    const T drho = e.rho * fs + corr[3];
    const T du = afcf * Fm + ascs * Sm;
    const T dvpar = afcf * Sm - ascs * Fm;     // times sgn(B_n), folded into Ssr below
    const T dvperp = Ap;
    const T dbpar = bp[BP_ASR * bstride] * (als * Fp - alf * Sp);
    const T ssr = bp[BP_SSR * bstride];
    const T S = ssr < T(0) ? T(-1) : T(1);
    const T dbperp = -ssr * Am;
    const T dp = bp[BP_RA2 * bstride] * fs;
    const T dv1 = e.be1 * S * dvpar - e.be2 * dvperp;
    const T dv2 = e.be2 * S * dvpar + e.be1 * dvperp;
    const T db1 = e.be1 * dbpar - e.be2 * dbperp;
    const T db2 = e.be2 * dbpar + e.be1 * dbperp;
    {
        T f1[7], f2[7], f3[7], f4[7];
        load7(sm, nc, SF, id[1], f1);
        load7(sm, nc, SF, id[2], f2);
        load7(sm, nc, SF, id[3], f3);
        load7(sm, nc, SF, id[4], f4);
#pragma unroll
        for (int f = 0; f < 7; f++)
            out[f] = (T(7) * (f2[f] + f3[f]) - (f1[f] + f4[f])) * T(1.0 / 12.0);
    }
    out[0] += drho;
    out[1] += e.u * drho + e.rho * du;
    out[2] += e.v1 * drho + e.rho * dv1;
    out[3] += e.v2 * drho + e.rho * dv2;
    out[4] += db1;
    out[5] += db2;
    out[6] += e.hv2 * drho + e.rho * (e.u * du + e.v1 * dv1 + e.v2 * dv2)
            + e.b1 * db1 + e.b2 * db2 + dp * bp[BP_IGM1 * bstride];
}

// ---- the kernel -------------------------------------------------------------
// Tile shapes (interfaces along the axis x pencils) and the
// number of resident blocks per SM the FP32 register budget is shaped for.
#ifndef WB_SWEEP_TA_X
#define WB_SWEEP_TA_X 32
#endif
#ifndef WB_SWEEP_TA_YZ
#define WB_SWEEP_TA_YZ 16
#endif
#ifndef WB_SWEEP_MINB_F32
#define WB_SWEEP_MINB_F32 2        // in 256-thread units (four 128-thread blocks)
#endif
// threads (= interfaces) per block of the Jiang-Shu / WENO-Z sweeps; the
// register budget per thread is kept when it changes (blocks per SM scale)
#ifndef WB_SWEEP_NT
#define WB_SWEEP_NT 128
#endif
constexpr int kSweepNT = WB_SWEEP_NT;
constexpr int kSweepLgNT = kSweepNT == 512 ? 9 : (kSweepNT == 256 ? 8 : (kSweepNT == 128 ? 7 : 6));
static_assert((1 << kSweepLgNT) == kSweepNT, "sweep block size must be 64, 128, 256 or 512");
template <int AXIS> struct Shape;
template <> struct Shape<0> { static constexpr int TA = WB_SWEEP_TA_X, TP = 256 / WB_SWEEP_TA_X; };
template <> struct Shape<1> { static constexpr int TA = WB_SWEEP_TA_YZ, TP = 256 / WB_SWEEP_TA_YZ; };
template <> struct Shape<2> { static constexpr int TA = WB_SWEEP_TA_YZ, TP = 256 / WB_SWEEP_TA_YZ; };

template <class T> struct MinBlocks { static constexpr int value = 256 / kSweepNT > 1 ? 256 / kSweepNT : 1; };
#ifdef WB_SWEEP_BLOCKS_F32      // resident blocks per SM, overriding the above
template <> struct MinBlocks<float> { static constexpr int value = WB_SWEEP_BLOCKS_F32; };
#else
template <> struct MinBlocks<float> { static constexpr int value = WB_SWEEP_MINB_F32 * 256 / kSweepNT; };
#endif

// Tile shapes a tile may use, per axis: TA interfaces along the axis times
// TP = kSweepNT / TA pencils.  Shape 0 is the default; the host picks a shape per
// patch (fewest thread slots for the patch's sizes) and stores it in the top
// byte of the tile's patch field.
#ifndef WB_SWEEP_TA_X1
#define WB_SWEEP_TA_X1 8
#endif
__host__ __device__ constexpr int shape_ta(int axis, int s) {
    return axis == 0 ? (s == 0 ? WB_SWEEP_TA_X : (s == 1 ? WB_SWEEP_TA_X1 : 16))
                     : (s == 0 ? WB_SWEEP_TA_YZ : (s == 1 ? 8 : 32));
}
constexpr int kNShape = 3;
__host__ __device__ constexpr int nc_of(int ta) { return (ta + 5) * (kSweepNT / ta); }
__host__ __device__ constexpr int max_nc(int axis) {
    return nc_of(shape_ta(axis, 0)) > nc_of(shape_ta(axis, 1))
               ? (nc_of(shape_ta(axis, 0)) > nc_of(shape_ta(axis, 2)) ? nc_of(shape_ta(axis, 0)) : nc_of(shape_ta(axis, 2)))
               : (nc_of(shape_ta(axis, 1)) > nc_of(shape_ta(axis, 2)) ? nc_of(shape_ta(axis, 1)) : nc_of(shape_ta(axis, 2)));
}

// One tile: stage the TA+5 cells of each of the TP pencils, then one thread
// per interface.  TA_CT > 0 fixes the shape at compile time; TA_CT = 0 takes
// it from ta_rt (a power of two), so that one body, and one register
// allocation, serves every shape of a persistent launch.
template <class T, int AXIS, int TA_CT, int NCMAX, bool Z>
__device__ __forceinline__ void tile_body(const SweepArgs<T>& A, const Tile& tile, const PatchDev& P,
                                          T* __restrict__ sm, int tid, int ta_rt = 0) {
    const int TA = TA_CT > 0 ? TA_CT : ta_rt;
    const int lg_ta = TA_CT > 0 ? __builtin_ctz(TA_CT) : __ffs(ta_rt) - 1;
    const int TP = kSweepNT >> lg_ta;
    const int NS = TA + 5;
    const int NC = NS * TP;
    const int na = AXIS == 0 ? P.nx : (AXIS == 1 ? P.ny : P.nz);
    const int np = AXIS == 0 ? P.ny : P.nx;

    // staging: cells tile.y-3 .. tile.y+TA+1 along the axis, TP pencils
    constexpr int NIT = ((TA_CT > 0 ? (TA_CT + 5) * (kSweepNT / (TA_CT > 0 ? TA_CT : 1)) : NCMAX) + kSweepNT - 1)
                        / kSweepNT;
    RawCell<T> raw[NIT];
    long long rc[NIT];
    int ridx[NIT];
    bool rok[NIT], rown[NIT];
#pragma unroll
    for (int it = 0; it < NIT; it++) {
        const int e = tid + it * kSweepNT;
        int s, tp;
        if (AXIS == 0) { tp = e / NS; s = e - tp * NS; }
        else { s = e / TP; tp = e - s * TP; }
        const int cp = tile.z + tp;
        rok[it] = e < NC && cp < np;
        const int raw_a = tile.y - 3 + s;
        rown[it] = raw_a >= tile.y && raw_a < tile.y + TA && raw_a < na;
        ridx[it] = AXIS == 0 ? tp * NS + s : s * TP + tp;
        if (rok[it]) {
            const int ca = A.links ? raw_a : wrap(raw_a, na);
            int i, j, k;
            if (AXIS == 0) { i = ca; j = cp; k = tile.w; }
            else if (AXIS == 1) { i = cp; j = ca; k = tile.w; }
            else { i = cp; j = tile.w; k = ca; }
            if (A.links) load_cell_linked<T>(A, tile.x, P, i, j, k, raw[it], rc[it]);
            else load_cell<T>(A, P, i, j, k, raw[it], rc[it]);
        }
    }
#pragma unroll
    for (int it = 0; it < NIT; it++)
        if (rok[it]) derive_cell<T, AXIS>(A, raw[it], rc[it], sm, NC, ridx[it], rown[it] && A.er != nullptr);
    __syncthreads();

    int ta, tp;
    if (AXIS == 0) { ta = tid & (TA - 1); tp = tid >> lg_ta; }
    else { tp = tid & (TP - 1); ta = tid >> (kSweepLgNT - lg_ta); }
    const int ia = tile.y + ta, ip = tile.z + tp;
    if (ia >= na || ip >= np) return;
    int id[6];
#pragma unroll
    for (int m = 0; m < 6; m++) id[m] = (int)chk(AXIS == 0 ? tp * NS + ta + m : (ta + m) * TP + tp, NC, A.flag);
    T F[7];
    T* bp = sm + kNSlot * NCMAX + tid;      // this thread's back-projection slots
    JsWeights<T, Z> js;
    interface_flux<T, JsWeights<T, Z>, WB_SWEEP_PARK != 0>(sm, NC, id, T(A.gamma), bp, kSweepNT, js, F);

    // rotate back and store at the lower face of cell ia
    int i, j, k;
    if (AXIS == 0) { i = ia; j = ip; k = tile.w; }
    else if (AXIS == 1) { i = ip; j = ia; k = tile.w; }
    else { i = ip; j = tile.w; k = ia; }
    const long long N = A.ncells;
    const long long c = chk(P.off + ((long long)k * P.ny + j) * P.nx + i, N, A.flag);
    T* __restrict__ fo = A.flux;
    T fx, fy, fz;
    if (AXIS == 0) { fx = F[1]; fy = F[2]; fz = F[3]; }
    else if (AXIS == 1) { fy = F[1]; fz = F[2]; fx = F[3]; }
    else { fz = F[1]; fx = F[2]; fy = F[3]; }
    fo[c] = F[0];
    fo[N + c] = fx;
    fo[2 * N + c] = fy;
    fo[3 * N + c] = fz;
    fo[4 * N + c] = F[6];
    fo[5 * N + c] = F[4];
    fo[6 * N + c] = F[5];
}

// Persistent sweep: a grid of (SMs x resident blocks) strides over the tile
// table; each tile carries its shape, so patches of uneven sizes share one
// launch.  Each tile runs the body compiled for its shape (a block-uniform
// switch over the three shapes, so every body keeps its compile-time
// layout); WB_SWEEP_PERSIST_SWITCH=0 selects one body with the shape as a
// runtime value instead.
#ifndef WB_SWEEP_PERSIST_SWITCH
#define WB_SWEEP_PERSIST_SWITCH 1
#endif
// One shape's body; WB_SWEEP_PERSIST_SWITCH=2 keeps it out of line, so that
// each of the three bodies gets a register allocation of its own.
#if WB_SWEEP_PERSIST_SWITCH == 2
#define WB_SHAPE_INLINE __noinline__
#else
#define WB_SHAPE_INLINE __forceinline__
#endif
template <class T, int AXIS, int S, int NCMAX, bool Z>
__device__ WB_SHAPE_INLINE void tile_body_shape(const SweepArgs<T>& A, const Tile& tile, const PatchDev& P,
                                                T* __restrict__ sm, int tid) {
    tile_body<T, AXIS, shape_ta(AXIS, S), NCMAX, Z>(A, tile, P, sm, tid);
}
template <class T, int AXIS, bool Z>
__global__ void __launch_bounds__(kSweepNT, MinBlocks<T>::value) sweep_kernel(const SweepArgs<T> A, int ntiles) {
    constexpr int NCMAX = max_nc(AXIS);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int tid = threadIdx.x;
    __shared__ int next_tile;
    // work queue: each block starts on tile blockIdx.x and then takes the next
    // unclaimed tile from the launch's counter (zeroed before the launch), so
    // uneven tiles balance across SMs; without a counter, a fixed stride
    for (int t = blockIdx.x; t < ntiles;) {
        Tile tile = A.tiles[t];
        const int shape = (unsigned)tile.x >> 24;
        tile.x &= 0xffffff;
        const PatchDev P = A.patches[tile.x];
#if WB_SWEEP_PERSIST_SWITCH
        if (shape == 0) tile_body_shape<T, AXIS, 0, NCMAX, Z>(A, tile, P, sm, tid);
        else if (shape == 1) tile_body_shape<T, AXIS, 1, NCMAX, Z>(A, tile, P, sm, tid);
        else tile_body_shape<T, AXIS, 2, NCMAX, Z>(A, tile, P, sm, tid);
#else
        tile_body<T, AXIS, 0, NCMAX, Z>(A, tile, P, sm, tid, shape_ta(AXIS, shape));
#endif
        __syncthreads();
        if (A.queue) {
            if (tid == 0) next_tile = gridDim.x + atomicAdd(A.queue, 1);
            __syncthreads();
            t = next_tile;
        } else {
            t += gridDim.x;
        }
    }
}

// One tile per block of one shape S, Jiang-Shu weights: the launch for tile
// tables that use shape 0 throughout (a single grid, or patches tuned to
// it), and for each shape's range of a table sorted by shape.
template <class T, int AXIS, int S = 0>
__global__ void __launch_bounds__(kSweepNT, MinBlocks<T>::value) sweep_kernel_fixed(const SweepArgs<T> A) {
    constexpr int NC0 = nc_of(shape_ta(AXIS, S));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    Tile tile = A.tiles[blockIdx.x];
    tile.x &= 0xffffff;
    const PatchDev P = A.patches[tile.x];
    tile_body<T, AXIS, shape_ta(AXIS, S), NC0, false>(A, tile, P, sm, threadIdx.x);
}

template <class T, int AXIS, int S = 0>
constexpr size_t smem_bytes_fixed() {
    return sizeof(T) * (kNSlot * nc_of(shape_ta(AXIS, S)) + kNThreadSlots * kSweepNT);
}

template <class T, int AXIS>
constexpr size_t smem_bytes() {
    return sizeof(T) * (kNSlot * (Shape<AXIS>::TA + 5) * Shape<AXIS>::TP
                        + kNBack * Shape<AXIS>::TA * Shape<AXIS>::TP);
}

template <class T, int AXIS>
constexpr size_t smem_bytes_persistent() {
    return sizeof(T) * (kNSlot * max_nc(AXIS) + kNThreadSlots * kSweepNT);
}

}  // namespace

// Persistent grid sizes per axis, set by prepare_sweep_kernels (outside any
// stream capture).
template <class T>
struct PersistGrid {
    static inline int g[3] = {0, 0, 0};
};

// Resident blocks per SM of the persistent sweep of `axis` (for the grid size).
template <class T>
int sweep_blocks_per_sm(int axis) {
    int nb = 0;
    if (axis == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T, 0, false>, kSweepNT,
                                                      smem_bytes_persistent<T, 0>());
    else if (axis == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T, 1, false>, kSweepNT,
                                                      smem_bytes_persistent<T, 1>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T, 2, false>, kSweepNT,
                                                      smem_bytes_persistent<T, 2>());
    return nb > 0 ? nb : 1;
}

template <class T>
cudaError_t prepare_sweep_kernels() {
    cudaError_t e;
    e = cudaFuncSetAttribute(sweep_kernel<T, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_persistent<T, 0>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<T, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_persistent<T, 0>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_persistent<T, 1>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_persistent<T, 1>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<T, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_persistent<T, 2>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<T, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_persistent<T, 2>());
    if (e != cudaSuccess) return e;
#define WB_FIXED_ATTR(AX, S)                                                                    \
    e = cudaFuncSetAttribute(sweep_kernel_fixed<T, AX, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem_bytes_fixed<T, AX, S>());                                 \
    if (e != cudaSuccess) return e;
    WB_FIXED_ATTR(0, 0) WB_FIXED_ATTR(0, 1) WB_FIXED_ATTR(0, 2)
    WB_FIXED_ATTR(1, 0) WB_FIXED_ATTR(1, 1) WB_FIXED_ATTR(1, 2)
    WB_FIXED_ATTR(2, 0) WB_FIXED_ATTR(2, 1) WB_FIXED_ATTR(2, 2)
#undef WB_FIXED_ATTR
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    for (int a = 0; a < 3; a++) PersistGrid<T>::g[a] = nsm * sweep_blocks_per_sm<T>(a);
    return cudaGetLastError();
}

template <class T, int S>
void launch_fixed_shape(int axis, const SweepArgs<T>& a, int ntiles, cudaStream_t s) {
    if (axis == 0) sweep_kernel_fixed<T, 0, S><<<ntiles, kSweepNT, smem_bytes_fixed<T, 0, S>(), s>>>(a);
    else if (axis == 1) sweep_kernel_fixed<T, 1, S><<<ntiles, kSweepNT, smem_bytes_fixed<T, 1, S>(), s>>>(a);
    else sweep_kernel_fixed<T, 2, S><<<ntiles, kSweepNT, smem_bytes_fixed<T, 2, S>(), s>>>(a);
}

template <class T>
cudaError_t launch_sweep(int axis, const SweepArgs<T>& a, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if ((a.split[0] | a.split[1] | a.split[2]) && !a.zweights) {
        // a table sorted by shape: one launch of the fixed kernel per shape
        SweepArgs<T> b = a;
        if (a.split[0]) launch_fixed_shape<T, 0>(axis, b, a.split[0], s);
        b.tiles = a.tiles + a.split[0];
        if (a.split[1]) launch_fixed_shape<T, 1>(axis, b, a.split[1], s);
        b.tiles = a.tiles + a.split[0] + a.split[1];
        if (a.split[2]) launch_fixed_shape<T, 2>(axis, b, a.split[2], s);
        return cudaGetLastError();
    }
    const int grid = PersistGrid<T>::g[axis] > 0 ? PersistGrid<T>::g[axis] : 152;
    const int nb = ntiles < grid ? ntiles : grid;
    if (a.queue) {
        const cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    if (a.zweights) {
        if (axis == 0) sweep_kernel<T, 0, true><<<nb, kSweepNT, smem_bytes_persistent<T, 0>(), s>>>(a, ntiles);
        else if (axis == 1) sweep_kernel<T, 1, true><<<nb, kSweepNT, smem_bytes_persistent<T, 1>(), s>>>(a, ntiles);
        else sweep_kernel<T, 2, true><<<nb, kSweepNT, smem_bytes_persistent<T, 2>(), s>>>(a, ntiles);
        return cudaGetLastError();
    }
    if (axis == 0) sweep_kernel<T, 0, false><<<nb, kSweepNT, smem_bytes_persistent<T, 0>(), s>>>(a, ntiles);
    else if (axis == 1) sweep_kernel<T, 1, false><<<nb, kSweepNT, smem_bytes_persistent<T, 1>(), s>>>(a, ntiles);
    else sweep_kernel<T, 2, false><<<nb, kSweepNT, smem_bytes_persistent<T, 2>(), s>>>(a, ntiles);
    return cudaGetLastError();
}

}  // namespace wb

// ---- training-record harvest -------------------------------------------------
// For each sampled interface (the lower face of cell `cells[t]` along `axis`
// of patch 0) and each characteristic field and side, one record of
// WB_MLP_RECORD floats: field, x[6], q[3], T, flag.  v is the split flux g+
// over the stencil cells i-2..i+3 ('-' side: g- reversed), x = (v - mean) /
// (max|v - mean| + 1e-12), q the three third-order candidate reconstructions
// of v at the face, T the face value of the split flux built from hU, hF (the
// exact face reconstructions of U and F, supplied by the caller) with the
// same left eigenvector and Lax-Friedrichs speed, q and T normalised like x;
// flag = 1 when the jump detector (largest of the four differences phi_N
// reads above kappa times the mean of the other three) or the pressure
// detector (max p > (1 + pjump) min p over the six cells) fires.
namespace wb {
namespace {

template <class T>
struct HarvestArgs {
    const T* src;
    long long ncells;
    PatchDev P;
    int axis;
    const long long* cells;
    long long n;
    const double* hU;
    const double* hF;
    double gamma, kappa, pjump;
    float* out;
};

template <class T, int AXIS>
__device__ void harvest_one(const HarvestArgs<T>& H, long long t, T* sm, int nc, int base, T* bp,
                            int bstride) {
    const PatchDev& P = H.P;
    const long long cell = H.cells[t];
    const int i0 = (int)(cell % P.nx), j0 = (int)((cell / P.nx) % P.ny), k0 = (int)(cell / ((long long)P.nx * P.ny));
    SweepArgs<T> A;
    A.src = H.src; A.flux = nullptr; A.er = nullptr; A.tiles = nullptr; A.patches = nullptr;
    A.ncells = H.ncells; A.gamma = H.gamma;
    const int na = AXIS == 0 ? P.nx : (AXIS == 1 ? P.ny : P.nz);
    const int a0 = AXIS == 0 ? i0 : (AXIS == 1 ? j0 : k0);
    T pmin = T(1e300), pmax = T(-1e300);
    int id[6];
    for (int m = 0; m < 6; m++) {
        const int a = wrap(a0 - 3 + m, na);
        int i = i0, j = j0, k = k0;
        if (AXIS == 0) i = a; else if (AXIS == 1) j = a; else k = a;
        RawCell<T> r;
        long long c;
        load_cell<T>(A, P, i, j, k, r, c);
        id[m] = base + m;
        derive_cell<T, AXIS>(A, r, c, sm, nc, id[m], false);
        const T p = sm[SP_P * nc + id[m]];
        pmin = p < pmin ? p : pmin;
        pmax = p > pmax ? p : pmax;
    }
    const bool pfire = pmax > (T(1) + T(H.pjump)) * pmin;
    Eig<T> e;
    {
        const int l = id[2], r = id[3];
        const T h = T(0.5);
        eigen<T>(h * (sm[SU * nc + l] + sm[SU * nc + r]), h * (sm[SP_U * nc + l] + sm[SP_U * nc + r]),
                 h * (sm[SP_V1 * nc + l] + sm[SP_V1 * nc + r]), h * (sm[SP_V2 * nc + l] + sm[SP_V2 * nc + r]),
                 h * (sm[SP_BN * nc + l] + sm[SP_BN * nc + r]), h * (sm[(SU + 4) * nc + l] + sm[(SU + 4) * nc + r]),
                 h * (sm[(SU + 5) * nc + l] + sm[(SU + 5) * nc + r]), h * (sm[SP_P * nc + l] + sm[SP_P * nc + r]),
                 T(H.gamma), e, bp, bstride);
    }
    T hu[7], hf[7];
    for (int f = 0; f < 7; f++) { hu[f] = T(H.hU[t * 7 + f]); hf[f] = T(H.hF[t * 7 + f]); }
    for (int G = 0; G < 4; G++) {
        T w[2][6], g[2][6], tu[2], tf[2];
        for (int m = 0; m < 6; m++) {
            T x[7], o[2];
            load7(sm, nc, SU, id[m], x);
            if (G == 0) project_pair<0>(e, x, o); else if (G == 1) project_pair<1>(e, x, o);
            else if (G == 2) project_pair<2>(e, x, o); else project_pair<3>(e, x, o);
            w[0][m] = o[0]; w[1][m] = o[1];
            load7(sm, nc, SF, id[m], x);
            if (G == 0) project_pair<0>(e, x, o); else if (G == 1) project_pair<1>(e, x, o);
            else if (G == 2) project_pair<2>(e, x, o); else project_pair<3>(e, x, o);
            g[0][m] = o[0]; g[1][m] = o[1];
        }
        {
            T o[2];
            if (G == 0) project_pair<0>(e, hu, o); else if (G == 1) project_pair<1>(e, hu, o);
            else if (G == 2) project_pair<2>(e, hu, o); else project_pair<3>(e, hu, o);
            tu[0] = o[0]; tu[1] = o[1];
            if (G == 0) project_pair<0>(e, hf, o); else if (G == 1) project_pair<1>(e, hf, o);
            else if (G == 2) project_pair<2>(e, hf, o); else project_pair<3>(e, hf, o);
            tf[0] = o[0]; tf[1] = o[1];
        }
        const int sl[2] = {G == 0 ? 0 : (G == 1 ? 2 : (G == 2 ? 1 : 3)), G == 0 ? 6 : (G == 1 ? 4 : (G == 2 ? 5 : 3))};
        const int nsl = G == 3 ? 1 : 2;
        for (int q = 0; q < nsl; q++) {
            const int s = sl[q];
            const T al = lf_speed(sm, nc, id, s, lam_avg(e, s));
            for (int side = 0; side < 2; side++) {
                const T sg = side == 0 ? T(1) : T(-1);
                T v[6];
                for (int m = 0; m < 6; m++) {
                    const int mm = side == 0 ? m : 5 - m;
                    v[m] = T(0.5) * (g[q][mm] + sg * al * w[q][mm]);
                }
                const T Tg = T(0.5) * (tf[q] + sg * al * tu[q]);
                T mean = T(0);
                for (int m = 0; m < 6; m++) mean += v[m];
                mean *= T(1.0 / 6.0);
                T mx = T(0);
                for (int m = 0; m < 6; m++) { const T d = tabs(v[m] - mean); mx = d > mx ? d : mx; }
                const T inv = T(1) / (mx + T(1e-12));
                T D[4];
                for (int m = 0; m < 4; m++) D[m] = tabs(v[m + 1] - v[m]);
                T dmax = D[0], dsum = D[0];
                for (int m = 1; m < 4; m++) { dmax = D[m] > dmax ? D[m] : dmax; dsum += D[m]; }
                const bool jfire = dmax > T(H.kappa) * (dsum - dmax) * T(1.0 / 3.0) + T(1e-300);
                float* o = H.out + ((t * 7 + s) * 2 + side) * WB_MLP_RECORD;
                o[0] = float(s);
                for (int m = 0; m < 6; m++) o[1 + m] = float((v[m] - mean) * inv);
                const T q0 = (T(2) * v[0] - T(7) * v[1] + T(11) * v[2]) * T(1.0 / 6.0);
                const T q1 = (-v[1] + T(5) * v[2] + T(2) * v[3]) * T(1.0 / 6.0);
                const T q2 = (T(2) * v[2] + T(5) * v[3] - v[4]) * T(1.0 / 6.0);
                o[7] = float((q0 - mean) * inv);
                o[8] = float((q1 - mean) * inv);
                o[9] = float((q2 - mean) * inv);
                o[10] = float((Tg - mean) * inv);
                o[11] = (jfire || pfire) ? 1.f : 0.f;
            }
        }
    }
}

template <class T>
__global__ void __launch_bounds__(32) harvest_kernel(const HarvestArgs<T> H) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int nc = 6 * 32;
    T* bp = sm + kNSlot * nc + threadIdx.x;
    const long long t = (long long)blockIdx.x * 32 + threadIdx.x;
    if (t >= H.n) return;
    const int base = threadIdx.x * 6;
    if (H.axis == 0) harvest_one<T, 0>(H, t, sm, nc, base, bp, 32);
    else if (H.axis == 1) harvest_one<T, 1>(H, t, sm, nc, base, bp, 32);
    else harvest_one<T, 2>(H, t, sm, nc, base, bp, 32);
}

// Rotated conserved 7-vector (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) and its
// physical flux along AXIS for every cell of a periodic patch: the sweep's
// own staging arithmetic (cell B from the faces, rotation, primitives, flux),
// written as FP64 arrays [7][cells] each.  The training pipeline reconstructs
// exact face values of these for its targets.
template <class T, int AXIS>
__global__ void __launch_bounds__(128) cell_state_flux_kernel(const SweepArgs<T> A, const PatchDev P,
                                                              double* __restrict__ X,
                                                              double* __restrict__ F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const long long np = (long long)P.nx * P.ny * P.nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int nc = blockDim.x;
    const int i = (int)(t % P.nx), j = (int)((t / P.nx) % P.ny), k = (int)(t / ((long long)P.nx * P.ny));
    RawCell<T> r;
    long long c;
    load_cell<T>(A, P, i, j, k, r, c);
    derive_cell<T, AXIS>(A, r, c, sm, nc, threadIdx.x, false);
    for (int f = 0; f < 7; f++) {
        X[f * np + t] = double(sm[(SU + f) * nc + threadIdx.x]);
        F[f * np + t] = double(sm[(SF + f) * nc + threadIdx.x]);
    }
}

}  // namespace

template <class T>
cudaError_t launch_cell_state_flux(const T* src, long long ncells, const PatchDev& P, int axis,
                                   double gamma, double* X, double* F, cudaStream_t s) {
    SweepArgs<T> A;
    A.src = src; A.flux = nullptr; A.er = nullptr; A.tiles = nullptr; A.patches = nullptr;
    A.ncells = ncells; A.gamma = gamma;
    const long long np = (long long)P.nx * P.ny * P.nz;
    const int nt = 128;
    const unsigned nb = (unsigned)((np + nt - 1) / nt);
    const size_t smem = sizeof(T) * kNSlot * nt;
    if (axis == 0) cell_state_flux_kernel<T, 0><<<nb, nt, smem, s>>>(A, P, X, F);
    else if (axis == 1) cell_state_flux_kernel<T, 1><<<nb, nt, smem, s>>>(A, P, X, F);
    else cell_state_flux_kernel<T, 2><<<nb, nt, smem, s>>>(A, P, X, F);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_harvest(const T* src, long long ncells, const PatchDev& P, int axis,
                           const long long* cells, long long n, const double* hU, const double* hF,
                           double gamma, double kappa, double pjump, float* out, cudaStream_t s) {
    HarvestArgs<T> H{src, ncells, P, axis, cells, n, hU, hF, gamma, kappa, pjump, out};
    const size_t smem = sizeof(T) * (kNSlot * 6 * 32 + kNBack * 32);
    cudaError_t e = cudaFuncSetAttribute(harvest_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    harvest_kernel<T><<<(unsigned)((n + 31) / 32), 32, smem, s>>>(H);
    return cudaGetLastError();
}

}  // namespace wb
