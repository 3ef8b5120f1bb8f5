/*
 * wb_oracle.c -- plain FP64 CPU oracle of the WENO-Wombat MHD hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the package smoke check
 * and by the benchmark's CPU-baseline leg, never by the product path.  It
 * shares no code with the CUDA kernels.
 *
 * Written to be read against the paper (Donnert et al. 2018), not to be fast:
 * one interface at a time, dense 7x7 eigenvector matrices, the left
 * eigenvectors obtained by inverting the right ones, plain loops.  OpenMP
 * only splits the outer z loop of grid sweeps (no reductions depend on it).
 * Compile with -ffp-contract=off.
 *
 * Pins: every function is checked in tests/ against something other than
 * itself (closed forms of the WENO interpolant, the flux Jacobian by finite
 * differences, exact solutions, invariants, brute force).  None is "parity
 * unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "wb_oracle.h"

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the oracle's loops use from now on (timing only; every cell's
 * arithmetic is the same with any count). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static long wrapi(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Sec. 2.1, nonlinear weights: smoothness indicators IS_0..2 as printed
 * (the alpha formula's "IC_k" is read as IS_k), linear weights 1:6:3,
 * epsilon = 1e-6 absolute, omega_k = alpha_k / sum(alpha). */
void orc_weno_weights(double a, double b, double c, double d,
                      double *w0, double *w1, double *w2)
{
    const double eps = 1e-6;
    double is0 = 13.0 * (a - b) * (a - b) + 3.0 * (a - 3.0 * b) * (a - 3.0 * b);
    double is1 = 13.0 * (b - c) * (b - c) + 3.0 * (b + c) * (b + c);
    double is2 = 13.0 * (c - d) * (c - d) + 3.0 * (3.0 * c - d) * (3.0 * c - d);
    double a0 = 1.0 / ((eps + is0) * (eps + is0));
    double a1 = 6.0 / ((eps + is1) * (eps + is1));
    double a2 = 3.0 / ((eps + is2) * (eps + is2));
    double s = a0 + a1 + a2;
    *w0 = a0 / s;
    *w1 = a1 / s;
    *w2 = a2 / s;
}

/* WENO-Z weights (the fifth-order-everywhere alternative Sec. 2.1 names,
 * Borges et al. 2008): the same smoothness indicators IS_k and linear
 * weights 1:6:3, tau5 = |IS_0 - IS_2|,
 * alpha_k = d_k (1 + tau5 / (eps + IS_k)), omega_k = alpha_k / sum(alpha). */
void orc_weno_weights_z(double a, double b, double c, double d,
                        double *w0, double *w1, double *w2)
{
    const double eps = 1e-6;
    double is0 = 13.0 * (a - b) * (a - b) + 3.0 * (a - 3.0 * b) * (a - 3.0 * b);
    double is1 = 13.0 * (b - c) * (b - c) + 3.0 * (b + c) * (b + c);
    double is2 = 13.0 * (c - d) * (c - d) + 3.0 * (3.0 * c - d) * (3.0 * c - d);
    double tau = fabs(is0 - is2);
    double a0 = 1.0 * (1.0 + tau / (eps + is0));
    double a1 = 6.0 * (1.0 + tau / (eps + is1));
    double a2 = 3.0 * (1.0 + tau / (eps + is2));
    double s = a0 + a1 + a2;
    *w0 = a0 / s;
    *w1 = a1 / s;
    *w2 = a2 / s;
}

double orc_phi_n_z(double a, double b, double c, double d)
{
    double w0, w1, w2;
    orc_weno_weights_z(a, b, c, d, &w0, &w1, &w2);
    return w0 * (a - 2.0 * b + c) / 3.0 + (w2 - 0.5) * (b - 2.0 * c + d) / 6.0;
}

/* Sec. 2.1, WENO5 interpolant
 * phi_N(a,b,c,d) = 1/3 w0 (a - 2b + c) + 1/6 (w2 - 1/2) (b - 2c + d). */
double orc_phi_n(double a, double b, double c, double d)
{
    double w0, w1, w2;
    orc_weno_weights(a, b, c, d, &w0, &w1, &w2);
    return w0 * (a - 2.0 * b + c) / 3.0 + (w2 - 0.5) * (b - 2.0 * c + d) / 6.0;
}

/* Sec. 2.1: the 8-field ideal-MHD state (rho, m_n, m_t1, m_t2, B_n, B_t1,
 * B_t2, E).  Units with the magnetic permeability absorbed (magnetic pressure
 * |B|^2/2), E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2.  The vector may be in any
 * rotated frame: the formula is frame independent. */
void orc_cons_to_prim(const double U[8], double gamma, double W[8])
{
    double rho = U[0];
    double u = U[1] / rho, v = U[2] / rho, w = U[3] / rho;
    double kin = 0.5 * rho * (u * u + v * v + w * w);
    double mag = 0.5 * (U[4] * U[4] + U[5] * U[5] + U[6] * U[6]);
    W[0] = rho;
    W[1] = u;
    W[2] = v;
    W[3] = w;
    W[4] = U[4];
    W[5] = U[5];
    W[6] = U[6];
    W[7] = (gamma - 1.0) * (U[7] - kin - mag);
}

void orc_prim_to_cons(const double W[8], double gamma, double U[8])
{
    double rho = W[0];
    U[0] = rho;
    U[1] = rho * W[1];
    U[2] = rho * W[2];
    U[3] = rho * W[3];
    U[4] = W[4];
    U[5] = W[5];
    U[6] = W[6];
    U[7] = W[7] / (gamma - 1.0)
         + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3])
         + 0.5 * (W[4] * W[4] + W[5] * W[5] + W[6] * W[6]);
}

/* Sec. 2.1: physical flux F(U) of the ideal-MHD system along the first
 * (normal) axis of the frame.  The normal-field flux is identically zero. */
void orc_flux_n(const double U[8], double gamma, double F[8])
{
    double W[8];
    orc_cons_to_prim(U, gamma, W);
    double rho = W[0], u = W[1], v = W[2], w = W[3];
    double bn = W[4], b1 = W[5], b2 = W[6], p = W[7];
    double pt = p + 0.5 * (bn * bn + b1 * b1 + b2 * b2);
    F[0] = rho * u;
    F[1] = rho * u * u + pt - bn * bn;
    F[2] = rho * u * v - bn * b1;
    F[3] = rho * u * w - bn * b2;
    F[4] = 0.0;
    F[5] = u * b1 - v * bn;
    F[6] = u * b2 - w * bn;
    F[7] = (U[7] + pt) * u - bn * (u * bn + v * b1 + w * b2);
}

/* Fast, Alfven and slow speeds along the normal axis for primitive W:
 * cf^2, cs^2 = (a^2 + b^2 +- D)/2 with D^2 = (a^2 + b^2)^2 - 4 a^2 ca^2, the
 * roots of the magnetosonic quartic (Sec. 2.1 eigen-system).  Evaluated
 * without cancellation: D^2 = (a^2 - ca^2)^2 + t (2 (a^2 + ca^2) + t) with
 * t = B_perp^2/rho (a sum of non-negative terms), cf^2 from the sum, and
 * cs^2 = a^2 ca^2 / cf^2 (the product of the roots), so that near the
 * triple point (B_perp -> 0, a^2 -> ca^2) the speeds keep full precision. */
void orc_wave_speeds(const double W[8], double gamma,
                     double *cf, double *ca, double *cs)
{
    double rho = W[0];
    double a2 = gamma * W[7] / rho;
    double ca2 = W[4] * W[4] / rho;
    double t = (W[5] * W[5] + W[6] * W[6]) / rho;
    double D = sqrt((a2 - ca2) * (a2 - ca2) + t * (2.0 * (a2 + ca2) + t));
    double cf2 = 0.5 * ((a2 + ca2 + t) + D);
    double cs2 = cf2 > 0.0 ? a2 * ca2 / cf2 : 0.0;
    *cf = sqrt(cf2);
    *ca = sqrt(ca2);
    *cs = sqrt(cs2);
}

/* Gauss-Jordan inverse of an n x n row-major matrix with partial pivoting.
 * Returns 0 on success, -1 if a pivot vanishes. */
static int invert(int n, const double *A, double *Ainv)
{
    double M[7][14];
    for (int r = 0; r < n; r++) {
        for (int c = 0; c < n; c++) {
            M[r][c] = A[r * n + c];
            M[r][n + c] = (r == c) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (M[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < 2 * n; k++) {
                double t = M[c][k];
                M[c][k] = M[piv][k];
                M[piv][k] = t;
            }
        }
        double inv = 1.0 / M[c][c];
        for (int k = 0; k < 2 * n; k++) M[c][k] *= inv;
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double f = M[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * n; k++) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) Ainv[r * n + c] = M[r][n + c];
    return 0;
}

/* Sec. 2.1 ("Roe-type Riemann solver ... decouple the system into independent
 * advection equations"; eigenvectors deferred by the paper to its companion
 * method paper).  Seven-wave system of the variables
 *     (rho, m_n, m_t1, m_t2, B_t1, B_t2, E)
 * at fixed B_n (B_n has zero normal flux and is evolved by constrained
 * transport instead).  Waves in the order
 *     u-cf, u-ca, u-cs, u, u+cs, u+ca, u+cf.
 * Right eigenvectors are first written in primitive variables
 * (rho, u, v, w, B_t1, B_t2, p) with the Roe-Balsara normalisation
 * (alpha_f, alpha_s, beta_1, beta_2, sign of B_n), mapped to conservative
 * variables by dU/dW, and the left eigenvectors are their inverse.
 * Degeneracy rules (identical on every implementation):
 *   beta = B_perp/|B_perp| if |B_perp|^2 > 1e-24 max(1,|B|^2), else 1/sqrt(2);
 *   if cf^2 - cs^2 <= 1e-12 (a^2 + b^2): (alpha_f, alpha_s) = (1,0) when
 *   a^2 >= ca^2, else (0,1); otherwise alpha_f^2 = (a^2 - cs^2)/(cf^2 - cs^2)
 *   and alpha_s^2 = (cf^2 - a^2)/(cf^2 - cs^2), evaluated without
 *   cancellation (below);
 *   sign(B_n) = +1 when B_n = 0.
 * With t = B_perp^2/rho, D = cf^2 - cs^2 = sqrt((a^2 - ca^2)^2 +
 * t (2 (a^2 + ca^2) + t)), x = a^2 - cs^2 = (D + a^2 - ca^2 - t)/2 and
 * y = cf^2 - a^2 = (D - a^2 + ca^2 + t)/2, where x + y = D and x y = a^2 t:
 * the larger of x, y is taken from its sum (relative error a few units of
 * rounding, as it is at least D/2) and the smaller from the product, so
 * that as B_perp -> 0 the vanishing weight goes to zero with B_perp instead
 * of being the square root of a rounding error.
 * RU and LU are row-major 7x7; column s of RU is the right eigenvector of
 * wave s, row s of LU the left one.  Returns -1 if RU is singular. */
int orc_eigen(const double W[8], double gamma, double lam[7],
              double RU[49], double LU[49])
{
    double rho = W[0], u = W[1], v = W[2], w = W[3];
    double bn = W[4], b1 = W[5], b2 = W[6], p = W[7];
    double a2 = gamma * p / rho;
    double a = sqrt(a2);
    double cf, ca, cs;
    orc_wave_speeds(W, gamma, &cf, &ca, &cs);
    double ca2 = bn * bn / rho;
    double bperp2 = b1 * b1 + b2 * b2;
    double btot2 = bn * bn + bperp2;
    double beta1, beta2;
    if (bperp2 > 1e-24 * (btot2 > 1.0 ? btot2 : 1.0)) {
        double bp = sqrt(bperp2);
        beta1 = b1 / bp;
        beta2 = b2 / bp;
    } else {
        beta1 = 1.0 / sqrt(2.0);
        beta2 = 1.0 / sqrt(2.0);
    }
    double alf, als;
    double bb2 = btot2 / rho;
    double t = bperp2 / rho;
    double dd = (a2 - ca2) * (a2 - ca2) + t * (2.0 * (a2 + ca2) + t);
    double D = sqrt(dd);
    if (D <= 1e-12 * (a2 + bb2)) {
        if (a2 >= ca2) { alf = 1.0; als = 0.0; }
        else           { alf = 0.0; als = 1.0; }
    } else {
        double x = 0.5 * (D + (a2 - ca2) - t);
        double y = 0.5 * (D - (a2 - ca2) + t);
        if (x >= y) y = a2 * t / x;
        else        x = a2 * t / y;
        alf = sqrt(x > 0.0 ? x / D : 0.0);
        als = sqrt(y > 0.0 ? y / D : 0.0);
    }
    double sgn = (bn >= 0.0) ? 1.0 : -1.0;
    double sr = sqrt(rho);

    lam[0] = u - cf;
    lam[1] = u - ca;
    lam[2] = u - cs;
    lam[3] = u;
    lam[4] = u + cs;
    lam[5] = u + ca;
    lam[6] = u + cf;

    /* right eigenvectors in primitive variables, RW[row*7 + wave] */
    double RW[49];
    memset(RW, 0, sizeof RW);
    for (int side = 0; side < 2; side++) {
        double sig = side == 0 ? -1.0 : 1.0;
        int f = side == 0 ? 0 : 6;   /* fast */
        int A = side == 0 ? 1 : 5;   /* Alfven */
        int s = side == 0 ? 2 : 4;   /* slow */
        RW[0 * 7 + f] = rho * alf;
        RW[1 * 7 + f] = sig * alf * cf;
        RW[2 * 7 + f] = -sig * als * cs * sgn * beta1;
        RW[3 * 7 + f] = -sig * als * cs * sgn * beta2;
        RW[4 * 7 + f] = als * a * sr * beta1;
        RW[5 * 7 + f] = als * a * sr * beta2;
        RW[6 * 7 + f] = rho * a2 * alf;

        RW[2 * 7 + A] = -beta2;
        RW[3 * 7 + A] = beta1;
        RW[4 * 7 + A] = sig * sgn * sr * beta2;
        RW[5 * 7 + A] = -sig * sgn * sr * beta1;

        RW[0 * 7 + s] = rho * als;
        RW[1 * 7 + s] = sig * als * cs;
        RW[2 * 7 + s] = sig * alf * cf * sgn * beta1;
        RW[3 * 7 + s] = sig * alf * cf * sgn * beta2;
        RW[4 * 7 + s] = -alf * a * sr * beta1;
        RW[5 * 7 + s] = -alf * a * sr * beta2;
        RW[6 * 7 + s] = rho * a2 * als;
    }
    RW[0 * 7 + 3] = 1.0;   /* entropy wave */

    /* dU/dW for U = (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) */
    double M[49];
    memset(M, 0, sizeof M);
    M[0 * 7 + 0] = 1.0;
    M[1 * 7 + 0] = u;   M[1 * 7 + 1] = rho;
    M[2 * 7 + 0] = v;   M[2 * 7 + 2] = rho;
    M[3 * 7 + 0] = w;   M[3 * 7 + 3] = rho;
    M[4 * 7 + 4] = 1.0;
    M[5 * 7 + 5] = 1.0;
    M[6 * 7 + 0] = 0.5 * (u * u + v * v + w * w);
    M[6 * 7 + 1] = rho * u;
    M[6 * 7 + 2] = rho * v;
    M[6 * 7 + 3] = rho * w;
    M[6 * 7 + 4] = b1;
    M[6 * 7 + 5] = b2;
    M[6 * 7 + 6] = 1.0 / (gamma - 1.0);

    for (int r = 0; r < 7; r++)
        for (int c = 0; c < 7; c++) {
            double acc = 0.0;
            for (int k = 0; k < 7; k++) acc += M[r * 7 + k] * RW[k * 7 + c];
            RU[r * 7 + c] = acc;
        }
    return invert(7, RU, LU);
}

/* indices of the seven characteristic variables inside the 8-vector */
static const int SYS[7] = {0, 1, 2, 3, 5, 6, 7};

/* Sec. 2.1, eq. FWENO, for one interface i+1/2 in the normal frame.
 * Us holds the six stencil cells i-2 .. i+3 (rotated conservative 8-vectors,
 * Us[k*8 + f]).  Steps, in the paper's order:
 *   1. physical fluxes F_k and primitives of the stencil cells;
 *   2. the interface state: arithmetic mean of the primitives of cells i and
 *      i+1 (the paper only says "Roe-type");
 *   3. eigen-system at that state (orc_eigen);
 *   4. projection of U_k and F_k on the left eigenvectors;
 *   5. local Lax-Friedrichs splitting g+- = (g +- alpha_s w)/2, alpha_s the
 *      largest |lambda_s| over the six cells and the interface state;
 *   6. differences of the split fluxes, Delta_{k+1/2} = g_{k+1} - g_k;
 *   7. F^s = -phi_N(D+_{i-3/2}, D+_{i-1/2}, D+_{i+1/2}, D+_{i+3/2})
 *            +phi_N(D-_{i+5/2}, D-_{i+3/2}, D-_{i+1/2}, D-_{i-1/2});
 *   8. back-projection with the right eigenvectors, added to the fourth-order
 *      central flux (-F_{i-1} + 7F_i + 7F_{i+1} - F_{i+2})/12, which is taken
 *      in physical variables (identical to projecting it, since R L = I).
 * Fhat[4] (normal B) is zero. */
void orc_interface_flux(const double Us[48], double gamma, double Fhat[8])
{
    orc_interface_flux_w(Us, gamma, 0, Fhat);
}

void orc_interface_flux_w(const double Us[48], double gamma, int weights, double Fhat[8])
{
    double (*phi)(double, double, double, double) = weights == 1 ? orc_phi_n_z : orc_phi_n;
    double W[6][8], F[6][8], lk[6][7];
    for (int k = 0; k < 6; k++) {
        orc_cons_to_prim(&Us[k * 8], gamma, W[k]);
        orc_flux_n(&Us[k * 8], gamma, F[k]);
        double cf, ca, cs;
        orc_wave_speeds(W[k], gamma, &cf, &ca, &cs);
        double u = W[k][1];
        lk[k][0] = u - cf;
        lk[k][1] = u - ca;
        lk[k][2] = u - cs;
        lk[k][3] = u;
        lk[k][4] = u + cs;
        lk[k][5] = u + ca;
        lk[k][6] = u + cf;
    }
    double Wm[8];
    for (int f = 0; f < 8; f++) Wm[f] = 0.5 * (W[2][f] + W[3][f]);
    double lam[7], RU[49], LU[49];
    orc_eigen(Wm, gamma, lam, RU, LU);

    double corr[7];
    for (int s = 0; s < 7; s++) {
        double alpha = fabs(lam[s]);
        for (int k = 0; k < 6; k++)
            if (fabs(lk[k][s]) > alpha) alpha = fabs(lk[k][s]);
        double gp[6], gm[6];
        for (int k = 0; k < 6; k++) {
            double wv = 0.0, gv = 0.0;
            for (int f = 0; f < 7; f++) {
                wv += LU[s * 7 + f] * Us[k * 8 + SYS[f]];
                gv += LU[s * 7 + f] * F[k][SYS[f]];
            }
            gp[k] = 0.5 * (gv + alpha * wv);
            gm[k] = 0.5 * (gv - alpha * wv);
        }
        double dp[5], dm[5];
        for (int j = 0; j < 5; j++) {
            dp[j] = gp[j + 1] - gp[j];
            dm[j] = gm[j + 1] - gm[j];
        }
        /* dp[0] is Delta_{i-3/2}, ..., dp[4] is Delta_{i+5/2} */
        corr[s] = -phi(dp[0], dp[1], dp[2], dp[3]) + phi(dm[4], dm[3], dm[2], dm[1]);
    }
    for (int f = 0; f < 7; f++) {
        int q = SYS[f];
        double central = (-F[1][q] + 7.0 * F[2][q] + 7.0 * F[3][q] - F[4][q]) / 12.0;
        double back = 0.0;
        for (int s = 0; s < 7; s++) back += RU[f * 7 + s] * corr[s];
        Fhat[q] = central + back;
    }
    Fhat[4] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */

#define IDX(g, i, j, k) ((((long)(k) * (g)->ny) + (j)) * (g)->nx + (i))

static long ncell(const orc_grid *g) { return (long)g->nx * g->ny * g->nz; }

/* Cell-centred B as the mean of the two faces (staggered mesh, Sec. 2.1). */
void orc_cell_b(const orc_grid *g, const double *bx, const double *by,
                const double *bz, double *U)
{
    long N = ncell(g);
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long c = IDX(g, i, j, k);
                U[4 * N + c] = 0.5 * (bx[c] + bx[IDX(g, wrapi(i + 1, g->nx), j, k)]);
                U[5 * N + c] = 0.5 * (by[c] + by[IDX(g, i, wrapi(j + 1, g->ny), k)]);
                U[6 * N + c] = 0.5 * (bz[c] + bz[IDX(g, i, j, wrapi(k + 1, g->nz))]);
            }
}

/* Sec. 2.2: one sweep along `axis` (0 x, 1 y, 2 z).  The stencil is gathered
 * into the frame (n, t1, t2) = (axis, axis+1, axis+2) mod 3 (the paper's
 * "rotation"), the interface flux is computed there and rotated back.
 * F[q*N + c] holds component q (global order) of the flux through the lower
 * face of cell c along axis, i.e. the interface (c - e_axis) + 1/2. */
void orc_face_fluxes(const orc_grid *g, const double *U, int axis, double *F)
{
    long N = ncell(g);
    int n = axis, t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
    int perm[8] = {0, 1 + n, 1 + t1, 1 + t2, 4 + n, 4 + t1, 4 + t2, 7};
    int dims[3] = {g->nx, g->ny, g->nz};
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                int pos[3] = {i, j, k};
                double Us[48], Fh[8];
                for (int m = 0; m < 6; m++) {
                    int q[3] = {pos[0], pos[1], pos[2]};
                    q[axis] = (int)wrapi(pos[axis] + m - 3, dims[axis]);
                    long c = IDX(g, q[0], q[1], q[2]);
                    for (int f = 0; f < 8; f++) Us[m * 8 + f] = U[perm[f] * N + c];
                }
                orc_interface_flux_w(Us, g->gamma, g->weights, Fh);
                long c = IDX(g, i, j, k);
                for (int f = 0; f < 8; f++) F[perm[f] * N + c] = Fh[f];
            }
}

/* Reference (cell-centred) electric field E = -v x B. */
static void cell_emf(const orc_grid *g, const double *U, long c, double e[3])
{
    long N = ncell(g);
    double rho = U[c];
    double u = U[N + c] / rho, v = U[2 * N + c] / rho, w = U[3 * N + c] / rho;
    double Bx = U[4 * N + c], By = U[5 * N + c], Bz = U[6 * N + c];
    e[0] = w * By - v * Bz;
    e[1] = u * Bz - w * Bx;
    e[2] = v * Bx - u * By;
}

/* Sec. 2.1, constrained transport on the staggered mesh.  Edge EMFs from the
 * upwind face fluxes of the magnetic field (E_z = -F_x(B_y) = F_y(B_x), and
 * cyclic).  emf_mode 0: E_edge = 1/2 (sum of the 4 face values)
 * - 1/4 (sum of the 4 cell values of -v x B), which equals the face value
 * exactly when the flow does not vary across it (so grid-aligned waves keep
 * the order of the flux); emf_mode 1: plain mean of the 4 face values.
 * Edge arrays: Ez[c] at (i-1/2, j-1/2, k), Ey[c] at (i-1/2, j, k-1/2),
 * Ex[c] at (i, j-1/2, k-1/2). */
static void edge_emfs(const orc_grid *g, const double *U, const double *Fx,
                      const double *Fy, const double *Fz,
                      double *Ex, double *Ey, double *Ez)
{
    long N = ncell(g);
    int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = IDX(g, i, j, k);
                int im = (int)wrapi(i - 1, nx), jm = (int)wrapi(j - 1, ny), km = (int)wrapi(k - 1, nz);
                double fz = -Fx[5 * N + IDX(g, i, jm, k)] - Fx[5 * N + c]
                          + Fy[4 * N + IDX(g, im, j, k)] + Fy[4 * N + c];
                double fy = Fx[6 * N + IDX(g, i, j, km)] + Fx[6 * N + c]
                          - Fz[4 * N + IDX(g, im, j, k)] - Fz[4 * N + c];
                double fx = -Fy[6 * N + IDX(g, i, j, km)] - Fy[6 * N + c]
                          + Fz[5 * N + IDX(g, i, jm, k)] + Fz[5 * N + c];
                if (g->emf_mode == 1) {
                    Ez[c] = 0.25 * fz;
                    Ey[c] = 0.25 * fy;
                    Ex[c] = 0.25 * fx;
                } else {
                    double e00[3], e10[3], e01[3], e11[3];
                    /* E_z edge: cells (i-1,j-1), (i,j-1), (i-1,j), (i,j) */
                    cell_emf(g, U, IDX(g, im, jm, k), e00);
                    cell_emf(g, U, IDX(g, i, jm, k), e10);
                    cell_emf(g, U, IDX(g, im, j, k), e01);
                    cell_emf(g, U, c, e11);
                    Ez[c] = 0.5 * fz - 0.25 * (e00[2] + e10[2] + e01[2] + e11[2]);
                    /* E_y edge: cells (i-1,k-1), (i,k-1), (i-1,k), (i,k) */
                    cell_emf(g, U, IDX(g, im, j, km), e00);
                    cell_emf(g, U, IDX(g, i, j, km), e10);
                    cell_emf(g, U, IDX(g, im, j, k), e01);
                    Ey[c] = 0.5 * fy - 0.25 * (e00[1] + e10[1] + e01[1] + e11[1]);
                    /* E_x edge: cells (j-1,k-1), (j,k-1), (j-1,k), (j,k) */
                    cell_emf(g, U, IDX(g, i, jm, km), e00);
                    cell_emf(g, U, IDX(g, i, j, km), e10);
                    cell_emf(g, U, IDX(g, i, jm, k), e01);
                    Ex[c] = 0.5 * fx - 0.25 * (e00[0] + e10[0] + e01[0] + e11[0]);
                }
            }
}

/* Semi-discrete operator L(U) (Sec. 2.2: sweeps in x, y, z, fluxes rotated
 * back, then the update).  LU[q*N + c] for q in {rho, mx, my, mz, E} is
 * -sum_d (F_d(c + e_d) - F_d(c)) / dx_d, accumulated in the order x, y, z;
 * the B rows of LU are zero because the field is evolved on the faces:
 * Lb[0..2] = -curl E at the bx, by, bz faces.  Fx, Fy, Fz (8*N each) receive
 * the face fluxes.  U must hold the cell B of the current faces. */
void orc_rhs(const orc_grid *g, const double *U, double *LU, double *Lb,
             double *Fx, double *Fy, double *Fz)
{
    long N = ncell(g);
    int nx = g->nx, ny = g->ny, nz = g->nz;
    orc_face_fluxes(g, U, 0, Fx);
    orc_face_fluxes(g, U, 1, Fy);
    orc_face_fluxes(g, U, 2, Fz);
    static const int CQ[5] = {0, 1, 2, 3, 7};
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = IDX(g, i, j, k);
                long cx = IDX(g, wrapi(i + 1, nx), j, k);
                long cy = IDX(g, i, wrapi(j + 1, ny), k);
                long cz = IDX(g, i, j, wrapi(k + 1, nz));
                for (int t = 0; t < 5; t++) {
                    int q = CQ[t];
                    double l = 0.0;
                    l -= (Fx[q * N + cx] - Fx[q * N + c]) / g->dx;
                    l -= (Fy[q * N + cy] - Fy[q * N + c]) / g->dy;
                    l -= (Fz[q * N + cz] - Fz[q * N + c]) / g->dz;
                    LU[q * N + c] = l;
                }
                LU[4 * N + c] = 0.0;
                LU[5 * N + c] = 0.0;
                LU[6 * N + c] = 0.0;
            }
    double *Ex = (double *)malloc(sizeof(double) * N);
    double *Ey = (double *)malloc(sizeof(double) * N);
    double *Ez = (double *)malloc(sizeof(double) * N);
    edge_emfs(g, U, Fx, Fy, Fz, Ex, Ey, Ez);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = IDX(g, i, j, k);
                long cx = IDX(g, wrapi(i + 1, nx), j, k);
                long cy = IDX(g, i, wrapi(j + 1, ny), k);
                long cz = IDX(g, i, j, wrapi(k + 1, nz));
                Lb[c]         = -((Ez[cy] - Ez[c]) / g->dy - (Ey[cz] - Ey[c]) / g->dz);
                Lb[N + c]     = -((Ex[cz] - Ex[c]) / g->dz - (Ez[cx] - Ez[c]) / g->dx);
                Lb[2 * N + c] = -((Ey[cx] - Ey[c]) / g->dx - (Ex[cy] - Ex[c]) / g->dy);
            }
    free(Ex);
    free(Ey);
    free(Ez);
}

/* One SSP-RK3 step in Shu-Osher form (the integrator the benchmark
 * configurations name; the paper itself uses classic RK4, see orc_rk4_step):
 *   U1 = Un + dt L(Un)
 *   U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
 *   Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2))
 * applied to (rho, m, E) and to the face fields; cell B follows the faces. */
void orc_ssprk3_step(const orc_grid *g, double dt, double *U,
                     double *bx, double *by, double *bz)
{
    long N = ncell(g);
    double *b[3] = {bx, by, bz};
    double *Uk = (double *)malloc(sizeof(double) * 8 * N);
    double *bk = (double *)malloc(sizeof(double) * 3 * N);
    double *L = (double *)malloc(sizeof(double) * 8 * N);
    double *Lb = (double *)malloc(sizeof(double) * 3 * N);
    double *F = (double *)malloc(sizeof(double) * 24 * N);
    static const int CQ[5] = {0, 1, 2, 3, 7};

    orc_cell_b(g, bx, by, bz, U);
    memcpy(Uk, U, sizeof(double) * 8 * N);
    for (int d = 0; d < 3; d++) memcpy(bk + d * N, b[d], sizeof(double) * N);

    for (int stage = 0; stage < 3; stage++) {
        orc_rhs(g, Uk, L, Lb, F, F + 8 * N, F + 16 * N);
        for (long c = 0; c < N; c++) {
            for (int t = 0; t < 5; t++) {
                long o = CQ[t] * N + c;
                if (stage == 0)      Uk[o] = U[o] + dt * L[o];
                else if (stage == 1) Uk[o] = 0.75 * U[o] + 0.25 * (Uk[o] + dt * L[o]);
                else                 Uk[o] = (1.0 / 3.0) * U[o] + (2.0 / 3.0) * (Uk[o] + dt * L[o]);
            }
            for (int d = 0; d < 3; d++) {
                long o = d * N + c;
                double bn = b[d][c];
                if (stage == 0)      bk[o] = bn + dt * Lb[o];
                else if (stage == 1) bk[o] = 0.75 * bn + 0.25 * (bk[o] + dt * Lb[o]);
                else                 bk[o] = (1.0 / 3.0) * bn + (2.0 / 3.0) * (bk[o] + dt * Lb[o]);
            }
        }
        orc_cell_b(g, bk, bk + N, bk + 2 * N, Uk);
    }
    memcpy(U, Uk, sizeof(double) * 8 * N);
    for (int d = 0; d < 3; d++) memcpy(b[d], bk + d * N, sizeof(double) * N);
    free(Uk); free(bk); free(L); free(Lb); free(F);
}

/* Sec. 2.1 "fourth order four-stage Runge Kutta": the classic scheme
 *   k1 = L(Un), k2 = L(Un + dt/2 k1), k3 = L(Un + dt/2 k2), k4 = L(Un + dt k3)
 *   Un+1 = Un + dt/6 (k1 + 2 k2 + 2 k3 + k4)
 * applied to (rho, m, E) and the face fields. */
void orc_rk4_step(const orc_grid *g, double dt, double *U,
                  double *bx, double *by, double *bz)
{
    long N = ncell(g);
    double *b[3] = {bx, by, bz};
    double *Us = (double *)malloc(sizeof(double) * 8 * N);
    double *bs = (double *)malloc(sizeof(double) * 3 * N);
    double *K = (double *)malloc(sizeof(double) * 8 * N * 4);
    double *Kb = (double *)malloc(sizeof(double) * 3 * N * 4);
    double *F = (double *)malloc(sizeof(double) * 24 * N);
    static const int CQ[5] = {0, 1, 2, 3, 7};
    static const double SUB[3] = {0.5, 0.5, 1.0};

    orc_cell_b(g, bx, by, bz, U);
    memcpy(Us, U, sizeof(double) * 8 * N);
    for (int d = 0; d < 3; d++) memcpy(bs + d * N, b[d], sizeof(double) * N);
    for (int stage = 0; stage < 4; stage++) {
        double *L = K + (long)stage * 8 * N;
        double *Lb = Kb + (long)stage * 3 * N;
        orc_rhs(g, Us, L, Lb, F, F + 8 * N, F + 16 * N);
        if (stage == 3) break;
        for (long c = 0; c < N; c++) {
            for (int t = 0; t < 5; t++) {
                long o = CQ[t] * N + c;
                Us[o] = U[o] + SUB[stage] * dt * L[o];
            }
            for (int d = 0; d < 3; d++) bs[d * N + c] = b[d][c] + SUB[stage] * dt * Lb[d * N + c];
        }
        orc_cell_b(g, bs, bs + N, bs + 2 * N, Us);
    }
    for (long c = 0; c < N; c++) {
        for (int t = 0; t < 5; t++) {
            long o = CQ[t] * N + c;
            double s = K[o] + 2.0 * K[8 * N + o] + 2.0 * K[16 * N + o] + K[24 * N + o];
            U[o] = U[o] + dt / 6.0 * s;
        }
        for (int d = 0; d < 3; d++) {
            long o = d * N + c;
            double s = Kb[o] + 2.0 * Kb[3 * N + o] + 2.0 * Kb[6 * N + o] + Kb[9 * N + o];
            b[d][c] = b[d][c] + dt / 6.0 * s;
        }
    }
    orc_cell_b(g, bx, by, bz, U);
    free(Us); free(bs); free(K); free(Kb); free(F);
}

/* CFL rule (not stated by the paper; reading): the largest over cells of
 * sum_d (|v_d| + c_f,d) / dx_d, with c_f,d the fast speed along axis d. */
double orc_cfl_speed(const orc_grid *g, const double *U)
{
    long N = ncell(g);
    double smax = 0.0;
    double dxs[3] = {g->dx, g->dy, g->dz};
#pragma omp parallel for reduction(max : smax) schedule(static)
    for (long c = 0; c < N; c++) {
        double Uc[8], W[8];
        for (int f = 0; f < 8; f++) Uc[f] = U[f * N + c];
        orc_cons_to_prim(Uc, g->gamma, W);
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
            double Wr[8] = {W[0], W[1 + d], W[1 + (d + 1) % 3], W[1 + (d + 2) % 3],
                            W[4 + d], W[4 + (d + 1) % 3], W[4 + (d + 2) % 3], W[7]};
            double cf, ca, cs;
            orc_wave_speeds(Wr, g->gamma, &cf, &ca, &cs);
            s += (fabs(Wr[1]) + cf) / dxs[d];
        }
        if (s > smax) smax = s;
    }
    return smax;
}

/* dt = C / max_cells sum_d (|v_d| + c_f,d) / dx_d. */
double orc_cfl_dt(const orc_grid *g, double cfl, const double *U)
{
    return cfl / orc_cfl_speed(g, U);
}

/* Conserved totals sum_cells U_q dV.  The sum over cells is compensated
 * (Neumaier 1974): the rounding error of every addition is recovered exactly
 * from the larger and the smaller operand and kept in a second double, which
 * is added back once at the end.  The result is within a few units in the
 * last place of the exact sum, and, being plain IEEE double arithmetic
 * without contraction, the same bits on every host. */
void orc_totals(const orc_grid *g, const double *U, double out[8])
{
    long N = ncell(g);
    double dV = g->dx * g->dy * g->dz;
    for (int q = 0; q < 8; q++) {
        double s = 0.0, comp = 0.0;
        for (long c = 0; c < N; c++) {
            double x = U[q * N + c];
            double t = s + x;
            if (fabs(s) >= fabs(x)) comp += (s - t) + x;
            else                    comp += (x - t) + s;
            s = t;
        }
        out[q] = (s + comp) * dV;
    }
}

/* Face-based divergence of b per cell. */
void orc_div_b(const orc_grid *g, const double *bx, const double *by,
               const double *bz, double *div)
{
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long c = IDX(g, i, j, k);
                div[c] = (bx[IDX(g, wrapi(i + 1, g->nx), j, k)] - bx[c]) / g->dx
                       + (by[IDX(g, i, wrapi(j + 1, g->ny), k)] - by[c]) / g->dy
                       + (bz[IDX(g, i, j, wrapi(k + 1, g->nz))] - bz[c]) / g->dz;
            }
}
