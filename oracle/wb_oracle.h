/*
 * wb_oracle.h -- plain FP64 CPU oracle of the WENO-Wombat MHD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA path (no header, no helper, no constant table).
 *
 * What it computes (Donnert et al. 2018, "Towards Exascale Simulations of the
 * ICM Dynamo with WENO-Wombat"):
 *   Sec. 2.1  ideal MHD, 8 conserved fields, characteristic (Roe-type)
 *             decomposition, Lax-Friedrichs splitting, fifth-order WENO flux
 *             (eq. FWENO), interpolant phi_N, Jiang-Shu nonlinear weights;
 *             constrained transport on a staggered mesh for the magnetic field.
 *   Sec. 2.2  dimension-by-dimension sweeps; fluxes rotated back before the
 *             update.
 * Readings of points the paper leaves open (averaged state, eigenvector
 * normalisation, degeneracy rules, LF speed, EMF averaging, CFL rule, SSP-RK3
 * integrator) are listed in the repository design notes; each function below
 * names the reading it follows.
 *
 * Layout: cell fields U[8][nz][ny][nx] (rho, mx, my, mz, Bx, By, Bz, E), x
 * fastest.  Face fields bx, by, bz [nz][ny][nx]: bx[k][j][i] sits on the face
 * (i-1/2, j, k), by[k][j][i] on (i, j-1/2, k), bz[k][j][i] on (i, j, k-1/2).
 * The domain is periodic in every direction.  Cell B is always the two-face
 * mean; the B entries of U are recomputed from the faces on every use.
 */
#ifndef WB_ORACLE_H
#define WB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double gamma;
    int emf_mode;   /* 0: 1-D-consistent EMF (twice the face mean minus the
                          cell mean), 1: plain mean of the four face EMFs   */
    int weights;    /* 0: Jiang-Shu nonlinear weights (Sec. 2.1),
                       1: WENO-Z weights (the alternative Sec. 2.1 names) */
} orc_grid;

/* --- point-wise pieces (Sec. 2.1) ---------------------------------------- */
double orc_phi_n(double a, double b, double c, double d);
double orc_phi_n_z(double a, double b, double c, double d);
void   orc_weno_weights_z(double a, double b, double c, double d,
                          double *w0, double *w1, double *w2);
void   orc_weno_weights(double a, double b, double c, double d,
                        double *w0, double *w1, double *w2);
void   orc_cons_to_prim(const double U[8], double gamma, double W[8]);
void   orc_prim_to_cons(const double W[8], double gamma, double U[8]);
void   orc_flux_n(const double U[8], double gamma, double F[8]);
void   orc_wave_speeds(const double W[8], double gamma,
                       double *cf, double *ca, double *cs);
int    orc_eigen(const double W[8], double gamma, double lam[7],
                 double RU[49], double LU[49]);
void   orc_interface_flux(const double Us[48], double gamma, double Fhat[8]);
void   orc_interface_flux_w(const double Us[48], double gamma, int weights, double Fhat[8]);

/* --- grid operators ------------------------------------------------------ */
void   orc_cell_b(const orc_grid *g, const double *bx, const double *by,
                  const double *bz, double *U);
void   orc_face_fluxes(const orc_grid *g, const double *U, int axis, double *F);
void   orc_rhs(const orc_grid *g, const double *U, double *LU, double *Lb,
               double *Fx, double *Fy, double *Fz);
void   orc_ssprk3_step(const orc_grid *g, double dt, double *U,
                       double *bx, double *by, double *bz);
void   orc_rk4_step(const orc_grid *g, double dt, double *U,
                    double *bx, double *by, double *bz);
double orc_cfl_speed(const orc_grid *g, const double *U);
double orc_cfl_dt(const orc_grid *g, double cfl, const double *U);
void   orc_totals(const orc_grid *g, const double *U, double out[8]);
void   orc_div_b(const orc_grid *g, const double *bx, const double *by,
                 const double *bz, double *div);
int    orc_num_threads(void);
void   orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
