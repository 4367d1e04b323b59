/*
 * Plain FP64 CPU oracle of the IB-LBM step (Jo, "Mechanism-Resolved Interface
 * Momentum Transfer in Immersed-Boundary Lattice Boltzmann Simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  This header and iblbm_oracle.c are the slow,
 * obviously-correct reference that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Units are lattice units throughout (dx = dt = 1, rho_f = 1), Sec. 2.1.
 * Populations are stored unshifted, one plane per direction:
 *   f[(i*ny + y)*nx + x],  i = 0..8,  D2Q9 numbering
 *   e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1)
 *   e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1).
 * The stored state between steps is the post-collision field (before streaming).
 */
#ifndef IBLBM_ORACLE_H
#define IBLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds per side (west, east, south, north) */
enum { ORC_PERIODIC = 0, ORC_VELOCITY = 1, ORC_NEUMANN = 2 };
/* collision operators, Sec. 2.2; ORC_STREAM_ONLY is the identity collision */
enum { ORC_BGK = 0, ORC_TRT = 1, ORC_CMMRT = 2, ORC_STREAM_ONLY = 3 };
/* delta kernels, Sec. 2.4 */
enum { ORC_HAT = 0, ORC_PESKIN4 = 1 };
/* boundary-enforcement schemes, Sec. 2.5 */
enum { ORC_DF = 0, ORC_MDF = 1, ORC_DFC = 2 };
/* body motion */
/* ORC_FREE_TRANSLATION: free in translation (Eq. 23), rotation held at rest (reading: the
 * paper calls the disks' rotational contribution negligible) */
enum { ORC_FIXED = 0, ORC_PRESCRIBED = 1, ORC_FREE = 2, ORC_FREE_TRANSLATION = 3 };

typedef struct {
    int nx, ny;
    int bc[4];          /* west, east, south, north */
    double ubc[4][2];   /* prescribed velocity per side (ORC_VELOCITY) */
    int collision;
    double tau;
    double trt_lambda;  /* TRT magic parameter Lambda_eo */
    double cm_sq, cm_se;/* CM-MRT third/fourth-order rates */
    double gfx, gfy;    /* uniform body-force density on the fluid (0 for IB cases) */
    int wall_closure;   /* 1: zero-velocity ORC_VELOCITY sides by on-node bounce-back */
} orc_lattice_params;

typedef struct {
    double xc, yc, radius, rho_ratio;
    int motion;
    double gx, gy;
    int internal_mass;          /* 0: scheme (A); 1: scheme (B-2), App. A.5 */
    int mdf_nmin, mdf_nmax;
    double mdf_tol, mdf_omega;  /* mdf_omega <= 0: 1/||A||_inf */
    double osc_amp, osc_period; /* prescribed x_c(t) = xc - A sin(2 pi t / T) */
} orc_body_params;

typedef struct orc_case orc_case;

orc_case* orc_create(const orc_lattice_params* p);
void      orc_destroy(orc_case* c);
int       orc_add_body(orc_case* c, const double* xy, int n, double ds, int kernel,
                       int scheme, const orc_body_params* bp);
void      orc_set_uniform(orc_case* c, double rho, double ux, double uy);
void      orc_set_populations(orc_case* c, const double* f);
void      orc_get_populations(const orc_case* c, double* f);
int       orc_step(orc_case* c, int nsteps);
/* rho, ux, uy used by the last collision (Eq. 4 velocity) */
void      orc_get_macro(const orc_case* c, double* rho, double* ux, double* uy);
void      orc_body_forces(const orc_case* c, int b, double out[3]);
void      orc_body_state(const orc_case* c, int b, double out[6]);
int       orc_force_history(const orc_case* c, int b, double* out, int cap);
/* per marker: X, Y, Udx, Udy, force x, force y, lambda (DFC) -> 7*n doubles */
void      orc_marker_data(const orc_case* c, int b, double* out);
void      orc_marker_stencils(const orc_case* c, int b, int* ij);
int       orc_mdf_iterations(const orc_case* c, int b);
double    orc_mdf_omega(const orc_case* c, int b);
double    orc_mdf_residual(const orc_case* c, int b);
/* coupled MDF path (two or more MDF bodies): relaxation factor when the last step's
 * iteration ended (omega_0 = min(0.8, omega_MDF of the bodies), halved per rejection) */
double    orc_mdf_omega_end(const orc_case* c, int b);

/* Fixed bodies: desired velocity of every marker (ud[2*n]) from the next step on,
 * or NULL for U_d = 0.  Returns 0, or 1 for a bad index or a moving body. */
int orc_set_marker_velocity(orc_case* c, int b, const double* ud);

/* Local boundary-fidelity diagnostics of Sec. 2.8 (with the bilinear probe of
 * Sec. 4.2) from node fields rho, ux, uy [ny*nx] and one body:
 *   md[7*n]   marker data as orc_marker_data writes it (X, Y, U_d, force, lambda)
 *   body[6]   centre xc, yc, rigid velocity vx, vy, omega, radius R
 * out[8]: mean and max over markers of |U(X_k) - U_d,k| / u_ref (U interpolated
 * with the body's kernel, Eq. 7); max of the same with a bilinear probe; net and
 * gross leakage sum_k rho(X_k) (U - U_d).n_k ds (resp. its absolute value) over
 * u_ref * n * ds; mean |u(x) - U_rigid(x)| / u_ref over nodes with
 * |x - X_c| < R - kappa, and their count; sum_k |F_k|.
 * pm[5*n] (may be NULL): per marker kernel slip, bilinear slip, (U - U_d).n_k /
 * u_ref, (rho_bilinear - 1) c_s^2, |F_k|.  Returns 0, or 1 if a stencil or probe
 * node lies outside the lattice. */
int orc_local_diagnostics_fields(int kernel, int nx, int ny, const double* rho, const double* ux,
                                 const double* uy, const double* md, int n, double ds,
                                 const double body[6], double u_ref, double kappa, double out[8],
                                 double* pm);
/* The same on the case's macro fields of the last collision and body b. */
int orc_local_diagnostics(const orc_case* c, int b, double u_ref, double kappa, double out[8],
                          double* pm);

/* primitives exposed for the pin tests */
double orc_phi(int kernel, double r);
void   orc_feq(double rho, double ux, double uy, double feq[9]);
void   orc_guo(double tau, double ux, double uy, double Fx, double Fy, double Fi[9]);
void   orc_collide_node(const orc_lattice_params* p, double f[9], double Fx, double Fy);
void   orc_interp(int kernel, int nx, int ny, const double* g, const double* xy, int n,
                  double* out);
void   orc_spread(int kernel, int nx, int ny, const double* Fk, const double* xy, int n,
                  double ds, double* out);
void   orc_dfc_lambda(int kernel, int nx, int ny, const double* xy, int n, double ds,
                      double* lambda);
double orc_mdf_norm_A(int kernel, int nx, int ny, const double* xy, int n, double ds);
void   orc_verlet_free_fall(double rho_ratio, double radius, double gx, double gy,
                            int internal_mass, int nsteps, double* out_v, double* out_x);

#ifdef __cplusplus
}
#endif
#endif
