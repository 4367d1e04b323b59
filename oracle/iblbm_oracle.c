/*
 * Plain FP64 CPU oracle of the IB-LBM step.  TEST INFRASTRUCTURE ONLY: it is
 * the reference the CUDA path is checked against and is never on the product
 * path.  Scalar loops, unshifted populations, two arrays (post-collision state
 * and post-streaming scratch), no blocking, no fusion.  Every function names
 * the equation of the paper it follows.  Where the paper is silent the reading
 * taken is stated beside the code.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add).  The three
 * whole-lattice node loops (streaming, moments, collision) carry OpenMP pragmas:
 * the tests build without -fopenmp (one thread, pragmas ignored); the all-cores
 * CPU baseline builds a second copy with it.  Every node is computed the same
 * way either way.
 */
#include "iblbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- D2Q9 lattice, Sec. 2.1 (Eq. 2 weights, c_s^2 = 1/3) ---------------- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
static const double PI = 3.14159265358979323846;

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

#define ORC_ERR_MARKER_OUT_OF_DOMAIN (-4)
#define ORC_MAX_COUPLED 64   /* MDF bodies of one lattice iterated together */

typedef struct {
    int n, kernel, scheme;
    double ds;
    orc_body_params p;
    double *X, *Y;      /* marker positions for the current step */
    double *r0x, *r0y;  /* marker offsets from the centre at theta = 0 */
    double *Udx, *Udy;  /* desired marker velocity */
    int ud_given;       /* fixed body whose U_d was set per marker (orc_set_marker_velocity) */
    double *Fx, *Fy;    /* DF/MDF: Lagrangian force F_L (MDF: F_total); DFC: F_s */
    double *lambda;     /* DFC scaling factor, Eq. 17 */
    /* rigid-body state, Sec. 2.7 */
    double xc, yc, vx, vy, om, theta;
    double Fhx, Fhy, Th;        /* hydrodynamic force / torque of the last step */
    double dFimx, dFimy;        /* internal-mass increment, Eq. A3 */
    double vhx, vhy, omh;       /* half-step velocities of the current step */
    double mdf_omega;
    int mdf_iters;
    double mdf_res;
    double mdf_omega_end;   /* coupled path: relaxation in use when the iteration ended */
    double* hist;
    int hist_n, hist_cap;
} orc_body;

struct orc_case {
    orc_lattice_params p;
    int nx, ny;
    long step;
    double* f;    /* post-collision state */
    double* fs;   /* post-streaming */
    double *rho, *uxr, *uyr;      /* raw moments of f* (no force) */
    double *Fx, *Fy;              /* Eulerian force density on the fluid, Eq. 8 */
    double* df;                   /* DFC correction field, Eq. 19 */
    double *mrho, *mux, *muy;     /* macro fields of the last collision */
    double *ucx, *ucy;            /* MDF working velocity u^(n) */
    orc_body* bodies;
    int nbodies;
};

static size_t IDX(const orc_case* c, int i, int x, int y) {
    return ((size_t)i * c->ny + y) * c->nx + x;
}

/* ---- Eq. 2: second-order equilibrium ------------------------------------ */
void orc_feq(double rho, double ux, double uy, double feq[9]) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = WT[i] * rho * (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* ---- Eq. 3 without its (1 - 1/2tau) prefactor --------------------------- */
static void guo_bracket(double ux, double uy, double Fx, double Fy, double S[9]) {
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double ax = (EX[i] - ux) / CS2 + eu * EX[i] / (CS2 * CS2);
        double ay = (EY[i] - uy) / CS2 + eu * EY[i] / (CS2 * CS2);
        S[i] = WT[i] * (ax * Fx + ay * Fy);
    }
}

/* ---- Eq. 3: Guo forcing term ------------------------------------------- */
void orc_guo(double tau, double ux, double uy, double Fx, double Fy, double Fi[9]) {
    double S[9];
    guo_bracket(ux, uy, Fx, Fy, S);
    for (int i = 0; i < 9; ++i) Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * S[i];
}

/* ---- Eq. 9 (hat) and Eq. 10 (Peskin 4-point) ----------------------------- */
double orc_phi(int kernel, double r) {
    double a = fabs(r);
    if (kernel == ORC_HAT) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* Footprint of one marker along one axis.  Reading: hat covers floor(X) and
 * floor(X)+1, Peskin 4-point floor(X)-1 .. floor(X)+2; these are exactly the
 * nodes with |x - X| < 1 (resp. < 2) plus a zero-weight node when X lies on a
 * node, so no node with non-zero weight is ever left out. */
static int stencil_origin(int kernel, double X, int* width) {
    int fl = (int)floor(X);
    *width = (kernel == ORC_HAT) ? 2 : 4;
    return (kernel == ORC_HAT) ? fl : fl - 1;
}

/* ---- Eq. 7: interpolation of a scalar node field to one marker ---------- */
static double interp_one(int kernel, int nx, const double* g, double X, double Y) {
    int w, i0 = stencil_origin(kernel, X, &w), j0 = stencil_origin(kernel, Y, &w);
    double acc = 0.0;
    for (int b = 0; b < w; ++b)
        for (int a = 0; a < w; ++a) {
            int x = i0 + a, y = j0 + b;
            double D = orc_phi(kernel, x - X) * orc_phi(kernel, y - Y);  /* Eq. 6, h = 1 */
            acc += g[(size_t)y * nx + x] * D;
        }
    return acc;
}

/* ---- Eq. 8: spreading of one marker value onto a node field ------------- */
static void spread_one(int kernel, int nx, double* out, double Fk, double X, double Y, double ds) {
    int w, i0 = stencil_origin(kernel, X, &w), j0 = stencil_origin(kernel, Y, &w);
    for (int b = 0; b < w; ++b)
        for (int a = 0; a < w; ++a) {
            int x = i0 + a, y = j0 + b;
            double D = orc_phi(kernel, x - X) * orc_phi(kernel, y - Y);
            out[(size_t)y * nx + x] += Fk * D * ds;
        }
}

static int stencil_inside(int kernel, int nx, int ny, double X, double Y) {
    int w, i0 = stencil_origin(kernel, X, &w), j0 = stencil_origin(kernel, Y, &w);
    return i0 >= 0 && j0 >= 0 && i0 + w <= nx && j0 + w <= ny;
}

void orc_interp(int kernel, int nx, int ny, const double* g, const double* xy, int n, double* out) {
    (void)ny;
    for (int k = 0; k < n; ++k) out[k] = interp_one(kernel, nx, g, xy[2 * k], xy[2 * k + 1]);
}

void orc_spread(int kernel, int nx, int ny, const double* Fk, const double* xy, int n, double ds,
                double* out) {
    memset(out, 0, sizeof(double) * (size_t)nx * ny);
    for (int k = 0; k < n; ++k) spread_one(kernel, nx, out, Fk[k], xy[2 * k], xy[2 * k + 1], ds);
}

/* ---- Eq. 17: lambda_k from W_total / W_sum (rho_f = 1) ------------------- */
void orc_dfc_lambda(int kernel, int nx, int ny, const double* xy, int n, double ds, double* lambda) {
    double* Wt = (double*)calloc((size_t)nx * ny, sizeof(double));
    /* W_total(x) = sum_k' D_h(x - X_k') */
    for (int k = 0; k < n; ++k) spread_one(kernel, nx, Wt, 1.0, xy[2 * k], xy[2 * k + 1], 1.0);
    for (int k = 0; k < n; ++k) {
        double Wsum = interp_one(kernel, nx, Wt, xy[2 * k], xy[2 * k + 1]);
        lambda[k] = 1.0 / (2.0 * 1.0 * ds * Wsum);
    }
    free(Wt);
}

/* ---- Sec. 2.5.2: ||A||_inf with A_lm = sum_x D(x-X_l) D(x-X_m) ds h^2 ----- */
double orc_mdf_norm_A(int kernel, int nx, int ny, const double* xy, int n, double ds) {
    (void)nx; (void)ny;
    double best = 0.0;
    for (int l = 0; l < n; ++l) {
        double Xl = xy[2 * l], Yl = xy[2 * l + 1];
        int w, i0 = stencil_origin(kernel, Xl, &w), j0 = stencil_origin(kernel, Yl, &w);
        double row = 0.0;
        for (int m = 0; m < n; ++m) {
            double Alm = 0.0;
            for (int b = 0; b < w; ++b)
                for (int a = 0; a < w; ++a) {
                    double x = i0 + a, y = j0 + b;
                    double Dl = orc_phi(kernel, x - Xl) * orc_phi(kernel, y - Yl);
                    double Dm = orc_phi(kernel, x - xy[2 * m]) * orc_phi(kernel, y - xy[2 * m + 1]);
                    Alm += Dl * Dm * ds;
                }
            row += fabs(Alm);
        }
        if (row > best) best = row;
    }
    return best;
}

/* ---- CM-MRT pieces, Eq. 5 ------------------------------------------------ */
/* moment order (k00,k10,k01,k20,k02,k11,k21,k12,k22) */
static const int MP[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MQ[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};

static double ipow(double v, int p) {
    double r = 1.0;
    for (int i = 0; i < p; ++i) r *= v;
    return r;
}

/* Solve A x = b (9x9) by Gaussian elimination with partial pivoting. */
static void solve9(double A[9][9], double b[9], double x[9]) {
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col) {
            for (int c2 = 0; c2 < 9; ++c2) {
                double t = A[col][c2]; A[col][c2] = A[piv][c2]; A[piv][c2] = t;
            }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < 9; ++r) {
            double m = A[r][col] / A[col][col];
            for (int c2 = col; c2 < 9; ++c2) A[r][c2] -= m * A[col][c2];
            b[r] -= m * b[col];
        }
    }
    for (int r = 8; r >= 0; --r) {
        double s = b[r];
        for (int c2 = r + 1; c2 < 9; ++c2) s -= A[r][c2] * x[c2];
        x[r] = s / A[r][r];
    }
}

/* ---- one-node collision: BGK (Eq. 1-3), TRT (Sec. 2.2), CM-MRT (Eq. 5) --- */
void orc_collide_node(const orc_lattice_params* p, double f[9], double Fx, double Fy) {
    if (p->collision == ORC_STREAM_ONLY) return;
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += f[i] * EX[i];
        jy += f[i] * EY[i];
    }
    /* Eq. 4: half-force velocity */
    double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
    double tau = p->tau;
    if (p->collision == ORC_BGK) {
        double feq[9], Fi[9];
        orc_feq(rho, ux, uy, feq);
        orc_guo(tau, ux, uy, Fx, Fy, Fi);
        for (int i = 0; i < 9; ++i) f[i] = f[i] - (f[i] - feq[i]) / tau + Fi[i];
        return;
    }
    if (p->collision == ORC_TRT) {
        /* Reading: s_e = 1/tau is the viscous (even) rate; s_o follows from
         * Lambda_eo = (1/s_e - 1/2)(1/s_o - 1/2). */
        double se = 1.0 / tau;
        double so = 1.0 / (0.5 + p->trt_lambda / (1.0 / se - 0.5));
        double feq[9], S[9], out[9];
        orc_feq(rho, ux, uy, feq);
        guo_bracket(ux, uy, Fx, Fy, S);
        for (int i = 0; i < 9; ++i) {
            int o = OPP[i];
            double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
            double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
            double Sp = 0.5 * (S[i] + S[o]), Sm = 0.5 * (S[i] - S[o]);
            out[i] = f[i] - se * (fp - ep) - so * (fm - em) + (1.0 - 0.5 * se) * Sp +
                     (1.0 - 0.5 * so) * Sm;
        }
        for (int i = 0; i < 9; ++i) f[i] = out[i];
        return;
    }
    /* CM-MRT.  Central moments k_pq = sum_i f_i (e_ix-u_x)^p (e_iy-u_y)^q.
     * Reading (the paper defers the forms to its ref. 38): equilibrium central
     * moments of the Maxwellian (rho,0,0,rho cs2,rho cs2,0,0,0,rho cs2^2) and
     * forcing central moments R = (0,Fx,Fy,0,0,0,cs2 Fy,cs2 Fx,0).  T(u) is
     * built from the monomials and inverted by an LU solve. */
    double T[9][9], k[9], keq[9], R[9], ks[9];
    for (int m = 0; m < 9; ++m)
        for (int i = 0; i < 9; ++i) T[m][i] = ipow(EX[i] - ux, MP[m]) * ipow(EY[i] - uy, MQ[m]);
    for (int m = 0; m < 9; ++m) {
        k[m] = 0.0;
        for (int i = 0; i < 9; ++i) k[m] += T[m][i] * f[i];
    }
    keq[0] = rho; keq[1] = 0.0; keq[2] = 0.0; keq[3] = rho * CS2; keq[4] = rho * CS2;
    keq[5] = 0.0; keq[6] = 0.0; keq[7] = 0.0; keq[8] = rho * CS2 * CS2;
    R[0] = 0.0; R[1] = Fx; R[2] = Fy; R[3] = 0.0; R[4] = 0.0; R[5] = 0.0;
    R[6] = CS2 * Fy; R[7] = CS2 * Fx; R[8] = 0.0;
    double om = 1.0 / tau;  /* omega = (nu/cs2 + 1/2)^-1 = 1/tau */
    double lam[9] = {0.0, 0.0, 0.0, om, om, om, p->cm_sq, p->cm_sq, p->cm_se};
    for (int m = 0; m < 9; ++m) ks[m] = (1.0 - lam[m]) * k[m] + lam[m] * keq[m] + (1.0 - 0.5 * lam[m]) * R[m];
    solve9(T, ks, f);
}

/* ---- domain boundary conditions (Sec. 2.9; readings stated) -------------- */
/* Zou-He velocity closures written out per side (textbook form, Zou and He). */
static void zou_he(int side, double f[9], double ux, double uy) {
    double rho;
    switch (side) {
    case SIDE_W:
        rho = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - ux);
        f[1] = f[3] + (2.0 / 3.0) * rho * ux;
        f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * ux + 0.5 * rho * uy;
        f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * ux - 0.5 * rho * uy;
        break;
    case SIDE_E:
        rho = (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / (1.0 + ux);
        f[3] = f[1] - (2.0 / 3.0) * rho * ux;
        f[7] = f[5] + 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * ux - 0.5 * rho * uy;
        f[6] = f[8] - 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * rho * ux + 0.5 * rho * uy;
        break;
    case SIDE_S:
        rho = (f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8])) / (1.0 - uy);
        f[2] = f[4] + (2.0 / 3.0) * rho * uy;
        f[5] = f[7] - 0.5 * (f[1] - f[3]) + 0.5 * rho * ux + (1.0 / 6.0) * rho * uy;
        f[6] = f[8] + 0.5 * (f[1] - f[3]) - 0.5 * rho * ux + (1.0 / 6.0) * rho * uy;
        break;
    default: /* SIDE_N */
        rho = (f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6])) / (1.0 + uy);
        f[4] = f[2] - (2.0 / 3.0) * rho * uy;
        f[7] = f[5] + 0.5 * (f[1] - f[3]) - 0.5 * rho * ux - (1.0 / 6.0) * rho * uy;
        f[8] = f[6] - 0.5 * (f[1] - f[3]) + 0.5 * rho * ux - (1.0 / 6.0) * rho * uy;
        break;
    }
}

/* A velocity side: the Zou-He closure, or (wall_closure = 1, zero wall velocity) the
 * populations pointing into the lattice equal to their opposites (on-node bounce-back):
 * W: 1, 5, 8 from 3, 7, 6;  E: 3, 7, 6 from 1, 5, 8;  S: 2, 5, 6 from 4, 7, 8;
 * N: 4, 7, 8 from 2, 5, 6. */
static void apply_velocity_side(const orc_case* c, int side, double f[9]) {
    const double ux = c->p.ubc[side][0], uy = c->p.ubc[side][1];
    if (c->p.wall_closure == 1 && ux == 0.0 && uy == 0.0) {
        switch (side) {
        case SIDE_W: f[1] = f[3]; f[5] = f[7]; f[8] = f[6]; break;
        case SIDE_E: f[3] = f[1]; f[7] = f[5]; f[6] = f[8]; break;
        case SIDE_S: f[2] = f[4]; f[5] = f[7]; f[6] = f[8]; break;
        default:     f[4] = f[2]; f[7] = f[5]; f[8] = f[6]; break;
        }
        return;
    }
    zou_he(side, f, ux, uy);
}

static void load9(const orc_case* c, const double* a, int x, int y, double v[9]) {
    for (int i = 0; i < 9; ++i) v[i] = a[IDX(c, i, x, y)];
}
static void store9(orc_case* c, double* a, int x, int y, const double v[9]) {
    for (int i = 0; i < 9; ++i) a[IDX(c, i, x, y)] = v[i];
}

/* Edges: Zou-He velocity, or zero-gradient copy of all nine post-streaming
 * populations from the adjacent interior node.  Corners (two non-periodic
 * sides): both zero-gradient -> copy all nine from the diagonal interior node;
 * otherwise equilibrium at the density of the diagonal interior node and the
 * prescribed velocity (the mean of both sides if both prescribe one). */
static void apply_bcs(orc_case* c) {
    const int nx = c->nx, ny = c->ny;
    const int* bc = c->p.bc;
    int xper = (bc[SIDE_W] == ORC_PERIODIC), yper = (bc[SIDE_S] == ORC_PERIODIC);
    int ylo = yper ? 0 : 1, yhi = yper ? ny - 1 : ny - 2;
    int xlo = xper ? 0 : 1, xhi = xper ? nx - 1 : nx - 2;
    double v[9];
    if (!xper) {
        for (int s = SIDE_W; s <= SIDE_E; ++s) {
            int x = (s == SIDE_W) ? 0 : nx - 1, xin = (s == SIDE_W) ? 1 : nx - 2;
            for (int y = ylo; y <= yhi; ++y) {
                if (bc[s] == ORC_NEUMANN) {
                    load9(c, c->fs, xin, y, v);
                } else {
                    load9(c, c->fs, x, y, v);
                    apply_velocity_side(c, s, v);
                }
                store9(c, c->fs, x, y, v);
            }
        }
    }
    if (!yper) {
        for (int s = SIDE_S; s <= SIDE_N; ++s) {
            int y = (s == SIDE_S) ? 0 : ny - 1, yin = (s == SIDE_S) ? 1 : ny - 2;
            for (int x = xlo; x <= xhi; ++x) {
                if (bc[s] == ORC_NEUMANN) {
                    load9(c, c->fs, x, yin, v);
                } else {
                    load9(c, c->fs, x, y, v);
                    apply_velocity_side(c, s, v);
                }
                store9(c, c->fs, x, y, v);
            }
        }
    }
    if (!xper && !yper) {
        for (int cx = 0; cx < 2; ++cx)
            for (int cy = 0; cy < 2; ++cy) {
                int sx = cx ? SIDE_E : SIDE_W, sy = cy ? SIDE_N : SIDE_S;
                int x = cx ? nx - 1 : 0, y = cy ? ny - 1 : 0;
                int xd = cx ? nx - 2 : 1, yd = cy ? ny - 2 : 1;
                load9(c, c->fs, xd, yd, v);
                if (!(bc[sx] == ORC_NEUMANN && bc[sy] == ORC_NEUMANN)) {
                    double rho = 0.0;
                    for (int i = 0; i < 9; ++i) rho += v[i];
                    double ux, uy;
                    if (bc[sx] == ORC_VELOCITY && bc[sy] == ORC_VELOCITY) {
                        ux = 0.5 * (c->p.ubc[sx][0] + c->p.ubc[sy][0]);
                        uy = 0.5 * (c->p.ubc[sx][1] + c->p.ubc[sy][1]);
                    } else if (bc[sx] == ORC_VELOCITY) {
                        ux = c->p.ubc[sx][0]; uy = c->p.ubc[sx][1];
                    } else {
                        ux = c->p.ubc[sy][0]; uy = c->p.ubc[sy][1];
                    }
                    orc_feq(rho, ux, uy, v);
                }
                store9(c, c->fs, x, y, v);
            }
    }
}

/* ---- streaming, Eq. 1 left-hand side (pull form of the same shift) ------- */
static void stream(orc_case* c) {
    const int nx = c->nx, ny = c->ny;
    int xper = (c->p.bc[SIDE_W] == ORC_PERIODIC), yper = (c->p.bc[SIDE_S] == ORC_PERIODIC);
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < 9; ++i)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int sx = x - EX[i], sy = y - EY[i];
                if (xper) sx = (sx + nx) % nx;
                if (yper) sy = (sy + ny) % ny;
                if (sx >= 0 && sx < nx && sy >= 0 && sy < ny)
                    c->fs[IDX(c, i, x, y)] = c->f[IDX(c, i, sx, sy)];
                else
                    c->fs[IDX(c, i, x, y)] = NAN; /* unknown: must be set by a BC */
            }
}

/* ---- case management ----------------------------------------------------- */
orc_case* orc_create(const orc_lattice_params* p) {
    if (p->nx < 3 || p->ny < 3) return NULL;
    if ((p->bc[SIDE_W] == ORC_PERIODIC) != (p->bc[SIDE_E] == ORC_PERIODIC)) return NULL;
    if ((p->bc[SIDE_S] == ORC_PERIODIC) != (p->bc[SIDE_N] == ORC_PERIODIC)) return NULL;
    orc_case* c = (orc_case*)calloc(1, sizeof(orc_case));
    c->p = *p;
    c->nx = p->nx;
    c->ny = p->ny;
    size_t N = (size_t)c->nx * c->ny;
    c->f = (double*)calloc(9 * N, sizeof(double));
    c->fs = (double*)calloc(9 * N, sizeof(double));
    c->df = (double*)calloc(9 * N, sizeof(double));
    c->rho = (double*)calloc(N, sizeof(double));
    c->uxr = (double*)calloc(N, sizeof(double));
    c->uyr = (double*)calloc(N, sizeof(double));
    c->Fx = (double*)calloc(N, sizeof(double));
    c->Fy = (double*)calloc(N, sizeof(double));
    c->mrho = (double*)calloc(N, sizeof(double));
    c->mux = (double*)calloc(N, sizeof(double));
    c->muy = (double*)calloc(N, sizeof(double));
    c->ucx = (double*)calloc(N, sizeof(double));
    c->ucy = (double*)calloc(N, sizeof(double));
    orc_set_uniform(c, 1.0, 0.0, 0.0);
    return c;
}

void orc_destroy(orc_case* c) {
    if (!c) return;
    for (int b = 0; b < c->nbodies; ++b) {
        orc_body* B = &c->bodies[b];
        free(B->X); free(B->Y); free(B->r0x); free(B->r0y); free(B->Udx); free(B->Udy);
        free(B->Fx); free(B->Fy); free(B->lambda); free(B->hist);
    }
    free(c->bodies);
    free(c->f); free(c->fs); free(c->df); free(c->rho); free(c->uxr); free(c->uyr);
    free(c->Fx); free(c->Fy); free(c->mrho); free(c->mux); free(c->muy); free(c->ucx); free(c->ucy);
    free(c);
}

void orc_set_uniform(orc_case* c, double rho, double ux, double uy) {
    double feq[9];
    orc_feq(rho, ux, uy, feq);
    for (int i = 0; i < 9; ++i)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) c->f[IDX(c, i, x, y)] = feq[i];
}

void orc_set_populations(orc_case* c, const double* f) {
    memcpy(c->f, f, sizeof(double) * 9 * (size_t)c->nx * c->ny);
}

void orc_get_populations(const orc_case* c, double* f) {
    memcpy(f, c->f, sizeof(double) * 9 * (size_t)c->nx * c->ny);
}

void orc_get_macro(const orc_case* c, double* rho, double* ux, double* uy) {
    size_t N = (size_t)c->nx * c->ny;
    memcpy(rho, c->mrho, sizeof(double) * N);
    memcpy(ux, c->mux, sizeof(double) * N);
    memcpy(uy, c->muy, sizeof(double) * N);
}

int orc_add_body(orc_case* c, const double* xy, int n, double ds, int kernel, int scheme,
                 const orc_body_params* bp) {
    if (n <= 0 || ds <= 0.0) return -1;
    for (int k = 0; k < n; ++k)
        if (!stencil_inside(kernel, c->nx, c->ny, xy[2 * k], xy[2 * k + 1]))
            return ORC_ERR_MARKER_OUT_OF_DOMAIN;
    c->bodies = (orc_body*)realloc(c->bodies, sizeof(orc_body) * (size_t)(c->nbodies + 1));
    orc_body* B = &c->bodies[c->nbodies];
    memset(B, 0, sizeof(*B));
    B->n = n; B->kernel = kernel; B->scheme = scheme; B->ds = ds; B->p = *bp;
    B->X = (double*)malloc(sizeof(double) * n);
    B->Y = (double*)malloc(sizeof(double) * n);
    B->r0x = (double*)malloc(sizeof(double) * n);
    B->r0y = (double*)malloc(sizeof(double) * n);
    B->Udx = (double*)calloc(n, sizeof(double));
    B->Udy = (double*)calloc(n, sizeof(double));
    B->Fx = (double*)calloc(n, sizeof(double));
    B->Fy = (double*)calloc(n, sizeof(double));
    B->lambda = (double*)calloc(n, sizeof(double));
    for (int k = 0; k < n; ++k) {
        B->X[k] = xy[2 * k];
        B->Y[k] = xy[2 * k + 1];
        B->r0x[k] = xy[2 * k] - bp->xc;
        B->r0y[k] = xy[2 * k + 1] - bp->yc;
    }
    B->xc = bp->xc; B->yc = bp->yc;
    if (scheme == ORC_MDF) {
        B->mdf_omega = bp->mdf_omega > 0.0 ? bp->mdf_omega
                                           : 1.0 / orc_mdf_norm_A(kernel, c->nx, c->ny, xy, n, ds);
    }
    c->nbodies++;
    return c->nbodies - 1;
}

/* Sec. 2.7 masses: m_s = rho_s pi r^2, I_s = m_s r^2 / 2, m_f = rho_f pi r^2 */
static double body_ms(const orc_body* B) { return B->p.rho_ratio * PI * B->p.radius * B->p.radius; }
static double body_mf(const orc_body* B) { return PI * B->p.radius * B->p.radius; }

/* Marker positions and desired velocities for the step about to run.
 * FREE: first half of Eq. 23 (half kick with F_total^n, drift), torque-only
 * rotation; markers follow the rigid motion.  U_d = v + Omega x (X - X_c)
 * evaluated at the half-step velocities.  PRESCRIBED: x_c(t) at t = n+1. */
static void prepare_body(orc_case* c, orc_body* B) {
    if (B->p.motion == ORC_FREE || B->p.motion == ORC_FREE_TRANSLATION) {
        double ms = body_ms(B), Is = 0.5 * ms * B->p.radius * B->p.radius;
        double dm = (B->p.rho_ratio - 1.0) * PI * B->p.radius * B->p.radius;  /* Eq. 22 */
        double Ftx = B->Fhx + dm * B->p.gx + B->dFimx, Fty = B->Fhy + dm * B->p.gy + B->dFimy;
        B->vhx = B->vx + Ftx / (2.0 * ms);
        B->vhy = B->vy + Fty / (2.0 * ms);
        B->omh = B->p.motion == ORC_FREE ? B->om + B->Th / (2.0 * Is) : 0.0;
        B->xc += B->vhx;
        B->yc += B->vhy;
        B->theta += B->omh;
        double ct = cos(B->theta), st = sin(B->theta);
        for (int k = 0; k < B->n; ++k) {
            double rx = ct * B->r0x[k] - st * B->r0y[k], ry = st * B->r0x[k] + ct * B->r0y[k];
            B->X[k] = B->xc + rx;
            B->Y[k] = B->yc + ry;
            B->Udx[k] = B->vhx - B->omh * ry;
            B->Udy[k] = B->vhy + B->omh * rx;
        }
    } else if (B->p.motion == ORC_PRESCRIBED) {
        double t = (double)(c->step + 1);
        double w = 2.0 * PI / B->p.osc_period;
        double xc = B->p.xc - B->p.osc_amp * sin(w * t);
        double vx = -B->p.osc_amp * w * cos(w * t);
        B->xc = xc;
        B->vx = vx;
        for (int k = 0; k < B->n; ++k) {
            B->X[k] = xc + B->r0x[k];
            B->Y[k] = B->p.yc + B->r0y[k];
            B->Udx[k] = vx;
            B->Udy[k] = 0.0;
        }
    } else if (!B->ud_given) {
        for (int k = 0; k < B->n; ++k) { B->Udx[k] = 0.0; B->Udy[k] = 0.0; }
    }
}

/* Desired velocity per marker of a fixed body (App. D.1 drives the markers with
 * the analytical Taylor-Green field); NULL returns to U_d = 0. */
int orc_set_marker_velocity(orc_case* c, int b, const double* ud) {
    if (b < 0 || b >= c->nbodies) return 1;
    orc_body* B = &c->bodies[b];
    if (B->p.motion != ORC_FIXED) return 1;
    B->ud_given = ud != NULL;
    for (int k = 0; k < B->n; ++k) {
        B->Udx[k] = ud ? ud[2 * k] : 0.0;
        B->Udy[k] = ud ? ud[2 * k + 1] : 0.0;
    }
    return 0;
}

/* Second half of Eq. 23 and the internal-mass increment of Eq. A3. */
static void finish_body(orc_body* B, double Fhx, double Fhy, double Th) {
    if (B->p.motion == ORC_FREE || B->p.motion == ORC_FREE_TRANSLATION) {
        double ms = body_ms(B), Is = 0.5 * ms * B->p.radius * B->p.radius;
        double dm = (B->p.rho_ratio - 1.0) * PI * B->p.radius * B->p.radius;
        double vnx = B->vhx + (Fhx + dm * B->p.gx + B->dFimx) / (2.0 * ms);
        double vny = B->vhy + (Fhy + dm * B->p.gy + B->dFimy) / (2.0 * ms);
        double omn = B->p.motion == ORC_FREE ? B->omh + Th / (2.0 * Is) : 0.0;
        if (B->p.internal_mass) {
            B->dFimx = body_mf(B) * (vnx - B->vx);
            B->dFimy = body_mf(B) * (vny - B->vy);
        } else {
            B->dFimx = 0.0;
            B->dFimy = 0.0;
        }
        B->vx = vnx; B->vy = vny; B->om = omn;
    }
    B->Fhx = Fhx; B->Fhy = Fhy; B->Th = Th;
    if (B->hist_n == B->hist_cap) {
        B->hist_cap = B->hist_cap ? 2 * B->hist_cap : 1024;
        B->hist = (double*)realloc(B->hist, sizeof(double) * 3 * (size_t)B->hist_cap);
    }
    B->hist[3 * B->hist_n + 0] = Fhx;
    B->hist[3 * B->hist_n + 1] = Fhy;
    B->hist[3 * B->hist_n + 2] = Th;
    B->hist_n++;
}

/* ---- IB stage of one body (Sec. 2.5) ------------------------------------ */
static void ib_df(orc_case* c, orc_body* B) {
    /* Eq. 7 on rho and on u_raw (no force yet), Eq. 11, Eq. 8 */
    for (int k = 0; k < B->n; ++k) {
        double rk = interp_one(B->kernel, c->nx, c->rho, B->X[k], B->Y[k]);
        double Ux = interp_one(B->kernel, c->nx, c->uxr, B->X[k], B->Y[k]);
        double Uy = interp_one(B->kernel, c->nx, c->uyr, B->X[k], B->Y[k]);
        B->Fx[k] = 2.0 * rk * (B->Udx[k] - Ux);
        B->Fy[k] = 2.0 * rk * (B->Udy[k] - Uy);
    }
    for (int k = 0; k < B->n; ++k) {
        spread_one(B->kernel, c->nx, c->Fx, B->Fx[k], B->X[k], B->Y[k], B->ds);
        spread_one(B->kernel, c->nx, c->Fy, B->Fy[k], B->X[k], B->Y[k], B->ds);
    }
}

/* Eqs. 12-14 with omega_MDF ~ 1/||A||_inf, L_inf slip stop and the 1.5x guard.
 * Readings: at least N_min increments are applied before the tolerance may
 * stop the loop; tolerance and guard are tested on U^(n) before increment n
 * is applied, and a diverging iterate is not applied; rho(x) and rho(X_k) stay
 * frozen over the iterations (Eq. 14 leaves density unchanged). */
static void ib_mdf(orc_case* c, orc_body* B) {
    size_t N = (size_t)c->nx * c->ny;
    memcpy(c->ucx, c->uxr, sizeof(double) * N);
    memcpy(c->ucy, c->uyr, sizeof(double) * N);
    int n = B->n;
    double* rk = (double*)malloc(sizeof(double) * n);
    double* Fnx = (double*)malloc(sizeof(double) * n);
    double* Fny = (double*)malloc(sizeof(double) * n);
    double* sx = (double*)malloc(sizeof(double) * N);
    double* sy = (double*)malloc(sizeof(double) * N);
    for (int k = 0; k < n; ++k) {
        rk[k] = interp_one(B->kernel, c->nx, c->rho, B->X[k], B->Y[k]);
        B->Fx[k] = 0.0;
        B->Fy[k] = 0.0;
    }
    double om = B->mdf_omega, rprev = 0.0, r = 0.0;
    int applied = 0;
    for (int it = 1; it <= B->p.mdf_nmax; ++it) {
        r = 0.0;
        for (int k = 0; k < n; ++k) {
            double Ux = interp_one(B->kernel, c->nx, c->ucx, B->X[k], B->Y[k]);
            double Uy = interp_one(B->kernel, c->nx, c->ucy, B->X[k], B->Y[k]);
            double dx = B->Udx[k] - Ux, dy = B->Udy[k] - Uy;
            double e = sqrt(dx * dx + dy * dy);
            if (e > r) r = e;
            Fnx[k] = 2.0 * rk[k] * dx;  /* Eq. 13 */
            Fny[k] = 2.0 * rk[k] * dy;
        }
        if (applied >= B->p.mdf_nmin && r < B->p.mdf_tol) break;
        if (it >= 2 && r > 1.5 * rprev) break;
        memset(sx, 0, sizeof(double) * N);
        memset(sy, 0, sizeof(double) * N);
        for (int k = 0; k < n; ++k) {
            spread_one(B->kernel, c->nx, sx, Fnx[k], B->X[k], B->Y[k], B->ds);
            spread_one(B->kernel, c->nx, sy, Fny[k], B->X[k], B->Y[k], B->ds);
        }
        for (size_t q = 0; q < N; ++q) {  /* Eq. 14 (applied on the footprint; zero elsewhere) */
            c->ucx[q] += om / (2.0 * c->rho[q]) * sx[q];
            c->ucy[q] += om / (2.0 * c->rho[q]) * sy[q];
        }
        for (int k = 0; k < n; ++k) {
            B->Fx[k] += om * Fnx[k];
            B->Fy[k] += om * Fny[k];
        }
        rprev = r;
        applied++;
    }
    B->mdf_iters = applied;
    B->mdf_res = r;
    for (int k = 0; k < n; ++k) {
        spread_one(B->kernel, c->nx, c->Fx, B->Fx[k], B->X[k], B->Y[k], B->ds);
        spread_one(B->kernel, c->nx, c->Fy, B->Fy[k], B->X[k], B->Y[k], B->ds);
    }
    free(rk); free(Fnx); free(Fny); free(sx); free(sy);
}

/* Residual of Eq. 12-13 at every marker of the coupled bodies for the iterate (ux, uy):
 * r = max_k |U_d,k - U(X_k)|_2 over all of them, and F = 2 rho_k (U_d,k - U(X_k)). */
static double coupled_residual(orc_case* c, orc_body** Bs, int nb, const double* ux, const double* uy,
                               double** rk, double** Fx, double** Fy) {
    double r = 0.0;
    for (int b = 0; b < nb; ++b) {
        orc_body* B = Bs[b];
        for (int k = 0; k < B->n; ++k) {
            double Ux = interp_one(B->kernel, c->nx, ux, B->X[k], B->Y[k]);
            double Uy = interp_one(B->kernel, c->nx, uy, B->X[k], B->Y[k]);
            double dx = B->Udx[k] - Ux, dy = B->Udy[k] - Uy;
            double e = sqrt(dx * dx + dy * dy);
            if (e > r) r = e;
            Fx[b][k] = 2.0 * rk[b][k] * dx;
            Fy[b][k] = 2.0 * rk[b][k] * dy;
        }
    }
    return r;
}

/* Sec. 2.5.2, coupled path (two or more MDF bodies in one lattice): the bodies' marker
 * forces share one fluid update per iteration, u^(n) = u^(n-1) + omega/(2 rho) sum_b
 * spread_b(F_b^(n)), and one L_inf residual over all their markers decides.  The
 * relaxation starts at omega_0 = min(0.8, omega_MDF of every body); a trial iteration
 * whose residual exceeds 1.2 times the residual of the iterate it started from is
 * rejected (the iterate is kept) and omega halved, and the iteration ends once omega
 * has come down to 0.125 omega_0.  Readings: every trial counts as one of the N_max
 * iterations; at least N_min accepted increments come before the tolerance may stop
 * the loop; N_min, N_max and tol are those of the first MDF body. */
static void ib_mdf_coupled(orc_case* c, orc_body** Bs, int nb) {
    size_t N = (size_t)c->nx * c->ny;
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* tx = (double*)malloc(sizeof(double) * N);
    double* ty = (double*)malloc(sizeof(double) * N);
    double* sx = (double*)malloc(sizeof(double) * N);
    double* sy = (double*)malloc(sizeof(double) * N);
    memcpy(ux, c->uxr, sizeof(double) * N);   /* u^(0): post-streaming velocity */
    memcpy(uy, c->uyr, sizeof(double) * N);
    double *rk[ORC_MAX_COUPLED], *Fx[ORC_MAX_COUPLED], *Fy[ORC_MAX_COUPLED], *Gx[ORC_MAX_COUPLED],
        *Gy[ORC_MAX_COUPLED];
    double om0 = 0.8;
    for (int b = 0; b < nb; ++b) {
        orc_body* B = Bs[b];
        rk[b] = (double*)malloc(sizeof(double) * B->n);
        Fx[b] = (double*)malloc(sizeof(double) * B->n);
        Fy[b] = (double*)malloc(sizeof(double) * B->n);
        Gx[b] = (double*)malloc(sizeof(double) * B->n);
        Gy[b] = (double*)malloc(sizeof(double) * B->n);
        for (int k = 0; k < B->n; ++k) {
            rk[b][k] = interp_one(B->kernel, c->nx, c->rho, B->X[k], B->Y[k]);
            B->Fx[k] = 0.0;
            B->Fy[k] = 0.0;
        }
        if (B->mdf_omega < om0) om0 = B->mdf_omega;
    }
    const int nmin = Bs[0]->p.mdf_nmin, nmax = Bs[0]->p.mdf_nmax;
    const double tol = Bs[0]->p.mdf_tol;
    double om = om0;
    double ra = coupled_residual(c, Bs, nb, ux, uy, rk, Fx, Fy);
    int applied = 0, trials = 0;
    for (;;) {
        if (applied >= nmin && ra < tol) break;
        if (trials >= nmax) break;
        /* trial iterate from the accepted one (Eq. 14 with the shared update) */
        memset(sx, 0, sizeof(double) * N);
        memset(sy, 0, sizeof(double) * N);
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < Bs[b]->n; ++k) {
                spread_one(Bs[b]->kernel, c->nx, sx, Fx[b][k], Bs[b]->X[k], Bs[b]->Y[k], Bs[b]->ds);
                spread_one(Bs[b]->kernel, c->nx, sy, Fy[b][k], Bs[b]->X[k], Bs[b]->Y[k], Bs[b]->ds);
            }
        for (size_t q = 0; q < N; ++q) {
            tx[q] = ux[q] + om / (2.0 * c->rho[q]) * sx[q];
            ty[q] = uy[q] + om / (2.0 * c->rho[q]) * sy[q];
        }
        ++trials;
        double rt = coupled_residual(c, Bs, nb, tx, ty, rk, Gx, Gy);
        if (rt > 1.2 * ra) {          /* rejected: keep the iterate, halve the relaxation */
            om *= 0.5;
            if (om <= 0.125 * om0) break;
            continue;
        }
        for (int b = 0; b < nb; ++b)  /* accepted */
            for (int k = 0; k < Bs[b]->n; ++k) {
                Bs[b]->Fx[k] += om * Fx[b][k];
                Bs[b]->Fy[k] += om * Fy[b][k];
                Fx[b][k] = Gx[b][k];
                Fy[b][k] = Gy[b][k];
            }
        memcpy(ux, tx, sizeof(double) * N);
        memcpy(uy, ty, sizeof(double) * N);
        ra = rt;
        ++applied;
    }
    for (int b = 0; b < nb; ++b) {
        orc_body* B = Bs[b];
        B->mdf_iters = trials;
        B->mdf_res = ra;
        B->mdf_omega_end = om;
        for (int k = 0; k < B->n; ++k) {
            spread_one(B->kernel, c->nx, c->Fx, B->Fx[k], B->X[k], B->Y[k], B->ds);
            spread_one(B->kernel, c->nx, c->Fy, B->Fy[k], B->X[k], B->Y[k], B->ds);
        }
        free(rk[b]); free(Fx[b]); free(Fy[b]); free(Gx[b]); free(Gy[b]);
    }
    free(ux); free(uy); free(tx); free(ty); free(sx); free(sy);
}

/* Eq. 17 across every DFC marker of the case: W_total sums over all of them. */
static void dfc_lambdas(orc_case* c) {
    size_t N = (size_t)c->nx * c->ny;
    double* Wt = (double*)calloc(N, sizeof(double));
    int any = 0;
    for (int b = 0; b < c->nbodies; ++b) {
        orc_body* B = &c->bodies[b];
        if (B->scheme != ORC_DFC) continue;
        any = 1;
        for (int k = 0; k < B->n; ++k) spread_one(B->kernel, c->nx, Wt, 1.0, B->X[k], B->Y[k], 1.0);
    }
    if (any)
        for (int b = 0; b < c->nbodies; ++b) {
            orc_body* B = &c->bodies[b];
            if (B->scheme != ORC_DFC) continue;
            for (int k = 0; k < B->n; ++k) {
                double Wsum = interp_one(B->kernel, c->nx, Wt, B->X[k], B->Y[k]);
                B->lambda[k] = 1.0 / (2.0 * 1.0 * B->ds * Wsum);
            }
        }
    free(Wt);
}

/* Eqs. 15, 16, 18, 19, 20 (rho_f = 1, cs2 = 1/3 so 2 w_i/cs2 = 6 w_i). */
static void ib_dfc(orc_case* c, orc_body* B) {
    double fst[9], fbar[9], dfk[9];
    size_t N = (size_t)c->nx * c->ny;
    for (int k = 0; k < B->n; ++k) {
        for (int i = 0; i < 9; ++i)
            fst[i] = interp_one(B->kernel, c->nx, c->fs + (size_t)i * N, B->X[k], B->Y[k]);
        double Fsx = 0.0, Fsy = 0.0;
        for (int i = 0; i < 9; ++i) {
            fbar[i] = fst[OPP[i]] + 2.0 * WT[i] * 1.0 * (EX[i] * B->Udx[k] + EY[i] * B->Udy[k]) / CS2;
            dfk[i] = B->lambda[k] * (fbar[i] - fst[i]);
            Fsx += EX[i] * dfk[i];
            Fsy += EY[i] * dfk[i];
        }
        B->Fx[k] = -B->ds * Fsx;
        B->Fy[k] = -B->ds * Fsy;
        for (int i = 0; i < 9; ++i)
            spread_one(B->kernel, c->nx, c->df + (size_t)i * N, dfk[i], B->X[k], B->Y[k], B->ds);
    }
}

/* Per-body force and torque on the body, Sec. 2.7:
 * DF/MDF F_h = -sum_k F_L ds, T = -sum_k (X_k - X_c) x F_L ds;
 * DFC    F_h =  sum_k F_s,    T =  sum_k (X_k - X_c) x F_s. */
static void body_force(const orc_body* B, double* Fhx, double* Fhy, double* Th) {
    double fx = 0.0, fy = 0.0, t = 0.0;
    for (int k = 0; k < B->n; ++k) {
        double rx = B->X[k] - B->xc, ry = B->Y[k] - B->yc;
        double gx, gy;
        if (B->scheme == ORC_DFC) { gx = B->Fx[k]; gy = B->Fy[k]; }
        else { gx = -B->Fx[k] * B->ds; gy = -B->Fy[k] * B->ds; }
        fx += gx;
        fy += gy;
        t += rx * gy - ry * gx;
    }
    *Fhx = fx; *Fhy = fy; *Th = t;
}

static int step_once(orc_case* c) {
    const int nx = c->nx, ny = c->ny;
    size_t N = (size_t)nx * ny;
    for (int b = 0; b < c->nbodies; ++b) {
        prepare_body(c, &c->bodies[b]);
        orc_body* B = &c->bodies[b];
        for (int k = 0; k < B->n; ++k)
            if (!stencil_inside(B->kernel, nx, ny, B->X[k], B->Y[k])) return ORC_ERR_MARKER_OUT_OF_DOMAIN;
    }
    stream(c);
    apply_bcs(c);
#pragma omp parallel for schedule(static)
    for (size_t q = 0; q < N; ++q) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            double v = c->fs[(size_t)i * N + q];
            r += v;
            jx += v * EX[i];
            jy += v * EY[i];
        }
        c->rho[q] = r;
        c->uxr[q] = jx / r;
        c->uyr[q] = jy / r;
    }
    for (size_t q = 0; q < N; ++q) {
        c->Fx[q] = c->p.gfx;
        c->Fy[q] = c->p.gfy;
    }
    memset(c->df, 0, sizeof(double) * 9 * N);
    int any_dfc = 0;
    for (int b = 0; b < c->nbodies; ++b) any_dfc |= (c->bodies[b].scheme == ORC_DFC);
    if (any_dfc) dfc_lambdas(c);
    orc_body* coupled[ORC_MAX_COUPLED];
    int nmdf = 0;
    for (int b = 0; b < c->nbodies; ++b)
        if (c->bodies[b].scheme == ORC_MDF && nmdf < ORC_MAX_COUPLED) coupled[nmdf++] = &c->bodies[b];
    for (int b = 0; b < c->nbodies; ++b) {
        orc_body* B = &c->bodies[b];
        if (B->scheme == ORC_DF) ib_df(c, B);
        else if (B->scheme == ORC_MDF) { if (nmdf == 1) ib_mdf(c, B); }
        else ib_dfc(c, B);
    }
    if (nmdf >= 2) ib_mdf_coupled(c, coupled, nmdf);
#pragma omp parallel for collapse(2) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t q = (size_t)y * nx + x;
            double v[9];
            for (int i = 0; i < 9; ++i) v[i] = c->fs[(size_t)i * N + q] + c->df[(size_t)i * N + q];
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) { r += v[i]; jx += v[i] * EX[i]; jy += v[i] * EY[i]; }
            c->mrho[q] = r;
            c->mux[q] = (jx + 0.5 * c->Fx[q]) / r;
            c->muy[q] = (jy + 0.5 * c->Fy[q]) / r;
            orc_collide_node(&c->p, v, c->Fx[q], c->Fy[q]);
            for (int i = 0; i < 9; ++i) c->f[(size_t)i * N + q] = v[i];
        }
    for (int b = 0; b < c->nbodies; ++b) {
        double fx, fy, t;
        body_force(&c->bodies[b], &fx, &fy, &t);
        finish_body(&c->bodies[b], fx, fy, t);
    }
    c->step++;
    return 0;
}

int orc_step(orc_case* c, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        int rc = step_once(c);
        if (rc) return rc;
    }
    return 0;
}

void orc_body_forces(const orc_case* c, int b, double out[3]) {
    const orc_body* B = &c->bodies[b];
    out[0] = B->Fhx; out[1] = B->Fhy; out[2] = B->Th;
}

void orc_body_state(const orc_case* c, int b, double out[6]) {
    const orc_body* B = &c->bodies[b];
    out[0] = B->xc; out[1] = B->yc; out[2] = B->vx; out[3] = B->vy; out[4] = B->om; out[5] = B->theta;
}

int orc_force_history(const orc_case* c, int b, double* out, int cap) {
    const orc_body* B = &c->bodies[b];
    int n = B->hist_n < cap ? B->hist_n : cap;
    int first = B->hist_n - n;
    memcpy(out, B->hist + 3 * (size_t)first, sizeof(double) * 3 * (size_t)n);
    return n;
}

void orc_marker_data(const orc_case* c, int b, double* out) {
    const orc_body* B = &c->bodies[b];
    for (int k = 0; k < B->n; ++k) {
        out[7 * k + 0] = B->X[k];
        out[7 * k + 1] = B->Y[k];
        out[7 * k + 2] = B->Udx[k];
        out[7 * k + 3] = B->Udy[k];
        out[7 * k + 4] = B->Fx[k];
        out[7 * k + 5] = B->Fy[k];
        out[7 * k + 6] = B->lambda[k];
    }
}

void orc_marker_stencils(const orc_case* c, int b, int* ij) {
    const orc_body* B = &c->bodies[b];
    int w;
    for (int k = 0; k < B->n; ++k) {
        ij[2 * k] = stencil_origin(B->kernel, B->X[k], &w);
        ij[2 * k + 1] = stencil_origin(B->kernel, B->Y[k], &w);
    }
}

int orc_mdf_iterations(const orc_case* c, int b) { return c->bodies[b].mdf_iters; }
double orc_mdf_omega(const orc_case* c, int b) { return c->bodies[b].mdf_omega; }
double orc_mdf_residual(const orc_case* c, int b) { return c->bodies[b].mdf_res; }
double orc_mdf_omega_end(const orc_case* c, int b) { return c->bodies[b].mdf_omega_end; }

/* ---- Sec. 2.8 local diagnostics ------------------------------------------------
 * Readings (the paper names the three metrics and their normalisations only):
 *  - slip is |U(X_k) - U_d,k| with U interpolated by the body's own kernel (Eq. 7)
 *    from the Eq. 4 velocity of the last collision; U_d,k is the marker's desired
 *    velocity (zero for a fixed body, so this is the paper's |U| / U_inf);
 *  - the bilinear probe (Sec. 4.2, Fig. 5) interpolates from the four nodes
 *    around X_k; the pressure residual is (rho - 1) c_s^2 at the probe;
 *  - leakage is the net flux sum_k rho(X_k) (U - U_d).n_k ds over the marker
 *    polygon, n_k the outward normal of the chord X_{k+1} - X_{k-1}, normalised by
 *    U_inf times the polygon length n ds (pi D for a circle); the gross flux with
 *    |.| is reported beside it;
 *  - the kappa = 2 buffer keeps the nodes with |x - X_c| < R - kappa (strict);
 *    inside the solid the residual is taken against the rigid velocity
 *    v + omega x (x - X_c), which is zero for a fixed body. */
static double bilinear_at(int nx, const double* g, double X, double Y) {
    int i0 = (int)floor(X), j0 = (int)floor(Y);
    double fx = X - i0, fy = Y - j0;
    return (1.0 - fx) * (1.0 - fy) * g[(size_t)j0 * nx + i0] + fx * (1.0 - fy) * g[(size_t)j0 * nx + i0 + 1]
         + (1.0 - fx) * fy * g[(size_t)(j0 + 1) * nx + i0] + fx * fy * g[(size_t)(j0 + 1) * nx + i0 + 1];
}

int orc_local_diagnostics_fields(int kernel, int nx, int ny, const double* rho, const double* ux,
                                 const double* uy, const double* md, int n, double ds,
                                 const double body[6], double u_ref, double kappa, double out[8],
                                 double* pm) {
    const double xc = body[0], yc = body[1], vx = body[2], vy = body[3], om = body[4], R = body[5];
    double slip_sum = 0.0, slip_max = 0.0, bl_max = 0.0, net = 0.0, gross = 0.0, fsum = 0.0;
    for (int k = 0; k < n; ++k) {
        const double X = md[7 * k], Y = md[7 * k + 1], Udx = md[7 * k + 2], Udy = md[7 * k + 3];
        const double Fkx = md[7 * k + 4], Fky = md[7 * k + 5];
        int w, i0 = stencil_origin(kernel, X, &w), j0 = stencil_origin(kernel, Y, &w);
        int b0 = (int)floor(X), c0 = (int)floor(Y);
        if (i0 < 0 || j0 < 0 || i0 + w > nx || j0 + w > ny || b0 < 0 || c0 < 0 || b0 + 2 > nx || c0 + 2 > ny)
            return 1;
        /* Eq. 7 with the body's kernel */
        const double U = interp_one(kernel, nx, ux, X, Y), V = interp_one(kernel, nx, uy, X, Y);
        const double rk = interp_one(kernel, nx, rho, X, Y);
        /* bilinear probe */
        const double Ub = bilinear_at(nx, ux, X, Y), Vb = bilinear_at(nx, uy, X, Y);
        const double rb = bilinear_at(nx, rho, X, Y);
        /* outward normal */
        double nxk, nyk;
        if (n >= 3) {
            const int kp = (k + 1) % n, km = (k + n - 1) % n;
            const double tx = md[7 * kp] - md[7 * km], ty = md[7 * kp + 1] - md[7 * km + 1];
            const double t = sqrt(tx * tx + ty * ty);
            nxk = t > 0.0 ? ty / t : 0.0;
            nyk = t > 0.0 ? -tx / t : 0.0;
            if (nxk * (X - xc) + nyk * (Y - yc) < 0.0) { nxk = -nxk; nyk = -nyk; }
        } else {
            const double r = sqrt((X - xc) * (X - xc) + (Y - yc) * (Y - yc));
            nxk = r > 0.0 ? (X - xc) / r : 0.0;
            nyk = r > 0.0 ? (Y - yc) / r : 0.0;
        }
        const double s = sqrt((U - Udx) * (U - Udx) + (V - Udy) * (V - Udy)) / u_ref;
        const double sb = sqrt((Ub - Udx) * (Ub - Udx) + (Vb - Udy) * (Vb - Udy)) / u_ref;
        const double un = (U - Udx) * nxk + (V - Udy) * nyk;
        const double fm = sqrt(Fkx * Fkx + Fky * Fky);
        slip_sum += s;
        if (s > slip_max) slip_max = s;
        if (sb > bl_max) bl_max = sb;
        net += rk * un * ds;
        gross += rk * fabs(un) * ds;
        fsum += fm;
        if (pm) {
            pm[5 * k + 0] = s;
            pm[5 * k + 1] = sb;
            pm[5 * k + 2] = un / u_ref;
            pm[5 * k + 3] = (rb - 1.0) / 3.0;
            pm[5 * k + 4] = fm;
        }
    }
    /* interior nodes beyond the kappa buffer */
    double in_sum = 0.0;
    long cnt = 0;
    const double ri = R - kappa;
    if (ri > 0.0) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const double dx = x - xc, dy = y - yc;
                if (dx * dx + dy * dy < ri * ri) {
                    const size_t q = (size_t)y * nx + x;
                    const double ex_ = ux[q] - (vx - om * dy), ey_ = uy[q] - (vy + om * dx);
                    in_sum += sqrt(ex_ * ex_ + ey_ * ey_);
                    ++cnt;
                }
            }
    }
    out[0] = n > 0 ? slip_sum / n : 0.0;
    out[1] = slip_max;
    out[2] = bl_max;
    out[3] = n > 0 ? net / (u_ref * n * ds) : 0.0;
    out[4] = n > 0 ? gross / (u_ref * n * ds) : 0.0;
    out[5] = cnt > 0 ? in_sum / cnt / u_ref : 0.0;
    out[6] = (double)cnt;
    out[7] = fsum;
    return 0;
}

int orc_local_diagnostics(const orc_case* c, int b, double u_ref, double kappa, double out[8], double* pm) {
    const orc_body* B = &c->bodies[b];
    double* md = (double*)malloc(sizeof(double) * 7 * (size_t)(B->n > 0 ? B->n : 1));
    orc_marker_data(c, b, md);
    const double body[6] = {B->xc, B->yc, B->vx, B->vy, B->om, B->p.radius};
    int rc = orc_local_diagnostics_fields(B->kernel, c->nx, c->ny, c->mrho, c->mux, c->muy, md, B->n,
                                          B->ds, body, u_ref, kappa, out, pm);
    free(md);
    return rc;
}

/* Verlet of Eq. 23 with F_hydro = 0 (no fluid): gravity and internal mass only. */
void orc_verlet_free_fall(double rho_ratio, double radius, double gx, double gy, int internal_mass,
                          int nsteps, double* out_v, double* out_x) {
    orc_body B;
    memset(&B, 0, sizeof(B));
    B.p.rho_ratio = rho_ratio;
    B.p.radius = radius;
    B.p.gx = gx;
    B.p.gy = gy;
    B.p.internal_mass = internal_mass;
    B.p.motion = ORC_FREE;
    B.n = 0;
    orc_case dummy;
    memset(&dummy, 0, sizeof(dummy));
    for (int s = 0; s < nsteps; ++s) {
        prepare_body(&dummy, &B);
        finish_body(&B, 0.0, 0.0, 0.0);
        out_v[2 * s] = B.vx; out_v[2 * s + 1] = B.vy;
        out_x[2 * s] = B.xc; out_x[2 * s + 1] = B.yc;
    }
    free(B.hist);
}
