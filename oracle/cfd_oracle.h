/*
 * cfd_oracle.h -- plain FP64 CPU oracle for the per-stage right-hand side
 * and TVD-RK3 step of the OpenCFD-SCU method (arXiv:2209.15333, Sections
 * 2.1-2.4, Eqs. 1-45).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Layout: every field is structure-of-arrays, [var][k][j][i], i (xi)
 * fastest, N = nx*ny*nz nodes.  Metrics are [10][N]:
 *   xi_x, xi_y, xi_z, eta_x, eta_y, eta_z, zeta_x, zeta_y, zeta_z, J
 * (Eq. 3 and Eq. 4; J = |d(xi,eta,zeta)/d(x,y,z)|).
 */
#ifndef CFD_ORACLE_H
#define CFD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_WALL = 1, ORC_BC_INFLOW = 2, ORC_BC_OUTFLOW = 3, ORC_BC_NONREFLECT = 5 };
enum { ORC_SUTHERLAND = 0, ORC_POWER = 1 };
enum { ORC_UD7 = 0, ORC_WENO5 = 1, ORC_WENO7 = 2, ORC_HYBRID = 3 };
enum { ORC_METRIC_NODAL = 0, ORC_METRIC_FSP = 1 };
enum { ORC_RECON_COMPONENT = 0, ORC_RECON_CHARACTERISTIC = 1 };

typedef struct orc_params {
    int nx, ny, nz;
    int bc_lo[3], bc_hi[3];       /* per direction xi, eta, zeta */
    double gamma, Re, Ma, Pr;     /* Re <= 0: inviscid */
    double T_wall, T_ref;         /* T_wall nondimensional, T_ref in K */
    int visc_law;                 /* ORC_SUTHERLAND or ORC_POWER */
    double visc_omega;
    int scheme;                   /* ORC_UD7 .. ORC_HYBRID */
    double theta1, theta2;
    int visc_order;               /* 6 or 8 */
    int metric_mode;              /* ORC_METRIC_NODAL or ORC_METRIC_FSP */
    double weno_eps;
    int nthreads;                 /* <= 0: library default */
    const unsigned char* forced_cls;  /* node classes to use instead of the sensor, or NULL */
    const double* inflow;         /* [5][ny]: rho,u,v,w,p on the xi-low face, or NULL */
    double blow_amp, blow_x0, blow_x1, blow_omega, blow_Lz;
    int blow_m;
    const double* wall_x;         /* [nx] x of the eta-low wall nodes (blowing), or NULL */
    const double* wall_z;         /* [nz] z of the eta-low wall nodes (blowing), or NULL */
    int recon_vars;               /* ORC_RECON_COMPONENT or ORC_RECON_CHARACTERISTIC (Sec. 2.2.2) */
} orc_params;

/* ---- whole-field operations ---- */
int orc_primitives(const orc_params* P, const double* U, double* prim /* [7][N]: rho,u,v,w,p,T,c */);
int orc_sensor(const orc_params* P, const double* U, double* theta /* [N] or NULL */,
               unsigned char* cls /* [N] */);
int orc_rhs(const orc_params* P, const double* metrics, const double* U, double* L,
            unsigned char* cls_out /* [N] or NULL */);
int orc_apply_bc(const orc_params* P, const double* metrics, double* U, double t);
int orc_rk3_stage(int stage, long n, const double* Un, const double* Uk, const double* L,
                  double dt, double* out);
int orc_step(const orc_params* P, const double* metrics, double* U, double dt, int nsteps,
             double t0);
double orc_cfl_dt(const orc_params* P, const double* metrics, const double* U, double cfl);

/* ---- building blocks, exported for the pin tests ---- */
void orc_sw_split(double gamma, double rho, double u, double v, double w, double c,
                  double a1, double a2, double a3, double fp[5], double fm[5]);
double orc_ud7(const double a[7]);
int orc_weno_tables(int r, double* c /* [r][r] */, double* d /* [r] */, double* Q /* [r][r][r] */,
                    double* cfull /* [2r-1] */);
/* WENO value at j+1/2 from a[0..2r-2] = f_{j-r+1..j+r-1}.  The
   smoothness indicators are measured on a/s (s > 0: the face-area scale of
   the flux, 1 for a plain function), so the weights do not depend on the
   scaling of the flux. */
double orc_weno(int r, const double* a /* [2r-1] */, const int* mask /* [r] or NULL */, double eps,
                double s, double* omega_out /* [r] or NULL */);
double orc_weno_beta(int r, int k, const double* a /* [r] */);
/* Eigenvector matrices of Sec. 2.2.2 (Eq. 34-40) at the conserved state
   U = (rho, rho u, rho v, rho w, E) for the unit normal n: S (rows: left
   eigenvectors, Eq. 35) and Sinv (columns: right eigenvectors, Eq. 34),
   both row-major [5][5]; the fields are ordered as the eigenvalues of
   Eq. 33: u_n (entropy), u_n (shear along l), u_n (shear along m), u_n - c,
   u_n + c.  Returns -1 for a non-physical state. */
int orc_char_matrices(double gamma, const double U[5], const double n[3], double S[25], double Sinv[25]);
int orc_central_deriv(int order, int n, int periodic, const double* g, double* dg);
int orc_midpoint_weights(double* w /* [8] */);
double orc_viscosity(const orc_params* P, double T);

#ifdef __cplusplus
}
#endif
#endif
