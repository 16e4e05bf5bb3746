/*
 * cfd_oracle.c -- plain, slow FP64 CPU oracle of the OpenCFD-SCU right-hand
 * side L(U) and TVD-RK3 step (arXiv:2209.15333, Sections 2.1-2.4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code with the
 * CUDA path.  Compile with -ffp-contract=off and without -ffast-math so that
 * every operation is a separately rounded IEEE double operation.
 *
 * Readings of the paper taken here (where it is garbled or silent):
 *  R1  Eq. 8 is read as E = p/(gamma-1) + rho(u^2+v^2+w^2)/2.
 *      Nondimensional gas: p = rho T/(gamma Ma^2), c = sqrt(T)/Ma.
 *  R2  sensor classes: theta <= theta1 -> UD7; theta1 < theta <= theta2 ->
 *      WENO7; theta > theta2 -> WENO5 (Eq. 43 and the thresholds after it).
 *  R3  interface m+1/2 takes the largest class of the nodes m-3..m+4.
 *  R4  phi_d = 0 at a node on a non-periodic boundary in direction d.
 *  R6  direction d uses alpha = (d_x, d_y, d_z)/J of its own coordinate.
 *  R7  Eq. 23/24 corrected so that f+ + f- equals the flux of Eq. 6:
 *      k_i (not k_1) in the momentum rows, energy row
 *      (gamma-1) l1 |u|^2 + W + l4 |u-ck|^2/2 + l5 |u+ck|^2/2.
 *  R8  WENO: alpha_k = d_k/(eps+beta_k)^2 with Jiang-Shu smoothness
 *      indicators; the tables are derived here from their definitions.
 *  R10 an interface whose stencil m-3..m+4 leaves a non-periodic line uses
 *      WENO5 with the out-of-range sub-stencils given weight zero (Sec. 2.2.4).
 *  R11 viscous closures (Sec. 2.3): one-sided 2nd order at the boundary
 *      node, then 2nd/4th/6th-order central at the next three nodes.
 *  R12 boundary conditions (isothermal wall, inflow, extrapolation) and the
 *      paper's undefined "non-reflecting" boundary as characteristic
 *      extrapolation with frozen incoming waves (nonreflect_node below).
 *  R13 tau_ij = (mu/Re)(du_i/dx_j + du_j/dx_i - 2/3 delta_ij div u) (Eq. 13).
 *  R14 Theta_i = u_j tau_ij + k dT/dx_i (Eq. 12), k from Eq. 14.
 *  R15 Sutherland: mu = T^1.5 (1+S/T_ref)/(T+S/T_ref), S = 110.4 K (Eq. 15).
 *  R16 dt = CFL / max_n sum_d (|U_d| + c |grad d|), computed once.
 *  R17 optional free-stream-preserving metric mode (FSP): interface metrics
 *      interpolated to m+1/2 and frozen over the whole stencil.
 */
#include "cfd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 5

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static long nnodes(const orc_params* P) { return (long)P->nx * P->ny * P->nz; }

static int dim_n(const orc_params* P, int d) { return d == 0 ? P->nx : (d == 1 ? P->ny : P->nz); }

static long dim_stride(const orc_params* P, int d)
{
    return d == 0 ? 1L : (d == 1 ? (long)P->nx : (long)P->nx * P->ny);
}

static int is_periodic(const orc_params* P, int d) { return P->bc_lo[d] == ORC_BC_PERIODIC; }

static int wrap(int m, int n)
{
    int r = m % n;
    return r < 0 ? r + n : r;
}

static void set_threads(const orc_params* P)
{
#ifdef _OPENMP
    if (P->nthreads > 0) omp_set_num_threads(P->nthreads);
#else
    (void)P;
#endif
}

/* position (i,j,k) of node n */
static void node_ijk(const orc_params* P, long n, int* i, int* j, int* k)
{
    *i = (int)(n % P->nx);
    *j = (int)((n / P->nx) % P->ny);
    *k = (int)(n / ((long)P->nx * P->ny));
}

/* a node is a boundary node when it lies on a non-periodic face */
static int is_boundary_node(const orc_params* P, int i, int j, int k)
{
    int pos[3] = {i, j, k};
    for (int d = 0; d < 3; ++d) {
        if (is_periodic(P, d)) continue;
        if (pos[d] == 0 || pos[d] == dim_n(P, d) - 1) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* primitives (Eq. 5, Eq. 8 read as R1, Eq. 16, Eq. 17)                 */
/* ------------------------------------------------------------------ */

static void cons_to_prim(const orc_params* P, const double q[5], double out[7])
{
    double g = P->gamma, Ma = P->Ma;
    double rho = q[0];
    double u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
    double p = (g - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));
    double T = g * Ma * Ma * p / rho;
    double c = sqrt(T) / Ma;
    out[0] = rho; out[1] = u; out[2] = v; out[3] = w; out[4] = p; out[5] = T; out[6] = c;
}

static void prim_to_cons(const orc_params* P, double rho, double u, double v, double w, double p,
                         double q[5])
{
    q[0] = rho;
    q[1] = rho * u;
    q[2] = rho * v;
    q[3] = rho * w;
    q[4] = p / (P->gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
}

int orc_primitives(const orc_params* P, const double* U, double* prim)
{
    long N = nnodes(P);
    set_threads(P);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double q[5], o[7];
        for (int v = 0; v < NV; ++v) q[v] = U[v * N + n];
        cons_to_prim(P, q, o);
        for (int v = 0; v < 7; ++v) prim[v * N + n] = o[v];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* viscosity law (Eq. 15 read as R15; power law)                       */
/* ------------------------------------------------------------------ */

double orc_viscosity(const orc_params* P, double T)
{
    if (P->visc_law == ORC_POWER) return pow(T, P->visc_omega);
    double s = 110.4 / P->T_ref;
    return pow(T, 1.5) * (1.0 + s) / (T + s);
}

/* ------------------------------------------------------------------ */
/* modified Jameson sensor (Eqs. 42-43; R2, R4)                         */
/* ------------------------------------------------------------------ */

static double sensor_phi(double pm, double p0, double pp)
{
    return fabs(-pm + 2.0 * p0 - pp) / (pm + 2.0 * p0 + pp);
}

int orc_sensor(const orc_params* P, const double* U, double* theta, unsigned char* cls)
{
    long N = nnodes(P);
    double* prim = (double*)malloc(sizeof(double) * 7 * N);
    if (!prim) return -2;
    orc_primitives(P, U, prim);
    const double* p = prim + 4 * N;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int pos[3];
        node_ijk(P, n, &pos[0], &pos[1], &pos[2]);
        double phi[3];
        for (int d = 0; d < 3; ++d) {
            int nd = dim_n(P, d);
            long s = dim_stride(P, d);
            int m = pos[d];
            if (!is_periodic(P, d) && (m == 0 || m == nd - 1)) {
                phi[d] = 0.0;
                continue;
            }
            long nm = n + (long)(wrap(m - 1, nd) - m) * s;
            long np = n + (long)(wrap(m + 1, nd) - m) * s;
            phi[d] = sensor_phi(p[nm], p[n], p[np]);
        }
        double th = phi[0] + phi[1] + phi[2];
        if (theta) theta[n] = th;
        unsigned char c;
        if (th <= P->theta1) c = 0;
        else if (th <= P->theta2) c = 1;
        else c = 2;
        cls[n] = c;
    }
    free(prim);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Steger-Warming flux-vector splitting (Eqs. 19-30, R7)                */
/* ------------------------------------------------------------------ */

/* Eq. 23 with the eigenvalues l1 (= l2 = l3), l4, l5 of one sign. */
static void sw_flux(double g, double rho, double u, double v, double w, double c, double k1,
                    double k2, double k3, double l1, double l4, double l5, double f[5])
{
    double a = rho / (2.0 * g);
    f[0] = a * (2.0 * (g - 1.0) * l1 + l4 + l5);
    f[1] = a * (2.0 * (g - 1.0) * l1 * u + l4 * (u - c * k1) + l5 * (u + c * k1));
    f[2] = a * (2.0 * (g - 1.0) * l1 * v + l4 * (v - c * k2) + l5 * (v + c * k2));
    f[3] = a * (2.0 * (g - 1.0) * l1 * w + l4 * (w - c * k3) + l5 * (w + c * k3));
    double um = (u - c * k1) * (u - c * k1) + (v - c * k2) * (v - c * k2) + (w - c * k3) * (w - c * k3);
    double up = (u + c * k1) * (u + c * k1) + (v + c * k2) * (v + c * k2) + (w + c * k3) * (w + c * k3);
    double W = (3.0 - g) * (l4 + l5) * c * c / (2.0 * (g - 1.0));        /* Eq. 26 */
    f[4] = a * ((g - 1.0) * l1 * (u * u + v * v + w * w) + W + 0.5 * l4 * um + 0.5 * l5 * up);
}

void orc_sw_split(double g, double rho, double u, double v, double w, double c, double a1,
                  double a2, double a3, double fp[5], double fm[5])
{
    double sig = sqrt(a1 * a1 + a2 * a2 + a3 * a3);               /* Eq. 22 */
    double k1 = a1 / sig, k2 = a2 / sig, k3 = a3 / sig;           /* Eq. 27 */
    double V = a1 * u + a2 * v + a3 * w;                          /* Eq. 21 */
    double lam[3] = {V, V - c * sig, V + c * sig};                /* Eq. 20: l1, l4, l5 */
    double lp[3], lm[3];
    for (int e = 0; e < 3; ++e) {                                 /* Eq. 29 */
        lp[e] = (lam[e] + fabs(lam[e])) / 2.0;
        lm[e] = (lam[e] - fabs(lam[e])) / 2.0;
    }
    sw_flux(g, rho, u, v, w, c, k1, k2, k3, lp[0], lp[1], lp[2], fp);
    sw_flux(g, rho, u, v, w, c, k1, k2, k3, lm[0], lm[1], lm[2], fm);
}

/* ------------------------------------------------------------------ */
/* reconstructions (Eq. 41; WENO5 and WENO7 of the cited references)    */
/* ------------------------------------------------------------------ */

/* Eq. 41: a[0..6] = f_{j-3} .. f_{j+3}, value at j+1/2 */
double orc_ud7(const double a[7])
{
    return (-3.0 * a[0] + 25.0 * a[1] - 101.0 * a[2] + 319.0 * a[3] + 214.0 * a[4] - 38.0 * a[5] +
            4.0 * a[6]) / 420.0;
}

/*
 * WENO tables derived from their definitions (R8).  In the conservative
 * finite-difference form the node values are cell averages of a function h
 * over cells of unit width; the reconstruction on a sub-stencil is the
 * polynomial q_k of degree r-1 with those cell averages, evaluated at the
 * right cell face x = 1/2 (cell j spans [-1/2, 1/2]).  The smoothness
 * indicator is beta_k = sum_{l=1}^{r-1} int_{-1/2}^{1/2} (d^l q_k/dx^l)^2 dx
 * (Jiang and Shu), a quadratic form in the sub-stencil values.  The linear
 * weights d_k make sum_k d_k q_k equal the reconstruction of the full
 * (2r-1)-cell stencil.
 */
typedef struct {
    int r;
    double c[4][4];      /* c[k][l]: q_k(1/2) = sum_l c[k][l] a[k+l] */
    double d[4];
    double P[4][4][4];   /* P[k][p][l]: coefficient of x^p of q_k = sum_l P[k][p][l] a[k+l] */
    double B[4][4];      /* beta = sum_{p,q >= 1} B[p][q] coef_p coef_q */
    double Q[4][4][4];   /* the same indicator as a quadratic form in a (exported for tests) */
    double cfull[7];
} weno_tab;

static weno_tab g_w5, g_w7;
static int g_tabs_ready = 0;

/* invert an n x n matrix by Gauss-Jordan elimination with partial pivoting */
static int mat_inverse(int n, const double* A, double* Ainv)
{
    double M[7][14];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            M[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(M[i][col]) > fabs(M[piv][col])) piv = i;
        if (M[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) {
                double t = M[piv][j]; M[piv][j] = M[col][j]; M[col][j] = t;
            }
        double inv = 1.0 / M[col][col];
        for (int j = 0; j < 2 * n; ++j) M[col][j] *= inv;
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            double f = M[i][col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[col][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i][j + n];
    return 0;
}

/*
 * polynomial with the given cell averages: returns C (np x np) with
 * coefficient a_p = sum_l C[p][l] f_l of x^p; cells are centred at offs[l].
 */
static int cell_average_poly(int np, const double* offs, double* C)
{
    double M[49];
    for (int l = 0; l < np; ++l)
        for (int p = 0; p < np; ++p)
            M[l * np + p] = (pow(offs[l] + 0.5, p + 1) - pow(offs[l] - 0.5, p + 1)) / (p + 1);
    return mat_inverse(np, M, C);
}

static double falling(int p, int l) /* p!/(p-l)! */
{
    double r = 1.0;
    for (int t = 0; t < l; ++t) r *= (double)(p - t);
    return r;
}

static double int_pow_sym(int e) /* int_{-1/2}^{1/2} x^e dx */
{
    if (e % 2) return 0.0;
    return 2.0 * pow(0.5, e + 1) / (e + 1);
}

static int build_tab(int r, weno_tab* T)
{
    memset(T, 0, sizeof(*T));
    T->r = r;
    double C[49];
    for (int k = 0; k < r; ++k) {
        double offs[4];
        for (int l = 0; l < r; ++l) offs[l] = (double)(-(r - 1) + k + l);
        if (cell_average_poly(r, offs, C)) return -1;
        for (int l = 0; l < r; ++l) {
            double s = 0.0;
            for (int p = 0; p < r; ++p) s += pow(0.5, p) * C[p * r + l];
            T->c[k][l] = s;
        }
        for (int p = 0; p < r; ++p)
            for (int l = 0; l < r; ++l) T->P[k][p][l] = C[p * r + l];
        double (*B)[4] = T->B;
        for (int p = 0; p < r; ++p)
            for (int q = 0; q < r; ++q) {
                double s = 0.0;
                for (int l = 1; l <= r - 1; ++l) {
                    if (p < l || q < l) continue;
                    s += falling(p, l) * falling(q, l) * int_pow_sym(p + q - 2 * l);
                }
                B[p][q] = s;
            }
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) {
                double s = 0.0;
                for (int p = 0; p < r; ++p)
                    for (int q = 0; q < r; ++q) s += C[p * r + a] * B[p][q] * C[q * r + b];
                T->Q[k][a][b] = s;
            }
    }
    int nf = 2 * r - 1;
    double offs[7];
    for (int l = 0; l < nf; ++l) offs[l] = (double)(-(r - 1) + l);
    if (cell_average_poly(nf, offs, C)) return -1;
    for (int l = 0; l < nf; ++l) {
        double s = 0.0;
        for (int p = 0; p < nf; ++p) s += pow(0.5, p) * C[p * nf + l];
        T->cfull[l] = s;
    }
    /* linear weights: sub-stencil k is the only one reaching cell k of the
       full stencil among sub-stencils k..r-1, so solve from the left */
    for (int k = 0; k < r; ++k) {
        double s = T->cfull[k];
        for (int kk = 0; kk < k; ++kk) s -= T->d[kk] * T->c[kk][k - kk];
        T->d[k] = s / T->c[k][0];
    }
    return 0;
}

static void ensure_tabs(void)
{
    if (g_tabs_ready) return;
    build_tab(3, &g_w5);
    build_tab(4, &g_w7);
    g_tabs_ready = 1;
}

int orc_weno_tables(int r, double* c, double* d, double* Q, double* cfull)
{
    ensure_tabs();
    const weno_tab* T = r == 3 ? &g_w5 : (r == 4 ? &g_w7 : NULL);
    if (!T) return -1;
    for (int k = 0; k < r; ++k) {
        d[k] = T->d[k];
        for (int l = 0; l < r; ++l) {
            c[k * r + l] = T->c[k][l];
            for (int m = 0; m < r; ++m) Q[(k * r + l) * r + m] = T->Q[k][l][m];
        }
    }
    for (int l = 0; l < 2 * r - 1; ++l) cfull[l] = T->cfull[l];
    return 0;
}

/* beta_k from its definition: the derivative coefficients of the
   sub-stencil polynomial first, then the integrals of the squared
   derivatives (a[0..r-1] are the sub-stencil values) */
static double beta_of(const weno_tab* T, int k, const double* a)
{
    int r = T->r;
    double co[4];
    for (int p = 1; p < r; ++p) {
        double s = 0.0;
        for (int l = 0; l < r; ++l) s += T->P[k][p][l] * a[l];
        co[p] = s;
    }
    double b = 0.0;
    for (int p = 1; p < r; ++p)
        for (int q = 1; q < r; ++q) b += T->B[p][q] * co[p] * co[q];
    return b;
}

double orc_weno_beta(int r, int k, const double* a)
{
    ensure_tabs();
    return beta_of(r == 3 ? &g_w5 : &g_w7, k, a);
}

/* a[0..2r-2] = f_{j-r+1} .. f_{j+r-1}; value at j+1/2.  Sec. 2.2.3:
   candidates q_k, indicators beta_k, alpha_k = d_k/(eps + beta_k)^2,
   omega_k = alpha_k / sum alpha.  The indicators are taken of a/s: beta is
   quadratic in the values, so beta_k(a/s) = beta_k(a)/s^2 (reading R23: the
   paper's fluxes carry the face area |grad d|/J, and eps is meant for the
   flux per unit area, whose size does not depend on the grid's scaling). */
double orc_weno(int r, const double* a, const int* mask, double eps, double fs, double* omega_out)
{
    ensure_tabs();
    const weno_tab* T = r == 3 ? &g_w5 : &g_w7;
    double q[4], alpha[4], sum = 0.0;
    for (int k = 0; k < r; ++k) {
        double s = 0.0;
        for (int l = 0; l < r; ++l) s += T->c[k][l] * a[k + l];
        q[k] = s;
        double b = beta_of(T, k, a + k) / (fs * fs);
        alpha[k] = (mask && mask[k]) ? 0.0 : T->d[k] / ((eps + b) * (eps + b));
        sum += alpha[k];
    }
    double f = 0.0;
    for (int k = 0; k < r; ++k) {
        double om = alpha[k] / sum;
        if (omega_out) omega_out[k] = om;
        f += om * q[k];
    }
    return f;
}

/* 8-point Lagrange interpolation to the midpoint 1/2 from nodes -3..4 */
int orc_midpoint_weights(double* w)
{
    for (int l = 0; l < 8; ++l) {
        double xl = (double)(l - 3), s = 1.0;
        for (int m = 0; m < 8; ++m) {
            if (m == l) continue;
            double xm = (double)(m - 3);
            s *= (0.5 - xm) / (xl - xm);
        }
        w[l] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* central first derivatives with boundary closures (Sec. 2.3, R11)     */
/* ------------------------------------------------------------------ */

static double central_at(int order, int n, int periodic, const double* g, long s, int m)
{
#define G(idx) g[(long)(idx) * s]
    if (periodic) {
#define GP(off) G(wrap(m + (off), n))
        if (order == 8)
            return (672.0 * (GP(1) - GP(-1)) - 168.0 * (GP(2) - GP(-2)) + 32.0 * (GP(3) - GP(-3)) -
                    3.0 * (GP(4) - GP(-4))) / 840.0;
        return (45.0 * (GP(1) - GP(-1)) - 9.0 * (GP(2) - GP(-2)) + (GP(3) - GP(-3))) / 60.0;
#undef GP
    }
    if (m == 0) return (-3.0 * G(0) + 4.0 * G(1) - G(2)) / 2.0;
    if (m == n - 1) return (3.0 * G(n - 1) - 4.0 * G(n - 2) + G(n - 3)) / 2.0;
    if (m == 1 || m == n - 2) return (G(m + 1) - G(m - 1)) / 2.0;
    if (m == 2 || m == n - 3) return (8.0 * (G(m + 1) - G(m - 1)) - (G(m + 2) - G(m - 2))) / 12.0;
    if (m == 3 || m == n - 4 || order == 6)
        return (45.0 * (G(m + 1) - G(m - 1)) - 9.0 * (G(m + 2) - G(m - 2)) + (G(m + 3) - G(m - 3))) /
               60.0;
    return (672.0 * (G(m + 1) - G(m - 1)) - 168.0 * (G(m + 2) - G(m - 2)) +
            32.0 * (G(m + 3) - G(m - 3)) - 3.0 * (G(m + 4) - G(m - 4))) / 840.0;
#undef G
}

int orc_central_deriv(int order, int n, int periodic, const double* g, double* dg)
{
    for (int m = 0; m < n; ++m) dg[m] = central_at(order, n, periodic, g, 1, m);
    return 0;
}

/* ------------------------------------------------------------------ */
/* boundary conditions (R12)                                           */
/* ------------------------------------------------------------------ */

static void node_prim(const orc_params* P, const double* U, long N, long n, double o[7])
{
    double q[5];
    for (int v = 0; v < NV; ++v) q[v] = U[v * N + n];
    cons_to_prim(P, q, o);
}

static void store_prim(const orc_params* P, double* U, long N, long n, double rho, double u,
                       double v, double w, double p)
{
    double q[5];
    prim_to_cons(P, rho, u, v, w, p, q);
    for (int c = 0; c < NV; ++c) U[c * N + n] = q[c];
}

static double blowing_velocity(const orc_params* P, int i, int k, double t)
{
    if (P->blow_amp == 0.0 || !P->wall_x || !P->wall_z) return 0.0;
    double x = P->wall_x[i], z = P->wall_z[k];
    if (x < P->blow_x0 || x > P->blow_x1) return 0.0;
    const double pi = 3.14159265358979323846;
    return P->blow_amp * sin(2.0 * pi * (x - P->blow_x0) / (P->blow_x1 - P->blow_x0)) *
           cos(2.0 * pi * P->blow_m * z / P->blow_Lz) * sin(P->blow_omega * t);
}

/* Non-reflecting boundary (the paper names one for the ramp's outlet and top
 * without defining it; this is the characteristic form of Thompson, J. Comput.
 * Phys. 68 (1987), written as an update of the boundary node).  Linearise
 * about the boundary node's current state (rho_b, c_b) with the outward unit
 * normal n of the face.  The changes from the boundary node to the first
 * interior node of the five characteristic variables
 *     entropy        dp - c^2 drho        speed u_n
 *     shear (x2)     dv - (dv.n) n        speed u_n
 *     acoustic +     dp + rho c (dv.n)    speed u_n + c
 *     acoustic -     dp - rho c (dv.n)    speed u_n - c
 * are applied where the characteristic leaves the domain (speed > 0) and
 * dropped where it enters: the boundary takes what the interior sends out and
 * admits no incoming wave.  Supersonic outflow reduces to zeroth-order
 * extrapolation.  met: metrics; nrm_row: 0, 3 or 6 (grad of xi, eta, zeta). */
static void nonreflect_node(const orc_params* P, const double* met, double* U, long N, long n, long n1,
                            int nrm_row, double sgn)
{
    double ob[7], o1[7];
    node_prim(P, U, N, n, ob);
    node_prim(P, U, N, n1, o1);
    double g0 = met[(nrm_row + 0) * N + n], g1 = met[(nrm_row + 1) * N + n], g2 = met[(nrm_row + 2) * N + n];
    double gn = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    double nx = sgn * g0 / gn, ny = sgn * g1 / gn, nz = sgn * g2 / gn;
    double rho = ob[0], c = sqrt(P->gamma * ob[4] / ob[0]);
    double un = ob[1] * nx + ob[2] * ny + ob[3] * nz;
    double drho = o1[0] - ob[0], du = o1[1] - ob[1], dv = o1[2] - ob[2], dw = o1[3] - ob[3];
    double dp = o1[4] - ob[4];
    double dvn = du * nx + dv * ny + dw * nz;
    /* characteristic changes, each kept only if its wave leaves the domain */
    double e_ent = dp - c * c * drho;
    double e_tx = du - dvn * nx, e_ty = dv - dvn * ny, e_tz = dw - dvn * nz;
    double e_ap = dp + rho * c * dvn;
    double e_am = dp - rho * c * dvn;
    if (!(un > 0.0)) { e_ent = 0.0; e_tx = 0.0; e_ty = 0.0; e_tz = 0.0; }
    if (!(un + c > 0.0)) e_ap = 0.0;
    if (!(un - c > 0.0)) e_am = 0.0;
    /* back to primitive changes */
    double dp2 = 0.5 * (e_ap + e_am);
    double dvn2 = (e_ap - e_am) / (2.0 * rho * c);
    double drho2 = (dp2 - e_ent) / (c * c);
    store_prim(P, U, N, n, ob[0] + drho2, ob[1] + e_tx + dvn2 * nx, ob[2] + e_ty + dvn2 * ny,
               ob[3] + e_tz + dvn2 * nz, ob[4] + dp2);
}

/* apply the boundary condition of face (d, side) to every node of the face */
static void bc_face(const orc_params* P, const double* met, double* U, int d, int side, double t)
{
    int type = side ? P->bc_hi[d] : P->bc_lo[d];
    if (type == ORC_BC_PERIODIC) return;
    long N = nnodes(P);
    int nd = dim_n(P, d);
    long s = dim_stride(P, d);
    int a = (d + 1) % 3, b = (d + 2) % 3;
    int na = dim_n(P, a), nb = dim_n(P, b);
    int mb = side ? nd - 1 : 0;          /* boundary index */
    int m1 = side ? nd - 2 : 1;          /* first interior index */
    int m2 = side ? nd - 3 : 2;
    for (int ib = 0; ib < nb; ++ib)
        for (int ia = 0; ia < na; ++ia) {
            int pos[3];
            pos[d] = mb; pos[a] = ia; pos[b] = ib;
            long n = pos[0] + (long)P->nx * (pos[1] + (long)P->ny * pos[2]);
            long n1 = n + (long)(m1 - mb) * s, n2 = n + (long)(m2 - mb) * s;
            if (type == ORC_BC_OUTFLOW) {
                double o[7];
                node_prim(P, U, N, n1, o);
                store_prim(P, U, N, n, o[0], o[1], o[2], o[3], o[4]);
            } else if (type == ORC_BC_NONREFLECT) {
                nonreflect_node(P, met, U, N, n, n1, 3 * d, side ? 1.0 : -1.0);
            } else if (type == ORC_BC_INFLOW) {
                if (!P->inflow) continue;
                int jj = pos[1];
                const double* f = P->inflow;
                store_prim(P, U, N, n, f[0 * P->ny + jj], f[1 * P->ny + jj], f[2 * P->ny + jj],
                           f[3 * P->ny + jj], f[4 * P->ny + jj]);
            } else if (type == ORC_BC_WALL) {
                double o1[7], o2[7];
                node_prim(P, U, N, n1, o1);
                node_prim(P, U, N, n2, o2);
                double pw = (4.0 * o1[4] - o2[4]) / 3.0;
                double Tw = P->T_wall;
                double rhow = P->gamma * P->Ma * P->Ma * pw / Tw;
                double u = 0.0, v = 0.0, w = 0.0;
                if (d == 1 && side == 0) {
                    double vn = blowing_velocity(P, pos[0], pos[2], t);
                    if (vn != 0.0) {
                        /* wall normal along grad(eta) */
                        double ex = met[3 * N + n], ey = met[4 * N + n], ez = met[5 * N + n];
                        double nrm = sqrt(ex * ex + ey * ey + ez * ez);
                        u = vn * ex / nrm; v = vn * ey / nrm; w = vn * ez / nrm;
                    }
                }
                store_prim(P, U, N, n, rhow, u, v, w, pw);
            }
        }
}

int orc_apply_bc(const orc_params* P, const double* metrics, double* U, double t)
{
    for (int d = 0; d < 3; ++d) {
        bc_face(P, metrics, U, d, 0, t);
        bc_face(P, metrics, U, d, 1, t);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* the right-hand side L(U) of one stage                               */
/* ------------------------------------------------------------------ */

/* inviscid flux at interface j+1/2 of one line (NODAL or FSP metrics) */
/* ------------------------------------------------------------------ */
/* characteristic variables (Sec. 2.2.2, Eq. 31-40)                    */
/* ------------------------------------------------------------------ */

int orc_char_matrices(double gamma, const double U[5], const double n[3], double S[25], double Sinv[25])
{
    double rho = U[0];
    if (!(rho > 0.0)) return -1;
    double u = U[1] / rho, v = U[2] / rho, w = U[3] / rho;
    double V = 0.5 * (u * u + v * v + w * w);                      /* Eq. 25 */
    double p = (gamma - 1.0) * (U[4] - rho * V);
    if (!(p > 0.0)) return -1;
    double c2 = gamma * p / rho, c = sqrt(c2);
    double H = V + c2 / (gamma - 1.0);                             /* Eq. 36 */
    double kap = (gamma - 1.0) / c2, kap1 = 0.5 * kap, chi = 0.5 / c; /* Eq. 37 */
    double n1 = n[0], n2 = n[1], n3 = n[2];
    double l1, l2, l3;                                             /* Eq. 39 */
    if (fabs(n3) <= fabs(n2)) {
        double r = sqrt(n1 * n1 + n2 * n2);
        l1 = -n2 / r; l2 = n1 / r; l3 = 0.0;
    } else {
        double r = sqrt(n1 * n1 + n3 * n3);
        l1 = -n3 / r; l2 = 0.0; l3 = n1 / r;
    }
    double m1 = n2 * l3 - n3 * l2, m2 = n3 * l1 - n1 * l3, m3 = n1 * l2 - n2 * l1; /* Eq. 40 */
    double un = u * n1 + v * n2 + w * n3;                          /* Eq. 38 */
    double ul = u * l1 + v * l2 + w * l3;
    double um = u * m1 + v * m2 + w * m3;
    double Si[25] = {                                              /* Eq. 34 */
        1.0, 0.0, 0.0, 1.0, 1.0,
        u,   l1,  m1,  u - c * n1, u + c * n1,
        v,   l2,  m2,  v - c * n2, v + c * n2,
        w,   l3,  m3,  w - c * n3, w + c * n3,
        V,   ul,  um,  H - c * un, H + c * un};
    double Sl[25] = {                                              /* Eq. 35 */
        1.0 - kap * V, kap * u, kap * v, kap * w, -kap,
        -ul, l1, l2, l3, 0.0,
        -um, m1, m2, m3, 0.0,
        kap1 * V + chi * un, -chi * n1 - kap1 * u, -chi * n2 - kap1 * v, -chi * n3 - kap1 * w, kap1,
        kap1 * V - chi * un, chi * n1 - kap1 * u, chi * n2 - kap1 * v, chi * n3 - kap1 * w, kap1};
    memcpy(S, Sl, sizeof(Sl));
    memcpy(Sinv, Si, sizeof(Si));
    return 0;
}

/* fs: face-area scale sigma_{j+1/2} of the interface (R23) */
/* chU (U_j and U_{j+1}, [2][5]) and chn (unit normal of the interface):
   characteristic reconstruction of the WENO faces (Sec. 2.2.2), or NULL */
static int interface_flux(const orc_params* P, int n, int periodic, int j,
                          const double* fp /* [n][5] */, const double* fm, const unsigned char* lcls,
                          double fs, const double* chU, const double* chn, double out[5])
{
    int scheme = P->scheme;
    int masked_edge = !periodic && (j - 3 < 0 || j + 4 > n - 1);
    int use; /* 0 UD7, 1 WENO7, 2 WENO5 */
    if (masked_edge) {
        use = 2;
    } else if (scheme == ORC_UD7) {
        use = 0;
    } else if (scheme == ORC_WENO7) {
        use = 1;
    } else if (scheme == ORC_WENO5) {
        use = 2;
    } else {
        int c = 0;
        for (int o = -3; o <= 4; ++o) {
            int cc = lcls[wrap(j + o, n)];
            if (cc > c) c = cc;
        }
        use = c;
    }
    /* Eq. 31: with characteristic reconstruction the WENO faces work on
       g = S f of every stencil node (UD7 is linear, so projecting would
       not change it); the result is mapped back with S^-1 */
    int chr = chU && use != 0;
    double char_S[25], char_Sinv[25];
    if (chr) {
        double Uh[5];
        for (int q = 0; q < NV; ++q) Uh[q] = 0.5 * (chU[q] + chU[NV + q]);   /* Eq. 32 */
        if (orc_char_matrices(P->gamma, Uh, chn, char_S, char_Sinv) != 0) return -1;
    }
    double gout[5];
    for (int q = 0; q < NV; ++q) {
        double a[7], b[7];
        int inrange_p[7], inrange_m[7];
        for (int o = -3; o <= 3; ++o) {
            int ip = j + o, im = j + 1 - o;
            inrange_p[o + 3] = periodic || (ip >= 0 && ip < n);
            inrange_m[o + 3] = periodic || (im >= 0 && im < n);
            a[o + 3] = 0.0;
            b[o + 3] = 0.0;
            if (chr) {
                for (int e = 0; e < NV; ++e) {
                    if (inrange_p[o + 3]) a[o + 3] += char_S[q * NV + e] * fp[wrap(ip, n) * NV + e];
                    if (inrange_m[o + 3]) b[o + 3] += char_S[q * NV + e] * fm[wrap(im, n) * NV + e];
                }
            } else {
                if (inrange_p[o + 3]) a[o + 3] = fp[wrap(ip, n) * NV + q];
                if (inrange_m[o + 3]) b[o + 3] = fm[wrap(im, n) * NV + q];
            }
        }
        double vp, vm;
        if (use == 0) {
            vp = orc_ud7(a);
            vm = orc_ud7(b);
        } else if (use == 1) {
            vp = orc_weno(4, a, NULL, P->weno_eps, fs, NULL);
            vm = orc_weno(4, b, NULL, P->weno_eps, fs, NULL);
        } else {
            int mp[3], mm[3];
            for (int k = 0; k < 3; ++k) {
                /* WENO5 sub-stencil k covers offsets -2+k .. k */
                mp[k] = mm[k] = 0;
                for (int l = 0; l < 3; ++l) {
                    if (!inrange_p[1 + k + l]) mp[k] = 1;
                    if (!inrange_m[1 + k + l]) mm[k] = 1;
                }
            }
            vp = orc_weno(3, a + 1, mp, P->weno_eps, fs, NULL);
            vm = orc_weno(3, b + 1, mm, P->weno_eps, fs, NULL);
        }
        gout[q] = vp + vm;
    }
    for (int q = 0; q < NV; ++q) {
        if (!chr) {
            out[q] = gout[q];
            continue;
        }
        double s = 0.0;
        for (int e = 0; e < NV; ++e) s += char_Sinv[q * NV + e] * gout[e];
        out[q] = s;
    }
    return 0;
}

/* does node position m along a line receive a right-hand side */
static int rhs_node(int periodic, int n, int m) { return periodic || (m > 0 && m < n - 1); }

static int inviscid_direction(const orc_params* P, const double* met, const double* U, const double* prim,
                              const unsigned char* cls, double* R, int d)
{
    int status = 0;
    long N = nnodes(P);
    int nd = dim_n(P, d);
    long s = dim_stride(P, d);
    int periodic = is_periodic(P, d);
    int a = (d + 1) % 3, b = (d + 2) % 3;
    int na = dim_n(P, a), nb = dim_n(P, b);
    double wmid[8];
    orc_midpoint_weights(wmid);
    long nlines = (long)na * nb;
#pragma omp parallel for schedule(dynamic, 16)
    for (long line = 0; line < nlines; ++line) {
        int ia = (int)(line % na), ib = (int)(line / na);
        int pos[3];
        pos[d] = 0; pos[a] = ia; pos[b] = ib;
        long base = pos[0] + (long)P->nx * (pos[1] + (long)P->ny * pos[2]);
        double* fp = (double*)malloc(sizeof(double) * NV * nd);
        double* fm = (double*)malloc(sizeof(double) * NV * nd);
        double* fh = (double*)malloc(sizeof(double) * NV * (nd + 1));
        unsigned char* lcls = (unsigned char*)malloc(nd);
        double* alpha = (double*)malloc(sizeof(double) * 3 * nd);
        for (int m = 0; m < nd; ++m) {
            long nn = base + m * s;
            double J = met[9 * N + nn];
            for (int e = 0; e < 3; ++e) alpha[3 * m + e] = met[(3 * d + e) * N + nn] / J; /* Eq. 19 */
            lcls[m] = cls ? cls[nn] : 0;
            orc_sw_split(P->gamma, prim[0 * N + nn], prim[1 * N + nn], prim[2 * N + nn],
                         prim[3 * N + nn], prim[6 * N + nn], alpha[3 * m], alpha[3 * m + 1],
                         alpha[3 * m + 2], fp + NV * m, fm + NV * m);
        }
        /* interfaces j+1/2, j = -1 .. nd-1, stored at fh[j+1] */
        int jlo = periodic ? -1 : 0, jhi = periodic ? nd - 1 : nd - 2;
        int chr = P->recon_vars == ORC_RECON_CHARACTERISTIC;
        for (int j = jlo; j <= jhi; ++j) {
            double out[5];
            /* characteristic reconstruction: conserved states of the two
               nodes of the interface (Eq. 32 averages them) */
            double chU[10];
            int ja = wrap(j, nd), jb = wrap(j + 1, nd);
            for (int q = 0; q < NV; ++q) {
                chU[q] = U[q * N + base + ja * s];
                chU[NV + q] = U[q * N + base + jb * s];
            }
            int rc;
            if (P->metric_mode == ORC_METRIC_FSP) {
                /* R17: interface metric, frozen over the stencil nodes j-3..j+4 */
                double ai[3] = {0.0, 0.0, 0.0};
                for (int l = 0; l < 8; ++l) {
                    int mm = wrap(j - 3 + l, nd);
                    for (int e = 0; e < 3; ++e) ai[e] += wmid[l] * alpha[3 * mm + e];
                }
                double lfp[8 * NV], lfm[8 * NV];
                unsigned char lc[8];
                for (int l = 0; l < 8; ++l) {
                    int mm = wrap(j - 3 + l, nd);
                    long nn = base + mm * s;
                    orc_sw_split(P->gamma, prim[0 * N + nn], prim[1 * N + nn], prim[2 * N + nn],
                                 prim[3 * N + nn], prim[6 * N + nn], ai[0], ai[1], ai[2],
                                 lfp + NV * l, lfm + NV * l);
                    lc[l] = lcls[mm];
                }
                /* local line of the 8 stencil nodes j-3..j+4: interface at local 3+1/2,
                   whose stencil stays inside the local line */
                double fs = sqrt(ai[0] * ai[0] + ai[1] * ai[1] + ai[2] * ai[2]);
                double nrm[3] = {ai[0] / fs, ai[1] / fs, ai[2] / fs};
                rc = interface_flux(P, 8, 1, 3, lfp, lfm, lc, fs, chr ? chU : NULL, nrm, out);
            } else {
                /* R23: sigma_{j+1/2} = (sigma_j + sigma_{j+1})/2, sigma = |alpha| (Eq. 22) */
                double fs = 0.5 * (sqrt(alpha[3 * ja] * alpha[3 * ja] + alpha[3 * ja + 1] * alpha[3 * ja + 1] +
                                        alpha[3 * ja + 2] * alpha[3 * ja + 2]) +
                                   sqrt(alpha[3 * jb] * alpha[3 * jb] + alpha[3 * jb + 1] * alpha[3 * jb + 1] +
                                        alpha[3 * jb + 2] * alpha[3 * jb + 2]));
                /* R25: interface normal from the two nodes' metric vectors */
                double sa[3], sn = 0.0;
                for (int e = 0; e < 3; ++e) {
                    sa[e] = alpha[3 * ja + e] + alpha[3 * jb + e];
                    sn += sa[e] * sa[e];
                }
                sn = sqrt(sn);
                double nrm[3] = {sa[0] / sn, sa[1] / sn, sa[2] / sn};
                rc = interface_flux(P, nd, periodic, periodic ? wrap(j, nd) : j, fp, fm, lcls, fs,
                                    chr ? chU : NULL, nrm, out);
            }
            if (rc != 0) {
#pragma omp atomic write
                status = -3;
            }
            for (int q = 0; q < NV; ++q) fh[NV * (j + 1) + q] = out[q];
        }
        for (int m = 0; m < nd; ++m) {
            if (!rhs_node(periodic, nd, m)) continue;
            long nn = base + m * s;
            for (int q = 0; q < NV; ++q)
                R[q * N + nn] -= fh[NV * (m + 1) + q] - fh[NV * m + q];
        }
        free(fp); free(fm); free(fh); free(lcls); free(alpha);
    }
    return status;
}

static void viscous_terms(const orc_params* P, const double* met, const double* prim, double* R)
{
    long N = nnodes(P);
    double g = P->gamma, Ma = P->Ma, Re = P->Re, Pr = P->Pr;
    int ord = P->visc_order;
    /* derivatives of u, v, w, T along xi, eta, zeta: dq[(3*var+d)*N + n] */
    double* dq = (double*)malloc(sizeof(double) * 12 * N);
    double* Fv = (double*)malloc(sizeof(double) * 12 * N); /* [(4*d + row-1)][N] */
    const int pvar[4] = {1, 2, 3, 5};
    for (int var = 0; var < 4; ++var)
        for (int d = 0; d < 3; ++d) {
            const double* f = prim + pvar[var] * N;
            double* out = dq + (3 * var + d) * N;
            int nd = dim_n(P, d);
            long s = dim_stride(P, d);
            int per = is_periodic(P, d);
#pragma omp parallel for schedule(static)
            for (long n = 0; n < N; ++n) {
                int pos[3];
                node_ijk(P, n, &pos[0], &pos[1], &pos[2]);
                long base = n - (long)pos[d] * s;
                out[n] = central_at(ord, nd, per, f + base, s, pos[d]);
            }
        }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double m[9];
        for (int e = 0; e < 9; ++e) m[e] = met[e * N + n];
        double J = met[9 * N + n];
        /* Cartesian gradients: dq/dx_i = sum_d (d)_{x_i} dq/dd */
        double gr[4][3];
        for (int var = 0; var < 4; ++var)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int d = 0; d < 3; ++d) s += m[3 * d + i] * dq[(3 * var + d) * N + n];
                gr[var][i] = s;
            }
        double T = prim[5 * N + n];
        double mu = orc_viscosity(P, T);
        double div = gr[0][0] + gr[1][1] + gr[2][2];
        double tau[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                tau[i][j] = (mu / Re) * (gr[i][j] + gr[j][i] - (i == j ? 2.0 / 3.0 * div : 0.0));
        double kc = mu / ((g - 1.0) * Ma * Ma * Pr * Re);                 /* Eq. 14 */
        double vel[3] = {prim[1 * N + n], prim[2 * N + n], prim[3 * N + n]};
        double Th[3];
        for (int i = 0; i < 3; ++i)
            Th[i] = vel[0] * tau[i][0] + vel[1] * tau[i][1] + vel[2] * tau[i][2] + kc * gr[3][i];
        for (int d = 0; d < 3; ++d) {                                    /* Eqs. 9-11 */
            double a0 = m[3 * d] / J, a1 = m[3 * d + 1] / J, a2 = m[3 * d + 2] / J;
            for (int row = 0; row < 3; ++row)
                Fv[(4 * d + row) * N + n] = a0 * tau[0][row] + a1 * tau[1][row] + a2 * tau[2][row];
            Fv[(4 * d + 3) * N + n] = a0 * Th[0] + a1 * Th[1] + a2 * Th[2];
        }
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int pos[3];
        node_ijk(P, n, &pos[0], &pos[1], &pos[2]);
        if (is_boundary_node(P, pos[0], pos[1], pos[2])) continue;
        for (int d = 0; d < 3; ++d) {
            int nd = dim_n(P, d);
            long s = dim_stride(P, d);
            long base = n - (long)pos[d] * s;
            for (int row = 0; row < 4; ++row) {
                const double* f = Fv + (4 * d + row) * N + base;
                R[(row + 1) * N + n] += central_at(ord, nd, is_periodic(P, d), f, s, pos[d]);
            }
        }
    }
    free(dq);
    free(Fv);
}

int orc_rhs(const orc_params* P, const double* met, const double* U, double* L,
            unsigned char* cls_out)
{
    ensure_tabs();
    set_threads(P);
    if (P->metric_mode == ORC_METRIC_FSP)
        for (int d = 0; d < 3; ++d)
            if (!is_periodic(P, d)) return -1; /* FSP mode is defined for periodic lines only */
    long N = nnodes(P);
    double* prim = (double*)malloc(sizeof(double) * 7 * N);
    double* R = (double*)calloc((size_t)NV * N, sizeof(double));
    unsigned char* cls = (unsigned char*)calloc((size_t)N, 1);
    if (!prim || !R || !cls) return -2;
    orc_primitives(P, U, prim);                                           /* step 1 */
    if (P->scheme == ORC_HYBRID) {                                        /* step 3 */
        if (P->forced_cls) memcpy(cls, P->forced_cls, (size_t)N);
        else orc_sensor(P, U, NULL, cls);
    }
    if (cls_out) memcpy(cls_out, cls, (size_t)N);
    int st = 0;
    for (int d = 0; d < 3 && st == 0; ++d) st = inviscid_direction(P, met, U, prim, cls, R, d); /* steps 4-7 */
    if (st != 0) {
        free(prim); free(R); free(cls);
        return st;
    }
    if (P->Re > 0.0) viscous_terms(P, met, prim, R);                      /* step 8 */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {                                        /* step 9 */
        int i, j, k;
        node_ijk(P, n, &i, &j, &k);
        int bnd = is_boundary_node(P, i, j, k);
        double J = met[9 * N + n];
        for (int q = 0; q < NV; ++q) L[q * N + n] = bnd ? 0.0 : J * R[q * N + n];
    }
    free(prim); free(R); free(cls);
    return 0;
}

/* ------------------------------------------------------------------ */
/* TVD Runge-Kutta (Eq. 45)                                            */
/* ------------------------------------------------------------------ */

int orc_rk3_stage(int stage, long n, const double* Un, const double* Uk, const double* L,
                  double dt, double* out)
{
    for (long i = 0; i < n; ++i) {
        if (stage == 1) out[i] = Un[i] + dt * L[i];
        else if (stage == 2) out[i] = 0.75 * Un[i] + 0.25 * (Uk[i] + dt * L[i]);
        else out[i] = Un[i] / 3.0 + 2.0 / 3.0 * (Uk[i] + dt * L[i]);
    }
    return 0;
}

int orc_step(const orc_params* P, const double* met, double* U, double dt, int nsteps, double t0)
{
    long N = nnodes(P), n5 = NV * N;
    double* Un = (double*)malloc(sizeof(double) * n5);
    double* Uk = (double*)malloc(sizeof(double) * n5);
    double* L = (double*)malloc(sizeof(double) * n5);
    if (!Un || !Uk || !L) return -2;
    const double tstage[3] = {1.0, 0.5, 1.0};
    double t = t0;
    for (int s = 0; s < nsteps; ++s) {
        memcpy(Un, U, sizeof(double) * n5);
        memcpy(Uk, U, sizeof(double) * n5);
        for (int st = 1; st <= 3; ++st) {
            int rc = orc_rhs(P, met, Uk, L, NULL);
            if (rc != 0) {
                free(Un); free(Uk); free(L);
                return rc;
            }
            orc_rk3_stage(st, n5, Un, Uk, L, dt, Uk);
            orc_apply_bc(P, met, Uk, t + tstage[st - 1] * dt);
        }
        memcpy(U, Uk, sizeof(double) * n5);
        t += dt;
    }
    free(Un); free(Uk); free(L);
    return 0;
}

/* R16: time step from the CFL condition */
double orc_cfl_dt(const orc_params* P, const double* met, const double* U, double cfl)
{
    long N = nnodes(P);
    double mx = 0.0;
    for (long n = 0; n < N; ++n) {
        double q[5], o[7];
        for (int v = 0; v < NV; ++v) q[v] = U[v * N + n];
        cons_to_prim(P, q, o);
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            double dx = met[(3 * d) * N + n], dy = met[(3 * d + 1) * N + n], dz = met[(3 * d + 2) * N + n];
            s += fabs(dx * o[1] + dy * o[2] + dz * o[3]) + o[6] * sqrt(dx * dx + dy * dy + dz * dz);
        }
        if (s > mx) mx = s;
    }
    return cfl / mx;
}
