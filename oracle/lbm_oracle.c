/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the two D2Q9 multiphase time steps
 * compared in "Fundamental comparison between the pseudopotential and the free
 * energy lattice Boltzmann methods" (Czelusniak et al., arXiv:2403.11167).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes, in the paper's order and notation (lattice units,
 * dx = dt = c = 1, c_s^2 = 1/3, G = -1):
 *
 *   Eq. (1)  MRT lattice Boltzmann equation
 *              f_i(x + c_i, t+1) = f_i - [M^-1 L M](f - f^eq)
 *                                      + [M^-1 (I - L/2) M] F' + C_i
 *            with the moment matrix M of Eq. (S48), M^-1 obtained by a plain
 *            Gauss-Jordan inversion of M (checked against the printed Eq. (S49)
 *            by the tests) and L = diag of Eq. (3).
 *   Modified pseudopotential model (MP-LBM, Sec. 4):
 *            Eq. (28) EOS, Eq. (11) psi, Eq. (10) Shan-Chen force,
 *            Eqs. (30a/b, 31a/b) Q tensor, Eq. (13) source MC,
 *            Eq. (32) forcing moments MF', Eq. (4) equilibrium, Eq. (6) macros.
 *            Reading of Eq. (30b): the C2 term carries the factor G like the
 *            C1 and kappa^Li terms, as the continuum form Eq. (S41b) requires.
 *   Improved well-balanced free-energy model (IWB-FE-LBM, Sec. 2.2):
 *            Eq. (29) bulk chemical potential, Eq. (24) 9-point stencils
 *            (gradient stencil read with the weights w_i), mu = mu_b - kappa lap rho,
 *            F = -rho grad mu, Eq. (20) equilibrium (A = 0, p_g = 0),
 *            Eq. (21) forcing with d = 2 and grad p_g = 0.
 *
 * Everything is done cell by cell with explicit 9x9 matrix products; no fusion,
 * no reordering beyond the equations.  Fields are SoA: f[i*ny*nx + y*nx + x],
 * periodic in x, and in y either periodic or bounded by no-slip walls on rows 0 and ny-1
 * (the parallel-plate flow of Sec. 5.3, Zou and He's condition; see wall_fill).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q9 9

/* Eq. (2): D2Q9 velocities, i = 0 rest, 1..4 axes, 5..8 diagonals. */
static const int CX[Q9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Weights below Eq. (4). */
static const double WI[Q9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* Eq. (S48): Lallemand-Luo moment matrix; rows rho, e, zeta, jx, qx, jy, qy, pxx, pxy. */
static const double MM[Q9][Q9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},  {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

typedef struct {
    double a, b, R, T;  /* Carnahan-Starling EOS, Eq. (28) */
    double G;           /* interaction strength, -1 (text below Eq. 11) */
    double tau_rho, tau_e, tau_zeta, tau_j, tau_q, tau_nu; /* Eq. (3) */
    double kappa_P, kappa_Li, sigma_Li; /* MP-LBM, Eqs. (30)-(32) */
    double kappa;       /* FE-LBM surface-tension parameter, mu = mu_b - kappa lap rho */
    double fx, fy;      /* constant body force added to the total force */
    double walls;       /* 0: periodic in y; 1: no-slip walls on rows 0 and ny-1 (Sec. 5.3);
                           2: the same walls with the free-energy wall rows' normal mu
                           gradient one-sided (see fe_wall_density) */
    double drive;       /* 1: add the droplet-collision force of Sec. 5.4 (drive_force) */
    double drive_ax_lo, drive_ax_hi, drive_x_split;
    double A;           /* FE viscosity-tuning term of Eqs. (20), (23) */
    double g, rho_g, y_ref; /* FE gravity (acting along -y), reference density rho_0 and the
                               reference height of p_g = rho_0 g (y - y_ref) (Eqs. 20, 21) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* M^-1 by Gauss-Jordan elimination with partial pivoting.                  */
static void invert9(const double A[Q9][Q9], double Ainv[Q9][Q9]) {
    double a[Q9][2 * Q9];
    for (int r = 0; r < Q9; ++r)
        for (int c = 0; c < 2 * Q9; ++c)
            a[r][c] = c < Q9 ? A[r][c] : (c - Q9 == r ? 1.0 : 0.0);
    for (int col = 0; col < Q9; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * Q9; ++c) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double d = a[col][col];
        for (int c = 0; c < 2 * Q9; ++c) a[col][c] /= d;
        for (int r = 0; r < Q9; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m != 0.0)
                for (int c = 0; c < 2 * Q9; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < Q9; ++r)
        for (int c = 0; c < Q9; ++c) Ainv[r][c] = a[r][Q9 + c];
}

static double MINV[Q9][Q9];
static int minv_ready = 0;
static void ensure_minv(void) {
    if (!minv_ready) {
        invert9(MM, MINV);
        minv_ready = 1;
    }
}

void orc_moment_matrix(double* out81) {
    for (int r = 0; r < Q9; ++r)
        for (int c = 0; c < Q9; ++c) out81[r * Q9 + c] = MM[r][c];
}
void orc_moment_matrix_inverse(double* out81) {
    ensure_minv();
    for (int r = 0; r < Q9; ++r)
        for (int c = 0; c < Q9; ++c) out81[r * Q9 + c] = MINV[r][c];
}

/* ------------------------------------------------------------------------ */
/* Thermodynamics.                                                          */
/* Eq. (28): Carnahan-Starling pressure. */
static double p_eos(const orc_params* p, double rho) {
    double eta = p->b * rho / 4.0;
    return rho * p->R * p->T * (1.0 + eta + eta * eta - eta * eta * eta) /
               ((1.0 - eta) * (1.0 - eta) * (1.0 - eta)) -
           p->a * rho * rho;
}
/* Eq. (29): bulk chemical potential. */
static double mu_bulk(const orc_params* p, double rho) {
    double eta = p->b * rho / 4.0;
    double RT = p->R * p->T;
    return RT * (3.0 - eta) / ((1.0 - eta) * (1.0 - eta) * (1.0 - eta)) + RT * log(rho) + RT -
           2.0 * p->a * rho;
}
double orc_p_eos(const orc_params* p, double rho) { return p_eos(p, rho); }
double orc_mu_bulk(const orc_params* p, double rho) { return mu_bulk(p, rho); }

/* Eq. (11): psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2 dt^2)).  Returns -1 if the
 * radicand is negative (the pseudopotential does not exist there). */
static double psi_of(const orc_params* p, double rho) {
    double rad = 2.0 * (p_eos(p, rho) - rho * CS2) / p->G;
    if (!(rad >= 0.0)) return -1.0;
    return sqrt(rad);
}

static inline int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* Row of a y neighbour: periodic, or, with walls, mirrored through the wall node (the
 * reading of this oracle: row -1 is row 1 and row ny is row ny-2, i.e. zero normal
 * gradient of psi, rho and mu at a wall node; the paper does not specify it). */
static inline int yrow(int y, int ny, int walls) {
    if (!walls) return wrap(y, ny);
    if (y < 0) return -y;
    if (y > ny - 1) return 2 * (ny - 1) - y;
    return y;
}

/* ------------------------------------------------------------------------ */
/* Equilibria.                                                               */
/* Eq. (4): standard second-order equilibrium (used by the pseudopotential model). */
static void feq_standard(double rho, double ux, double uy, double feq[Q9]) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < Q9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        /* (c_a c_b - c_s^2 d_ab) u_a u_b / (2 c_s^4) */
        double quad = (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2);
        feq[i] = WI[i] * rho * (1.0 + cu / CS2 + quad);
    }
}

/* Eq. (20) with A = 0 and p_g = 0: improved well-balanced equilibrium. */
/* Eq. (20) in full: p_g the gravitational reference pressure, A the viscosity-tuning term,
 * S_ab = d_a u_b + d_b u_a (Sxx, Sxy, Syy).  With X = u u + c_s^2 A S,
 *   f_0 = rho - (1 - w_0) p_g / c_s^2 - w_0 rho tr(X) / (2 c_s^2)
 *   f_i = w_i p_g / c_s^2 + w_i rho [c_i.u / c_s^2 + (c_i.X.c_i - c_s^2 tr X) / (2 c_s^4)]
 * (w_0 rho c_s^2 A tr(S) / (2 c_s^2) = w_0 rho A d_g u_g, the printed f_0 term). */
static void feq_iwb(double rho, double ux, double uy, double pg, double A, double Sxx, double Sxy, double Syy,
                    double feq[Q9]) {
    const double Xxx = ux * ux + CS2 * A * Sxx, Xyy = uy * uy + CS2 * A * Syy, Xxy = ux * uy + CS2 * A * Sxy;
    const double trX = Xxx + Xyy;
    feq[0] = rho - (1.0 - WI[0]) * pg / CS2 - WI[0] * rho * trX / (2.0 * CS2);
    for (int i = 1; i < Q9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        double cXc = CX[i] * CX[i] * Xxx + 2.0 * CX[i] * CY[i] * Xxy + CY[i] * CY[i] * Xyy;
        feq[i] = WI[i] * pg / CS2 + WI[i] * rho * (cu / CS2 + (cXc - CS2 * trX) / (2.0 * CS2 * CS2));
    }
}

/* Eq. (20) with A = 0 and p_g = 0. */
static void feq_wellbalanced(double rho, double ux, double uy, double feq[Q9]) {
    feq_iwb(rho, ux, uy, 0.0, 0.0, 0.0, 0.0, 0.0, feq);
}

/* p_g = rho_0 g (y - y_ref) of Eq. (20). */
static double p_grav(const orc_params* p, int y) { return p->rho_g * p->g * ((double)y - p->y_ref); }

/* FE initialisation with gravity: f = f^eq of Eq. (20) at rest, p_g included. */
void orc_init_iwb(const orc_params* p, int nx, int ny, const double* rho0, double* f) {
    size_t N = (size_t)nx * ny;
    for (size_t c = 0; c < N; ++c) {
        double feq[Q9];
        feq_iwb(rho0[c], 0.0, 0.0, p_grav(p, (int)(c / nx)), 0.0, 0.0, 0.0, 0.0, feq);
        for (int i = 0; i < Q9; ++i) f[(size_t)i * N + c] = feq[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Initialisation: f = f^eq(rho0, u = 0) of the model (model 0 = MP-LBM, 1 = FE). */
void orc_init(int model, int nx, int ny, const double* rho0, double* f) {
    size_t N = (size_t)nx * ny;
    for (size_t c = 0; c < N; ++c) {
        double feq[Q9];
        if (model == 0)
            feq_standard(rho0[c], 0.0, 0.0, feq);
        else
            feq_wellbalanced(rho0[c], 0.0, 0.0, feq);
        for (int i = 0; i < Q9; ++i) f[(size_t)i * N + c] = feq[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Pseudopotential (MP-LBM) pieces, cell-local given the psi field.          */

/* Eq. (10): Shan-Chen force, omega(1) = 1/3, omega(2) = 1/12. */
static double omega_of(int i) { return (CX[i] * CX[i] + CY[i] * CY[i]) == 1 ? 1.0 / 3.0 : 1.0 / 12.0; }

static void sc_force(const orc_params* p, const double* psi, int nx, int ny, int x, int y,
                     double* Fx, double* Fy) {
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < Q9; ++i) {
        double pn = psi[yrow(y + CY[i], ny, p->walls != 0.0) * nx + wrap(x + CX[i], nx)];
        sx += omega_of(i) * pn * CX[i];
        sy += omega_of(i) * pn * CY[i];
    }
    double pc = psi[y * nx + x];
    *Fx = -p->G * pc * sx;
    *Fy = -p->G * pc * sy;
}

/* Eqs. (30a), (30b), (31a), (31b): width-control tensor Q_ab. */
static void q_tensor(const orc_params* p, const double* psi, int nx, int ny, int x, int y,
                     double Q[2][2]) {
    double C1 = 5.0 / 6.0 * (p->kappa_P - 1.0);
    double C2 = 0.5 * (1.0 - p->kappa_P);
    double pc = psi[y * nx + x];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Q[a][b] = 0.0;
    for (int i = 1; i < Q9; ++i) {
        double pn = psi[yrow(y + CY[i], ny, p->walls != 0.0) * nx + wrap(x + CX[i], nx)];
        double c[2] = {(double)CX[i], (double)CY[i]};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double d = (a == b) ? 1.0 : 0.0;
                double Ciab = C1 * p->G * d + C2 * p->G * (c[a] * c[b] - CS2 * d) +
                              p->kappa_Li * p->G / 2.0 * c[a] * c[b];
                Q[a][b] += omega_of(i) * Ciab * (pn - pc);
            }
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Q[a][b] *= pc;
}

/* Relaxation rates, Eq. (3): L = diag(1/tau_rho, 1/tau_e, 1/tau_zeta, 1/tau_j,
 * 1/tau_q, 1/tau_j, 1/tau_q, 1/tau_nu, 1/tau_nu). */
static void lambda_diag(const orc_params* p, double L[Q9]) {
    L[0] = 1.0 / p->tau_rho;
    L[1] = 1.0 / p->tau_e;
    L[2] = 1.0 / p->tau_zeta;
    L[3] = 1.0 / p->tau_j;
    L[4] = 1.0 / p->tau_q;
    L[5] = 1.0 / p->tau_j;
    L[6] = 1.0 / p->tau_q;
    L[7] = 1.0 / p->tau_nu;
    L[8] = 1.0 / p->tau_nu;
}

/* ------------------------------------------------------------------------ */
/* No-slip walls on rows 0 and ny-1 (Sec. 5.3: Zou and He's velocity condition).  After
 * streaming, a wall node lacks the populations that would come from beyond the wall
 * (bottom: i = 2, 5, 6; top: i = 4, 7, 8).  They are set so that the node's momentum is
 * J = rho u - F/2 with u = 0, i.e. J = -F/2 (Eq. 6b), Zou-He style:
 *   bottom  f2 = f4 + 2/3 Jy,  f5 = f7 - (f1 - f3)/2 + Jx/2 + Jy/6,  f6 = f8 + (f1 - f3)/2 - Jx/2 + Jy/6
 *   top     f4 = f2 - 2/3 Jy,  f7 = f5 + (f1 - f3)/2 - Jx/2 - Jy/6,  f8 = f6 - (f1 - f3)/2 + Jx/2 - Jy/6
 * The node's density sum_i f_i then depends on Jy only, and the wall-normal force is the
 * body force alone (the mirrored neighbours cancel the interaction part), so a first fill
 * with Jy = -fy/2 and Jx = 0 fixes rho exactly; once the forces are known the fill is
 * repeated with Jx = -Fx/2. */
static void wall_fill(const orc_params* p, int nx, int ny, double* f, const double* Fx, const double* Fy) {
    size_t N = (size_t)nx * ny;
    for (int side = 0; side < 2; ++side) {
        const int y = side == 0 ? 0 : ny - 1;
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double* g[Q9];
            for (int i = 0; i < Q9; ++i) g[i] = &f[(size_t)i * N + c];
            const double Jx = Fx ? -Fx[c] / 2.0 : 0.0;
            const double Jy = Fy ? -Fy[c] / 2.0 : -p->fy / 2.0;
            const double d13 = *g[1] - *g[3];
            if (side == 0) {
                *g[2] = *g[4] + 2.0 / 3.0 * Jy;
                *g[5] = *g[7] - d13 / 2.0 + Jx / 2.0 + Jy / 6.0;
                *g[6] = *g[8] + d13 / 2.0 - Jx / 2.0 + Jy / 6.0;
            } else {
                *g[4] = *g[2] - 2.0 / 3.0 * Jy;
                *g[7] = *g[5] + d13 / 2.0 - Jx / 2.0 - Jy / 6.0;
                *g[8] = *g[6] - d13 / 2.0 + Jx / 2.0 - Jy / 6.0;
            }
        }
    }
}

/* Sec. 5.4: the horizontal force a_x |rho - rho_ave| that drives two droplets together;
 * a_x = drive_ax_lo for x <= drive_x_split and drive_ax_hi beyond, rho_ave the mean density
 * of the domain (domain_mean, taken every step).  It is an external force: it enters the
 * total force but not the interaction force of the sigma^Li term. */
static double domain_mean(const double* rho, size_t N) {
    double s = 0.0;
    for (size_t c = 0; c < N; ++c) s += rho[c];
    return s / (double)N;
}
static double drive_force(const orc_params* p, int x, double rho, double rho_ave) {
    if (p->drive == 0.0) return 0.0;
    const double ax = (double)x <= p->drive_x_split ? p->drive_ax_lo : p->drive_ax_hi;
    return ax * fabs(rho - rho_ave);
}

static inline int is_wall_row(const orc_params* p, int y, int ny) {
    return p->walls != 0.0 && (y == 0 || y == ny - 1);
}

/* Density, psi, force and velocity of the pseudopotential model for the whole
 * lattice (Eqs. 6a, 11, 10, 6b). psi < 0 marks a negative radicand. */
static int pp_fields(const orc_params* p, int nx, int ny, double* f, double* rho,
                     double* psi, double* Fx, double* Fy, double* ux, double* uy) {
    size_t N = (size_t)nx * ny;
    int bad = 0;
    if (p->walls != 0.0) wall_fill(p, nx, ny, f, NULL, NULL);
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long c = 0; c < (long)N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q9; ++i) s += f[(size_t)i * N + c];
        rho[c] = s;
        psi[c] = psi_of(p, s);
        if (psi[c] < 0.0 || !(s > 0.0)) bad = 1;
    }
    if (bad) return -1;
    const double rave = p->drive != 0.0 ? domain_mean(rho, N) : 0.0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double fix, fiy;
            sc_force(p, psi, nx, ny, x, y, &fix, &fiy);
            Fx[c] = fix + p->fx + drive_force(p, x, rho[c], rave);
            Fy[c] = is_wall_row(p, y, ny) ? p->fy : fiy + p->fy;
        }
    if (p->walls != 0.0) wall_fill(p, nx, ny, f, Fx, NULL);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double jx = 0.0, jy = 0.0;
            for (int i = 0; i < Q9; ++i) {
                jx += f[(size_t)i * N + c] * CX[i];
                jy += f[(size_t)i * N + c] * CY[i];
            }
            ux[c] = (jx + Fx[c] / 2.0) / rho[c];
            uy[c] = (jy + Fy[c] / 2.0) / rho[c];
        }
    return 0;
}

/* One MP-LBM time step: collision per Eq. (1) with Eqs. (4), (13), (30)-(32), then
 * streaming f_i(x + c_i) <- f*_i(x).  f is read, fnew written.  Returns 0 or -1
 * if rho <= 0 or the psi radicand is negative somewhere. */
static int pp_step(const orc_params* p, int nx, int ny, double* f, double* fnew,
                   double* rho, double* psi, double* Fx, double* Fy, double* ux, double* uy) {
    size_t N = (size_t)nx * ny;
    if (pp_fields(p, nx, ny, f, rho, psi, Fx, Fy, ux, uy)) return -1;
    const double rave = p->drive != 0.0 ? domain_mean(rho, N) : 0.0;
    double L[Q9];
    lambda_diag(p, L);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double fc[Q9], feq[Q9], m[Q9], meq[Q9], MF[Q9], MC[Q9], dm[Q9];
            for (int i = 0; i < Q9; ++i) fc[i] = f[(size_t)i * N + c];
            feq_standard(rho[c], ux[c], uy[c], feq);
            for (int k = 0; k < Q9; ++k) {
                m[k] = 0.0;
                meq[k] = 0.0;
                for (int j = 0; j < Q9; ++j) {
                    m[k] += MM[k][j] * fc[j];
                    meq[k] += MM[k][j] * feq[j];
                }
            }
            /* Eq. (32): forcing in moment space.  The consistency term uses only the
             * interaction force F_int; the velocity terms use the total force. */
            double fix = Fx[c] - p->fx - drive_force(p, x, rho[c], rave), fiy = Fy[c] - p->fy;
            double Fint2 = fix * fix + fiy * fiy;
            double uF = ux[c] * Fx[c] + uy[c] * Fy[c];
            double ps2 = psi[c] * psi[c];
            MF[0] = 0.0;
            MF[1] = 6.0 * uF + 12.0 * p->kappa_P * p->sigma_Li * Fint2 / (ps2 * (p->tau_e - 0.5));
            MF[2] = -6.0 * uF - 12.0 * p->kappa_P * p->sigma_Li * Fint2 / (ps2 * (p->tau_zeta - 0.5));
            MF[3] = Fx[c];
            MF[4] = -Fx[c];
            MF[5] = Fy[c];
            MF[6] = -Fy[c];
            MF[7] = 2.0 * (ux[c] * Fx[c] - uy[c] * Fy[c]);
            MF[8] = ux[c] * Fy[c] + uy[c] * Fx[c];
            /* Eq. (13) with the modified Q of Eq. (30). */
            double Q[2][2];
            q_tensor(p, psi, nx, ny, x, y, Q);
            MC[0] = 0.0;
            MC[1] = 1.5 / p->tau_e * (Q[0][0] + Q[1][1]);
            MC[2] = -1.5 / p->tau_zeta * (Q[0][0] + Q[1][1]);
            MC[3] = MC[4] = MC[5] = MC[6] = 0.0;
            MC[7] = -1.0 / p->tau_nu * (Q[0][0] - Q[1][1]);
            MC[8] = -1.0 / p->tau_nu * Q[0][1];
            /* Eq. (1): f* = f - M^-1 L (m - m^eq) + M^-1 (I - L/2) MF' + M^-1 MC. */
            for (int k = 0; k < Q9; ++k)
                dm[k] = -L[k] * (m[k] - meq[k]) + (1.0 - L[k] / 2.0) * MF[k] + MC[k];
            for (int i = 0; i < Q9; ++i) {
                double s = 0.0;
                for (int k = 0; k < Q9; ++k) s += MINV[i][k] * dm[k];
                int xd = wrap(x + CX[i], nx), yd = wrap(y + CY[i], ny);
                if (p->walls != 0.0 && (y + CY[i] < 0 || y + CY[i] > ny - 1)) continue;  /* leaves through a wall */
                fnew[(size_t)i * N + (size_t)yd * nx + xd] = fc[i] + s;
            }
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Free-energy (IWB-FE-LBM) pieces.                                          */

/* Eq. (24): grad phi = (1/c_s^2) sum_i w_i phi(x + c_i) c_i;
 *           lap phi  = (2/c_s^2) sum_i w_i [phi(x + c_i) - phi(x)]. */
static void stencil_grad(const double* phi, int nx, int ny, int walls, int x, int y, double* gx, double* gy) {
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < Q9; ++i) {
        double v = phi[yrow(y + CY[i], ny, walls) * nx + wrap(x + CX[i], nx)];
        sx += WI[i] * v * CX[i];
        sy += WI[i] * v * CY[i];
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
}
static double stencil_lap(const double* phi, int nx, int ny, int walls, int x, int y) {
    double s = 0.0, pc = phi[y * nx + x];
    for (int i = 0; i < Q9; ++i) s += WI[i] * (phi[yrow(y + CY[i], ny, walls) * nx + wrap(x + CX[i], nx)] - pc);
    return 2.0 / CS2 * s;
}

/* Eq. (24) gradient of a velocity component.  Beyond a no-slip wall the velocity is the
 * negative of the mirrored row's (odd extension through u = 0 at the wall node). */
static void stencil_grad_vel(const double* phi, int nx, int ny, int walls, int x, int y, double* gx, double* gy) {
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < Q9; ++i) {
        const int yy = y + CY[i];
        const double sgn = (walls && (yy < 0 || yy > ny - 1)) ? -1.0 : 1.0;
        double v = sgn * phi[yrow(yy, ny, walls) * nx + wrap(x + CX[i], nx)];
        sx += WI[i] * v * CX[i];
        sy += WI[i] * v * CY[i];
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
}

/* Free-energy walls = 2: at a wall row the normal component of grad mu is taken one-sided,
 * through the ghost mu(-1) = 2 mu(0) - mu(1) (bottom; mirrored at the top), instead of through
 * the mirrored row (which makes it zero).  With a wall-normal force (fy, gravity) the mirrored
 * reading leaves the wall node's force unbalanced at hydrostatic equilibrium, and the free-energy
 * model's neutral period-2 density mode, which no central-difference stencil damps, grows from
 * the wall rows without bound; the one-sided gradient removes that source.  The wall node's
 * density then depends on its own normal force (sum_i f_i = K +- J_y, J_y = -F_y/2, F_y through
 * mu(0), mu(1)), so it is found by fixed-point iteration of fill and force. */
static double fe_wall_grad_y(const double* mu, int nx, int ny, int x, int y) {
    const int yi = y == 0 ? 1 : ny - 2;
    const double sgn = y == 0 ? 1.0 : -1.0;
    double s = 0.0;
    for (int dx = -1; dx <= 1; ++dx) {
        const double w = dx == 0 ? WI[2] : WI[5];  /* axis and diagonal weights */
        const int xx = wrap(x + dx, nx);
        s += w * 2.0 * (mu[yi * nx + xx] - mu[y * nx + xx]);
    }
    return sgn * s / CS2;
}

static void fe_wall_density(const orc_params* p, int nx, int ny, double* f, double* rho, double* mu,
                            double* Fy) {
    size_t N = (size_t)nx * ny;
    for (int it = 0; it < 200; ++it) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                mu[(size_t)y * nx + x] = mu_bulk(p, rho[(size_t)y * nx + x]) - p->kappa * stencil_lap(rho, nx, ny, 1, x, y);
        for (int side = 0; side < 2; ++side) {
            const int y = side == 0 ? 0 : ny - 1;
            for (int x = 0; x < nx; ++x) {
                size_t c = (size_t)y * nx + x;
                Fy[c] = -rho[c] * fe_wall_grad_y(mu, nx, ny, x, y) + p->fy - (rho[c] - p->rho_g) * p->g;
            }
        }
        wall_fill(p, nx, ny, f, NULL, Fy);
        double dmax = 0.0;
        for (int side = 0; side < 2; ++side) {
            const int y = side == 0 ? 0 : ny - 1;
            for (int x = 0; x < nx; ++x) {
                size_t c = (size_t)y * nx + x;
                double s = 0.0;
                for (int i = 0; i < Q9; ++i) s += f[(size_t)i * N + c];
                dmax = fmax(dmax, fabs(s - rho[c]) / s);
                rho[c] = s;
            }
        }
        if (dmax <= 4e-16) break;  /* rounding level (reached in 16-29 sweeps) */
    }
}

/* Density, chemical potential, gradients, force and velocity of the FE model. */
static int fe_fields(const orc_params* p, int nx, int ny, double* f, double* rho,
                     double* mu, double* Fx, double* Fy, double* ux, double* uy, double* drx,
                     double* dry) {
    size_t N = (size_t)nx * ny;
    int bad = 0;
    if (p->walls != 0.0) wall_fill(p, nx, ny, f, NULL, NULL);
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long c = 0; c < (long)N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q9; ++i) s += f[(size_t)i * N + c];
        rho[c] = s;
        if (!(s > 0.0) || !(p->b * s / 4.0 < 1.0)) bad = 1;
    }
    if (bad) return -1;
    if (p->walls == 2.0) fe_wall_density(p, nx, ny, f, rho, mu, Fy);
    if (p->walls == 1.0 && p->g != 0.0) {
        /* a wall node's normal force includes gravity, -(rho - rho_0) g, which depends on its
         * own density: sum_i f_i = K + Jy (bottom) or K - Jy (top), Jy = -F_y/2, solved for
         * rho in closed form from the first fill's density (Jy = -fy/2) and filled again */
        for (int side = 0; side < 2; ++side) {
            const int y = side == 0 ? 0 : ny - 1;
            const double sg = side == 0 ? 1.0 : -1.0;
            for (int x = 0; x < nx; ++x) {
                size_t c = (size_t)y * nx + x;
                const double rw = (rho[c] - sg * p->rho_g * p->g / 2.0) / (1.0 - sg * p->g / 2.0);
                Fy[c] = p->fy - (rw - p->rho_g) * p->g;
            }
        }
        wall_fill(p, nx, ny, f, NULL, Fy);
        for (int side = 0; side < 2; ++side) {
            const int y = side == 0 ? 0 : ny - 1;
            for (int x = 0; x < nx; ++x) {
                size_t c = (size_t)y * nx + x;
                double s = 0.0;
                for (int i = 0; i < Q9; ++i) s += f[(size_t)i * N + c];
                rho[c] = s;
            }
        }
    }
    const double rave = p->drive != 0.0 ? domain_mean(rho, N) : 0.0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            mu[c] = mu_bulk(p, rho[c]) - p->kappa * stencil_lap(rho, nx, ny, p->walls != 0.0, x, y);
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double gmx, gmy;
            stencil_grad(mu, nx, ny, p->walls != 0.0, x, y, &gmx, &gmy);
            stencil_grad(rho, nx, ny, p->walls != 0.0, x, y, &drx[c], &dry[c]);
            const double Fg = -(rho[c] - p->rho_g) * p->g;  /* buoyancy F_g of Eq. (21) */
            Fx[c] = -rho[c] * gmx + p->fx + drive_force(p, x, rho[c], rave);
            Fy[c] = -rho[c] * gmy + p->fy + Fg;
            if (is_wall_row(p, y, ny)) {
                /* walls = 1: mirrored neighbours, no normal gradient; walls = 2: one-sided */
                Fy[c] = p->walls == 2.0 ? -rho[c] * fe_wall_grad_y(mu, nx, ny, x, y) + p->fy + Fg : p->fy + Fg;
                dry[c] = 0.0;
            }
        }
    if (p->walls != 0.0) wall_fill(p, nx, ny, f, Fx, Fy);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double jx = 0.0, jy = 0.0;
            for (int i = 0; i < Q9; ++i) {
                jx += f[(size_t)i * N + c] * CX[i];
                jy += f[(size_t)i * N + c] * CY[i];
            }
            ux[c] = (jx + Fx[c] / 2.0) / rho[c];
            uy[c] = (jy + Fy[c] / 2.0) / rho[c];
        }
    return 0;
}

/* One IWB-FE-LBM step: Eq. (1) with Eq. (20) equilibrium, Eq. (21) forcing, C_i = 0. */
static int fe_step(const orc_params* p, int nx, int ny, double* f, double* fnew,
                   double* rho, double* mu, double* Fx, double* Fy, double* ux, double* uy,
                   double* drx, double* dry) {
    size_t N = (size_t)nx * ny;
    if (fe_fields(p, nx, ny, f, rho, mu, Fx, Fy, ux, uy, drx, dry)) return -1;
    double L[Q9];
    lambda_diag(p, L);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double fc[Q9], feq[Q9], Fi[Q9], m[Q9], meq[Q9], MF[Q9], dm[Q9];
            for (int i = 0; i < Q9; ++i) fc[i] = f[(size_t)i * N + c];
            /* Eq. (20) with S_ab from the Eq. (24) gradients of u (only when A != 0) */
            double Sxx = 0.0, Sxy = 0.0, Syy = 0.0;
            if (p->A != 0.0) {
                double dxux, dyux, dxuy, dyuy;
                stencil_grad_vel(ux, nx, ny, p->walls != 0.0, x, y, &dxux, &dyux);
                stencil_grad_vel(uy, nx, ny, p->walls != 0.0, x, y, &dxuy, &dyuy);
                Sxx = 2.0 * dxux;
                Syy = 2.0 * dyuy;
                Sxy = dxuy + dyux;
            }
            feq_iwb(rho[c], ux[c], uy[c], p_grav(p, y), p->A, Sxx, Sxy, Syy, feq);
            /* Eq. (21), d = 2, grad p_g = (0, rho_0 g):
             * F_i = w_i [ c_a F_a / c_s^2
             *           + (c_a c_b - c_s^2 d_ab) u_a (F_b - d_b p_g + c_s^2 d_b rho) / c_s^4
             *           + 1/2 (|c|^2 / c_s^2 - d) u_g d_g rho ] */
            const double dpg[2] = {0.0, p->rho_g * p->g};
            double u[2] = {ux[c], uy[c]}, F[2] = {Fx[c], Fy[c]}, gr[2] = {drx[c], dry[c]};
            double ugr = u[0] * gr[0] + u[1] * gr[1];
            for (int i = 0; i < Q9; ++i) {
                double ci[2] = {(double)CX[i], (double)CY[i]};
                double t1 = (ci[0] * F[0] + ci[1] * F[1]) / CS2;
                double t2 = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        double d = (a == b) ? 1.0 : 0.0;
                        t2 += (ci[a] * ci[b] - CS2 * d) * u[a] * (F[b] - dpg[b] + CS2 * gr[b]);
                    }
                t2 /= CS2 * CS2;
                double c2 = ci[0] * ci[0] + ci[1] * ci[1];
                double t3 = 0.5 * (c2 / CS2 - 2.0) * ugr;
                Fi[i] = WI[i] * (t1 + t2 + t3);
            }
            for (int k = 0; k < Q9; ++k) {
                m[k] = meq[k] = MF[k] = 0.0;
                for (int j = 0; j < Q9; ++j) {
                    m[k] += MM[k][j] * fc[j];
                    meq[k] += MM[k][j] * feq[j];
                    MF[k] += MM[k][j] * Fi[j];
                }
            }
            for (int k = 0; k < Q9; ++k) dm[k] = -L[k] * (m[k] - meq[k]) + (1.0 - L[k] / 2.0) * MF[k];
            for (int i = 0; i < Q9; ++i) {
                double s = 0.0;
                for (int k = 0; k < Q9; ++k) s += MINV[i][k] * dm[k];
                int xd = wrap(x + CX[i], nx), yd = wrap(y + CY[i], ny);
                if (p->walls != 0.0 && (y + CY[i] < 0 || y + CY[i] > ny - 1)) continue;  /* leaves through a wall */
                fnew[(size_t)i * N + (size_t)yd * nx + xd] = fc[i] + s;
            }
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Public entry points (ctypes).                                            */

typedef struct {
    double *rho, *aux, *Fx, *Fy, *ux, *uy, *drx, *dry, *ftmp;
} work_t;

static int work_alloc(work_t* w, size_t N) {
    memset(w, 0, sizeof(*w));
    w->rho = malloc(N * sizeof(double));
    w->aux = malloc(N * sizeof(double));
    w->Fx = malloc(N * sizeof(double));
    w->Fy = malloc(N * sizeof(double));
    w->ux = malloc(N * sizeof(double));
    w->uy = malloc(N * sizeof(double));
    w->drx = malloc(N * sizeof(double));
    w->dry = malloc(N * sizeof(double));
    w->ftmp = malloc(Q9 * N * sizeof(double));
    return (w->rho && w->aux && w->Fx && w->Fy && w->ux && w->uy && w->drx && w->dry && w->ftmp) ? 0 : -1;
}
static void work_free(work_t* w) {
    free(w->rho); free(w->aux); free(w->Fx); free(w->Fy); free(w->ux);
    free(w->uy); free(w->drx); free(w->dry); free(w->ftmp);
}

/* Advance f (in place, SoA [9][ny][nx]) by nsteps time steps of the given model.
 * nthreads <= 0 keeps the OpenMP default.  Returns the number of steps done
 * (< nsteps if the state became invalid: rho <= 0, eta >= 1 or psi^2 < 0). */
long orc_run(int model, const orc_params* p, int nx, int ny, double* f, long nsteps, int nthreads) {
    ensure_minv();
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    size_t N = (size_t)nx * ny;
    work_t w;
    if (work_alloc(&w, N)) {
        work_free(&w);
        return -1;
    }
    double *cur = f, *nxt = w.ftmp;
    long s;
    for (s = 0; s < nsteps; ++s) {
        int rc = model == 0 ? pp_step(p, nx, ny, cur, nxt, w.rho, w.aux, w.Fx, w.Fy, w.ux, w.uy)
                            : fe_step(p, nx, ny, cur, nxt, w.rho, w.aux, w.Fx, w.Fy, w.ux, w.uy,
                                      w.drx, w.dry);
        if (rc) break;
        double* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (p->walls != 0.0 && s == nsteps) {
        /* complete the wall nodes' incoming populations of the returned state */
        if (model == 0)
            pp_fields(p, nx, ny, cur, w.rho, w.aux, w.Fx, w.Fy, w.ux, w.uy);
        else
            fe_fields(p, nx, ny, cur, w.rho, w.aux, w.Fx, w.Fy, w.ux, w.uy, w.drx, w.dry);
    }
    if (cur != f) memcpy(f, cur, Q9 * N * sizeof(double));
    work_free(&w);
    return s;
}

/* Macroscopic fields of the current populations: rho (Eq. 6a), u including the
 * half-force shift (Eq. 6b), the total force, and the model's auxiliary field
 * (psi for the pseudopotential model, mu for the free-energy model). */
int orc_macro(int model, const orc_params* p, int nx, int ny, const double* f, double* rho,
              double* ux, double* uy, double* Fx, double* Fy, double* aux) {
    size_t N = (size_t)nx * ny;
    work_t w;
    if (work_alloc(&w, N)) {
        work_free(&w);
        return -1;
    }
    memcpy(w.ftmp, f, Q9 * N * sizeof(double));  /* the wall fill writes the populations */
    int rc = model == 0 ? pp_fields(p, nx, ny, w.ftmp, w.rho, w.aux, w.Fx, w.Fy, w.ux, w.uy)
                        : fe_fields(p, nx, ny, w.ftmp, w.rho, w.aux, w.Fx, w.Fy, w.ux, w.uy, w.drx, w.dry);
    if (rc == 0) {
        if (rho) memcpy(rho, w.rho, N * sizeof(double));
        if (ux) memcpy(ux, w.ux, N * sizeof(double));
        if (uy) memcpy(uy, w.uy, N * sizeof(double));
        if (Fx) memcpy(Fx, w.Fx, N * sizeof(double));
        if (Fy) memcpy(Fy, w.Fy, N * sizeof(double));
        if (aux) memcpy(aux, w.aux, N * sizeof(double));
    }
    work_free(&w);
    return rc;
}

/* Cell-local building blocks exposed for the moment tests (Eqs. 4, 20, 21, 32, 13). */
void orc_feq(int model, double rho, double ux, double uy, double* feq) {
    if (model == 0)
        feq_standard(rho, ux, uy, feq);
    else
        feq_wellbalanced(rho, ux, uy, feq);
}

/* Eq. (20) in full for given rho, u, p_g, A and S (Sxx, Sxy, Syy). */
void orc_feq_iwb(double rho, double ux, double uy, double pg, double A, double Sxx, double Sxy, double Syy,
                 double* feq) {
    feq_iwb(rho, ux, uy, pg, A, Sxx, Sxy, Syy, feq);
}

/* Population-space forcing of the FE model, Eq. (21), for given u, F, grad rho. */
void orc_fe_forcing(double ux, double uy, double Fx, double Fy, double gx, double gy, double* Fi) {
    double u[2] = {ux, uy}, F[2] = {Fx, Fy}, gr[2] = {gx, gy};
    double ugr = ux * gx + uy * gy;
    for (int i = 0; i < Q9; ++i) {
        double ci[2] = {(double)CX[i], (double)CY[i]};
        double t1 = (ci[0] * F[0] + ci[1] * F[1]) / CS2, t2 = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                t2 += (ci[a] * ci[b] - CS2 * (a == b)) * u[a] * (F[b] + CS2 * gr[b]);
        t2 /= CS2 * CS2;
        double c2 = ci[0] * ci[0] + ci[1] * ci[1];
        Fi[i] = WI[i] * (t1 + t2 + 0.5 * (c2 / CS2 - 2.0) * ugr);
    }
}

/* Population-space pieces S_i = [M^-1 (I - L/2) M] F' and C_i = M^-1 MC of the
 * pseudopotential model at one cell, for given u, F, F_int, psi and Q (Eqs. 32, 13). */
void orc_pp_sources(const orc_params* p, double ux, double uy, double Fx, double Fy,
                    double Fix, double Fiy, double psi, double Qxx, double Qyy, double Qxy,
                    double* S, double* C) {
    ensure_minv();
    double L[Q9], MF[Q9], MC[Q9];
    lambda_diag(p, L);
    double uF = ux * Fx + uy * Fy, Fint2 = Fix * Fix + Fiy * Fiy, ps2 = psi * psi;
    MF[0] = 0.0;
    MF[1] = 6.0 * uF + 12.0 * p->kappa_P * p->sigma_Li * Fint2 / (ps2 * (p->tau_e - 0.5));
    MF[2] = -6.0 * uF - 12.0 * p->kappa_P * p->sigma_Li * Fint2 / (ps2 * (p->tau_zeta - 0.5));
    MF[3] = Fx; MF[4] = -Fx; MF[5] = Fy; MF[6] = -Fy;
    MF[7] = 2.0 * (ux * Fx - uy * Fy);
    MF[8] = ux * Fy + uy * Fx;
    MC[0] = 0.0;
    MC[1] = 1.5 / p->tau_e * (Qxx + Qyy);
    MC[2] = -1.5 / p->tau_zeta * (Qxx + Qyy);
    MC[3] = MC[4] = MC[5] = MC[6] = 0.0;
    MC[7] = -1.0 / p->tau_nu * (Qxx - Qyy);
    MC[8] = -1.0 / p->tau_nu * Qxy;
    for (int i = 0; i < Q9; ++i) {
        double s = 0.0, c = 0.0;
        for (int k = 0; k < Q9; ++k) {
            s += MINV[i][k] * (1.0 - L[k] / 2.0) * MF[k];
            c += MINV[i][k] * MC[k];
        }
        S[i] = s;
        C[i] = c;
    }
}

/* Q tensor of Eq. (30) on a given psi field at (x, y): out = {Qxx, Qyy, Qxy}. */
void orc_q_tensor(const orc_params* p, const double* psi, int nx, int ny, int x, int y, double* out) {
    double Q[2][2];
    q_tensor(p, psi, nx, ny, x, y, Q);
    out[0] = Q[0][0];
    out[1] = Q[1][1];
    out[2] = Q[0][1];
}

/* Stencils of Eq. (24) on a given field at (x, y): out = {d_x, d_y, lap}. */
void orc_stencils(const double* phi, int nx, int ny, int x, int y, double* out) {
    stencil_grad(phi, nx, ny, 0, x, y, &out[0], &out[1]);
    out[2] = stencil_lap(phi, nx, ny, 0, x, y);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
