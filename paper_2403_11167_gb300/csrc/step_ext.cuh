// step_ext.cuh -- direct step and field kernels with the two extensions of the paper's flow
// tests: no-slip walls on rows 0 and ny-1 (periodic in x; the two-phase flow between
// parallel plates of Sec. 5.3, driven by the constant body force of StepParams::fx, fy) and
// the density-dependent drive of the droplet collision of Sec. 5.4 (Drive).
//
// Wall treatment (Zou and He's velocity condition, cited in Sec. 5.3):
//   * a wall node lacks the populations that would stream in from beyond the wall (bottom:
//     i = 2, 5, 6; top: i = 4, 7, 8).  They are set so that the node momentum is J = -F/2,
//     i.e. u = 0 including the half-force shift of Eq. (6b) (wall_fill);
//   * every stencil (psi, rho, mu and their gradients / Laplacian) sees beyond a wall the
//     row mirrored through it (row -1 is row 1, row ny is row ny-2).  The wall-normal
//     component of each central-difference gradient is then exactly zero, so a wall node's
//     normal force is the body force alone and its density, sum_i f_i, depends on J_y only:
//     a first fill with J = (0, -fy/2) fixes rho, psi and mu; after the forces are known the
//     fill is repeated with J_x = -F_x/2 before the collision.
//   * populations that stream out through a wall are dropped: in the pull layout (a buffer
//     holds S_i(y) = f_i(y + c_i)) their slots are exactly the slots a wall node pulls its
//     unknowns from, which the fill overwrites.
//
// Droplet-collision drive (Sec. 5.4): the force a_x |rho - rho_ave| along x, a_x = ax_lo for
// x <= x_split and ax_hi beyond, rho_ave the mean density of the state being collided, from
// block sums of every stored population (mass_partials_kernel and mass_final_kernel, launched
// before the step: the pull layout holds each population of a periodic lattice exactly once).  It is an external
// force: it adds to the total force like the body force and stays out of the interaction
// force of Eq. (32)'s sigma^Li term.
//
// Full free-energy model (fe_step_iwb): the viscosity-tuning term A of Eqs. (20)/(23), which
// needs the strain rate of u and so u at the neighbours (one more ring level: rho -> mu -> u ->
// collision), and gravity: p_g = rho_g g (y - y_ref) in the equilibrium, -grad p_g in the
// forcing's second-order term, and the buoyancy F_g = -(rho - rho_g) g in the force (Eq. 21).
// Beyond a wall, velocities are odd (u = 0 at the wall node).
//
// The kernels follow the direct step kernels of lbm_kernels.cuh (one column per thread,
// shared-memory rings of the neighbour fields, one halo warp).  With WALLS the pulled rows
// map through mirror_row, wall rows get the two fills, and a wall row's collision sees its
// neighbour fields mirrored; without, rows wrap.  Requirements (checked on the host): with
// walls ny >= 4.
//
// band > 0 launches only the rows next to the walls: grid.y = 2, CTA row 0 updates rows
// [0, band), CTA row 1 rows [ny - band, ny).  This completes a step whose interior was
// updated by a periodic step kernel: a periodic stencil is exact on every row whose
// neighbourhood holds neither a wall row (whose density needs the fill) nor a row beyond
// the wall (mirrored, not wrapped).  The pseudopotential collision reads psi one row away
// (rows 0 and 1 differ, band = 2); the free-energy collision reads mu one row away and mu
// reads rho one row further (rows 0, 1, 2 differ, band = 3).
#pragma once
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbmk {

// Row seen by a stencil: rows beyond a wall are mirrored through the wall node.
__host__ __device__ __forceinline__ int mirror_row(int y, int ny) {
    return y < 0 ? -y : (y > ny - 1 ? 2 * (ny - 1) - y : y);
}

// Zou-He completion of a wall node for the node momentum (Jx, Jy):
//   bottom  f2 = f4 + 2/3 Jy,  f5 = f7 - (f1 - f3)/2 + Jx/2 + Jy/6,  f6 = f8 + (f1 - f3)/2 - Jx/2 + Jy/6
//   top     f4 = f2 - 2/3 Jy,  f7 = f5 + (f1 - f3)/2 - Jx/2 - Jy/6,  f8 = f6 - (f1 - f3)/2 + Jx/2 - Jy/6
// (sum_i f_i c_i = J follows from these and the known populations).
template <typename real>
__device__ __forceinline__ void wall_fill(real v[9], bool top, real Jx, real Jy) {
    const real h = real(0.5) * (v[1] - v[3]);
    const real hx = real(0.5) * Jx, sy = Jy * real(1.0 / 6.0), ty = Jy * real(2.0 / 3.0);
    if (!top) {
        v[2] = v[4] + ty;
        v[5] = (v[7] - h) + (hx + sy);
        v[6] = (v[8] + h) - (hx - sy);
    } else {
        v[4] = v[2] - ty;
        v[7] = (v[5] + h) - (hx + sy);
        v[8] = (v[6] - h) + (hx - sy);
    }
}

// Neighbour values n[i] at x + c_i of a wall node with the rows beyond the wall replaced by
// their mirror images (bottom: 4 <- 2, 7 <- 6, 8 <- 5; top: 2 <- 4, 5 <- 8, 6 <- 7).
template <typename real>
__device__ __forceinline__ void mirror_neighbours(real n[9], bool top) {
    if (!top) {
        n[4] = n[2];
        n[7] = n[6];
        n[8] = n[5];
    } else {
        n[2] = n[4];
        n[5] = n[8];
        n[6] = n[7];
    }
}

// x component of the Eq. (24) gradient weights (sum_i w_i phi_i c_ix / c_s^2), as in the
// collision functions.
template <typename real>
__device__ __forceinline__ real grad_x(const real n[9]) {
    return (n[1] - n[3]) * real(1.0 / 3.0) + ((n[5] - n[7]) + (n[8] - n[6])) * real(1.0 / 12.0);
}

// Row seen by a stencil: mirrored through a wall, or wrapped (periodic; any ny >= 1).
template <bool WALLS>
__device__ __forceinline__ int stencil_row(int y, int ny) {
    return WALLS ? mirror_row(y, ny) : ((y % ny) + ny) % ny;
}

// Pulled populations of row y (already mapped) of column x; with walls a wall row gets the
// first fill, J = (0, -fy/2).  The pull of a wall row reads its unknowns from the wrapped
// row: in bounds, and overwritten by the fill.
template <bool WALLS, typename real>
__device__ __forceinline__ void pull_row_ext(const real* __restrict__ f, const StepParams<real>& P, int x, int xm,
                                             int xp, int y, real v[9], const real* __restrict__ wjy = nullptr) {
    const int ny = P.ny, nx = P.nx;
    const long long om = (long long)(y == 0 ? ny - 1 : y - 1) * nx, o0 = (long long)y * nx,
                    op = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
    pull9(f, P.pitch, x, xm, xp, om, o0, op, v);
    // wjy: the wall rows' solved J_y (one-sided reading, fe_wall_solve_kernel), bottom then top
    if (WALLS && (y == 0 || y == ny - 1))
        wall_fill(v, y != 0, real(0), wjy ? wjy[(y != 0 ? nx : 0) + x] : real(-0.5) * P.fy);
}

// One-sided reading of the free-energy walls: the wall-normal Eq. (24) gradient of mu at a
// wall node through the ghost mu(-1) = 2 mu(0) - mu(1) (bottom; mu(ny) = 2 mu(ny-1) - mu(ny-2)
// at the top), n[i] = mu at x + c_i (only the entries inside the lattice are read).  With the
// mirrored reading a wall-normal force (fy, gravity) is left unbalanced at the wall node and
// drives the free-energy model's neutral period-2 mode; this reading removes that source.
template <typename real>
__device__ __forceinline__ real wall_grad_y_onesided(const real n[9], bool top) {
    const real a = real(2.0 / 9.0), d = real(1.0 / 18.0);
    if (!top) return real(3) * (a * (n[2] - n[0]) + d * ((n[5] - n[1]) + (n[6] - n[3])));
    return -real(3) * (a * (n[4] - n[0]) + d * ((n[8] - n[1]) + (n[7] - n[3])));
}

// Full improved well-balanced free-energy terms (Eqs. 20, 21): the viscosity-tuning A and
// gravity g along -y with reference density rho_g, p_g = rho_g g (y - y_ref).  on == 0: none.
template <typename real>
struct Ext {
    int on;
    real A, g, rho_g, y_ref;
};

// With gravity a wall node's normal force, fy - (rho - rho_g) g, depends on its own density:
// sum_i f_i = K + Jy (bottom) or K - Jy (top) with Jy = -F_y/2.  Solved in closed form from
// the density after the first fill (Jy = -fy/2), then filled again.
template <typename real>
__device__ __forceinline__ void wall_gravity_refill(real v[9], bool top, const StepParams<real>& P,
                                                    const Ext<real>& E) {
    const real rp = sum9(v);
    const real sg = top ? real(-1) : real(1);
    const real rw = (rp - sg * E.rho_g * E.g * real(0.5)) / (real(1) - sg * E.g * real(0.5));
    wall_fill(v, top, real(0), real(-0.5) * (P.fy - (rw - E.rho_g) * E.g));
}

// Parameters of one cell's collision with the drive added to the body force.
template <typename real>
__device__ __forceinline__ StepParams<real> with_drive(const StepParams<real>& P, const Drive<real>& D, int x,
                                                       real rho, real rho_ave) {
    StepParams<real> Q = P;
    const real d = rho > rho_ave ? rho - rho_ave : rho_ave - rho;
    Q.fx = P.fx + (x <= D.x_split ? D.ax_lo : D.ax_hi) * d;
    return Q;
}

// Block sums of every stored population (9 planes of n cells) into out[blockIdx.x]: per thread
// a plane-by-plane strided sum (in the storage precision within a plane, FP64 across planes and
// in the block tree).  Fixed grid and order: deterministic.
template <typename real>
__global__ void __launch_bounds__(256) mass_partials_kernel(const real* __restrict__ f, long long pitch, long long n,
                                                            double* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
        const real* p = f + i * pitch;
        real a = real(0), b = real(0);
        long long k = t0;
        for (; k + stride < n; k += 2 * stride) {
            a += __ldg(p + k);
            b += __ldg(p + k + stride);
        }
        if (k < n) a += __ldg(p + k);
        s += (double)a + (double)b;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        out[blockIdx.x] = t;
    }
}

// rho_ave = (sum of nparts block sums) * inv_cells into *rho_ave; one warp, fixed order.
__global__ void mass_final_kernel(const double* __restrict__ parts, int nparts, double inv_cells,
                                  double* __restrict__ rho_ave) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 32) s += parts[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *rho_ave = s * inv_cells;
}

// ---------------------------------------------------------------------------------
// Pseudopotential step (Eqs. 1, 4, 6, 10, 11, 13, 30-32) with walls and/or the drive.
template <typename real, int TX, bool WALLS>
__global__ void __launch_bounds__(TX + 32) pp_step_ext(const real* __restrict__ fin, real* __restrict__ fout,
                                                       const StepParams<real> P, int band, const Drive<real> D) {
    __shared__ real s_psi[4][TX + 2];
    const real s_rave = D.rho_ave ? real(*D.rho_ave) : real(0);
    const int nx = P.nx, ny = P.ny;
    const long long pitch = P.pitch;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int y0 = band > 0 ? (blockIdx.y == 0 ? 0 : ny - band) : blockIdx.y * P.rows;
    const int y1 = band > 0 ? y0 + band : min(y0 + P.rows, ny);
    const int t = threadIdx.x;
    const bool is_main = t < TX;
    bool has_col;
    int x, sc;
    if (is_main) {
        has_col = t < w;
        x = x0 + (has_col ? t : 0);
        sc = t + 1;
    } else {
        const int lane = t - TX;
        has_col = lane < 2;
        x = lane == 0 ? wrap_idx(x0 - 1, nx) : wrap_idx(x0 + w, nx);
        sc = lane == 0 ? 0 : w + 1;
    }
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;

    real cur[9], prv[9];
    real rho_cur = real(1), rho_prv = real(1);
    if (has_col) {
        pull_row_ext<WALLS>(fin, P, x, xm, xp, stencil_row<WALLS>(y0 - 1, ny), cur);
        rho_cur = sum9(cur);
    }
#pragma unroll 1
    for (int r = y0 - 1; r <= y1; ++r) {
        real nxt[9];
        real rho_nxt = real(1);
        if (has_col && r < y1) {
            pull_row_ext<WALLS>(fin, P, x, xm, xp, stencil_row<WALLS>(r + 1, ny), nxt);
            rho_nxt = sum9(nxt);
        }
        if (has_col) s_psi[r & 3][sc] = pseudo_psi(rho_cur, P);
        __syncthreads();
        if (is_main && has_col && r > y0) {
            // centre row c = r - 1: neighbours in rows c-1 (slot r-2), c (r-1), c+1 (r)
            const int c = r - 1;
            const real* sm = s_psi[(r - 2) & 3];
            const real* s0 = s_psi[(r - 1) & 3];
            const real* sp = s_psi[r & 3];
            real pn[9];
            pn[0] = s0[sc];
            pn[1] = s0[sc + 1];
            pn[2] = sp[sc];
            pn[3] = s0[sc - 1];
            pn[4] = sm[sc];
            pn[5] = sp[sc + 1];
            pn[6] = sp[sc - 1];
            pn[7] = sm[sc - 1];
            pn[8] = sm[sc + 1];
            if (WALLS && (c == 0 || c == ny - 1)) {
                mirror_neighbours(pn, c != 0);
                const real Fx = pn[0] * grad_x(pn) + P.fx;  // F_int,x + body force (Eq. 10)
                wall_fill(prv, c != 0, real(-0.5) * Fx, real(-0.5) * P.fy);
            }
            const long long o = (long long)c * nx + x;
            const StepParams<real> Pd = D.rho_ave ? with_drive(P, D, x, rho_prv, s_rave) : P;
            if constexpr (std::is_same<real, float>::value) {
                int q = rest_lo_plane(fin, pitch)[o];  // compensated rest population
                pp_collide_comp(prv, q, rho_prv, pn[0], pn, Pd);
                rest_lo_plane(fout, pitch)[o] = (short)q;
            } else {
                pp_collide(prv, rho_prv, pn[0], pn, Pd);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) fout[i * pitch + o] = prv[i];
        }
        if (has_col) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                prv[i] = cur[i];
                cur[i] = nxt[i];
            }
            rho_prv = rho_cur;
            rho_cur = rho_nxt;
        }
    }
}

// ---------------------------------------------------------------------------------
// Free-energy step (Eqs. 1, 6, 20, 21, 24, 29) with walls and/or the drive.  Rings as in fe_step_kernel:
// rho (8 rows, 2 halo columns each side), mu (4 rows, 1 halo column).
template <typename real, int TX, bool WALLS>
__global__ void __launch_bounds__(TX + 32) fe_step_ext(const real* __restrict__ fin, real* __restrict__ fout,
                                                       const StepParams<real> P, int band, const Drive<real> D,
                                                       const real* __restrict__ wjy) {
    __shared__ real s_rho[8][TX + 4];
    __shared__ real s_mu[4][TX + 2];
    const real s_rave = D.rho_ave ? real(*D.rho_ave) : real(0);
    const int nx = P.nx, ny = P.ny;
    const long long pitch = P.pitch;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int y0 = band > 0 ? (blockIdx.y == 0 ? 0 : ny - band) : blockIdx.y * P.rows;
    const int y1 = band > 0 ? y0 + band : min(y0 + P.rows, ny);
    const int t = threadIdx.x;
    const bool is_main = t < TX;
    bool has_col, has_mu;
    int x, rc, mc;  // global column, rho-ring column, mu-ring column
    if (is_main) {
        has_col = t < w;
        has_mu = has_col;
        x = x0 + (has_col ? t : 0);
        rc = t + 2;
        mc = t + 1;
    } else {
        const int lane = t - TX;
        has_col = lane < 4;
        has_mu = lane == 1 || lane == 2;
        const int off = lane == 0 ? -2 : lane == 1 ? -1 : lane == 2 ? w : w + 1;
        x = wrap_idx(x0 + off, nx);
        rc = lane == 0 ? 0 : lane == 1 ? 1 : lane == 2 ? w + 2 : w + 3;
        mc = lane == 1 ? 0 : w + 1;
    }
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    real p0[9], p1[9], p2[9];  // pulled populations of rows r-2, r-1, r
    if (has_col) pull_row_ext<WALLS>(fin, P, x, xm, xp, stencil_row<WALLS>(y0 - 2, ny), p2, wjy);
#pragma unroll 1
    for (int r = y0 - 2; r <= y1 + 1; ++r) {
        real nxt[9];
        if (has_col && r <= y1) pull_row_ext<WALLS>(fin, P, x, xm, xp, stencil_row<WALLS>(r + 1, ny), nxt, wjy);
        if (has_col) s_rho[r & 7][rc] = sum9(p2);
        __syncthreads();
        if (has_mu && r >= y0) {
            // mu at row r - 1 from rho rows r-2, r-1, r (mirrored rows hold mirrored rho)
            const real* rm = s_rho[(r - 2) & 7];
            const real* r0 = s_rho[(r - 1) & 7];
            const real* rp = s_rho[r & 7];
            real rn[9];
            rn[1] = r0[rc + 1];
            rn[2] = rp[rc];
            rn[3] = r0[rc - 1];
            rn[4] = rm[rc];
            rn[5] = rp[rc + 1];
            rn[6] = rp[rc - 1];
            rn[7] = rm[rc - 1];
            rn[8] = rm[rc + 1];
            rn[0] = r0[rc];  // every entry defined: the FP32 overload copies all nine
            s_mu[(r - 1) & 3][mc] = fe_mu(r0[rc], rn, P);
        }
        __syncthreads();
        if (is_main && has_col && r >= y0 + 2) {
            // centre row c = r - 2
            const int c = r - 2;
            const real* mm = s_mu[(r - 3) & 3];
            const real* m0 = s_mu[(r - 2) & 3];
            const real* mp = s_mu[(r - 1) & 3];
            const real* rm = s_rho[(r - 3) & 7];
            const real* r0 = s_rho[(r - 2) & 7];
            const real* rp = s_rho[(r - 1) & 7];
            real mn[9], rn[9];
            mn[1] = m0[mc + 1]; mn[2] = mp[mc]; mn[3] = m0[mc - 1]; mn[4] = mm[mc];
            mn[5] = mp[mc + 1]; mn[6] = mp[mc - 1]; mn[7] = mm[mc - 1]; mn[8] = mm[mc + 1];
            rn[1] = r0[rc + 1]; rn[2] = rp[rc]; rn[3] = r0[rc - 1]; rn[4] = rm[rc];
            rn[5] = rp[rc + 1]; rn[6] = rp[rc - 1]; rn[7] = rm[rc - 1]; rn[8] = rm[rc + 1];
            const real rho_c = r0[rc];
            mn[0] = m0[mc];
            rn[0] = rho_c;
            StepParams<real> Pc = P;
            if (WALLS && (c == 0 || c == ny - 1)) {
                // one-sided reading: the normal force -rho d_y mu enters through fy (the
                // mirrored mu below makes the collision's own normal gradient zero)
                if (wjy) Pc.fy = P.fy - rho_c * wall_grad_y_onesided(mn, c != 0);
                // mu beyond the wall is mu of the mirrored row (the ring holds the value
                // recomputed from mirrored rho, equal up to rounding order)
                mirror_neighbours(mn, c != 0);
                mirror_neighbours(rn, c != 0);
                const real Fx = -rho_c * grad_x(mn) + P.fx;  // F = -rho grad mu + body force
                wall_fill(p0, c != 0, real(-0.5) * Fx, real(-0.5) * Pc.fy);
            }
            const long long o = (long long)c * nx + x;
            const StepParams<real> Pd = D.rho_ave ? with_drive(Pc, D, x, rho_c, s_rave) : Pc;
            if constexpr (std::is_same<real, float>::value) {
                int q = rest_lo_plane(fin, pitch)[o];  // compensated rest population
                fe_collide_comp(p0, q, rho_c, mn, rn, Pd);
                rest_lo_plane(fout, pitch)[o] = (short)q;
            } else {
                fe_collide(p0, rho_c, mn, rn, Pd);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) fout[i * pitch + o] = p0[i];
        }
        if (has_col) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                p0[i] = p1[i];
                p1[i] = p2[i];
                p2[i] = nxt[i];
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Fields of the current state of a walled channel (observables, not on the step path).

// Values at x + c_i with rows beyond a wall mirrored (walls) or wrapped; n[0] is the cell.
template <typename real>
__device__ __forceinline__ void gather8_ext(const real* __restrict__ a, int x, int y, int nx, int ny, bool walls,
                                            real n[9]) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int rm = walls ? mirror_row(y - 1, ny) : (y == 0 ? ny - 1 : y - 1);
    const int rp = walls ? mirror_row(y + 1, ny) : (y == ny - 1 ? 0 : y + 1);
    const long long ym = (long long)rm * nx, y0 = (long long)y * nx, yp = (long long)rp * nx;
    n[0] = a[y0 + x];
    n[1] = a[y0 + xp];
    n[2] = a[yp + x];
    n[3] = a[y0 + xm];
    n[4] = a[ym + x];
    n[5] = a[yp + xp];
    n[6] = a[yp + xm];
    n[7] = a[ym + xm];
    n[8] = a[ym + xp];
}

// rho (Eq. 6a, wall rows after the first fill) and aux = psi (P) or rho (FE).
template <typename real>
__global__ void rho_walls_kernel(const real* __restrict__ f, real* __restrict__ rho, real* __restrict__ aux,
                                 const StepParams<real> P, int model, const Ext<real> E,
                                 const real* __restrict__ wjy) {
    const long long n = (long long)P.nx * P.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % P.nx), y = (int)(c / P.nx);
        real v[9];
        pull_row_ext<true>(f, P, x, x == 0 ? P.nx - 1 : x - 1, x == P.nx - 1 ? 0 : x + 1, y, v, wjy);
        if (!wjy && E.on && E.g != real(0) && (y == 0 || y == P.ny - 1)) wall_gravity_refill(v, y != 0, P, E);
        real r;
        if constexpr (std::is_same<real, float>::value)
            r = sum9_rest(v, rest_lo_plane(f, P.pitch)[c], P);
        else
            r = sum9(v);
        rho[c] = r;
        aux[c] = model == 0 ? pseudo_psi(r, P) : r;
    }
}

// FE: mu from rho with mirrored rows (writes into mu).
template <typename real>
__global__ void mu_walls_kernel(const real* __restrict__ rho, real* __restrict__ mu, const StepParams<real> P) {
    const long long n = (long long)P.nx * P.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        real rn[9];
        gather8_ext(rho, (int)(c % P.nx), (int)(c / P.nx), P.nx, P.ny, true, rn);
        mu[c] = fe_mu(rn[0], rn, P);
    }
}

// Completes the wall nodes of the stored state: the final fill (J = -F/2) of each wall node,
// written into the slots its unknowns are pulled from (the dropped outgoing populations),
// so that pulling any cell returns the full state.  Each thread reads and writes only its
// own node's unknown slots.  aux = psi (P) or mu (FE).
template <typename real>
__global__ void walls_complete_kernel(real* __restrict__ f, const real* __restrict__ rho,
                                      const real* __restrict__ aux, const StepParams<real> P, int model,
                                      const Ext<real> E, int onesided) {
    const int nx = P.nx, ny = P.ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * nx; k += gridDim.x * blockDim.x) {
        const bool top = k >= nx;
        const int x = top ? k - nx : k, y = top ? ny - 1 : 0;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        real v[9], an[9];
        pull_row_ext<true>(f, P, x, xm, xp, y, v);
        gather8_ext(aux, x, y, nx, ny, true, an);
        const long long c = (long long)y * nx + x;
        const real Fx = (model == 0 ? an[0] : -rho[c]) * grad_x(an) + P.fx;
        const real Fy = P.fy - (E.on ? (rho[c] - E.rho_g) * E.g : real(0)) -
                        (onesided ? rho[c] * wall_grad_y_onesided(an, top) : real(0));
        wall_fill(v, top, real(-0.5) * Fx, real(-0.5) * Fy);
        // f_i(x, y) = S_i(x - c_i): bottom unknowns 2 (0,1), 5 (1,1), 6 (-1,1) sit in row ny-1;
        // top unknowns 4 (0,-1), 7 (-1,-1), 8 (1,-1) in row 0
        const long long ro = top ? 0 : (long long)(ny - 1) * nx;
        if (!top) {
            f[2 * P.pitch + ro + x] = v[2];
            f[5 * P.pitch + ro + xm] = v[5];
            f[6 * P.pitch + ro + xp] = v[6];
        } else {
            f[4 * P.pitch + ro + x] = v[4];
            f[7 * P.pitch + ro + xp] = v[7];
            f[8 * P.pitch + ro + xm] = v[8];
        }
    }
}

// u of Eq. (6b) with the total force: walls -- of the completed state, mirrored neighbour
// fields (the wall-normal interaction force vanishes at wall nodes, so u = 0 there up to
// rounding); D.rho_ave -- the drive of the state included.
template <typename real>
__global__ void velocity_ext_kernel(const real* __restrict__ f, const real* __restrict__ rho,
                                    const real* __restrict__ aux, real* __restrict__ ux, real* __restrict__ uy,
                                    const StepParams<real> P, int model, int walls, const Drive<real> D,
                                    const Ext<real> E, int onesided) {
    const long long n = (long long)P.nx * P.ny;
    const real rave = D.rho_ave ? real(*D.rho_ave) : real(0);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % P.nx), y = (int)(c / P.nx);
        real v[9], an[9];
        pull_cell(f, P.pitch, x, y, P.nx, P.ny, v);
        gather8_ext(aux, x, y, P.nx, P.ny, walls != 0, an);
        const real w1 = real(1.0 / 3.0), w2 = real(1.0 / 12.0);
        const real gx = (an[1] - an[3]) * w1 + ((an[5] - an[7]) + (an[8] - an[6])) * w2;
        const real gy = (an[2] - an[4]) * w1 + ((an[5] - an[7]) + (an[6] - an[8])) * w2;
        const real r = rho[c];
        const real s = model == 0 ? an[0] : -r;
        const real Fx = s * gx + (D.rho_ave ? with_drive(P, D, x, r, rave).fx : P.fx);
        const bool wrow = walls && (y == 0 || y == P.ny - 1);
        const real Fy = (onesided && wrow ? -r * wall_grad_y_onesided(an, y != 0) : s * gy) + P.fy -
                        (E.on ? (r - E.rho_g) * E.g : real(0));
        const real jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
        const real jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
        ux[c] = (jx + real(0.5) * Fx) / r;
        uy[c] = (jy + real(0.5) * Fy) / r;
    }
}

// ---------------------------------------------------------------------------------
// Full improved well-balanced free-energy model (Eqs. 1, 6, 20, 21, 24, 29 with A != 0 and/or
// gravity; walls and the drive as above).
//
// Collision of one cell: mn, rn -- mu and rho at x + c_i; uxn, uyn -- u at x + c_i (the
// strain rate S_ab = d_a u_b + d_b u_a of Eq. 20 by the Eq. 24 gradient); Fxe, Fye -- the
// external force (body force, drive, buoyancy F_g = -(rho - rho_g) g); pg -- p_g at the cell.
// The moments of Eq. (20)'s extra terms: e^eq += rho A tr S + 6 p_g, zeta^eq -= rho A tr S +
// 9 p_g, p_xx^eq += rho c_s^2 A (S_xx - S_yy), p_xy^eq += rho c_s^2 A S_xy; the forcing's
// second-order term carries F - grad p_g + c_s^2 grad rho, grad p_g = (0, rho_g g).
template <typename real>
__device__ __forceinline__ void fe_collide_iwb(real v[9], real rho, const real mn[9], const real rn[9],
                                               const real uxn[9], const real uyn[9], real Fxe, real Fye, real pg,
                                               const StepParams<real>& P, const Ext<real>& E, real* d0 = nullptr) {
    const real w1 = real(1.0 / 3.0), w2 = real(1.0 / 12.0);
    const real gmx = grad_x(mn);
    const real gmy = (mn[2] - mn[4]) * w1 + ((mn[5] - mn[7]) + (mn[6] - mn[8])) * w2;
    const real grx = grad_x(rn);
    const real gry = (rn[2] - rn[4]) * w1 + ((rn[5] - rn[7]) + (rn[6] - rn[8])) * w2;
    const real Fx = -rho * gmx + Fxe, Fy = -rho * gmy + Fye;
    const real jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const real jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
    const real ux = (jx + real(0.5) * Fx) / rho;
    const real uy = (jy + real(0.5) * Fy) / rho;
    // S from the velocity stencil (Eq. 24)
    const real dxux = grad_x(uxn), dxuy = grad_x(uyn);
    const real dyux = (uxn[2] - uxn[4]) * w1 + ((uxn[5] - uxn[7]) + (uxn[6] - uxn[8])) * w2;
    const real dyuy = (uyn[2] - uyn[4]) * w1 + ((uyn[5] - uyn[7]) + (uyn[6] - uyn[8])) * w2;
    const real Sxx = real(2) * dxux, Syy = real(2) * dyuy, Sxy = dxuy + dyux;
    const real rA = rho * E.A;
    const real sax = (v[1] + v[2]) + (v[3] + v[4]);
    const real sdg = (v[5] + v[6]) + (v[7] + v[8]);
    const real e = -real(4) * v[0] - sax + real(2) * sdg;
    const real z = real(4) * v[0] - real(2) * sax + sdg;
    const real qx = real(2) * (v[3] - v[1]) + (v[5] - v[6]) + (v[8] - v[7]);
    const real qy = real(2) * (v[4] - v[2]) + (v[5] + v[6]) - (v[7] + v[8]);
    const real pxx = (v[1] + v[3]) - (v[2] + v[4]);
    const real pxy = (v[5] + v[7]) - (v[6] + v[8]);
    const real uu = ux * ux + uy * uy;
    const real dpg = E.rho_g * E.g;  // d_y p_g
    const real uG = ux * Fx + uy * (Fy - dpg);
    const real s = ux * grx + uy * gry;  // u . grad rho
    const real Gx = Fx + grx * real(1.0 / 3.0), Gy = Fy - dpg + gry * real(1.0 / 3.0);
    const real fe = real(6) * uG + real(4) * s;
    const real trS = Sxx + Syy;
    const real e_eq = rho * (real(3) * uu - real(4)) + rA * trS + real(6) * pg;
    const real z_eq = rho * (real(4) - real(3) * uu) - rA * trS - real(9) * pg;
    const real pxx_eq = rho * (ux * ux - uy * uy) + rA * real(1.0 / 3.0) * (Sxx - Syy);
    const real pxy_eq = rho * ux * uy + rA * real(1.0 / 3.0) * Sxy;
    const real de = -P.s_e * (e - e_eq) + (real(1) - real(0.5) * P.s_e) * fe;
    const real dz = -P.s_z * (z - z_eq) - (real(1) - real(0.5) * P.s_z) * fe;
    const real dqx = -P.s_q * (qx + rho * ux) - (real(1) - real(0.5) * P.s_q) * Fx;
    const real dqy = -P.s_q * (qy + rho * uy) - (real(1) - real(0.5) * P.s_q) * Fy;
    const real dpxx = -P.s_nu * (pxx - pxx_eq) + (real(1) - real(0.5) * P.s_nu) * real(2) * (ux * Gx - uy * Gy);
    const real dpxy = -P.s_nu * (pxy - pxy_eq) + (real(1) - real(0.5) * P.s_nu) * (ux * Gy + uy * Gx);
    apply_dm(v, de, dz, Fx, dqx, Fy, dqy, dpxx, dpxy, d0);
}

// One column per thread plus a halo warp whose lanes 0..5 hold the columns x0-3, x0-2, x0-1,
// x0+w, x0+w+1, x0+w+2.  Row pipeline of iteration r: pull row r+1; rho(r) into the rho ring;
// mu(r-1) (columns x0-2 .. x0+w+1); u(r-2) (columns x0-1 .. x0+w; at a wall row after the
// final fill, J = -F/2); collision of row r-3.  Rings: rho 8 rows, mu and u 4 rows.
template <typename real, int TX, bool WALLS>
__global__ void __launch_bounds__(TX + 32) fe_step_iwb(const real* __restrict__ fin, real* __restrict__ fout,
                                                       const StepParams<real> P, const Drive<real> D,
                                                       const Ext<real> E, const real* __restrict__ wjy) {
    __shared__ real s_rho[8][TX + 6];
    __shared__ real s_mu[4][TX + 4];
    __shared__ real s_ux[4][TX + 2];
    __shared__ real s_uy[4][TX + 2];
    const real s_rave = D.rho_ave ? real(*D.rho_ave) : real(0);
    const int nx = P.nx, ny = P.ny;
    const long long pitch = P.pitch;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, ny);
    const int t = threadIdx.x;
    const bool is_main = t < TX;
    bool has_col, has_mu, has_u;
    int off;  // column offset from x0
    if (is_main) {
        has_col = t < w;
        has_mu = has_u = has_col;
        off = t;
    } else {
        const int lane = t - TX;
        has_col = lane < 6;
        has_mu = lane >= 1 && lane <= 4;
        has_u = lane == 2 || lane == 3;
        off = lane < 3 ? lane - 3 : w + (lane - 3);
    }
    const int x = has_col ? wrap_idx(x0 + off, nx) : x0;
    const int rc = off + 3, mc = off + 2, uc = off + 1;  // ring columns
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    // pulled populations of one row (mapped), with the wall fills of the first kind
    auto pull = [&](int r, real v[9]) {
        const int y = stencil_row<WALLS>(r, ny);
        pull_row_ext<WALLS>(fin, P, x, xm, xp, y, v, wjy);
        if (WALLS && !wjy && E.on && E.g != real(0) && (y == 0 || y == ny - 1)) wall_gravity_refill(v, y != 0, P, E);
    };
    // external force of a cell of row r (mapped row y) with density rho
    auto ext_fx = [&](real rho) { return D.rho_ave ? with_drive(P, D, x, rho, s_rave).fx : P.fx; };
    auto ext_fy = [&](real rho) { return P.fy - (E.on ? (rho - E.rho_g) * E.g : real(0)); };
    real p0[9], p1[9], p2[9], p3[9];  // rows r-3, r-2, r-1, r
    if (has_col) pull(y0 - 3, p3);
#pragma unroll 1
    for (int r = y0 - 3; r <= y1 + 2; ++r) {
        real nxt[9];
        if (has_col && r + 1 <= y1 + 2) pull(r + 1, nxt);
        if (has_col) s_rho[r & 7][rc] = sum9(p3);
        __syncthreads();
        if (has_mu && r >= y0 - 1) {  // mu(r-1)
            const real* rm = s_rho[(r - 2) & 7];
            const real* r0 = s_rho[(r - 1) & 7];
            const real* rp = s_rho[r & 7];
            real rn[9];
            rn[1] = r0[rc + 1]; rn[2] = rp[rc]; rn[3] = r0[rc - 1]; rn[4] = rm[rc];
            rn[5] = rp[rc + 1]; rn[6] = rp[rc - 1]; rn[7] = rm[rc - 1]; rn[8] = rm[rc + 1];
            rn[0] = r0[rc];  // every entry defined (the FP32 overload reads all nine)
            s_mu[(r - 1) & 3][mc] = fe_mu<real>(r0[rc], rn, P);
        }
        __syncthreads();
        if (has_u && r >= y0 + 1) {  // u(r-2) from this column's populations of row r-2 (p1)
            const int cu = r - 2;
            const real* mm = s_mu[(cu - 1) & 3];
            const real* m0 = s_mu[cu & 3];
            const real* mp = s_mu[(cu + 1) & 3];
            real mn[9];
            mn[1] = m0[mc + 1]; mn[2] = mp[mc]; mn[3] = m0[mc - 1]; mn[4] = mm[mc];
            mn[5] = mp[mc + 1]; mn[6] = mp[mc - 1]; mn[7] = mm[mc - 1]; mn[8] = mm[mc + 1];
            mn[0] = m0[mc];
            const real rho = s_rho[cu & 7][rc];
            const bool wall = WALLS && (cu == 0 || cu == ny - 1);
            // one-sided reading: the wall node's normal -rho d_y mu (zero when mirrored)
            const real fy_w = (wall && wjy) ? -rho * wall_grad_y_onesided(mn, cu != 0) : real(0);
            if (wall) mirror_neighbours(mn, cu != 0);
            const real w1 = real(1.0 / 3.0), w2 = real(1.0 / 12.0);
            const real Fx = -rho * grad_x(mn) + ext_fx(rho);
            const real Fy = -rho * ((mn[2] - mn[4]) * w1 + ((mn[5] - mn[7]) + (mn[6] - mn[8])) * w2) + ext_fy(rho) + fy_w;
            if (wall) wall_fill(p1, cu != 0, real(-0.5) * Fx, real(-0.5) * Fy);
            const real jx = (p1[1] - p1[3]) + (p1[5] - p1[6]) + (p1[8] - p1[7]);
            const real jy = (p1[2] - p1[4]) + (p1[5] + p1[6]) - (p1[7] + p1[8]);
            s_ux[cu & 3][uc] = (jx + real(0.5) * Fx) / rho;
            s_uy[cu & 3][uc] = (jy + real(0.5) * Fy) / rho;
        }
        __syncthreads();
        if (is_main && has_col && r >= y0 + 3) {
            const int c = r - 3;
            const real* mm = s_mu[(c - 1) & 3];
            const real* m0 = s_mu[c & 3];
            const real* mp = s_mu[(c + 1) & 3];
            const real* rm = s_rho[(c - 1) & 7];
            const real* r0 = s_rho[c & 7];
            const real* rp = s_rho[(c + 1) & 7];
            const real* xm_ = s_ux[(c - 1) & 3];
            const real* x0_ = s_ux[c & 3];
            const real* xp_ = s_ux[(c + 1) & 3];
            const real* ym_ = s_uy[(c - 1) & 3];
            const real* y0_ = s_uy[c & 3];
            const real* yp_ = s_uy[(c + 1) & 3];
            real mn[9], rn[9], un[9], vn[9];
            mn[1] = m0[mc + 1]; mn[2] = mp[mc]; mn[3] = m0[mc - 1]; mn[4] = mm[mc];
            mn[5] = mp[mc + 1]; mn[6] = mp[mc - 1]; mn[7] = mm[mc - 1]; mn[8] = mm[mc + 1];
            rn[1] = r0[rc + 1]; rn[2] = rp[rc]; rn[3] = r0[rc - 1]; rn[4] = rm[rc];
            rn[5] = rp[rc + 1]; rn[6] = rp[rc - 1]; rn[7] = rm[rc - 1]; rn[8] = rm[rc + 1];
            un[1] = x0_[uc + 1]; un[2] = xp_[uc]; un[3] = x0_[uc - 1]; un[4] = xm_[uc];
            un[5] = xp_[uc + 1]; un[6] = xp_[uc - 1]; un[7] = xm_[uc - 1]; un[8] = xm_[uc + 1];
            vn[1] = y0_[uc + 1]; vn[2] = yp_[uc]; vn[3] = y0_[uc - 1]; vn[4] = ym_[uc];
            vn[5] = yp_[uc + 1]; vn[6] = yp_[uc - 1]; vn[7] = ym_[uc - 1]; vn[8] = ym_[uc + 1];
            const real rho_c = r0[rc];
            mn[0] = m0[mc];
            rn[0] = rho_c;
            un[0] = x0_[uc];
            vn[0] = y0_[uc];
            real fy_w = real(0);
            if (WALLS && (c == 0 || c == ny - 1)) {
                const bool top = c != 0;
                if (wjy) fy_w = -rho_c * wall_grad_y_onesided(mn, top);
                mirror_neighbours(mn, top);
                mirror_neighbours(rn, top);
                // velocity beyond a no-slip wall: odd extension through u = 0 at the wall node
                if (!top) {
                    un[4] = -un[2]; un[7] = -un[6]; un[8] = -un[5];
                    vn[4] = -vn[2]; vn[7] = -vn[6]; vn[8] = -vn[5];
                } else {
                    un[2] = -un[4]; un[5] = -un[8]; un[6] = -un[7];
                    vn[2] = -vn[4]; vn[5] = -vn[8]; vn[6] = -vn[7];
                }
            }
            const real pg = E.on ? E.rho_g * E.g * (real(c) - E.y_ref) : real(0);
            const long long o = (long long)c * nx + x;
            if constexpr (std::is_same<real, float>::value) {
                // compensated rest population
                int q = rest_lo_plane(fin, pitch)[o];
                float d0;
                fe_collide_iwb(p0, rho_c, mn, rn, un, vn, ext_fx(rho_c), ext_fy(rho_c) + fy_w, pg, P, E, &d0);
                rest_update(p0[0], q, d0, P);
                rest_lo_plane(fout, pitch)[o] = (short)q;
            } else {
                fe_collide_iwb(p0, rho_c, mn, rn, un, vn, ext_fx(rho_c), ext_fy(rho_c) + fy_w, pg, P, E);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) fout[i * pitch + o] = p0[i];
        }
        if (has_col) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                p0[i] = p1[i];
                p1[i] = p2[i];
                p2[i] = p3[i];
                p3[i] = nxt[i];
            }
        }
    }
}

// f = f^eq of Eq. (20) at rest with p_g, stored as S_i(y) = f^eq_i(y + c_i) (rows beyond a
// wall hold slots no step reads; the row is wrapped there).
template <typename real, typename src_t>
__global__ void init_iwb_kernel(const src_t* __restrict__ rho0, real* __restrict__ S, int nx, int ny,
                                long long pitch, double pg_coef, double y_ref, float rest_inv) {
    const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cys[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double w[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                         1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ys = (y + cys[i] + ny) % ny;
            const double pg = pg_coef * ((double)ys - y_ref);
            const double r = (double)rho0[shifted_cell(x, y, cxs[i], cys[i], nx, ny)];
            const double f = i == 0 ? r - (1.0 - w[0]) * 3.0 * pg : w[i] * 3.0 * pg;
            S[i * pitch + c] = (real)f;
            if constexpr (std::is_same<real, float>::value)
                if (i == 0) rest_lo_plane(S, pitch)[c] = rest_encode(f, (float)f, rest_inv);
        }
    }
}

// One-sided reading of the free-energy walls, the wall rows' densities: a wall node's density
// is K +- J_y (bottom +, top -) with J_y = -F_y/2 and F_y = -rho d_y mu + fy - (rho - rho_g) g,
// where d_y mu (wall_grad_y_onesided) depends on mu of the wall row and the next row, which
// depend on the wall row's densities through the chemical potential and its Laplacian.  One
// CTA per wall (blockIdx.x: 0 bottom, 1 top; 1024 threads) iterates the fixed point `iters` times over the
// whole row (Jacobi sweeps between CTA barriers; each sweep contracts by about rho c_T^2 / 2)
// and leaves the converged J_y in wall[0, 2 nx) (bottom then top) for the step and field
// kernels.  wall[2 nx, 14 nx) is scratch: per wall the first-fill density, the current wall
// densities, the densities of the next two rows, and mu of the wall row and the next row.
template <typename real>
__global__ void __launch_bounds__(1024) fe_wall_solve_kernel(const real* __restrict__ fin, const StepParams<real> P,
                                                            const Ext<real> E, real* __restrict__ wall, int iters) {
    const int nx = P.nx, ny = P.ny;
    const bool top = blockIdx.x == 1;
    const int yw = top ? ny - 1 : 0, y1 = top ? ny - 2 : 1, y2 = top ? ny - 3 : 2;
    const real sg = top ? real(-1) : real(1);
    real* Jy = wall + (top ? nx : 0);
    real* w = wall + 2 * nx + (top ? 6 * nx : 0);
    real* Kp = w;
    real* r0 = w + nx;
    real* r1 = w + 2 * nx;
    real* r2 = w + 3 * nx;
    real* m0 = w + 4 * nx;
    real* m1 = w + 5 * nx;
    const real jy0 = real(-0.5) * P.fy;  // the first fill's J_y
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        real v[9];
        pull_row_ext<true>(fin, P, x, xm, xp, yw, v);
        Kp[x] = r0[x] = sum9(v);
        pull_row_ext<true>(fin, P, x, xm, xp, y1, v);
        r1[x] = sum9(v);
        pull_row_ext<true>(fin, P, x, xm, xp, y2, v);
        r2[x] = sum9(v);
    }
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            real rn[9];
            // wall row: the row beyond the wall is the next row, mirrored (Laplacian symmetric)
            rn[0] = r0[x]; rn[1] = r0[xp]; rn[3] = r0[xm];
            rn[2] = r1[x]; rn[4] = r1[x]; rn[5] = r1[xp]; rn[8] = r1[xp]; rn[6] = r1[xm]; rn[7] = r1[xm];
            m0[x] = fe_mu<real>(r0[x], rn, P);
            // next row: the wall row on one side, the row after on the other
            rn[0] = r1[x]; rn[1] = r1[xp]; rn[3] = r1[xm];
            rn[2] = r2[x]; rn[5] = r2[xp]; rn[6] = r2[xm];
            rn[4] = r0[x]; rn[8] = r0[xp]; rn[7] = r0[xm];
            m1[x] = fe_mu<real>(r1[x], rn, P);
        }
        __syncthreads();
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            const real g = real(3) * (real(2.0 / 9.0) * (m1[x] - m0[x]) +
                                      real(1.0 / 18.0) * ((m1[xp] - m0[xp]) + (m1[xm] - m0[xm])));
            const real Fy = -r0[x] * (top ? -g : g) + P.fy - (E.on ? (r0[x] - E.rho_g) * E.g : real(0));
            const real jy = real(-0.5) * Fy;
            Jy[x] = jy;
            r0[x] = Kp[x] + sg * (jy - jy0);
        }
        __syncthreads();
    }
}

}  // namespace lbmk
