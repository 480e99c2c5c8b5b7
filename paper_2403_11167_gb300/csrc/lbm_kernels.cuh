// lbm_kernels.cuh -- sm_103a kernels of the fused D2Q9 multiphase time step.
//
// Layout: populations are 9 planes f_i[y][x] (structure of arrays), plane i at
// offset i * pitch, velocity order of Eq. (2).  Streaming is done by pulling:
// the kernel reading buffer A gathers f_i(x - c_i) (the post-collision values of
// the previous step), collides, and writes f*_i(x) to buffer B at x, so A is
// read-only and B write-only inside a launch (ping-pong).  Periodic in x and y.
//
// Fusion: every quantity needed at neighbours (psi for the pseudopotential model,
// rho and mu for the free-energy model) is recomputed from the pulled populations
// inside the CTA that needs it, so the step moves only 9 loads + 9 stores of
// populations per cell through HBM.  A CTA owns a strip of TX columns and walks
// down `rows` rows; the per-row neighbour fields live in small shared-memory
// rings (sliding window), and one extra warp computes the x-halo columns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbmk {

// D2Q9, Eq. (2): 0 rest; 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1); 5 (1,1); 6 (-1,1); 7 (-1,-1); 8 (1,-1).

template <typename real>
struct StepParams {
    int nx, ny, rows;  // lattice, rows per CTA
    long long pitch;   // plane pitch (elements)
    real RT, a, b4;    // Carnahan-Starling: R*T, a, b/4  (Eq. 28)
    real kA, kB;       // Q tensor (Eq. 30): G (C1 - C2/3) and G (C2 + kappa_Li/2)
    real li;           // 12 kappa_P sigma_Li  (Eq. 32, consistency term; G^2 = 1)
    real kappa;        // free energy: mu = mu_b - kappa lap rho
    real rho_ref_v, rho_ref_l, rho_split;  // coexistence densities (reference points of mu_b) and midpoint
    real mu_off_l;     // mu_b(rho_ref_l) - mu_b(rho_ref_v) at the rounded references (host FP64)
    real ur_v, ur_l;   // 1 - b rho_ref / 4 of each reference
    real ur3_v, ur3_l; // its cube
    real irr_v, irr_l; // 1 / rho_ref
    real s_e, s_z, s_q, s_nu;  // relaxation rates 1/tau (Eq. 3); tau_rho, tau_j drop out
    real fx, fy;       // body force
    real rest_unit, rest_inv;  // FP32: unit of the rest population's extension and its inverse
    // 1 - s/2 of e, zeta, q, nu and 6 (1 - s/2) of e, zeta (forcing factors of Eq. 1), rounded
    // once on the host: computed in the kernels, a compiler may fuse them differently in two
    // kernels and the same cell would then differ by an ulp of the increments between routes
    real h_e, h_z, h_q, h_nu, h6_e, h6_z;
};

// Correctly rounded reciprocal (FP32: one hardware-assisted sequence instead of a full division).
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }


template <typename real>
__device__ __forceinline__ real cs_pressure(real rho, real RT, real a, real b4) {
    const real e = b4 * rho;
    const real r = rcp(real(1) - e);
    const real num = real(1) + e * (real(1) + e * (real(1) - e));
    return rho * RT * num * (r * r * r) - a * rho * rho;
}

// Eq. (11) with G = -1: psi = sqrt(2 (rho c_s^2 - p_EOS)).  NaN for a negative radicand
// (propagates into the populations and is caught by the divergence check).
template <typename real>
__device__ __forceinline__ real pseudo_psi(real rho, const StepParams<real>& P) {
    return sqrt(real(2) * (rho * real(1.0 / 3.0) - cs_pressure(rho, P.RT, P.a, P.b4)));
}

// Eq. (29): mu_b = RT (3 - e)/(1 - e)^3 + RT ln rho + RT - 2 a rho, e = b rho / 4.
// Only differences of mu enter the method (F = -rho grad mu), so the kernels use
// mu_b(rho) - mu_b(rho_r) with rho_r the Maxwell density of the same phase
// (mu_b(rho_v) = mu_b(rho_l)): one constant offset for every cell.  Written as a
// divided difference it has no cancellation between the O(0.1) terms of Eq. (29),
// which in FP32 would leave O(1e-8) noise on a chemical potential of O(1e-3):
//   ln(rho/rho_r) = log1p(d/rho_r),  d = rho - rho_r,
//   g(e) - g(e_r) = (e - e_r) [2 (ur^2 + ur u + u^2)/(u^3 ur^3) + (ur + u)/(u^2 ur^2)],
// with g(e) = (3 - e)/(1 - e)^3 = 2/u^3 + 1/u^2, u = 1 - e.
template <typename real>
__device__ __forceinline__ real mu_bulk_rel(real rho, const StepParams<real>& P) {
    const bool liq = rho >= P.rho_split;
    const real rr = liq ? P.rho_ref_l : P.rho_ref_v;
    const real ur = liq ? P.ur_l : P.ur_v;
    const real ur3 = liq ? P.ur3_l : P.ur3_v;
    const real irr = liq ? P.irr_l : P.irr_v;
    const real d = rho - rr;
    const real u = real(1) - P.b4 * rho;
    // g(e) - g(e_r) = (e - e_r) [2 (ur^2 + ur u + u^2) + (ur + u) u ur] / (u^3 ur^3)
    const real num = real(2) * (ur * ur + ur * u + u * u) + (ur + u) * u * ur;
    const real dg = P.b4 * d * num * rcp(u * u * u * ur3);
    return P.RT * (dg + log1p(d * irr)) - real(2) * P.a * d + (liq ? P.mu_off_l : real(0));
}

__device__ __forceinline__ int wrap_idx(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Pulled populations of cell (x, r): v_i = f_i(x - c_i).  xm = x-1, xp = x+1 (wrapped);
// om, o0, op = row offsets of rows r-1, r, r+1 (wrapped).
template <typename real>
__device__ __forceinline__ void pull9(const real* __restrict__ f, long long pitch, int x, int xm, int xp,
                                      long long om, long long o0, long long op, real v[9]) {
    v[0] = __ldg(f + 0 * pitch + o0 + x);
    v[1] = __ldg(f + 1 * pitch + o0 + xm);
    v[2] = __ldg(f + 2 * pitch + om + x);
    v[3] = __ldg(f + 3 * pitch + o0 + xp);
    v[4] = __ldg(f + 4 * pitch + op + x);
    v[5] = __ldg(f + 5 * pitch + om + xm);
    v[6] = __ldg(f + 6 * pitch + om + xp);
    v[7] = __ldg(f + 7 * pitch + op + xp);
    v[8] = __ldg(f + 8 * pitch + op + xm);
}

// rho = sum_i f_i (Eq. 6a), summed in mirror pairs (1,3), (2,4), (5,7), (6,8): reflecting the
// lattice in x or in y (or transposing it) maps every partial sum onto itself, so mirror-image
// cells get bitwise equal densities and a mirror-symmetric state stays symmetric in FP32.
template <typename real>
__device__ __forceinline__ real sum9(const real v[9]) {
    return v[0] + (((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8])));
}

// f* = f + M^-1 dm for the moment increments dm (rho increment is zero); M^-1 of Eq. (S49).
// d0: if not null, receives the rest population's increment, and v[0] is left unchanged (the
// caller applies it to a compensated rest population; see rest_update).
template <typename real>
__device__ __forceinline__ void apply_dm(real v[9], real de, real dz, real djx, real dqx, real djy, real dqy,
                                         real dpxx, real dpxy, real* d0 = nullptr) {
    const real A = -de * real(1.0 / 36.0) - dz * real(1.0 / 18.0);
    const real B = de * real(1.0 / 18.0) + dz * real(1.0 / 36.0);
    const real X1 = (djx - dqx) * real(1.0 / 6.0);
    const real Y1 = (djy - dqy) * real(1.0 / 6.0);
    const real X2 = djx * real(1.0 / 6.0) + dqx * real(1.0 / 12.0);
    const real Y2 = djy * real(1.0 / 6.0) + dqy * real(1.0 / 12.0);
    const real Pp = dpxx * real(0.25);
    const real Z = dpxy * real(0.25);
    if (d0)
        *d0 = (dz - de) * real(1.0 / 9.0);
    else
        v[0] += (dz - de) * real(1.0 / 9.0);
    v[1] += A + X1 + Pp;
    v[2] += A + Y1 - Pp;
    v[3] += A - X1 + Pp;
    v[4] += A - Y1 - Pp;
    v[5] += B + X2 + Y2 + Z;
    v[6] += B - X2 + Y2 - Z;
    v[7] += B - X2 - Y2 + Z;
    v[8] += B + X2 - Y2 - Z;
}

// ---------------------------------------------------------------------------------
// Modified pseudopotential collision of one cell (Eqs. 1, 4, 6, 10, 13, 30-32).
//   v  : pulled populations (in: f, out: f*)
//   pc : psi at the cell; pn[i] : psi at x + c_i (i = 1..8)
template <typename real>
__device__ __forceinline__ void pp_collide(real v[9], real rho, real pc, const real pn[9],
                                           const StepParams<real>& P) {
    const real w1 = real(1.0 / 3.0), w2 = real(1.0 / 12.0);
    // Eq. (10): F_int = -G psi sum_i omega_i psi(x + c_i) c_i, G = -1
    const real Sx = (pn[1] - pn[3]) * w1 + ((pn[5] - pn[7]) + (pn[8] - pn[6])) * w2;
    const real Sy = (pn[2] - pn[4]) * w1 + ((pn[5] - pn[7]) + (pn[6] - pn[8])) * w2;
    const real Fix = pc * Sx, Fiy = pc * Sy;
    const real Fx = Fix + P.fx, Fy = Fiy + P.fy;
    // Eq. (30): Q_ab = psi sum_i omega_i C_iab (psi_i - psi), C2 term carrying G
    const real d1 = pn[1] - pc, d2 = pn[2] - pc, d3 = pn[3] - pc, d4 = pn[4] - pc;
    const real d5 = pn[5] - pc, d6 = pn[6] - pc, d7 = pn[7] - pc, d8 = pn[8] - pc;
    const real dd = ((d5 + d6) + (d7 + d8)) * w2;
    const real sxx = (d1 + d3) * w1 + dd;
    const real syy = (d2 + d4) * w1 + dd;
    const real sa = sxx + syy - dd;  // sum_i omega_i d_i
    const real sxy = ((d5 - d6) + (d7 - d8)) * w2;
    const real Qxx = pc * (P.kA * sa + P.kB * sxx);
    const real Qyy = pc * (P.kA * sa + P.kB * syy);
    const real Qxy = pc * (P.kB * sxy);
    // Eq. (32) consistency term: 12 kappa_P sigma_Li |F_int|^2/psi^2 = li |S|^2 (G^2 = 1)
    const real L = P.li * (Sx * Sx + Sy * Sy);
    // Eq. (6b) and the moments m = M f (Eq. S48)
    const real jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const real jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
    const real inv_rho = rcp(rho);
    const real ux = (jx + real(0.5) * Fx) * inv_rho;
    const real uy = (jy + real(0.5) * Fy) * inv_rho;
    const real sax = (v[1] + v[2]) + (v[3] + v[4]);
    const real sdg = (v[5] + v[6]) + (v[7] + v[8]);
    const real e = -real(4) * v[0] - sax + real(2) * sdg;
    const real z = real(4) * v[0] - real(2) * sax + sdg;
    const real qx = real(2) * (v[3] - v[1]) + (v[5] - v[6]) + (v[8] - v[7]);
    const real qy = real(2) * (v[4] - v[2]) + (v[5] + v[6]) - (v[7] + v[8]);
    const real pxx = (v[1] + v[3]) - (v[2] + v[4]);
    const real pxy = (v[5] + v[7]) - (v[6] + v[8]);
    const real uu = ux * ux + uy * uy;
    const real uF = ux * Fx + uy * Fy;
    const real trQ = Qxx + Qyy;
    // m* - m = -L (m - m^eq) + (I - L/2) MF' + MC  (Eqs. 1, 4/S66, 32, 13)
    const real de = -P.s_e * (e - rho * (real(3) * uu - real(2))) + (real(1) - real(0.5) * P.s_e) * real(6) * uF +
                    P.s_e * (L + real(1.5) * trQ);
    const real dz = -P.s_z * (z - rho * (real(1) - real(3) * uu)) - (real(1) - real(0.5) * P.s_z) * real(6) * uF -
                    P.s_z * (L + real(1.5) * trQ);
    const real dqx = -P.s_q * (qx + rho * ux) - (real(1) - real(0.5) * P.s_q) * Fx;
    const real dqy = -P.s_q * (qy + rho * uy) - (real(1) - real(0.5) * P.s_q) * Fy;
    const real dpxx = -P.s_nu * (pxx - rho * (ux * ux - uy * uy)) +
                      (real(1) - real(0.5) * P.s_nu) * real(2) * (ux * Fx - uy * Fy) - P.s_nu * (Qxx - Qyy);
    const real dpxy = -P.s_nu * (pxy - rho * ux * uy) + (real(1) - real(0.5) * P.s_nu) * (ux * Fy + uy * Fx) -
                      P.s_nu * Qxy;
    // j* - j = F exactly (tau_j drops out)
    apply_dm(v, de, dz, Fx, dqx, Fy, dqy, dpxx, dpxy);
}

// ---------------------------------------------------------------------------------
// Improved well-balanced free-energy collision of one cell (Eqs. 1, 6, 20, 21, 24).
//   mn[i] : mu at x + c_i, rn[i] : rho at x + c_i (i = 1..8)
template <typename real>
__device__ __forceinline__ void fe_collide(real v[9], real rho, const real mn[9], const real rn[9],
                                           const StepParams<real>& P) {
    const real w1 = real(1.0 / 3.0), w2 = real(1.0 / 12.0);
    // Eq. (24) gradient with weights: d_a phi = 3 sum_i w_i phi_i c_ia
    const real gmx = (mn[1] - mn[3]) * w1 + ((mn[5] - mn[7]) + (mn[8] - mn[6])) * w2;
    const real gmy = (mn[2] - mn[4]) * w1 + ((mn[5] - mn[7]) + (mn[6] - mn[8])) * w2;
    const real grx = (rn[1] - rn[3]) * w1 + ((rn[5] - rn[7]) + (rn[8] - rn[6])) * w2;
    const real gry = (rn[2] - rn[4]) * w1 + ((rn[5] - rn[7]) + (rn[6] - rn[8])) * w2;
    const real Fx = -rho * gmx + P.fx, Fy = -rho * gmy + P.fy;
    const real jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const real jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
    const real inv_rho = rcp(rho);
    const real ux = (jx + real(0.5) * Fx) * inv_rho;
    const real uy = (jy + real(0.5) * Fy) * inv_rho;
    const real sax = (v[1] + v[2]) + (v[3] + v[4]);
    const real sdg = (v[5] + v[6]) + (v[7] + v[8]);
    const real e = -real(4) * v[0] - sax + real(2) * sdg;
    const real z = real(4) * v[0] - real(2) * sax + sdg;
    const real qx = real(2) * (v[3] - v[1]) + (v[5] - v[6]) + (v[8] - v[7]);
    const real qy = real(2) * (v[4] - v[2]) + (v[5] + v[6]) - (v[7] + v[8]);
    const real pxx = (v[1] + v[3]) - (v[2] + v[4]);
    const real pxy = (v[5] + v[7]) - (v[6] + v[8]);
    const real uu = ux * ux + uy * uy;
    const real uF = ux * Fx + uy * Fy;
    const real s = ux * grx + uy * gry;  // u . grad rho
    const real Gx = Fx + grx * real(1.0 / 3.0), Gy = Fy + gry * real(1.0 / 3.0);  // F + c_s^2 grad rho
    // M F_i of Eq. (21): (0, 6uF + 4s, -6uF - 4s, Fx, -Fx, Fy, -Fy, 2(uxGx - uyGy), uxGy + uyGx)
    const real fe = real(6) * uF + real(4) * s;
    // m^eq of Eq. (20): (rho, rho(-4 + 3uu), rho(4 - 3uu), rho u, -rho u, ..., rho(ux^2-uy^2), rho ux uy)
    const real de = -P.s_e * (e - rho * (real(3) * uu - real(4))) + (real(1) - real(0.5) * P.s_e) * fe;
    const real dz = -P.s_z * (z - rho * (real(4) - real(3) * uu)) - (real(1) - real(0.5) * P.s_z) * fe;
    const real dqx = -P.s_q * (qx + rho * ux) - (real(1) - real(0.5) * P.s_q) * Fx;
    const real dqy = -P.s_q * (qy + rho * uy) - (real(1) - real(0.5) * P.s_q) * Fy;
    const real dpxx = -P.s_nu * (pxx - rho * (ux * ux - uy * uy)) +
                      (real(1) - real(0.5) * P.s_nu) * real(2) * (ux * Gx - uy * Gy);
    const real dpxy = -P.s_nu * (pxy - rho * ux * uy) + (real(1) - real(0.5) * P.s_nu) * (ux * Gy + uy * Gx);
    apply_dm(v, de, dz, Fx, dqx, Fy, dqy, dpxx, dpxy);
}

// Chemical potential (up to the constant mu_b(rho_v)) at one cell from rho at the cell (rc) and
// its 8 neighbours; Eq. (24) Laplacian summed over differences.
template <typename real>
__device__ __forceinline__ real fe_mu(real rc, const real rn[9], const StepParams<real>& P) {
    const real lap = (((rn[1] - rc) + (rn[2] - rc)) + ((rn[3] - rc) + (rn[4] - rc))) * real(2.0 / 3.0) +
                     (((rn[5] - rc) + (rn[6] - rc)) + ((rn[7] - rc) + (rn[8] - rc))) * real(1.0 / 6.0);
    return mu_bulk_rel(rc, P) - P.kappa * lap;
}

// ---------------------------------------------------------------------------------
// FP32 arithmetic of both models, written once for one cell (F1) or two cells at a time (F2,
// Blackwell's packed FP32: one instruction computes both lanes).  Every operation is an
// explicit correctly rounded add / multiply / fused multiply-add, never re-associated or
// contracted by the compiler, so the single-cell and the two-cell kernels produce bitwise
// identical cells.  The algebra is that of pp_collide / fe_collide / fe_mu above (Eqs. 10-13,
// 20, 21, 24, 29-32), arranged for FP32 in three ways:
//  * Mirror equivariance.  Every sum over velocities is grouped so that reflecting the lattice
//    in x (1<->3, 5<->6, 7<->8) or in y (2<->4, 5<->8, 6<->7) maps each partial result onto
//    itself or onto its exact negative (IEEE addition is commutative and a - b = -(b - a)).
//    A mirror-symmetric state therefore stays bitwise symmetric: its momentum is exactly zero
//    and a static droplet or slab cannot drift rigidly from rounding (in FP32 it otherwise
//    wanders by ~1e-5 cells per 1e4 steps).
//  * Scale-exact constants.  c_s^2 = 1/3 and the stencil weights 1/3, 1/12 round up by 3e-8 in
//    FP32.  In the pseudopotential model the lattice pressure rho c_s^2 must cancel the rho c_s^2
//    inside psi^2 (Eq. 11) against a force of exactly the stencil's scale, so these roundings act
//    as a spurious -3e-8 rho term in the equation of state (a 1.6e-6 relative change of the
//    temperature at Tr = 0.8, shifting the vapour density by ~1e-5).  psi^2 therefore uses 1/3
//    as a hi + lo pair, the force stencil integer weights times a hi + lo 1/12, and the
//    momentum increments of M^-1 are formed so that they sum to the force up to one rounding.
//  * No rest population in small differences.  In the free-energy model f_0 = rho carries
//    almost all of the mass, so e - e^eq and zeta - zeta^eq are formed from the moving
//    populations alone (rho = f_0 + sum of the others substituted exactly).
struct F1 {
    float v;
    __device__ __forceinline__ F1() {}
    __device__ __forceinline__ explicit F1(float x) : v(x) {}
    static __device__ __forceinline__ F1 c(float s) { return F1(s); }
};
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1(__fsub_rn(a.v, b.v)); }
// a product is a fused multiply-add with +0 (the rounded product, a zero product taken as +0),
// for the reason given at F2
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return F1(__fmaf_rn(a.v, b.v, 0.0f)); }
__device__ __forceinline__ F1 operator-(F1 a) { return F1(-a.v); }
__device__ __forceinline__ F1 fmav(F1 a, F1 b, F1 c) { return F1(__fmaf_rn(a.v, b.v, c.v)); }

struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    static __device__ __forceinline__ F2 c(float s) { return F2(s, s); }
};
// Packed FP32 (one instruction for both lanes).  The packed add and fused multiply-add round
// like their scalar _rn counterparts, but a packed multiply whose only use is a packed add is
// fused with it by the compiler -- whatever the rounding modifier or -fmad setting -- where the
// scalar __fmul_rn never is, so the one-cell and two-cell instantiations of the step rounded
// differently.  A product is therefore a fused multiply-add with +0, which no compiler may
// treat as a multiply (it maps a -0 product to +0), in both types; the arithmetic writes fmav
// wherever it wants a product fused into a sum.
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__ffma2_rn(a.v, b.v, make_float2(0.0f, 0.0f))); }
__device__ __forceinline__ F2 fmav(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

__device__ __forceinline__ F1 rcp_v(F1 x) { return F1(__frcp_rn(x.v)); }
__device__ __forceinline__ F2 rcp_v(F2 x) { return F2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }
__device__ __forceinline__ F1 log1p_v(F1 x) { return F1(log1pf(x.v)); }
__device__ __forceinline__ F2 log1p_v(F2 x) { return F2(log1pf(x.v.x), log1pf(x.v.y)); }
// per lane: l where rho >= split (liquid branch), v elsewhere
__device__ __forceinline__ F1 pick_v(F1 rho, float split, float l, float v) { return F1(rho.v >= split ? l : v); }
__device__ __forceinline__ F2 pick_v(F2 rho, float split, float l, float v) {
    return F2(rho.v.x >= split ? l : v, rho.v.y >= split ? l : v);
}

// Eq. (29) relative to the coexistence reference (see mu_bulk_rel), explicit ops; the
// reference (liquid or vapour branch), log1p and the reciprocal are taken per lane.
template <class F>
__device__ __forceinline__ F mu_bulk_v(F rho, const StepParams<float>& P) {
    const F rr = pick_v(rho, P.rho_split, P.rho_ref_l, P.rho_ref_v);
    const F U = pick_v(rho, P.rho_split, P.ur_l, P.ur_v);
    const F ur3 = pick_v(rho, P.rho_split, P.ur3_l, P.ur3_v);
    const F irr = pick_v(rho, P.rho_split, P.irr_l, P.irr_v);
    const F off = pick_v(rho, P.rho_split, P.mu_off_l, 0.0f);
    const F d = rho - rr;
    const F u = fmav(F::c(-P.b4), rho, F::c(1.0f));
    const F num = fmav(F::c(2.0f), fmav(U, U, fmav(U, u, u * u)), (U + u) * u * U);
    const F dg = F::c(P.b4) * d * num * rcp_v(u * u * u * ur3);
    const F lg = log1p_v(d * irr);
    return fmav(F::c(P.RT), dg + lg, F::c(-2.0f * P.a) * d) + off;
}

template <class F>
__device__ __forceinline__ F sum9_v(const F v[9]) {
    return v[0] + (((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8])));
}

// 1/3 and 1/12 as FP32 hi + lo pairs (hi the rounded value, lo the rounded remainder; the pair
// is exact to 3e-16).
constexpr float kThirdHi = 0x1.555556p-2f, kThirdLo = -0x1.555556p-27f;
constexpr float kTwelfthHi = 0x1.555556p-4f, kTwelfthLo = -0x1.555556p-29f;

// Sums over the lattice velocities in mirror-equivariant grouping (see above).
//   jx = f1 - f3 + f5 - f6 - f7 + f8, jy = f2 - f4 + f5 + f6 - f7 - f8, sax = f1 + f2 + f3 + f4.
template <class F>
__device__ __forceinline__ F mom_jx(const F v[9]) { return (v[1] - v[3]) + ((v[5] - v[6]) + (v[8] - v[7])); }
template <class F>
__device__ __forceinline__ F mom_jy(const F v[9]) { return (v[2] - v[4]) + ((v[5] - v[8]) + (v[6] - v[7])); }
template <class F>
__device__ __forceinline__ F sum_axes(const F v[9]) { return (v[1] + v[3]) + (v[2] + v[4]); }

// 12 sum_i omega_i phi(x + c_i) c_i with omega = 1/3 (axes), 1/12 (diagonals): integer weights,
// exact up to the rounding of the last operation.
template <class F>
__device__ __forceinline__ F stencil12_x(const F n[9]) {
    return fmav(F::c(4.0f), n[1] - n[3], (n[5] - n[7]) + (n[8] - n[6]));
}
template <class F>
__device__ __forceinline__ F stencil12_y(const F n[9]) {
    return fmav(F::c(4.0f), n[2] - n[4], (n[5] - n[7]) + (n[6] - n[8]));
}
template <class F>
__device__ __forceinline__ F div12(F t) { return fmav(t, F::c(kTwelfthHi), t * F::c(kTwelfthLo)); }

// mu at the cell from rho at the cell (rc) and at x + c_i (rn[1..8]).
template <class F>
__device__ __forceinline__ F fe_mu_v(F rc, const F rn[9], const StepParams<float>& P) {
    const F lap = fmav(((rn[1] - rc) + (rn[3] - rc)) + ((rn[2] - rc) + (rn[4] - rc)), F::c(2.0f / 3.0f),
                       ((rn[5] - rc) + (rn[6] - rc) + ((rn[7] - rc) + (rn[8] - rc))) * F::c(1.0f / 6.0f));
    return fmav(F::c(-P.kappa), lap, mu_bulk_v(rc, P));
}

// f* = f + M^-1 dm (Eq. S49) in the FP32 arithmetic.  COMP: the rest population's increment
// goes to *d0 and v[0] is left unchanged (compensated rest population, see rest_update).
// ABSORB (with COMP): each moving population's rounding error, inc - (fl(f + inc) - f) (exact
// by Fast2Sum when |f| >= |inc|), is added to *d0 as well, so the rest population takes up
// what the moving ones lost and the cell's mass changes only by rounding of the increments
// (relative ~1e-7 of them) -- needed where the moving populations carry much of the mass
// (pseudopotential model, f_i = w_i rho at rest).  The errors are summed in mirror pairs.
template <class F, bool COMP = false, bool ABSORB = false>
__device__ __forceinline__ void apply_dm_v(F v[9], F de, F dz, F djx, F dqx, F djy, F dqy, F dpxx, F dpxy,
                                           F* d0 = nullptr) {
    const F A = fmav(de, F::c(-1.0f / 36.0f), dz * F::c(-1.0f / 18.0f));
    const F B = fmav(de, F::c(1.0f / 18.0f), dz * F::c(1.0f / 36.0f));
    const F X1 = (djx - dqx) * F::c(1.0f / 6.0f);
    const F Y1 = (djy - dqy) * F::c(1.0f / 6.0f);
    // X2 = djx / 6 + dqx / 12 taken as (djx - 2 X1) / 4, so that 2 X1 + 4 X2 (the x momentum
    // added to the populations) equals djx up to one rounding, without the 3e-8 scale error of a
    // rounded 1/6
    const F X2 = fmav(F::c(-2.0f), X1, djx) * F::c(0.25f);
    const F Y2 = fmav(F::c(-2.0f), Y1, djy) * F::c(0.25f);
    const F Pp = dpxx * F::c(0.25f);
    const F Z = dpxy * F::c(0.25f);
    if constexpr (COMP)
        *d0 = (dz - de) * F::c(1.0f / 9.0f);
    else
        v[0] = fmav(dz - de, F::c(1.0f / 9.0f), v[0]);
    F inc[9];
    inc[1] = (A + X1) + Pp;
    inc[2] = (A + Y1) - Pp;
    inc[3] = (A - X1) + Pp;
    inc[4] = (A - Y1) - Pp;
    inc[5] = ((B + X2) + Y2) + Z;
    inc[6] = ((B - X2) + Y2) - Z;
    inc[7] = ((B - X2) - Y2) + Z;
    inc[8] = ((B + X2) - Y2) - Z;
    if constexpr (COMP && ABSORB) {
        F err[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const F n = v[i] + inc[i];
            err[i] = inc[i] - (n - v[i]);
            v[i] = n;
        }
        *d0 = *d0 + (((err[1] + err[3]) + (err[2] + err[4])) + ((err[5] + err[7]) + (err[6] + err[8])));
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) v[i] = v[i] + inc[i];
    }
}

// Improved well-balanced free-energy collision (Eqs. 1, 6, 20, 21, 24); mn, rn: mu and rho
// at x + c_i (i = 1..8).  COMP: the rest population's increment goes to *d0, v[0] unchanged.
// fx: the x body force of the cell (P.fx, or P.fx plus the droplet-collision drive).
template <class F, bool COMP = false>
__device__ __forceinline__ void fe_collide_fx_v(F v[9], F rho, const F mn[9], const F rn[9], F fx,
                                                const StepParams<float>& P, F* d0) {
    const F w1 = F::c(1.0f / 3.0f), w2 = F::c(1.0f / 12.0f);
    const F gmx = fmav(mn[1] - mn[3], w1, ((mn[5] - mn[7]) + (mn[8] - mn[6])) * w2);
    const F gmy = fmav(mn[2] - mn[4], w1, ((mn[5] - mn[7]) + (mn[6] - mn[8])) * w2);
    const F grx = fmav(rn[1] - rn[3], w1, ((rn[5] - rn[7]) + (rn[8] - rn[6])) * w2);
    const F gry = fmav(rn[2] - rn[4], w1, ((rn[5] - rn[7]) + (rn[6] - rn[8])) * w2);
    const F Fx = fmav(-rho, gmx, fx), Fy = fmav(-rho, gmy, F::c(P.fy));
    const F jx = mom_jx(v);
    const F jy = mom_jy(v);
    const F inv_rho = rcp_v(rho);
    const F ux = fmav(F::c(0.5f), Fx, jx) * inv_rho;
    const F uy = fmav(F::c(0.5f), Fy, jy) * inv_rho;
    const F sax = sum_axes(v);
    const F sdg = (v[5] + v[6]) + (v[7] + v[8]);
    const F qx = fmav(F::c(2.0f), v[3] - v[1], (v[5] - v[6]) + (v[8] - v[7]));
    const F qy = fmav(F::c(2.0f), v[4] - v[2], (v[5] + v[6]) - (v[7] + v[8]));
    const F pxx = (v[1] + v[3]) - (v[2] + v[4]);
    const F pxy = (v[5] + v[7]) - (v[6] + v[8]);
    const F uu = fmav(ux, ux, uy * uy);
    const F uF = fmav(ux, Fx, uy * Fy);
    const F s = fmav(ux, grx, uy * gry);                                      // u . grad rho
    const F Gx = fmav(grx, F::c(1.0f / 3.0f), Fx), Gy = fmav(gry, F::c(1.0f / 3.0f), Fy);  // F + c_s^2 grad rho
    const F fe = fmav(F::c(6.0f), uF, F::c(4.0f) * s);
    const float he = P.h_e, hz = P.h_z, hq = P.h_q, hn = P.h_nu;
    // e - e^eq = (-4 f0 - sax + 2 sdg) - rho (3 uu - 4) and zeta - zeta^eq = (4 f0 - 2 sax + sdg)
    // - rho (4 - 3 uu) with rho = f0 + sax + sdg: f0 cancels exactly
    const F rhouu = F::c(3.0f) * rho * uu;
    const F ene = fmav(F::c(3.0f), sax, fmav(F::c(6.0f), sdg, -rhouu));
    const F zne = fmav(F::c(-6.0f), sax, fmav(F::c(-3.0f), sdg, rhouu));
    const F de = fmav(F::c(he), fe, F::c(-P.s_e) * ene);
    const F dz = fmav(F::c(-hz), fe, F::c(-P.s_z) * zne);
    const F dqx = fmav(F::c(-hq), Fx, F::c(-P.s_q) * fmav(rho, ux, qx));
    const F dqy = fmav(F::c(-hq), Fy, F::c(-P.s_q) * fmav(rho, uy, qy));
    const F dpxx = fmav(F::c(2.0f * hn), fmav(ux, Gx, -(uy * Gy)), F::c(-P.s_nu) * (pxx - rho * fmav(ux, ux, -(uy * uy))));
    const F dpxy = fmav(F::c(hn), fmav(ux, Gy, uy * Gx), F::c(-P.s_nu) * (pxy - rho * ux * uy));
    apply_dm_v<F, COMP>(v, de, dz, Fx, dqx, Fy, dqy, dpxx, dpxy, d0);
}
template <class F, bool COMP = false>
__device__ __forceinline__ void fe_collide_v(F v[9], F rho, const F mn[9], const F rn[9],
                                             const StepParams<float>& P, F* d0 = nullptr) {
    fe_collide_fx_v<F, COMP>(v, rho, mn, rn, F::c(P.fx), P, d0);
}

// Carnahan-Starling pressure (Eq. 28) and pseudopotential (Eq. 11, G = -1), explicit ops.
template <class F>
__device__ __forceinline__ F cs_pressure_v(F rho, const StepParams<float>& P) {
    const F e = F::c(P.b4) * rho;
    const F r = rcp_v(F::c(1.0f) - e);
    const F num = fmav(e, fmav(e, F::c(1.0f) - e, F::c(1.0f)), F::c(1.0f));  // 1 + e (1 + e (1 - e))
    return fmav(rho * F::c(P.RT) * num, r * r * r, -(F::c(P.a) * rho * rho));
}
__device__ __forceinline__ F1 sqrt_v(F1 x) { return F1(__fsqrt_rn(x.v)); }
__device__ __forceinline__ F2 sqrt_v(F2 x) { return F2(__fsqrt_rn(x.v.x), __fsqrt_rn(x.v.y)); }
template <class F>
__device__ __forceinline__ F pseudo_psi_v(F rho, const StepParams<float>& P) {
    // rho c_s^2 - p with c_s^2 = 1/3 as a hi + lo pair (scale-exact; see above)
    return sqrt_v(F::c(2.0f) * fmav(rho, F::c(kThirdHi), fmav(rho, F::c(kThirdLo), -cs_pressure_v(rho, P))));
}

// Modified pseudopotential collision (Eqs. 1, 4, 6, 10, 13, 30-32) in the algebra of pp_collide:
// pc = psi at the cell, pn[i] = psi at x + c_i (i = 1..8).
// COMP: compensated rest population with the moving populations' rounding absorbed (the rest
// increment goes to *d0, v[0] unchanged; see apply_dm_v and rest_update).
// fx: the x body force of the cell (P.fx, or P.fx plus the droplet-collision drive).
template <class F, bool COMP = false>
__device__ __forceinline__ void pp_collide_fx_v(F v[9], F rho, F pc, const F pn[9], F fx,
                                                const StepParams<float>& P, F* d0) {
    const F w1 = F::c(1.0f / 3.0f), w2 = F::c(1.0f / 12.0f);
    const F Sx = div12(stencil12_x(pn));
    const F Sy = div12(stencil12_y(pn));
    const F Fx = fmav(pc, Sx, fx), Fy = fmav(pc, Sy, F::c(P.fy));
    const F d1 = pn[1] - pc, d2 = pn[2] - pc, d3 = pn[3] - pc, d4 = pn[4] - pc;
    const F d5 = pn[5] - pc, d6 = pn[6] - pc, d7 = pn[7] - pc, d8 = pn[8] - pc;
    const F dd = ((d5 + d6) + (d7 + d8)) * w2;
    const F sxx = fmav(d1 + d3, w1, dd);
    const F syy = fmav(d2 + d4, w1, dd);
    const F sa = (sxx + syy) - dd;
    const F sxy = ((d5 - d6) + (d7 - d8)) * w2;
    const F Qxx = pc * fmav(F::c(P.kA), sa, F::c(P.kB) * sxx);
    const F Qyy = pc * fmav(F::c(P.kA), sa, F::c(P.kB) * syy);
    const F Qxy = pc * (F::c(P.kB) * sxy);
    const F L = F::c(P.li) * fmav(Sx, Sx, Sy * Sy);
    const F jx = mom_jx(v);
    const F jy = mom_jy(v);
    const F inv_rho = rcp_v(rho);
    const F ux = fmav(F::c(0.5f), Fx, jx) * inv_rho;
    const F uy = fmav(F::c(0.5f), Fy, jy) * inv_rho;
    const F sax = sum_axes(v);
    const F sdg = (v[5] + v[6]) + (v[7] + v[8]);
    const F e = fmav(F::c(-4.0f), v[0], fmav(F::c(2.0f), sdg, -sax));
    const F z = fmav(F::c(4.0f), v[0], fmav(F::c(-2.0f), sax, sdg));
    const F qx = fmav(F::c(2.0f), v[3] - v[1], (v[5] - v[6]) + (v[8] - v[7]));
    const F qy = fmav(F::c(2.0f), v[4] - v[2], (v[5] + v[6]) - (v[7] + v[8]));
    const F pxx = (v[1] + v[3]) - (v[2] + v[4]);
    const F pxy = (v[5] + v[7]) - (v[6] + v[8]);
    const F uu = fmav(ux, ux, uy * uy);
    const F uF = fmav(ux, Fx, uy * Fy);
    const F Ls = fmav(F::c(1.5f), Qxx + Qyy, L);  // L + 1.5 tr Q
    const float hq = P.h_q, hn = P.h_nu;
    // m* - m = -L (m - m^eq) + (I - L/2) MF' + MC  (Eqs. 1, 4/S66, 32, 13)
    const F de = fmav(F::c(P.h6_e), uF, fmav(F::c(P.s_e), Ls, F::c(-P.s_e) * (e - rho * fmav(F::c(3.0f), uu, F::c(-2.0f)))));
    const F dz = fmav(F::c(-P.h6_z), uF, fmav(F::c(-P.s_z), Ls, F::c(-P.s_z) * (z - rho * fmav(F::c(-3.0f), uu, F::c(1.0f)))));
    const F dqx = fmav(F::c(-hq), Fx, F::c(-P.s_q) * fmav(rho, ux, qx));
    const F dqy = fmav(F::c(-hq), Fy, F::c(-P.s_q) * fmav(rho, uy, qy));
    const F dpxx = fmav(F::c(2.0f * hn), fmav(ux, Fx, -(uy * Fy)),
                        F::c(-P.s_nu) * ((pxx - rho * fmav(ux, ux, -(uy * uy))) + (Qxx - Qyy)));
    const F dpxy = fmav(F::c(hn), fmav(ux, Fy, uy * Fx), F::c(-P.s_nu) * ((pxy - rho * ux * uy) + Qxy));
    // j* - j = F exactly (tau_j drops out)
    apply_dm_v<F, COMP, COMP>(v, de, dz, Fx, dqx, Fy, dqy, dpxx, dpxy, d0);
}
template <class F, bool COMP = false>
__device__ __forceinline__ void pp_collide_v(F v[9], F rho, F pc, const F pn[9], const StepParams<float>& P,
                                             F* d0 = nullptr) {
    pp_collide_fx_v<F, COMP>(v, rho, pc, pn, F::c(P.fx), P, d0);
}

// Droplet-collision drive (Sec. 5.4): the force a_x |rho - rho_ave| along x, a_x = ax_lo for
// x <= x_split and ax_hi beyond, rho_ave the mean density of the state being collided (a device
// scalar).  rho_ave == nullptr: no drive.
template <typename real>
struct Drive {
    const double* rho_ave;
    int x_split;
    real ax_lo, ax_hi;
};

// ---------------------------------------------------------------------------------
// Compensated rest population of the FP32 step (both models).
//
// FP32 rounds every population of every cell at each step; in a static state the roundings
// repeat step after step, so the cells' masses drift (linearly in the number of steps) and
// the interfaces follow: measured 1e-5 .. 4e-4 relative density error after 1e4 static steps,
// largest at low Tr where the liquid's rounding lands on a vapour ~700 times less dense.  In
// the free-energy model the rest population carries almost all of a cell's mass (f_0 = rho at
// rest, Eq. 20); in the pseudopotential model it carries 4/9 (f_i = w_i rho, Eq. 4).  FP32
// buffers therefore carry a tenth plane of int16 q per cell: the rest population is hi + q u,
// hi the FP32 value of plane 0 and u = 2^(e - 38) a per-lattice unit, e the binary exponent of
// the Carnahan-Starling packing limit 4/b (every density is below it, so |hi| < 2^(e+1), the
// rounding residual of hi is below 2^(e-24) = 2^14 u and q never leaves its 16 bits; for the
// smallest vapour densities u is still 1e-8 of the value).  Every collision adds its rest
// increment with an error-free transformation (rest_update); the pseudopotential collision
// also hands the moving populations' rounding errors to it (apply_dm_v, ABSORB), so a cell's
// stored mass changes only by the rounding of the small increments.  The arithmetic of the
// step reads hi only (rho = sum f_i in FP32); the observables and the host population views
// add q u.

// Nearest integer of each lane (the packed unit has no rounding instruction).
__device__ __forceinline__ F1 rint_v(F1 x) { return F1(rintf(x.v)); }
__device__ __forceinline__ F2 rint_v(F2 x) { return F2(rintf(x.v.x), rintf(x.v.y)); }

// (hi + qf u) + d -> (hi, qf), qf the extension held as an integer-valued float: TwoSum of hi
// and d, the old extension carried in the error term, Fast2Sum renormalisation, the residual
// rounded to a multiple of u.  The pair is then made canonical -- hi the FP32 value nearest to
// hi + qf u, ties to even -- so that a host round trip through FP64 (lbm_get_populations /
// lbm_set_populations, checkpoints) restores it bit for bit: rounding the residual can carry
// |qf u| up to u/2 past half an ulp of hi, and the last fused multiply-add moves that excess
// (a whole ulp, an exact multiple of u) into hi.  Written once for one cell (F1) or two (F2).
template <class F>
__device__ __forceinline__ void rest_update_v(F& hi, F& qf, F d, const StepParams<float>& P) {
    const F lo = qf * F::c(P.rest_unit);
    const F s = hi + d;
    const F bb = s - hi;
    const F err = (hi - (s - bb)) + (d - bb);  // hi + d = s + err exactly
    const F t = err + lo;
    const F h2 = s + t;
    const F l2 = t - (h2 - s);  // s + t = h2 + l2
    const F q2 = rint_v(l2 * F::c(P.rest_inv));
    const F h3 = fmav(q2, F::c(P.rest_unit), h2);  // nearest FP32 to h2 + q2 u
    qf = fmav(h2 - h3, F::c(P.rest_inv), q2);      // exact: h2 - h3 is 0 or one ulp
    hi = h3;
}

// Extension <-> int16 storage (rounded to nearest, clamped to +-32767).
__device__ __forceinline__ float rest_q_float(int q) { return (float)q; }
__device__ __forceinline__ int rest_q_int(float qf) { return max(-32767, min(32767, __float2int_rn(qf))); }

// Single cell: hi and its int16 q updated by the rest increment d.
__device__ __forceinline__ void rest_update(float& hi, int& q, float d, const StepParams<float>& P) {
    F1 h(hi), qf(rest_q_float(q));
    rest_update_v(h, qf, F1(d), P);
    hi = h.v;
    q = rest_q_int(qf.v);
}

// Two cells of a lane (packed FP32): w holds both int16 extensions (first cell low half).
__device__ __forceinline__ unsigned rest_update_pair(F2& hi, unsigned w, F2 d, const StepParams<float>& P) {
    F2 qf(rest_q_float((int)(short)(w & 0xffffu)), rest_q_float((int)w >> 16));
    rest_update_v(hi, qf, d, P);
    return ((unsigned)rest_q_int(qf.v.x) & 0xffffu) | ((unsigned)rest_q_int(qf.v.y) << 16);
}

// The rest-population plane of an FP32 buffer (plane 9, int16).
__device__ __forceinline__ short* rest_lo_plane(float* f, long long pitch) {
    return reinterpret_cast<short*>(f + 9 * pitch);
}
__device__ __forceinline__ const short* rest_lo_plane(const float* f, long long pitch) {
    return reinterpret_cast<const short*>(f + 9 * pitch);
}

// q of a value v (FP64) given its FP32 rounding hi and the inverse unit of the lattice.
__device__ __forceinline__ short rest_encode(double v, float hi, float rest_inv) {
    const double q = rint((v - (double)hi) * (double)rest_inv);
    return (short)fmax(-32767.0, fmin(32767.0, q));
}

// rho of pulled FP32 populations including the rest population's extension q.
__device__ __forceinline__ float sum9_rest(const float v[9], int q, const StepParams<float>& P) {
    return v[0] + ((((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]))) +
                   __fmul_rn((float)q, P.rest_unit));
}

// FP32 single-cell entry points used by every FP32 pseudopotential kernel (step, batch,
// observables); the templates above serve FP64.
__device__ __forceinline__ float pseudo_psi(float rho, const StepParams<float>& P) {
    return pseudo_psi_v(F1(rho), P).v;
}
__device__ __forceinline__ void pp_collide(float v[9], float rho, float pc, const float pn[9],
                                           const StepParams<float>& P) {
    F1 vv[9], n[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        vv[i] = F1(v[i]);
        n[i] = F1(pn[i]);
    }
    pp_collide_v(vv, F1(rho), F1(pc), n, P);
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = vv[i].v;
}

// The same collision with a compensated rest population (v[0] and q updated together).
__device__ __forceinline__ void pp_collide_comp(float v[9], int& q, float rho, float pc, const float pn[9],
                                                const StepParams<float>& P) {
    F1 vv[9], n[9], d0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        vv[i] = F1(v[i]);
        n[i] = F1(pn[i]);
    }
    pp_collide_v<F1, true>(vv, F1(rho), F1(pc), n, P, &d0);
#pragma unroll
    for (int i = 1; i < 9; ++i) v[i] = vv[i].v;
    rest_update(v[0], q, d0.v, P);
}

// FP32 single-cell entry points used by every FP32 free-energy kernel (the templates above
// serve FP64).
__device__ __forceinline__ void fe_collide(float v[9], float rho, const float mn[9], const float rn[9],
                                           const StepParams<float>& P) {
    // entry 0 of mn, rn (the cell itself) is not used and callers need not set it
    F1 vv[9], m[9], r[9];
    m[0] = r[0] = F1(0.0f);
#pragma unroll
    for (int i = 0; i < 9; ++i) vv[i] = F1(v[i]);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        m[i] = F1(mn[i]);
        r[i] = F1(rn[i]);
    }
    fe_collide_v(vv, F1(rho), m, r, P);
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = vv[i].v;
}
// The same collision with a compensated rest population: v[0] (hi) and q of the cell are
// updated together (see rest_update).
__device__ __forceinline__ void fe_collide_comp(float v[9], int& q, float rho, const float mn[9], const float rn[9],
                                                const StepParams<float>& P) {
    F1 vv[9], m[9], r[9], d0;
    m[0] = r[0] = F1(0.0f);
#pragma unroll
    for (int i = 0; i < 9; ++i) vv[i] = F1(v[i]);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        m[i] = F1(mn[i]);
        r[i] = F1(rn[i]);
    }
    fe_collide_v<F1, true>(vv, F1(rho), m, r, P, &d0);
#pragma unroll
    for (int i = 1; i < 9; ++i) v[i] = vv[i].v;
    rest_update(v[0], q, d0.v, P);
}
__device__ __forceinline__ float fe_mu(float rc, const float rn[9], const StepParams<float>& P) {
    // rn[0] is not used and callers need not set it
    F1 r[9];
    r[0] = F1(rc);
#pragma unroll
    for (int i = 1; i < 9; ++i) r[i] = F1(rn[i]);
    return fe_mu_v(F1(rc), r, P).v;
}

// ---------------------------------------------------------------------------------
// Pseudopotential step.  Block = TX main threads (one column each) + one halo warp.
template <typename real, int TX>
__global__ void __launch_bounds__(TX + 32) pp_step_kernel(const real* __restrict__ fin, real* __restrict__ fout,
                                                          const StepParams<real> P) {
    __shared__ real s_psi[4][TX + 2];
    const int nx = P.nx, ny = P.ny;
    const long long pitch = P.pitch;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, ny);
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
    auto row_offsets = [&](int r, long long& om, long long& o0, long long& op) {
        om = (long long)wrap_idx(r - 1, ny) * nx;
        o0 = (long long)wrap_idx(r, ny) * nx;
        op = (long long)wrap_idx(r + 1, ny) * nx;
    };
    if (has_col) {
        long long om, o0, op;
        row_offsets(y0 - 1, om, o0, op);
        pull9(fin, pitch, x, xm, xp, om, o0, op, cur);
    }
#pragma unroll 1
    for (int r = y0 - 1; r <= y1; ++r) {
        real nxt[9];
        const bool more = r < y1;
        if (has_col && more) {
            long long om, o0, op;
            row_offsets(r + 1, om, o0, op);
            pull9(fin, pitch, x, xm, xp, om, o0, op, nxt);
        }
        real rho = real(0);
        if (has_col) {
            rho = sum9(cur);
            s_psi[r & 3][sc] = pseudo_psi(rho, P);
        }
        __syncthreads();
        if (is_main && has_col && r > y0) {
            // centre row c = r - 1: neighbours in rows c-1 (slot r-2), c (r-1), c+1 (r)
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
            const real rho_c = sum9(prv);
            const long long o = (long long)(r - 1) * nx + x;
            if constexpr (std::is_same<real, float>::value) {
                int q = rest_lo_plane(fin, pitch)[o];  // compensated rest population
                pp_collide_comp(prv, q, rho_c, pn[0], pn, P);
                rest_lo_plane(fout, pitch)[o] = (short)q;
            } else {
                pp_collide(prv, rho_c, pn[0], pn, P);
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
        }
    }
}

// ---------------------------------------------------------------------------------
// Free-energy step.  rho ring (8 rows, 2 halo columns each side), mu ring (4 rows, 1 halo).
// Halo warp lanes: 0 -> x0-2, 1 -> x0-1 (also mu), 2 -> x0+w (also mu), 3 -> x0+w+1.
template <typename real, int TX>
__global__ void __launch_bounds__(TX + 32) fe_step_kernel(const real* __restrict__ fin, real* __restrict__ fout,
                                                          const StepParams<real> P) {
    __shared__ real s_rho[8][TX + 4];
    __shared__ real s_mu[4][TX + 2];
    const int nx = P.nx, ny = P.ny;
    const long long pitch = P.pitch;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, ny);
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
    auto row_offsets = [&](int r, long long& om, long long& o0, long long& op) {
        om = (long long)wrap_idx(r - 1, ny) * nx;
        o0 = (long long)wrap_idx(r, ny) * nx;
        op = (long long)wrap_idx(r + 1, ny) * nx;
    };
    real p0[9], p1[9], p2[9];  // pulled populations of rows r-2, r-1, r
    if (has_col) {
        long long om, o0, op;
        row_offsets(y0 - 2, om, o0, op);
        pull9(fin, pitch, x, xm, xp, om, o0, op, p2);
    }
#pragma unroll 1
    for (int r = y0 - 2; r <= y1 + 1; ++r) {
        real nxt[9];
        if (has_col && r <= y1) {
            long long om, o0, op;
            row_offsets(r + 1, om, o0, op);
            pull9(fin, pitch, x, xm, xp, om, o0, op, nxt);
        }
        if (has_col) s_rho[r & 7][rc] = sum9(p2);
        __syncthreads();
        if (has_mu && r >= y0) {
            // mu at row r - 1 from rho rows r-2, r-1, r
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
            s_mu[(r - 1) & 3][mc] = fe_mu(r0[rc], rn, P);
        }
        __syncthreads();
        if (is_main && has_col && r >= y0 + 2) {
            // centre row c = r - 2
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
            const long long o = (long long)(r - 2) * nx + x;
            if constexpr (std::is_same<real, float>::value) {
                int q = rest_lo_plane(fin, pitch)[o];  // compensated rest population
                fe_collide_comp(p0, q, rho_c, mn, rn, P);
                rest_lo_plane(fout, pitch)[o] = (short)q;
            } else {
                fe_collide(p0, rho_c, mn, rn, P);
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
// Storage convention of the pull scheme: buffer S holds S_i(y) = f_i(y + c_i), i.e. the
// population that the next step pulls into y + c_i.  The state f of the method is recovered
// as f_i(x) = S_i(x - c_i).
__device__ __forceinline__ long long shifted_cell(int x, int y, int cx, int cy, int nx, int ny) {
    int xs = x + cx, ys = y + cy;
    xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    return (long long)ys * nx + xs;
}

// Pulled populations of cell (x, y) from populations in shared memory (plain loads; the
// read-only global path of pull9 must not be given a shared-memory address).
template <typename real>
__device__ __forceinline__ void pull_cell_shared(const real* S, int N, int x, int y, int nx, int ny, real v[9]) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int om = (y == 0 ? ny - 1 : y - 1) * nx, o0 = y * nx, op = (y == ny - 1 ? 0 : y + 1) * nx;
    v[0] = S[0 * N + o0 + x];
    v[1] = S[1 * N + o0 + xm];
    v[2] = S[2 * N + om + x];
    v[3] = S[3 * N + o0 + xp];
    v[4] = S[4 * N + op + x];
    v[5] = S[5 * N + om + xm];
    v[6] = S[6 * N + om + xp];
    v[7] = S[7 * N + op + xp];
    v[8] = S[8 * N + op + xm];
}

// Pulled populations of cell (x, y) from global memory: v_i = S_i(x - c_i) = f_i(x).
template <typename real>
__device__ __forceinline__ void pull_cell(const real* __restrict__ S, long long pitch, int x, int y, int nx, int ny,
                                          real v[9]) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const long long om = (long long)(y == 0 ? ny - 1 : y - 1) * nx, o0 = (long long)y * nx,
                    op = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
    pull9(S, pitch, x, xm, xp, om, o0, op, v);
}

// f = f^eq(rho0, u = 0): Eq. (4) (weights w_i rho) or Eq. (20) (f_0 = rho, others 0),
// stored as S_i(y) = f^eq_i(rho0(y + c_i)).
template <typename real, typename src_t>
__global__ void init_kernel(const src_t* __restrict__ rho0, real* __restrict__ S, int model, int nx, int ny,
                            long long pitch, float rest_inv) {
    const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cys[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        if (model == 0) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const real w = i == 0 ? real(4.0 / 9.0) : (i < 5 ? real(1.0 / 9.0) : real(1.0 / 36.0));
                S[i * pitch + c] = w * (real)rho0[shifted_cell(x, y, cxs[i], cys[i], nx, ny)];
            }
            if constexpr (std::is_same<real, float>::value)  // the rest population to ~40 bits
                rest_lo_plane(S, pitch)[c] = rest_encode(4.0 / 9.0 * (double)rho0[c], S[c], rest_inv);
        } else {
            S[c] = (real)rho0[c];
#pragma unroll
            for (int i = 1; i < 9; ++i) S[i * pitch + c] = real(0);
            if constexpr (std::is_same<real, float>::value)
                rest_lo_plane(S, pitch)[c] = rest_encode((double)rho0[c], S[c], rest_inv);
        }
    }
}

// ---------------------------------------------------------------------------------
// Macroscopic fields for observables (not on the time-stepping path).
// rho of the current populations (Eq. 6a), and aux = psi (P) or rho itself (FE).
template <typename real>
__global__ void rho_kernel(const real* __restrict__ f, real* __restrict__ rho, real* __restrict__ aux,
                           const StepParams<real> P, int model) {
    const long long n = (long long)P.nx * P.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        real v[9];
        pull_cell(f, P.pitch, (int)(c % P.nx), (int)(c / P.nx), P.nx, P.ny, v);
        real r;
        if constexpr (std::is_same<real, float>::value)
            r = sum9_rest(v, rest_lo_plane(f, P.pitch)[c], P);
        else
            r = sum9(v);
        rho[c] = r;
        aux[c] = model == 0 ? pseudo_psi(r, P) : r;
    }
}

template <typename real>
__device__ __forceinline__ void gather8(const real* __restrict__ a, int x, int y, int nx, int ny, real n[9]) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const long long ym = (long long)(y == 0 ? ny - 1 : y - 1) * nx, y0 = (long long)y * nx,
                    yp = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
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

// FE: mu from rho (writes into mu).
template <typename real>
__global__ void mu_kernel(const real* __restrict__ rho, real* __restrict__ mu, const StepParams<real> P) {
    const long long n = (long long)P.nx * P.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % P.nx), y = (int)(c / P.nx);
        real rn[9];
        gather8(rho, x, y, P.nx, P.ny, rn);
        mu[c] = fe_mu(rn[0], rn, P);
    }
}

// u of Eq. (6b) with the model's total force; aux = psi (P) or mu (FE); rho field given.
template <typename real>
__global__ void velocity_kernel(const real* __restrict__ f, const real* __restrict__ rho,
                                const real* __restrict__ aux, real* __restrict__ ux, real* __restrict__ uy,
                                const StepParams<real> P, int model) {
    const long long n = (long long)P.nx * P.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % P.nx), y = (int)(c / P.nx);
        real v[9], an[9];
        pull_cell(f, P.pitch, x, y, P.nx, P.ny, v);
        gather8(aux, x, y, P.nx, P.ny, an);
        const real w1 = real(1.0 / 3.0), w2 = real(1.0 / 12.0);
        const real gx = (an[1] - an[3]) * w1 + ((an[5] - an[7]) + (an[8] - an[6])) * w2;
        const real gy = (an[2] - an[4]) * w1 + ((an[5] - an[7]) + (an[6] - an[8])) * w2;
        const real r = rho[c];
        real Fx, Fy;
        if (model == 0) {
            Fx = an[0] * gx + P.fx;
            Fy = an[0] * gy + P.fy;
        } else {
            Fx = -r * gx + P.fx;
            Fy = -r * gy + P.fy;
        }
        const real jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
        const real jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
        ux[c] = (jx + real(0.5) * Fx) / r;
        uy[c] = (jy + real(0.5) * Fy) / r;
    }
}

// Block partials of the observables reduction: [mass, max|u|^2, bad count] per block.
template <typename real>
__global__ void obs_partial_kernel(const real* __restrict__ rho, const real* __restrict__ ux,
                                   const real* __restrict__ uy, long long n, double* __restrict__ partials) {
    double m = 0.0, u2 = 0.0, bad = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double r = (double)rho[c], a = (double)ux[c], b = (double)uy[c];
        const double q = a * a + b * b;
        if (!(r > 0.0) || !isfinite(r) || !isfinite(q)) bad += 1.0;
        m += r;
        u2 = fmax(u2, isfinite(q) ? q : 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_down_sync(0xffffffffu, m, o);
        u2 = fmax(u2, __shfl_down_sync(0xffffffffu, u2, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    __shared__ double sm[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sm[0][wid] = m;
        sm[1][wid] = u2;
        sm[2][wid] = bad;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        m = lane < nw ? sm[0][lane] : 0.0;
        u2 = lane < nw ? sm[1][lane] : 0.0;
        bad = lane < nw ? sm[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_down_sync(0xffffffffu, m, o);
            u2 = fmax(u2, __shfl_down_sync(0xffffffffu, u2, o));
            bad += __shfl_down_sync(0xffffffffu, bad, o);
        }
        if (lane == 0) {
            partials[3 * blockIdx.x + 0] = m;
            partials[3 * blockIdx.x + 1] = u2;
            partials[3 * blockIdx.x + 2] = bad;
        }
    }
}

struct ObsConst {
    int nx, ny, geometry, nblocks;
    double RT, a, b4;
};

__device__ __forceinline__ double cs_p_d(double rho, const ObsConst& C) {
    const double e = C.b4 * rho, om = 1.0 - e;
    return rho * C.RT * (1.0 + e + e * e - e * e * e) / (om * om * om) - C.a * rho * rho;
}

// One block: combine partials, probe means, tangent width, pressure jump, radius.
// out: [rho_l, rho_v, width, dp, u_max, mass, radius, bad]
template <typename real>
__global__ void obs_final_kernel(const real* __restrict__ rho, const double* __restrict__ partials, ObsConst C,
                                 double* __restrict__ out) {
    __shared__ double red[4][256];
    const int t = threadIdx.x;
    double m = 0.0, u2 = 0.0, bad = 0.0, liq = 0.0, vap = 0.0, dmax = 0.0;
    for (int b = t; b < C.nblocks; b += blockDim.x) {
        m += partials[3 * b];
        u2 = fmax(u2, partials[3 * b + 1]);
        bad += partials[3 * b + 2];
    }
    const int nx = C.nx, ny = C.ny;
    double nl, nv;
    if (C.geometry == 0) {
        const int xl0 = nx / 2 - 1 < 0 ? 0 : nx / 2 - 1, xl1 = nx / 2, xv1 = nx - 1;
        for (int y = t; y < ny; y += blockDim.x) {
            liq += (double)rho[(long long)y * nx + xl0] + (double)rho[(long long)y * nx + xl1];
            vap += (double)rho[(long long)y * nx + 0] + (double)rho[(long long)y * nx + xv1];
        }
        nl = nv = 2.0 * ny;
    } else {
        const int cx0 = nx / 2 - 2, cy0 = ny / 2 - 2;
        if (t < 16) {
            const int dx = t & 3, dy = t >> 2;
            liq = (double)rho[(long long)wrap_idx(cy0 + dy, ny) * nx + wrap_idx(cx0 + dx, nx)];
        }
        if (t < 64) {
            const int k = t >> 4, dx = t & 3, dy = (t >> 2) & 3;
            const int xx = (k & 1) ? nx - 4 + dx : dx, yy = (k & 2) ? ny - 4 + dy : dy;
            vap = (double)rho[(long long)wrap_idx(yy, ny) * nx + wrap_idx(xx, nx)];
        }
        nl = 16.0;
        nv = 64.0;
    }
    const int prow = C.geometry == 0 ? 0 : ny / 2;
    for (int x = t; x < nx; x += blockDim.x) {
        const double a = (double)rho[(long long)prow * nx + (x == nx - 1 ? 0 : x + 1)];
        const double b = (double)rho[(long long)prow * nx + (x == 0 ? nx - 1 : x - 1)];
        dmax = fmax(dmax, fabs(a - b) * 0.5);
    }
    red[0][t] = m;
    red[1][t] = liq;
    red[2][t] = vap;
    red[3][t] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) {
            red[0][t] += red[0][t + s];
            red[1][t] += red[1][t + s];
            red[2][t] += red[2][t + s];
            red[3][t] += red[3][t + s];
        }
        __syncthreads();
    }
    const double msum = red[0][0], lsum = red[1][0], vsum = red[2][0], bsum = red[3][0];
    __syncthreads();
    red[0][t] = u2;
    red[1][t] = dmax;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) {
            red[0][t] = fmax(red[0][t], red[0][t + s]);
            red[1][t] = fmax(red[1][t], red[1][t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double rl = lsum / nl, rv = vsum / nv;
        out[0] = rl;
        out[1] = rv;
        out[2] = (rl - rv) / red[1][0];
        out[3] = cs_p_d(rl, C) - cs_p_d(rv, C);
        out[4] = sqrt(red[0][0]);
        out[5] = msum;
        const double ex = msum - rv * (double)nx * (double)ny;
        out[6] = C.geometry == 1 ? sqrt(fmax(ex, 0.0) / (3.14159265358979323846 * (rl - rv))) : nan("");
        out[7] = bsum;
    }
}

}  // namespace lbmk
