// step_iwb_pair.cuh -- FP32 strip kernel of the full improved well-balanced free-energy model
// (Eqs. 20-24: the viscosity-tuning A, whose strain rate needs u at the neighbours, and gravity
// with reference density 0, i.e. the buoyancy force -rho g and no p_g) on a periodic lattice.
//
// The data movement is that of the strip kernels of step_pair.cuh (one producer warp feeding a
// row ring through TMA bulk copies, consumer warps in warp windows, two cells per lane in packed
// FP32), with one more level in each consumer's row pipeline: iteration q pulls row q -> rho(q);
// mu(q-1) from rho rows q-2..q; u(q-2) (Eq. 6b with the full force) from the re-pulled
// populations of row q-2, mu rows q-3..q-1 and rho(q-2); collides row q-3 with rho, mu and u
// rows q-4..q-2, re-pulling its populations from the ring; releases the stage of row q-4.  The
// chain rho -> mu -> u -> collision reaches three columns beyond the cells it updates, so a
// warp's lanes cover four columns on each side of its 56-column run, and the ring stages eight
// halo columns on each side of the strip (multiples of 4 keep every bulk copy 16-byte aligned).
//
// The direct kernel fe_step_iwb (step_ext.cuh) serves FP64, walls, the drive and gravity with a
// non-zero reference density; it writes the same equations with plain arithmetic, so the two
// agree to rounding, not bit for bit.
//
// Requirements (checked on the host): nx % 4 == 0, nx >= 8, ny >= 4; every wait bounded.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"
#include "ring.cuh"
#include "step_ext.cuh"
#include "step_pair.cuh"

namespace lbmk {

// Velocity of Eq. (6b) with the full force F = -rho grad mu + (fx, fy): the same operations, in
// the same order, as inside fe_collide_iwb_v, so a cell's stored u equals the u of its collision.
template <class F>
__device__ __forceinline__ void fe_velocity_v(const F v[9], F rho, const F mn[9], F fx, F fy, F& ux, F& uy) {
    const F w1 = F::c(1.0f / 3.0f), w2 = F::c(1.0f / 12.0f);
    const F gmx = fmav(mn[1] - mn[3], w1, ((mn[5] - mn[7]) + (mn[8] - mn[6])) * w2);
    const F gmy = fmav(mn[2] - mn[4], w1, ((mn[5] - mn[7]) + (mn[6] - mn[8])) * w2);
    const F Fx = fmav(-rho, gmx, fx), Fy = fmav(-rho, gmy, fy);
    const F inv_rho = rcp_v(rho);
    ux = fmav(F::c(0.5f), Fx, mom_jx(v)) * inv_rho;
    uy = fmav(F::c(0.5f), Fy, mom_jy(v)) * inv_rho;
}

// Full improved well-balanced collision (Eqs. 1, 6, 20, 21, 23, 24) in the FP32 algebra of
// fe_collide_fx_v: un, wn -- u_x and u_y at x + c_i (i = 0..8, entry 0 the cell's own); fx, fy --
// the external force (body force and buoyancy); pg, dpg -- p_g at the cell and d_y p_g; A -- the
// viscosity-tuning coefficient.  With X = uu + c_s^2 A S (S = grad u + grad u^T from the Eq. 24
// stencil) the equilibrium is the plain one with uu -> X plus p_g: its moments gain
// e += rho A tr S + 6 p_g, zeta -= rho A tr S + 9 p_g, p_xx += rho A (S_xx - S_yy) / 3,
// p_xy += rho A S_xy / 3.  COMP: the rest increment goes to *d0, v[0] unchanged.
// Velocity derivatives of Eq. (24) at the cell from u_x (un) and u_y (wn) at x + c_i.
template <class F>
struct Strain {
    F dxux, dyux, dxuy, dyuy;
};
template <class F>
__device__ __forceinline__ Strain<F> strain_v(const F un[9], const F wn[9]) {
    const F w1 = F::c(1.0f / 3.0f), w2 = F::c(1.0f / 12.0f);
    Strain<F> g;
    g.dxux = fmav(un[1] - un[3], w1, ((un[5] - un[7]) + (un[8] - un[6])) * w2);
    g.dyux = fmav(un[2] - un[4], w1, ((un[5] - un[7]) + (un[6] - un[8])) * w2);
    g.dxuy = fmav(wn[1] - wn[3], w1, ((wn[5] - wn[7]) + (wn[8] - wn[6])) * w2);
    g.dyuy = fmav(wn[2] - wn[4], w1, ((wn[5] - wn[7]) + (wn[6] - wn[8])) * w2);
    return g;
}

// st: the velocity derivatives of strain_v (taken before the populations are pulled, so that
// the neighbours' velocities are no longer live during the collision).
template <class F, bool COMP = false>
__device__ __forceinline__ void fe_collide_iwb_v(F v[9], F rho, const F mn[9], const F rn[9], const Strain<F>& st,
                                                 F fx, F fy, F pg, float dpg, float A,
                                                 const StepParams<float>& P, F* d0 = nullptr) {
    const F w1 = F::c(1.0f / 3.0f), w2 = F::c(1.0f / 12.0f);
    const F gmx = fmav(mn[1] - mn[3], w1, ((mn[5] - mn[7]) + (mn[8] - mn[6])) * w2);
    const F gmy = fmav(mn[2] - mn[4], w1, ((mn[5] - mn[7]) + (mn[6] - mn[8])) * w2);
    const F grx = fmav(rn[1] - rn[3], w1, ((rn[5] - rn[7]) + (rn[8] - rn[6])) * w2);
    const F gry = fmav(rn[2] - rn[4], w1, ((rn[5] - rn[7]) + (rn[6] - rn[8])) * w2);
    const F Fx = fmav(-rho, gmx, fx), Fy = fmav(-rho, gmy, fy);
    const F jx = mom_jx(v);
    const F jy = mom_jy(v);
    const F inv_rho = rcp_v(rho);
    const F ux = fmav(F::c(0.5f), Fx, jx) * inv_rho;
    const F uy = fmav(F::c(0.5f), Fy, jy) * inv_rho;
    // strain rate from the velocity stencil (Eq. 24)
    const F dxux = st.dxux, dyux = st.dyux, dxuy = st.dxuy, dyuy = st.dyuy;
    const F rA = rho * F::c(A);
    const F trS = F::c(2.0f) * (dxux + dyuy);
    const F rA3 = rA * F::c(1.0f / 3.0f);
    const F sax = sum_axes(v);
    const F sdg = (v[5] + v[6]) + (v[7] + v[8]);
    const F qx = fmav(F::c(2.0f), v[3] - v[1], (v[5] - v[6]) + (v[8] - v[7]));
    const F qy = fmav(F::c(2.0f), v[4] - v[2], (v[5] + v[6]) - (v[7] + v[8]));
    const F pxx = (v[1] + v[3]) - (v[2] + v[4]);
    const F pxy = (v[5] + v[7]) - (v[6] + v[8]);
    const F uu = fmav(ux, ux, uy * uy);
    const F Fyg = Fy - F::c(dpg);
    const F uG = fmav(ux, Fx, uy * Fyg);
    const F s = fmav(ux, grx, uy * gry);                                        // u . grad rho
    const F Gx = fmav(grx, F::c(1.0f / 3.0f), Fx), Gy = fmav(gry, F::c(1.0f / 3.0f), Fyg);  // F + c_s^2 grad rho
    const F fe = fmav(F::c(6.0f), uG, F::c(4.0f) * s);
    const float he = P.h_e, hz = P.h_z, hq = P.h_q, hn = P.h_nu;
    // e - e^eq and zeta - zeta^eq with f0 cancelled exactly (see fe_collide_fx_v), then the A and
    // p_g terms of the equilibrium
    const F rhouu = F::c(3.0f) * rho * uu;
    const F ene = fmav(F::c(-6.0f), pg, fmav(-rA, trS, fmav(F::c(3.0f), sax, fmav(F::c(6.0f), sdg, -rhouu))));
    const F zne = fmav(F::c(9.0f), pg, fmav(rA, trS, fmav(F::c(-6.0f), sax, fmav(F::c(-3.0f), sdg, rhouu))));
    const F de = fmav(F::c(he), fe, F::c(-P.s_e) * ene);
    const F dz = fmav(F::c(-hz), fe, F::c(-P.s_z) * zne);
    const F dqx = fmav(F::c(-hq), Fx, F::c(-P.s_q) * fmav(rho, ux, qx));
    const F dqy = fmav(F::c(-hq), Fy, F::c(-P.s_q) * fmav(rho, uy, qy));
    const F nxx = fmav(-rA3, F::c(2.0f) * (dxux - dyuy), pxx - rho * fmav(ux, ux, -(uy * uy)));
    const F nxy = fmav(-rA3, dxuy + dyux, pxy - rho * ux * uy);
    const F dpxx = fmav(F::c(2.0f * hn), fmav(ux, Gx, -(uy * Gy)), F::c(-P.s_nu) * nxx);
    const F dpxy = fmav(F::c(hn), fmav(ux, Gy, uy * Gx), F::c(-P.s_nu) * nxy);
    apply_dm_v<F, COMP>(v, de, dz, Fx, dqx, Fy, dqy, dpxx, dpxy, d0);
}

// Shared memory of one CTA: S staged rows of the strip (its columns plus 8 halo columns on each
// side, all nine planes), the ring's full/empty barriers, and each lane's slots for the
// rest-population extensions of the last four pulled rows (read three rows later).
template <int NW, int S>
struct IwbStripSmem {
    static constexpr int TXW = 56;        // columns updated per warp
    static constexpr int TX = NW * TXW;   // widest strip
    static constexpr int WH = TX + 16;    // staged row
    float stage[S][9 * WH];
    uint64_t full[S];
    uint64_t empty[S];
    uint32_t qext[4][NW][32];
};

// Issue the bulk copies of one source row into a stage: columns x0-8 .. x0+w+7 of the nine
// planes (periodic in x), completing on bar.  x0, w and nx are multiples of 4 and nx >= 8, so
// every source address, destination offset and size is a multiple of 16 bytes.
template <int WH>
__device__ __forceinline__ void issue_row_h8(const float* __restrict__ fin, long long pitch, int nx, int row, int x0,
                                            int w, float* stage, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, 9u * (uint32_t)(w + 16) * 4u);
    const float* src = fin + (long long)row * nx;
    const bool interior = x0 >= 8 && x0 + w + 8 <= nx;
    const int xl = x0 >= 8 ? x0 - 8 : nx - 8;
    const int xr = x0 + w < nx ? x0 + w : 0;
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
        const float* pl = src + i * pitch;
        float* d = stage + i * WH;
        if (interior) {
            bulk_g2s(d, pl + (x0 - 8), (uint32_t)(w + 16) * 4u, bar);
        } else {
            bulk_g2s(d, pl + xl, 32u, bar);
            bulk_g2s(d + 8, pl + x0, (uint32_t)w * 4u, bar);
            bulk_g2s(d + 8 + w, pl + xr, 32u, bar);
        }
    }
}

// Producer side of the ring (one thread), as ring_produce with the 8-column halo.
template <int S, int WH>
__device__ __forceinline__ bool iwb_ring_produce(const float* __restrict__ fin, const StepParams<float>& P, int rbase,
                                                 int nsrc, int x0, int w, float (*stage)[9 * WH], uint64_t* full,
                                                 uint64_t* empty, int* issued) {
    for (int k = 0; k < S && k < nsrc; ++k) {
        issue_row_h8<WH>(fin, P.pitch, P.nx, wrap_once(rbase + k, P.ny), x0, w, stage[k], &full[k]);
        *issued = k + 1;
    }
    for (int k = S; k < nsrc; ++k) {
        const int s = k % S;
        if (!mbar_wait_bounded(&empty[s], (uint32_t)(((k / S) - 1) & 1))) return false;
        fence_proxy_async_smem();
        issue_row_h8<WH>(fin, P.pitch, P.nx, wrap_once(rbase + k, P.ny), x0, w, stage[s], &full[s]);
        *issued = k + 1;
    }
    return true;
}

// E.rho_g must be 0 (checked on the host): the buoyancy is -rho g and p_g vanishes.
template <int NW, int S>
__global__ void __launch_bounds__((NW + 1) * 32, 3) fe_iwb_pair(const float* __restrict__ fin,
                                                                float* __restrict__ fout, const StepParams<float> P,
                                                                const Ext<float> E, int* __restrict__ err) {
    static_assert(S >= 6, "a consumer warp reads staged rows q-4 .. q+1 in one iteration");
    using Smem = IwbStripSmem<NW, S>;
    constexpr int TXW = Smem::TXW, WH = Smem::WH;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int nx = P.nx;
    const int wb = warp_strip_width(nx, gridDim.x);
    const int x0 = blockIdx.x * wb;
    const int w = min(wb, nx - x0);
    if (w <= 0) return;
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, P.ny);
    const int rbase = y0 - 4;
    const int nsrc = y1 - y0 + 8;  // source rows y0-4 .. y1+3 (rho rows y0-3 .. y1+2)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwa = min(NW, (w + TXW - 1) / TXW);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], nwa);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == NW) {  // producer warp
        if (lane == 0) {
            int issued = 0;
            if (!iwb_ring_produce<S, WH>(fin, P, rbase, nsrc, x0, w, sm.stage, sm.full, sm.empty, &issued)) {
                atomicExch(err, 1);
                drain_stages<S>(sm.full, issued);
            }
        }
        return;
    }
    if (warp >= nwa) return;
    // consumer warp: columns [cw, cw + nw) of the strip (nw a multiple of 4, > 0); lane l at
    // columns cw - 4 + 2l and cw - 3 + 2l, staged at sc = col + 8 (reads sc - 1 .. sc + 2, within
    // the staged row for every lane).  rho is right on columns cw-4 .. cw+nw+3, mu one column in
    // from each end, u two, the collision three: enough for the run.
    const int cw = warp * TXW;
    const int nw = min(TXW, w - cw);
    const int col = cw - 4 + 2 * lane;
    const bool act = 2 * lane < nw + 8;                // rho, mu and u lanes
    const bool out = lane >= 2 && 2 * lane < nw + 4;   // both cells inside the warp's run
    const int sc = col + 8;
    Row2 r1, r2, r3, r4;      // rho of rows q-1 .. q-4
    Row2 m2, m3, m4;          // mu of rows q-2 .. q-4
    Row2 ux3, uy3, ux4, uy4;  // u of rows q-3, q-4
    r1.c = r2.c = r3.c = r4.c = r1.xm = r2.xm = r3.xm = r4.xm = r1.xp = r2.xp = r3.xp = r4.xp = F2::c(1.0f);
    m2.c = m3.c = m4.c = m2.xm = m3.xm = m4.xm = m2.xp = m3.xp = m4.xp = F2::c(0.0f);
    ux3.c = ux4.c = uy3.c = uy4.c = ux3.xm = ux4.xm = uy3.xm = uy4.xm = F2::c(0.0f);
    ux3.xp = ux4.xp = uy3.xp = uy4.xp = F2::c(0.0f);
    const unsigned* qin = reinterpret_cast<const unsigned*>(rest_lo_plane(fin, P.pitch));
    unsigned* qout = reinterpret_cast<unsigned*>(rest_lo_plane(fout, P.pitch));
    const F2 fx = F2::c(P.fx);
    // y force: body force plus the buoyancy -rho g (reference density 0)
    auto fy_of = [&](F2 rho) { return fmav(F2::c(-E.g), rho, F2::c(P.fy)); };
    bool ok = mbar_wait_bounded(&sm.full[0], 0) && mbar_wait_bounded(&sm.full[1], 0);
#pragma unroll 1
    for (int q = y0 - 3; q <= y1 + 2 && ok; ++q) {
        const int k = q + 1 - rbase;  // ring index of row q+1
        ok = mbar_wait_bounded(&sm.full[k % S], (uint32_t)((k / S) & 1));
        if (!ok) break;
        if (out && q >= y0 && q < y1)
            cp_async4(&sm.qext[(q - y0 + 4) & 3][warp][lane], qin + (((long long)q * nx + x0 + col) >> 1));
        cp_async_commit();
        // pull row q, rho(q)
        F2 rho0 = F2::c(1.0f);
        if (act) {
            F2 v[9];
            pull_pair<WH>(sm.stage[(k - 2) % S], sm.stage[(k - 1) % S], sm.stage[k % S], sc, v);
            rho0 = sum9_v(v);
        }
        const Row2 r0 = with_shifted(rho0);
        // mu(q-1) from rho rows q-2 .. q
        Row2 m1;
        {
            F2 rn[9];
            neighbours_pair(r2, r1, r0, rn);
            const F2 mu = (act && q >= y0 - 1) ? fe_mu_v(r1.c, rn, P) : F2::c(0.0f);
            m1 = with_shifted(mu);
        }
        // u(q-2) from its populations (ring indices k-4 .. k-2 hold source rows q-3 .. q-1), mu
        // rows q-3 .. q-1 and rho(q-2)
        Row2 ux2, uy2;
        {
            F2 ux = F2::c(0.0f), uy = F2::c(0.0f);
            if (act && q >= y0 + 1) {
                F2 v[9], mn[9];
                pull_pair<WH>(sm.stage[(k - 4) % S], sm.stage[(k - 3) % S], sm.stage[(k - 2) % S], sc, v);
                neighbours_pair(m3, m2, m1, mn);
                fe_velocity_v(v, r2.c, mn, fx, fy_of(r2.c), ux, uy);
            }
            ux2 = with_shifted(ux);
            uy2 = with_shifted(uy);
        }
        // collide row q-3 (ring indices k-5 .. k-3 hold source rows q-4 .. q-2)
        if (out && q >= y0 + 3) {
            Strain<F2> st;
            {
                F2 un[9], wn[9];
                neighbours_pair(ux4, ux3, ux2, un);
                neighbours_pair(uy4, uy3, uy2, wn);
                st = strain_v(un, wn);
            }
            F2 v[9], mn[9], rn[9];
            pull_pair<WH>(sm.stage[(k - 5) % S], sm.stage[(k - 4) % S], sm.stage[(k - 3) % S], sc, v);
            neighbours_pair(m4, m3, m2, mn);
            neighbours_pair(r4, r3, r2, rn);
            F2 d0;
            fe_collide_iwb_v<F2, true>(v, r3.c, mn, rn, st, fx, fy_of(r3.c), F2::c(0.0f), 0.0f, E.A, P, &d0);
            cp_async_wait<3>();  // the copy of row q-3's extensions (three groups ago) has landed
            const unsigned ql3 = sm.qext[(q - 3 - y0 + 4) & 3][warp][lane];
            const unsigned qw = rest_update_pair(v[0], ql3, d0, P);  // compensated rest population
            const long long oc = (long long)(q - 3) * nx + x0 + col;
            float* o = fout + oc;
#pragma unroll
            for (int i = 0; i < 9; ++i) *reinterpret_cast<float2*>(o + i * P.pitch) = v[i].v;
            qout[oc >> 1] = qw;
        }
        // row q-4 (ring index k-5) is no longer read by this warp
        __syncwarp();
        if (lane == 0 && k >= 5) mbar_arrive(&sm.empty[(k - 5) % S]);
        r4 = r3;
        r3 = r2;
        r2 = r1;
        r1 = r0;
        m4 = m3;
        m3 = m2;
        m2 = m1;
        ux4 = ux3;
        ux3 = ux2;
        uy4 = uy3;
        uy3 = uy2;
    }
    cp_async_wait<0>();
    if (!ok) atomicExch(err, 1);
}

}  // namespace lbmk
