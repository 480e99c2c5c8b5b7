// step_pair.cuh -- FP32 step kernels of both models: warp-independent windows, two cells
// per lane.  (The free-energy kernel is described first; the pseudopotential kernel at the end.)
//
// Per-cell arithmetic: fe_mu_v / fe_collide_v (lbm_kernels.cuh) on F2, Blackwell's packed
// FP32, so one instruction updates both cells of a lane; results are bitwise those of the
// single-cell kernels.  Data movement: the row ring of ring.cuh (one producer warp,
// per-stage full/empty mbarriers, no CTA barrier per row).  Each consumer warp owns a run of
// 60 columns (the last one fewer; warps beyond the strip stay idle) plus two halo columns on each side, two adjacent columns per lane: it keeps rho
// of the last four rows and mu of the last three in registers, reads x-neighbours with warp
// shuffles, and re-pulls the populations of the row it collides (two rows behind the row it
// pulls) from the ring, which therefore holds rows q-3 .. q+1 of every warp plus prefetch.
//
// Iteration q of a consumer warp: pull row q (staged rows q-1..q+1), rho(q); mu(q-1) from rho
// rows q-2..q; collide row q-2 with mu rows q-3..q-1 and rho rows q-3..q-1, re-pulling its
// populations from staged rows q-3..q-1; release the stage of row q-3.
//
// Both kernels carry the compensated rest population (rest_update in lbm_kernels.cuh): each
// lane reads and writes one 32-bit word of the int16 rest plane per row (its two cells),
// loaded when the row is pulled and used when that row is collided (two iterations later for
// the free-energy kernel, one for the pseudopotential kernel).
//
// Requirements (checked on the host): nx % 4 == 0, nx >= 8, ny >= 4; every wait bounded.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"
#include "ring.cuh"

namespace lbmk {

// Populations of the two cells at staged columns sc, sc + 1 (sc even) pulled from the stages of
// rows q-1 (Rm), q (R0), q+1 (Rp): v_i = f_i(x - c_i).
template <int W8>
__device__ __forceinline__ void pull_pair(const float* Rm, const float* R0, const float* Rp, int sc, F2 v[9]) {
    v[0] = F2(*reinterpret_cast<const float2*>(R0 + 0 * W8 + sc));
    v[1] = F2(R0[1 * W8 + sc - 1], R0[1 * W8 + sc]);
    v[2] = F2(*reinterpret_cast<const float2*>(Rm + 2 * W8 + sc));
    v[3] = F2(R0[3 * W8 + sc + 1], R0[3 * W8 + sc + 2]);
    v[4] = F2(*reinterpret_cast<const float2*>(Rp + 4 * W8 + sc));
    v[5] = F2(Rm[5 * W8 + sc - 1], Rm[5 * W8 + sc]);
    v[6] = F2(Rm[6 * W8 + sc + 1], Rm[6 * W8 + sc + 2]);
    v[7] = F2(Rp[7 * W8 + sc + 1], Rp[7 * W8 + sc + 2]);
    v[8] = F2(Rp[8 * W8 + sc - 1], Rp[8 * W8 + sc]);
}

// A row of a field held as pairs (c: the lane's two cells) with its x-shifted pairs formed
// once from the adjacent lanes: the values at x - 1 (xm) and x + 1 (xp) of both cells, so that
// each use of the row reads them without re-pairing registers.
struct Row2 {
    F2 c, xm, xp;
};
__device__ __forceinline__ Row2 with_shifted(F2 c) {
    Row2 r;
    r.c = c;
    r.xm = F2(__shfl_up_sync(0xffffffffu, c.v.y, 1), c.v.x);
    r.xp = F2(c.v.y, __shfl_down_sync(0xffffffffu, c.v.x, 1));
    return r;
}
// Values at x + c_i (i = 1..8) of both cells of a lane, from the rows below (ym), at (y0) and
// above (yp); y grows with the row index.
__device__ __forceinline__ void neighbours_pair(const Row2& ym, const Row2& y0, const Row2& yp, F2 n[9]) {
    n[0] = y0.c;
    n[1] = y0.xp;  // (+1, 0)
    n[2] = yp.c;   // ( 0, +1)
    n[3] = y0.xm;  // (-1, 0)
    n[4] = ym.c;   // ( 0, -1)
    n[5] = yp.xp;  // (+1, +1)
    n[6] = yp.xm;  // (-1, +1)
    n[7] = ym.xm;  // (-1, -1)
    n[8] = ym.xp;  // (+1, -1)
}

// DRIVE: the droplet-collision drive of Sec. 5.4 adds a_x |rho - rho_ave| to each cell's x
// force (rho_ave from D.rho_ave), and every consumer warp writes the sum of the populations it
// stored -- the mass of the next state, which on a periodic lattice holds each stored population
// once -- to mass[((blockIdx.y * gridDim.x) + blockIdx.x) * NW + warp] (0 for idle warps), so
// that the next step's rho_ave needs no pass over the lattice.
template <int NW, bool DRIVE>
__device__ __forceinline__ void zero_mass_slots(double* mass) {
    if (DRIVE && threadIdx.x < NW) mass[(blockIdx.y * gridDim.x + blockIdx.x) * NW + threadIdx.x] = 0.0;
}
// The two cells' x force with the drive: P.fx + a_x |rho - rho_ave| (ax: a_x of both cells).
__device__ __forceinline__ F2 driven_fx(F2 rho, float rave, F2 ax, const StepParams<float>& P) {
    const F2 dr = rho - F2::c(rave);
    return fmav(ax, F2(fabsf(dr.v.x), fabsf(dr.v.y)), F2::c(P.fx));
}
// a_x of the cells at columns gx and gx + 1
__device__ __forceinline__ F2 drive_ax(const Drive<float>& D, int gx) {
    return F2(gx <= D.x_split ? D.ax_lo : D.ax_hi, gx + 1 <= D.x_split ? D.ax_lo : D.ax_hi);
}
// One warp's stored mass (two FP32 partial sums per lane) into its slot, fixed order.
__device__ __forceinline__ void store_warp_mass(F2 macc, double* slot) {
    double s = (double)macc.v.x + (double)macc.v.y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) *slot = s;
}

template <int NW, int S, bool DRIVE = false>
__global__ void __launch_bounds__((NW + 1) * 32, 1) fe_step_pair(const float* __restrict__ fin,
                                                                 float* __restrict__ fout, const StepParams<float> P,
                                                                 int* __restrict__ err, const Drive<float> D = {},
                                                                 double* __restrict__ mass = nullptr) {
    constexpr int TXW = 60;
    using Smem = WarpStripSmem<NW, S, TXW>;
    constexpr int W8 = Smem::W8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int nx = P.nx;
    const int wb = warp_strip_width(nx, gridDim.x);
    const int x0 = blockIdx.x * wb;
    const int w = min(wb, nx - x0);
    if (w <= 0) {
        zero_mass_slots<NW, DRIVE>(mass);
        return;
    }
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, P.ny);
    const int rbase = y0 - 3;
    const int nsrc = y1 - y0 + 6;  // source rows y0-3 .. y1+2 (rho rows y0-2 .. y1+1)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // consumer warps fill 60-column runs from the left; only the warps with columns run (a
    // narrow strip leaves the others idle instead of spreading few lanes over all of them)
    const int nwa = min(NW, (w + 59) / 60);
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
            if (!ring_produce<S, W8>(fin, P, rbase, nsrc, x0, w, sm.stage, sm.full, sm.empty, &issued)) {
                atomicExch(err, 1);
                drain_stages<S>(sm.full, issued);
            }
        }
        return;
    }
    double* const mslot = DRIVE ? mass + (blockIdx.y * gridDim.x + blockIdx.x) * NW + warp : nullptr;
    if (warp >= nwa) {
        if (DRIVE && lane == 0) *mslot = 0.0;
        return;
    }
    // consumer warp: columns [cw, cw + nw) of the strip (nw even, > 0), lane l at columns
    // cw - 2 + 2l and cw - 1 + 2l
    const int cw = warp * 60;
    const int nw = min(60, w - cw);
    const int col = cw - 2 + 2 * lane;
    const bool act = nw > 0 && 2 * lane <= nw + 2;           // rho and mu lanes
    const bool out = act && lane >= 1 && 2 * lane <= nw;     // both cells inside the warp's run
    const int sc = col + 4;
    Row2 r1, r2, r3;  // rho of rows q-1, q-2, q-3
    Row2 m2, m3;      // mu of rows q-2, q-3
    // rest-population extensions q (two int16 per lane): copied into slot (row mod 3) of the
    // lane's qext ring when the row is pulled, read two iterations later by its collision
    const unsigned* qin = reinterpret_cast<const unsigned*>(rest_lo_plane(fin, P.pitch));
    unsigned* qout = reinterpret_cast<unsigned*>(rest_lo_plane(fout, P.pitch));
    r1.c = r2.c = r3.c = m2.c = m3.c = F2::c(1.0f);
    r1.xm = r1.xp = r2.xm = r2.xp = r3.xm = r3.xp = F2::c(1.0f);
    m2.xm = m2.xp = m3.xm = m3.xp = F2::c(1.0f);
    const float rave = DRIVE ? (float)*D.rho_ave : 0.0f;
    const F2 ax = DRIVE ? drive_ax(D, x0 + col) : F2::c(0.0f);
    F2 macc = F2::c(0.0f);
    bool ok = mbar_wait_bounded(&sm.full[0], 0) && mbar_wait_bounded(&sm.full[1], 0);
#pragma unroll 1
    for (int q = y0 - 2; q <= y1 + 1 && ok; ++q) {
        const int k = q + 1 - rbase;  // ring index of row q+1
        ok = mbar_wait_bounded(&sm.full[k % S], (uint32_t)((k / S) & 1));
        if (!ok) break;
        if (out && q >= y0 && q < y1)
            cp_async4(&sm.qext[(q - y0 + 3) % 3][warp][lane], qin + (((long long)q * nx + x0 + col) >> 1));
        cp_async_commit();
        // pull row q, rho(q)
        F2 rho0 = F2::c(1.0f);
        if (act) {
            F2 v[9];
            pull_pair<W8>(sm.stage[(k - 2) % S], sm.stage[(k - 1) % S], sm.stage[k % S], sc, v);
            rho0 = sum9_v(v);
        }
        const Row2 r0 = with_shifted(rho0);
        // mu(q-1) from rho rows q-2, q-1, q
        Row2 m1;
        {
            F2 rn[9];
            neighbours_pair(r2, r1, r0, rn);
            const F2 mu = (act && q >= y0) ? fe_mu_v(r1.c, rn, P) : F2::c(0.0f);
            m1 = with_shifted(mu);
        }
        // collide row q-2 (ring indices k-4 .. k-2 hold source rows q-3 .. q-1)
        if (out && q >= y0 + 2) {
            F2 v[9], mn[9], rn[9];
            pull_pair<W8>(sm.stage[(k - 4) % S], sm.stage[(k - 3) % S], sm.stage[(k - 2) % S], sc, v);
            neighbours_pair(m3, m2, m1, mn);
            neighbours_pair(r3, r2, r1, rn);
            F2 d0;
            if constexpr (DRIVE)
                fe_collide_fx_v<F2, true>(v, r2.c, mn, rn, driven_fx(r2.c, rave, ax, P), P, &d0);
            else
                fe_collide_v<F2, true>(v, r2.c, mn, rn, P, &d0);
            cp_async_wait<2>();  // the copy of row q-2's extensions (two groups ago) has landed
            const unsigned ql2 = sm.qext[(q - 2 - y0 + 3) % 3][warp][lane];
            const unsigned qw = rest_update_pair(v[0], ql2, d0, P);  // compensated rest population
            if constexpr (DRIVE) macc = macc + sum9_v(v);
            const long long oc = (long long)(q - 2) * nx + x0 + col;
            float* o = fout + oc;
#pragma unroll
            for (int i = 0; i < 9; ++i) *reinterpret_cast<float2*>(o + i * P.pitch) = v[i].v;
            qout[oc >> 1] = qw;
        }
        // row q-3 (ring index k-4) is no longer read by this warp
        __syncwarp();
        if (lane == 0 && k >= 4) mbar_arrive(&sm.empty[(k - 4) % S]);
        r3 = r2;
        r2 = r1;
        r1 = r0;
        m3 = m2;
        m2 = m1;
    }
    cp_async_wait<0>();
    if constexpr (DRIVE) store_warp_mass(macc, mslot);
    if (!ok) atomicExch(err, 1);
}

// Pseudopotential step (Eqs. 1, 4, 6, 10, 11, 13, 28, 30-32), two cells per lane.
// Consumer warp iteration q: pull row q (staged rows q-1..q+1), psi(q); collide row q-1 with
// psi rows q-2..q, re-pulling its populations from staged rows q-2..q; release the stage of
// row q-2.  Lanes 0 and nw/2 + 1 supply the psi halo columns.
// One CTA's strip of the pseudopotential step: columns [x0, x0 + w) (w <= 60 NW, x0 and w
// multiples of 4), rows [y0, y1).  Called by every thread of the CTA.
// DRIVE: as for fe_step_pair; mass points to this CTA's NW slots.
template <int NW, int S, bool DRIVE = false>
__device__ __forceinline__ void pp_pair_strip(const float* __restrict__ fin, float* __restrict__ fout,
                                              const StepParams<float>& P, int x0, int w, int y0, int y1,
                                              WarpStripSmem<NW, S, 60>& sm, int* __restrict__ err,
                                              const Drive<float>* D = nullptr, double* mass = nullptr) {
    constexpr int W8 = WarpStripSmem<NW, S, 60>::W8;
    const int nx = P.nx;
    const int rbase = y0 - 2;
    const int nsrc = y1 - y0 + 4;  // source rows y0-2 .. y1+1 (psi rows y0-1 .. y1)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // consumer warps fill 60-column runs from the left; only the warps with columns run (a
    // narrow strip leaves the others idle instead of spreading few lanes over all of them)
    const int nwa = min(NW, (w + 59) / 60);
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
            if (!ring_produce<S, W8>(fin, P, rbase, nsrc, x0, w, sm.stage, sm.full, sm.empty, &issued)) {
                atomicExch(err, 1);
                drain_stages<S>(sm.full, issued);
            }
        }
        return;
    }
    if (warp >= nwa) {
        if (DRIVE && lane == 0) mass[warp] = 0.0;
        return;
    }
    const int cw = warp * 60;
    const int nw = min(60, w - cw);
    const int col = cw - 2 + 2 * lane;
    const bool act = nw > 0 && 2 * lane <= nw + 2;
    const bool out = act && lane >= 1 && 2 * lane <= nw;
    const int sc = col + 4;
    Row2 p1, p2;  // psi of rows q-1, q-2
    // rest-population extensions q (two int16 per lane): copied into slot (row mod 3) of the
    // lane's qext ring when the row is pulled, read by its collision in the next iteration
    const unsigned* qin = reinterpret_cast<const unsigned*>(rest_lo_plane(fin, P.pitch));
    unsigned* qout = reinterpret_cast<unsigned*>(rest_lo_plane(fout, P.pitch));
    p1.c = p2.c = F2::c(0.0f);
    p1.xm = p1.xp = p2.xm = p2.xp = F2::c(0.0f);
    F2 rho1 = F2::c(1.0f);  // rho of row q-1
    const float rave = DRIVE ? (float)*D->rho_ave : 0.0f;
    const F2 ax = DRIVE ? drive_ax(*D, x0 + col) : F2::c(0.0f);
    F2 macc = F2::c(0.0f);
    bool ok = mbar_wait_bounded(&sm.full[0], 0) && mbar_wait_bounded(&sm.full[1], 0);
#pragma unroll 1
    for (int q = y0 - 1; q <= y1 && ok; ++q) {
        const int k = q + 1 - rbase;  // ring index of row q+1
        ok = mbar_wait_bounded(&sm.full[k % S], (uint32_t)((k / S) & 1));
        if (!ok) break;
        if (out && q >= y0 && q < y1)
            cp_async4(&sm.qext[(q - y0 + 3) % 3][warp][lane], qin + (((long long)q * nx + x0 + col) >> 1));
        cp_async_commit();
        F2 rho0 = F2::c(1.0f), psi = F2::c(0.0f);
        if (act) {
            F2 v[9];
            pull_pair<W8>(sm.stage[(k - 2) % S], sm.stage[(k - 1) % S], sm.stage[k % S], sc, v);
            rho0 = sum9_v(v);
            psi = pseudo_psi_v(rho0, P);
        }
        const Row2 p0 = with_shifted(psi);
        // collide row q-1 (ring indices k-3 .. k-1 hold source rows q-2 .. q)
        if (out && q > y0) {
            F2 v[9], pn[9];
            pull_pair<W8>(sm.stage[(k - 3) % S], sm.stage[(k - 2) % S], sm.stage[(k - 1) % S], sc, v);
            neighbours_pair(p2, p1, p0, pn);
            F2 d0;
            if constexpr (DRIVE)
                pp_collide_fx_v<F2, true>(v, rho1, pn[0], pn, driven_fx(rho1, rave, ax, P), P, &d0);
            else
                pp_collide_v<F2, true>(v, rho1, pn[0], pn, P, &d0);
            cp_async_wait<1>();  // the copy of row q-1's extensions (one group ago) has landed
            const unsigned ql1 = sm.qext[(q - 1 - y0 + 3) % 3][warp][lane];
            const unsigned qw = rest_update_pair(v[0], ql1, d0, P);  // compensated rest population
            if constexpr (DRIVE) macc = macc + sum9_v(v);
            const long long oc = (long long)(q - 1) * nx + x0 + col;
            float* o = fout + oc;
#pragma unroll
            for (int i = 0; i < 9; ++i) *reinterpret_cast<float2*>(o + i * P.pitch) = v[i].v;
            qout[oc >> 1] = qw;
        }
        // row q-2 (ring index k-3) is no longer read by this warp
        __syncwarp();
        if (lane == 0 && k >= 3) mbar_arrive(&sm.empty[(k - 3) % S]);
        p2 = p1;
        p1 = p0;
        rho1 = rho0;
    }
    cp_async_wait<0>();
    if constexpr (DRIVE) store_warp_mass(macc, mass + warp);
    if (!ok) atomicExch(err, 1);
}

template <int NW, int S, bool DRIVE = false>
__global__ void __launch_bounds__((NW + 1) * 32, 1) pp_step_pair(const float* __restrict__ fin,
                                                                 float* __restrict__ fout, const StepParams<float> P,
                                                                 int* __restrict__ err, const Drive<float> D = {},
                                                                 double* __restrict__ mass = nullptr) {
    using Smem = WarpStripSmem<NW, S, 60>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int wb = warp_strip_width(P.nx, gridDim.x);
    const int x0 = blockIdx.x * wb;
    const int w = min(wb, P.nx - x0);
    if (w <= 0) {
        zero_mass_slots<NW, DRIVE>(mass);
        return;
    }
    const int y0 = blockIdx.y * P.rows;
    pp_pair_strip<NW, S, DRIVE>(fin, fout, P, x0, w, y0, min(y0 + P.rows, P.ny), sm, err, &D,
                                DRIVE ? mass + (blockIdx.y * gridDim.x + blockIdx.x) * NW : nullptr);
}

}  // namespace lbmk
