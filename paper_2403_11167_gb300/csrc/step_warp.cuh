// step_warp.cuh -- FP32 step kernels with warp-independent sliding windows.
//
// Same per-cell arithmetic as the other step kernels (lbm_kernels.cuh); what changes is
// the synchronisation.  One producer warp streams source rows of all 9 planes (columns
// [x0-4, x0+w+4) of the CTA's strip) into an S-stage shared-memory ring with 1-D bulk
// copies that complete on a per-stage "full" mbarrier.  Each consumer warp owns a run of
// at most 30 (pseudopotential) columns plus one halo column on each side, one column per
// lane: it keeps its neighbour field (psi) of the last rows in registers, reads
// x-neighbours with warp shuffles, and, once done with a staged row, arrives on that
// stage's "empty" mbarrier; the producer refills a stage when every consumer warp has
// released it.  There is no CTA-wide barrier per row: warps drift freely within the
// ring's depth.  The halo lanes cost 2 of 32 lanes of each warp.
//
// Requirements (checked on the host): nx % 4 == 0, nx >= 8, ny >= 4.  Every wait is
// bounded: on timeout a warp records the error in *err and stops; the producer waits
// (bounded) for its copies in flight before the CTA exits; the host reports
// LBM_ERR_TIMEOUT.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"
#include "step_tma.cuh"

namespace lbmk {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

template <int NW, int S, int TXW>
struct WarpStripSmem {
    static constexpr int TX = NW * TXW;  // widest strip
    static constexpr int W8 = TX + 8;    // staged row: 4 halo columns each side
    float stage[S][9 * W8];
    uint64_t full[S];
    uint64_t empty[S];
};

// Strip geometry shared by the host and the kernels: nx is split into gx strips of equal
// width rounded up to a multiple of 4 (at most NW * TXW columns); the last strip takes the
// remainder.
__host__ __device__ __forceinline__ int warp_strip_width(int nx, int gx) {
    return ((nx + gx - 1) / gx + 3) & ~3;
}

// Producer side of the ring, run by one thread: issue the first S rows, then refill each
// stage once all NW consumer warps have released it.  Returns false on timeout.
template <int S, int W8>
__device__ __forceinline__ bool ring_produce(const float* __restrict__ fin, const StepParams<float>& P, int rbase,
                                             int nsrc, int x0, int w, float (*stage)[9 * W8], uint64_t* full,
                                             uint64_t* empty, int* issued) {
    for (int k = 0; k < S && k < nsrc; ++k) {
        issue_row<W8>(fin, P.pitch, P.nx, wrap_once(rbase + k, P.ny), x0, w, stage[k], &full[k]);
        *issued = k + 1;
    }
    for (int k = S; k < nsrc; ++k) {
        const int s = k % S;
        if (!mbar_wait_bounded(&empty[s], (uint32_t)(((k / S) - 1) & 1))) return false;
        fence_proxy_async_smem();
        issue_row<W8>(fin, P.pitch, P.nx, wrap_once(rbase + k, P.ny), x0, w, stage[s], &full[s]);
        *issued = k + 1;
    }
    return true;
}

// Pseudopotential step (Eqs. 1, 4, 6, 10, 11, 13, 28, 30-32).
// Consumer warp iteration q: pull row q (staged rows q-1..q+1), psi(q); release the stage
// of row q-1; collide row q-1 with psi rows q-2..q (x-neighbours by shuffles).
template <int NW, int S>
__global__ void __launch_bounds__((NW + 1) * 32, 1) pp_step_warp(const float* __restrict__ fin,
                                                                 float* __restrict__ fout, const StepParams<float> P,
                                                                 int* __restrict__ err) {
    constexpr int TXW = 30;
    using Smem = WarpStripSmem<NW, S, TXW>;
    constexpr int W8 = Smem::W8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int nx = P.nx;
    const int wb = warp_strip_width(nx, gridDim.x);
    const int x0 = blockIdx.x * wb;
    const int w = min(wb, nx - x0);
    if (w <= 0) return;
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, P.ny);
    const int rbase = y0 - 2;
    const int nsrc = y1 - y0 + 4;  // source rows y0-2 .. y1+1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NW);
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
    // consumer warp: columns [cw, cw + nw) of the strip, lane l at column cw - 1 + l
    const int ww = (w + NW - 1) / NW;
    const int cw = warp * ww;
    const int nw = max(0, min(ww, w - cw));
    const int col = cw - 1 + lane;
    const bool act = nw > 0 && lane <= nw + 1;  // psi lanes (outputs and the two halo lanes)
    const bool out = act && lane >= 1 && lane <= nw;
    const int sc = col + 4;
    float prv[9], cur[9];
    float rho_prv = 1.0f, psm = 0.0f, ps0 = 0.0f;
    // rows 0 and 1 of the ring are read by the first iteration besides the one it waits for
    bool ok = mbar_wait_bounded(&sm.full[0], 0) && mbar_wait_bounded(&sm.full[1], 0);
#pragma unroll 1
    for (int q = y0 - 1; q <= y1 && ok; ++q) {
        const int k = q + 1 - rbase;  // ring index of row q+1
        const int sP = k % S, s0 = (k - 1) % S, sM = (k - 2) % S;
        ok = mbar_wait_bounded(&sm.full[sP], (uint32_t)((k / S) & 1));
        if (!ok) break;
        float rho_cur = 1.0f, psp = 0.0f;
        if (act) {
            pull_smem<W8>(sm.stage[sM], sm.stage[s0], sm.stage[sP], sc, cur);
            rho_cur = sum9(cur);
            psp = pseudo_psi(rho_cur, P);
        }
        // row q-1 (ring index k-2) is no longer read by this warp
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[sM]);
        // psi neighbours of row q-1: rows q-2 (psm), q-1 (ps0), q (psp)
        float pn[9];
        pn[0] = ps0;
        pn[1] = __shfl_down_sync(0xffffffffu, ps0, 1);
        pn[3] = __shfl_up_sync(0xffffffffu, ps0, 1);
        pn[2] = psp;
        pn[4] = psm;
        pn[5] = __shfl_down_sync(0xffffffffu, psp, 1);
        pn[6] = __shfl_up_sync(0xffffffffu, psp, 1);
        pn[7] = __shfl_up_sync(0xffffffffu, psm, 1);
        pn[8] = __shfl_down_sync(0xffffffffu, psm, 1);
        if (out && q > y0) {
            pp_collide(prv, rho_prv, pn[0], pn, P);
            float* o = fout + (long long)(q - 1) * nx + x0 + col;
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i * P.pitch] = prv[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) prv[i] = cur[i];
        rho_prv = rho_cur;
        psm = ps0;
        ps0 = psp;
    }
    if (!ok) atomicExch(err, 1);
}

}  // namespace lbmk
