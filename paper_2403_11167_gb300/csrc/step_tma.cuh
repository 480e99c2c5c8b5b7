// step_tma.cuh -- FP32 step kernels fed by a TMA (cp.async.bulk) row pipeline.
//
// Same arithmetic as pp_step_kernel / fe_step_kernel (lbm_kernels.cuh); what changes
// is how populations reach the CTA.  One elected thread streams whole source rows of
// all 9 planes -- columns [x0-4, x0+w+4) of the CTA's strip, so every pulled value
// and every halo column is present -- into an S-stage shared-memory ring with 1-D
// bulk copies that complete on a per-stage mbarrier.  The other threads read their
// pulled populations with shared-memory loads at constant offsets; no global-load
// latency sits on their critical path, no registers hold prefetched rows, and the
// ring keeps several rows of every CTA in flight.
//
// Requirements (checked on the host): nx % 4 == 0, nx >= 8, ny >= 4 (16-byte aligned
// rows for the bulk copies; the wrapped x halo is fetched as separate 16-byte pieces).
// Every mbarrier wait is bounded: on timeout the CTA records the error in *err, waits
// (bounded) for its own copies in flight and returns; the host reports LBM_ERR_TIMEOUT.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"

namespace lbmk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for a phase of an mbarrier for at most max_polls polls (with backoff after 64);
// false on timeout.
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* bar, uint32_t parity, uint32_t max_polls) {
    for (uint32_t it = 0; it < max_polls; ++it) {
        if (mbar_test_parity(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// Bounded wait of the step kernels (2^22 polls, well under a second); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    return mbar_wait_polls(bar, parity, 1u << 22);
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Issue the 9-plane copy of source row `row` (already wrapped into [0, ny)) into one stage:
// smem layout per plane: [4 left halo | w main | 4 right halo], plane stride W8 floats.
#ifdef LBM_TMA_CHECKS
// Self-check build: verify a bulk copy before issuing it; record the first bad one in
// err[1..7] and skip it (the stage then never completes and the bounded wait reports it).
__device__ __forceinline__ bool tma_copy_ok(const float* fin, long long total, const float* src, uint32_t bytes,
                                            const void* dst, const void* smem_lo, const void* smem_hi, int* err,
                                            int k, int i) {
    const long long off = (long long)(src - fin);
    const bool ok = off >= 0 && off * 4 + bytes <= total * 4 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) &&
                    (bytes & 15) == 0 && dst >= smem_lo && (const char*)dst + bytes <= (const char*)smem_hi &&
                    ((smem_u32(dst) & 15) == 0);
    if (!ok && atomicCAS(err + 1, 0, 1) == 0) {
        err[2] = (int)blockIdx.x;
        err[3] = (int)blockIdx.y;
        err[4] = k;
        err[5] = i;
        err[6] = (int)off;
        err[7] = (int)bytes;
    }
    return ok;
}
#endif

template <int W8>
__device__ __forceinline__ void issue_row(const float* __restrict__ fin, long long pitch, int nx, int row, int x0,
                                         int w, float* stage, uint64_t* bar, int* err = nullptr, int kdbg = 0,
                                         const void* smem_lo = nullptr, const void* smem_hi = nullptr) {
    mbar_arrive_expect_tx(bar, 9u * (uint32_t)(w + 8) * 4u);
    const float* src = fin + (long long)row * nx;
    const bool interior = x0 >= 4 && x0 + w + 4 <= nx;
    const int xl = x0 >= 4 ? x0 - 4 : nx - 4;
    const int xr = x0 + w < nx ? x0 + w : 0;
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
        const float* pl = src + i * pitch;
        float* d = stage + i * W8;
#ifdef LBM_TMA_CHECKS
        const long long tot = 9 * pitch;
#define LBM_BULK(D, SRC, B)                                                                 \
    do {                                                                                    \
        if (tma_copy_ok(fin, tot, (SRC), (B), (D), smem_lo, smem_hi, err, kdbg, i)) bulk_g2s((D), (SRC), (B), bar); \
    } while (0)
#else
#define LBM_BULK(D, SRC, B) bulk_g2s((D), (SRC), (B), bar)
#endif
        if (interior) {
            LBM_BULK(d, pl + (x0 - 4), (uint32_t)(w + 8) * 4u);
        } else {
            LBM_BULK(d, pl + xl, 16u);
            LBM_BULK(d + 4, pl + x0, (uint32_t)w * 4u);
            LBM_BULK(d + 4 + w, pl + xr, 16u);
        }
#undef LBM_BULK
    }
}

// Pulled populations of smem column sc from the stages holding rows q-1 (Rm), q (R0), q+1 (Rp).
template <int W8>
__device__ __forceinline__ void pull_smem(const float* Rm, const float* R0, const float* Rp, int sc, float v[9]) {
    v[0] = R0[0 * W8 + sc];
    v[1] = R0[1 * W8 + sc - 1];
    v[2] = Rm[2 * W8 + sc];
    v[3] = R0[3 * W8 + sc + 1];
    v[4] = Rp[4 * W8 + sc];
    v[5] = Rm[5 * W8 + sc - 1];
    v[6] = Rm[6 * W8 + sc + 1];
    v[7] = Rp[7 * W8 + sc + 1];
    v[8] = Rp[8 * W8 + sc - 1];
}

// After a timeout: wait (bounded) for the last fill issued into every stage, so no bulk
// copy still targets this CTA's shared memory when it exits.
template <int S>
__device__ __forceinline__ void drain_stages(uint64_t* bars, int issued) {
    for (int s = 0; s < S; ++s) {
        int last = -1;
        for (int k = issued - 1; k >= 0 && k >= issued - S; --k)
            if (k % S == s) {
                last = k;
                break;
            }
        if (last >= 0) mbar_wait_bounded(&bars[s], (uint32_t)((last / S) & 1));
    }
}

__device__ __forceinline__ int wrap_once(int r, int n) { return r < 0 ? r + n : (r >= n ? r - n : r); }

template <int TX, int S>
struct PPTmaSmem {
    static constexpr int W8 = TX + 8;
    float stage[S][9 * W8];
    float psi[4][TX + 2];
    uint64_t bar[S];
};

__device__ __forceinline__ int next_stage(int s, int S) { return s + 1 == S ? 0 : s + 1; }

// Pseudopotential step (Eqs. 1, 4, 6, 10, 11, 13, 28, 30-32), TMA-fed.
// Iteration q computes psi of row q (needs staged rows q-1..q+1), then, after the one
// barrier of the row, collides row q-1.
// Minimum resident CTAs per SM given to ptxas.  These kernels are issue-bound, and a
// register budget beats occupancy (measured: 1 block minimum, i.e. no register cap, was
// 10-25% faster than caps matching the shared-memory occupancy); an explicit bound also
// keeps ptxas from trading registers for spills, which a bare thread bound provoked.
#ifndef LBM_PP_MINB
#define LBM_PP_MINB 1
#endif
#ifndef LBM_FE_MINB
#define LBM_FE_MINB 1
#endif
#ifndef LBM_PP_UNROLL
#define LBM_PP_UNROLL 1
#endif
#ifndef LBM_FE_UNROLL
#define LBM_FE_UNROLL 1
#endif
constexpr int kPPUnroll = LBM_PP_UNROLL;  // row-loop unroll factors
constexpr int kFEUnroll = LBM_FE_UNROLL;

// One CTA's strip of the pseudopotential step: columns [x0, x0 + w), rows [y0, y1).
template <int TX, int S>
__device__ __forceinline__ void pp_strip_tma(const float* __restrict__ fin, float* __restrict__ fout,
                                             const StepParams<float>& P, int x0, int w, int y0, int y1,
                                             PPTmaSmem<TX, S>& sm, int* __restrict__ err) {
    constexpr int W8 = TX + 8;
    const int nx = P.nx, ny = P.ny;
    const int t = threadIdx.x;
    const bool is_main = t < TX;
    const bool producer = t == TX;
    bool has_col;
    int col;  // column relative to x0 (-1 and w are the halo columns)
    if (is_main) {
        has_col = t < w;
        col = t;
    } else {
        has_col = (t - TX) < 2;
        col = (t - TX) == 0 ? -1 : w;
    }
    const int sc = col + 4;  // column in a staged row
    const int rbase = y0 - 2;
    const int nsrc = y1 + 1 - rbase + 1;  // source rows y0-2 .. y1+1
    if (producer) {
        for (int s = 0; s < S; ++s) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;  // rows issued so far (producer only)
    if (producer) {
        for (int k = 0; k < S && k < nsrc; ++k)
            issue_row<W8>(fin, P.pitch, nx, wrap_once(rbase + k, ny), x0, w, sm.stage[k], &sm.bar[k], err, k,
                          sm.stage[0], sm.stage[0] + S * 9 * W8);
        issued = min(S, nsrc);
    }
    float prv[9], cur[9];
    float rho_prv = 1.0f, rho_cur = 1.0f;
    // The first iteration reads the stages of rows y0-2 and y0-1 (fills 0 and 1) besides the
    // one it waits for; wait for those two here, so every fill is waited on before it is read
    // and before its stage is re-armed for the next fill.
    bool failed = __syncthreads_or(!(mbar_wait_bounded(&sm.bar[0], 0) && mbar_wait_bounded(&sm.bar[1], 0)));
    int sm2 = 0, sm1 = 1, s0 = 2 % S;  // stages of rows q-1, q, q+1
    uint32_t par = 0;                  // parity of the fill being waited for (stage s0)
#pragma unroll(kPPUnroll)
    for (int q = y0 - 1; q <= y1 && !failed; ++q) {
        const int k = q + 1 - rbase;  // staged index of row q+1
        const bool ok = mbar_wait_bounded(&sm.bar[s0], par);
        if (ok && has_col) {
            pull_smem<W8>(sm.stage[sm2], sm.stage[sm1], sm.stage[s0], sc, cur);
            rho_cur = sum9(cur);
            sm.psi[q & 3][col + 1] = pseudo_psi(rho_cur, P);
        }
        if (__syncthreads_or(!ok)) {
#ifdef LBM_TMA_CHECKS
            if (!ok && atomicCAS(err + 8, 0, 1) == 0) {
                err[9] = (int)blockIdx.x;
                err[10] = (int)blockIdx.y;
                err[11] = q;
                err[12] = k;
            }
#endif
            failed = true;
            break;
        }
        if (producer && k - 2 + S < nsrc) {
            fence_proxy_async_smem();
            const int kk = k - 2 + S;
            issue_row<W8>(fin, P.pitch, nx, wrap_once(rbase + kk, ny), x0, w, sm.stage[sm2], &sm.bar[sm2], err,
                          kk, sm.stage[0], sm.stage[0] + S * 9 * W8);
            issued = kk + 1;
        }
        if (is_main && has_col && q > y0) {
            const float* pm = sm.psi[(q - 2) & 3];
            const float* p0 = sm.psi[(q - 1) & 3];
            const float* pp = sm.psi[q & 3];
            const int c1 = col + 1;
            float pn[9];
            pn[0] = p0[c1];
            pn[1] = p0[c1 + 1];
            pn[2] = pp[c1];
            pn[3] = p0[c1 - 1];
            pn[4] = pm[c1];
            pn[5] = pp[c1 + 1];
            pn[6] = pp[c1 - 1];
            pn[7] = pm[c1 - 1];
            pn[8] = pm[c1 + 1];
            pp_collide(prv, rho_prv, pn[0], pn, P);
            float* o = fout + (long long)(q - 1) * nx + x0 + col;
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i * P.pitch] = prv[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) prv[i] = cur[i];
        rho_prv = rho_cur;
        sm2 = sm1;
        sm1 = s0;
        s0 = next_stage(s0, S);
        if (s0 == 0) par ^= 1u;
    }
    if (failed && producer) {
        atomicExch(err, 1);
        drain_stages<S>(sm.bar, issued);
    }
}

template <int TX, int S>
__global__ void __launch_bounds__(TX + 32, LBM_PP_MINB) pp_step_tma(const float* __restrict__ fin, float* __restrict__ fout,
                                                       const StepParams<float> P, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PPTmaSmem<TX, S>& sm = *reinterpret_cast<PPTmaSmem<TX, S>*>(smem_raw);
    const int x0 = blockIdx.x * TX;
    const int y0 = blockIdx.y * P.rows;
    pp_strip_tma<TX, S>(fin, fout, P, x0, min(TX, P.nx - x0), y0, min(y0 + P.rows, P.ny), sm, err);
}

template <int TX, int S>
struct FETmaSmem {
    static constexpr int W8 = TX + 8;
    float stage[S][9 * W8];
    float rho[8][TX + 4];
    float mu[4][TX + 2];
    uint64_t bar[S];
};

// Free-energy step (Eqs. 1, 6, 20, 21, 24, 29), TMA-fed, one barrier per row:
// iteration q computes rho of row q and mu of row q-2 (whose rho rows q-3..q-1 were
// written in earlier iterations), then, after the barrier, collides row q-3.
template <int TX, int S>
__global__ void __launch_bounds__(TX + 32, LBM_FE_MINB) fe_step_tma(const float* __restrict__ fin, float* __restrict__ fout,
                                                       const StepParams<float> P, int* __restrict__ err) {
    constexpr int W8 = TX + 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FETmaSmem<TX, S>& sm = *reinterpret_cast<FETmaSmem<TX, S>*>(smem_raw);
    const int nx = P.nx, ny = P.ny;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int y0 = blockIdx.y * P.rows;
    const int y1 = min(y0 + P.rows, ny);
    const int t = threadIdx.x;
    const bool is_main = t < TX;
    const bool producer = t == TX;
    bool has_col, has_mu;
    int col;
    if (is_main) {
        has_col = t < w;
        has_mu = has_col;
        col = t;
    } else {
        const int lane = t - TX;
        has_col = lane < 4;
        has_mu = lane == 1 || lane == 2;
        col = lane == 0 ? -2 : lane == 1 ? -1 : lane == 2 ? w : w + 1;
    }
    const int sc = col + 4, rc = col + 2, mc = col + 1;
    const int rbase = y0 - 3;
    const int nsrc = y1 + 2 - rbase + 1;  // source rows y0-3 .. y1+2 (rho rows y0-2 .. y1+1)
    if (producer) {
        for (int s = 0; s < S; ++s) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (producer) {
        for (int k = 0; k < S && k < nsrc; ++k)
            issue_row<W8>(fin, P.pitch, nx, wrap_once(rbase + k, ny), x0, w, sm.stage[k], &sm.bar[k], err, k,
                          sm.stage[0], sm.stage[0] + S * 9 * W8);
        issued = min(S, nsrc);
    }
    float p3[9], p2[9], p1[9], cur[9];  // pulled populations of rows q-3, q-2, q-1, q
    // wait for fills 0 and 1 (rows y0-3, y0-2), read by the first iteration besides the one
    // it waits for (see pp_step_tma)
    bool failed = __syncthreads_or(!(mbar_wait_bounded(&sm.bar[0], 0) && mbar_wait_bounded(&sm.bar[1], 0)));
    int sm2 = 0, sm1 = 1, s0 = 2 % S;
    uint32_t par = 0;
#pragma unroll(kFEUnroll)
    for (int q = y0 - 2; q <= y1 + 2 && !failed; ++q) {
        const int k = q + 1 - rbase;
        const bool load = q <= y1 + 1;  // rho rows run to y1+1; the last iteration only finishes mu and collides
        bool ok = true;
        if (load) {
            ok = mbar_wait_bounded(&sm.bar[s0], par);
            if (ok && has_col) {
                pull_smem<W8>(sm.stage[sm2], sm.stage[sm1], sm.stage[s0], sc, cur);
                sm.rho[q & 7][rc] = sum9(cur);
            }
        }
        if (has_mu && q >= y0 + 1) {
            // mu of row q-2 from rho rows q-3, q-2, q-1 (written before the previous barrier)
            const float* rm = sm.rho[(q - 3) & 7];
            const float* r0 = sm.rho[(q - 2) & 7];
            const float* rp = sm.rho[(q - 1) & 7];
            float rn[9];
            rn[1] = r0[rc + 1];
            rn[2] = rp[rc];
            rn[3] = r0[rc - 1];
            rn[4] = rm[rc];
            rn[5] = rp[rc + 1];
            rn[6] = rp[rc - 1];
            rn[7] = rm[rc - 1];
            rn[8] = rm[rc + 1];
            sm.mu[(q - 2) & 3][mc] = fe_mu(r0[rc], rn, P);
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (producer && load && k - 2 + S < nsrc) {
            fence_proxy_async_smem();
            const int kk = k - 2 + S;
            issue_row<W8>(fin, P.pitch, nx, wrap_once(rbase + kk, ny), x0, w, sm.stage[sm2], &sm.bar[sm2], err,
                          kk, sm.stage[0], sm.stage[0] + S * 9 * W8);
            issued = kk + 1;
        }
        if (is_main && has_col && q >= y0 + 3) {
            // collide row c = q - 3: mu rows c-1..c+1 = q-4..q-2, rho rows q-4..q-2
            const float* mm = sm.mu[(q - 4) & 3];
            const float* m0 = sm.mu[(q - 3) & 3];
            const float* mp = sm.mu[(q - 2) & 3];
            const float* rm = sm.rho[(q - 4) & 7];
            const float* r0 = sm.rho[(q - 3) & 7];
            const float* rp = sm.rho[(q - 2) & 7];
            float mn[9], rn[9];
            mn[1] = m0[mc + 1]; mn[2] = mp[mc]; mn[3] = m0[mc - 1]; mn[4] = mm[mc];
            mn[5] = mp[mc + 1]; mn[6] = mp[mc - 1]; mn[7] = mm[mc - 1]; mn[8] = mm[mc + 1];
            rn[1] = r0[rc + 1]; rn[2] = rp[rc]; rn[3] = r0[rc - 1]; rn[4] = rm[rc];
            rn[5] = rp[rc + 1]; rn[6] = rp[rc - 1]; rn[7] = rm[rc - 1]; rn[8] = rm[rc + 1];
            fe_collide(p3, r0[rc], mn, rn, P);
            float* o = fout + (long long)(q - 3) * nx + x0 + col;
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i * P.pitch] = p3[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            p3[i] = p2[i];
            p2[i] = p1[i];
            p1[i] = cur[i];
        }
        if (load) {
            sm2 = sm1;
            sm1 = s0;
            s0 = next_stage(s0, S);
            if (s0 == 0) par ^= 1u;
        }
    }
    if (failed && producer) {
        atomicExch(err, 1);
        drain_stages<S>(sm.bar, issued);
    }
}

}  // namespace lbmk
