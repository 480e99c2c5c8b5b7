// ring.cuh -- the shared-memory row ring that feeds the FP32 strip kernels.
//
// One producer thread streams whole source rows of all nine population planes -- the strip's
// columns plus 4 halo columns on each side, so every pulled value and every halo column is
// present -- into an S-stage shared-memory ring with 1-D bulk copies (cp.async.bulk) that
// complete on a per-stage "full" mbarrier with an expected-transaction count.  Consumer warps
// arrive on a stage's "empty" mbarrier once they no longer read it; the producer refills a
// stage when every active consumer warp has released it.  There is no CTA-wide barrier per
// row: warps drift freely within the ring's depth.
//
// Copy rules (checked on the host): nx % 4 == 0, nx >= 8 (16-byte aligned rows for the bulk
// copies; the wrapped x halo is fetched as separate 16-byte pieces).  Every mbarrier wait is
// bounded: on timeout a warp records the error in *err and stops; the producer waits (bounded)
// for its copies in flight before the CTA exits; the host reports LBM_ERR_TIMEOUT.
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

// Per-thread asynchronous 4-byte copy global -> shared (cp.async, L1-allocating) and its
// group bookkeeping.  A thread sees its own copies in shared memory after cp.async.wait_group;
// no other thread reads them, so no barrier is needed.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NW, int S, int TXW>
struct WarpStripSmem {
    static constexpr int TX = NW * TXW;  // widest strip
    static constexpr int W8 = TX + 8;    // staged row: 4 halo columns each side
    float stage[S][9 * W8];
    uint64_t full[S];
    uint64_t empty[S];
    // rest-population extensions (two int16 per lane) of the last three pulled rows, each lane
    // its own word: copied asynchronously when a row is pulled and read by the same lane when
    // that row is collided one (pseudopotential) or two (free energy) rows later, so that no
    // register waits on the global load in between
    uint32_t qext[3][NW][32];
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

}  // namespace lbmk
