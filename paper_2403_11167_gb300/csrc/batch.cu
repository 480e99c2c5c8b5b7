// batch.cu -- batched calibration sweep: many independent pseudopotential lattices at once.
//
// The calibration runs the pseudopotential model needs (Sec. 3: sigma^Li, kappa^P and
// kappa^Li tuned against coexistence densities, interface width and surface tension; Secs.
// 5.1-5.2: its parameters are set from preliminary runs) are many small, independent
// lattices of uneven sizes and step counts.  Run one at a time, the small ones are
// launch-latency bound and the large ones leave most SMs idle.  Here they run together:
//
//   resident lattices  -- populations (9 N floats, the rest extensions N int16) + psi and
//                         rho (2 N floats) fit in one CTA's shared
//                         memory: one CTA per lattice runs every step of that lattice in
//                         shared memory, in one persistent launch (no HBM traffic per step);
//   tiled lattices     -- the rest: a work table of (lattice, strip) items; one launch per
//                         time step runs the two-cells-per-lane TMA strip of the context
//                         path (pp_pair_strip) over every active lattice,
//                         replayed as captured 64-step CUDA graphs on a second stream,
//                         concurrently with the resident launch.
//
// An autotuner picks the resident block size and the strip height by timing short trials
// (cached per shape class for the process), and orders work longest-first.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"
#include "ring.cuh"
#include "step_pair.cuh"
#include "rest_host.h"

namespace {

thread_local char g_batch_msg[256] = "";
int bfail(cudaError_t e, const char* what) {
    snprintf(g_batch_msg, sizeof(g_batch_msg), "%s: %s", what, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}
#define BCK(call)                                             \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bfail(e_, #call);       \
    } while (0)

constexpr int kBPWarps = 4;
constexpr int kBPStages = 6;
static_assert(kBPStages >= 4, "the pseudopotential strip ring needs at least 4 stages");
using BPSmem = lbmk::WarpStripSmem<kBPWarps, kBPStages, 60>;
constexpr int kBPTX = BPSmem::TX;  // widest pair strip (240 columns)
constexpr int kChunk = 64;       // steps per captured graph
constexpr size_t kResidentSmemMax = 200 * 1024;

struct BatchLattice {
    lbmk::StepParams<float> P;  // physics and geometry (nx, ny, rows, pitch)
    float* buf[2];              // ping-pong stored populations
    float* scratch;             // 2 N floats: rho and psi for observables / density staging
    double RT, a, b4;           // FP64 EOS constants for the observables (pressure jump)
    int nsteps;
    int geometry;
    int resident;
    int pad_;
};

struct BatchItem {
    int lat, x0, w, y0, y1;
};

size_t a256(size_t n) { return (n + 255) & ~size_t(255); }

// Shared memory of a resident lattice of N cells: 9 population planes, psi and rho (FP32), and
// the int16 extensions of the rest population.
size_t resident_bytes(size_t N) { return 11 * N * sizeof(float) + ((2 * N + 15) & ~size_t(15)); }

// One population buffer of a lattice: 9 FP32 planes plus the int16 rest plane (plane 9).
size_t buffer_bytes(long long pitch) { return a256(10 * (size_t)pitch * 4); }

}  // namespace

namespace lbmk {

// ------------------------------------------------------------------------------------
// Resident lattice: all steps in shared memory.  Stored layout S_i(x) (post-collision at
// the source cell, as in the tiled kernels).  Per step: (A) rho and psi of every cell into
// shared arrays; barrier; (B) collision of every cell from the pulled populations and the
// psi neighbours, f* written to the lattice's spare global buffer (L2-resident at these
// sizes); barrier; (C) each thread copies its own cells' f* back into S; barrier.  Nothing
// is held in registers across a barrier, so the block can be 1024 threads wide.
__global__ void __launch_bounds__(1024, 1)
    pp_resident_kernel(const BatchLattice* __restrict__ lats, const int* __restrict__ ids, int step_limit) {
    extern __shared__ __align__(16) float rsm[];
    const BatchLattice& L = lats[ids[blockIdx.x]];
    const StepParams<float> P = L.P;
    const int nx = P.nx, ny = P.ny, N = nx * ny;
    const long long pitch = P.pitch;
    float* S = rsm;            // 9 planes of N
    float* psi = rsm + 9 * N;  // N
    float* rho = psi + N;      // N
    short* Q = reinterpret_cast<short*>(rho + N);  // N: rest-population extensions
    const float* g0 = L.buf[0];
    float* G = L.buf[1];
    for (int idx = threadIdx.x; idx < 9 * N; idx += blockDim.x) {
        const int i = idx / N, c = idx - i * N;
        S[idx] = g0[i * pitch + c];
    }
    for (int c = threadIdx.x; c < N; c += blockDim.x) Q[c] = rest_lo_plane(g0, pitch)[c];
    __syncthreads();
    const int nsteps = step_limit >= 0 ? min(step_limit, L.nsteps) : L.nsteps;
    for (int s = 0; s < nsteps; ++s) {
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            float v[9];
            pull_cell_shared(S, N, c % nx, c / nx, nx, ny, v);
            const float r = sum9(v);
            rho[c] = r;
            psi[c] = pseudo_psi(r, P);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const int x = c % nx, y = c / nx;
            float v[9], pn[9];
            pull_cell_shared(S, N, x, y, nx, ny, v);
            gather8(psi, x, y, nx, ny, pn);
            int q = Q[c];  // compensated rest population (only this thread touches Q[c])
            pp_collide_comp(v, q, rho[c], pn[0], pn, P);
            Q[c] = (short)q;
#pragma unroll
            for (int i = 0; i < 9; ++i) G[i * pitch + c] = v[i];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
#pragma unroll
            for (int i = 0; i < 9; ++i) S[i * N + c] = G[i * pitch + c];
        }
        __syncthreads();
    }
    // final state to the buffer the tiled convention uses after nsteps steps
    float* g = L.buf[nsteps & 1];
    for (int idx = threadIdx.x; idx < 9 * N; idx += blockDim.x) {
        const int i = idx / N, c = idx - i * N;
        g[i * pitch + c] = S[idx];
    }
    for (int c = threadIdx.x; c < N; c += blockDim.x) rest_lo_plane(g, pitch)[c] = Q[c];
}

// Tiled lattices, two cells per lane: one strip of one lattice per CTA, one step per launch.
template <int NW, int S>
__global__ void __launch_bounds__((NW + 1) * 32, 1)
    pp_batch_pair(const BatchLattice* __restrict__ lats, const BatchItem* __restrict__ items,
                  const int* __restrict__ step_base, int k, int* __restrict__ err) {
    using Smem = WarpStripSmem<NW, S, 60>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const BatchItem it = items[blockIdx.x];
    const BatchLattice& L = lats[it.lat];
    const int step = *step_base + k;
    if (step >= L.nsteps) return;
    const StepParams<float> P = L.P;
    pp_pair_strip<NW, S>(L.buf[step & 1], L.buf[(step + 1) & 1], P, it.x0, it.w, it.y0, it.y1, sm, err);
}

__global__ void advance_step(int* step_base, int by) { *step_base += by; }

// Observables of every lattice (one CTA per lattice): rho and psi of the final state into
// the lattice scratch, then u (Eq. 6b with the Shan-Chen force), mass, u_max, probes,
// tangent width, pressure jump and equimolar radius -- the definitions of lbm_observables.
__global__ void batch_obs_kernel(const BatchLattice* __restrict__ lats, double* __restrict__ out) {
    const BatchLattice& L = lats[blockIdx.x];
    const StepParams<float> P = L.P;
    const int nx = P.nx, ny = P.ny, N = nx * ny;
    const float* f = L.buf[L.nsteps & 1];
    float* rho = L.scratch;
    float* ps = L.scratch + N;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        float v[9];
        pull_cell(f, P.pitch, c % nx, c / nx, nx, ny, v);
        const float r = sum9_rest(v, rest_lo_plane(f, P.pitch)[c], P);
        rho[c] = r;
        ps[c] = pseudo_psi(r, P);
    }
    __syncthreads();
    double m = 0.0, u2 = 0.0, bad = 0.0, liq = 0.0, vap = 0.0, dmax = 0.0;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const int x = c % nx, y = c / nx;
        float v[9], an[9];
        pull_cell(f, P.pitch, x, y, nx, ny, v);
        gather8(ps, x, y, nx, ny, an);
        const float w1 = 1.0f / 3.0f, w2 = 1.0f / 12.0f;
        const float gx = (an[1] - an[3]) * w1 + ((an[5] - an[7]) + (an[8] - an[6])) * w2;
        const float gy = (an[2] - an[4]) * w1 + ((an[5] - an[7]) + (an[6] - an[8])) * w2;
        const float r = rho[c];
        const float Fx = an[0] * gx + P.fx, Fy = an[0] * gy + P.fy;
        const float jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
        const float jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
        const double ux = (jx + 0.5f * Fx) / r, uy = (jy + 0.5f * Fy) / r;
        const double q = ux * ux + uy * uy;
        if (!(r > 0.0f) || !isfinite(r) || !isfinite(q)) bad += 1.0;
        m += r;
        u2 = fmax(u2, isfinite(q) ? q : 0.0);
        if (L.geometry == 0) {
            if (x == nx / 2 - 1 || x == nx / 2) liq += r;
            if (x == 0 || x == nx - 1) vap += r;
        } else {
            const int cx0 = nx / 2 - 2, cy0 = ny / 2 - 2;
            if (x >= cx0 && x < cx0 + 4 && y >= cy0 && y < cy0 + 4) liq += r;
            if ((x < 4 || x >= nx - 4) && (y < 4 || y >= ny - 4)) vap += r;
        }
        const int prow = L.geometry == 0 ? 0 : ny / 2;
        if (y == prow) {
            const double a = rho[y * nx + (x == nx - 1 ? 0 : x + 1)], b = rho[y * nx + (x == 0 ? nx - 1 : x - 1)];
            dmax = fmax(dmax, fabs(a - b) * 0.5);
        }
    }
    __shared__ double red[6][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_down_sync(0xffffffffu, m, o);
        liq += __shfl_down_sync(0xffffffffu, liq, o);
        vap += __shfl_down_sync(0xffffffffu, vap, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
        u2 = fmax(u2, __shfl_down_sync(0xffffffffu, u2, o));
        dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    }
    if (lane == 0) {
        red[0][wid] = m;
        red[1][wid] = liq;
        red[2][wid] = vap;
        red[3][wid] = bad;
        red[4][wid] = u2;
        red[5][wid] = dmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w) {
            for (int j = 0; j < 4; ++j) s[j] += red[j][w];
            s[4] = fmax(s[4], red[4][w]);
            s[5] = fmax(s[5], red[5][w]);
        }
        const double nl = L.geometry == 0 ? 2.0 * ny : 16.0, nv = L.geometry == 0 ? 2.0 * ny : 64.0;
        const double rl = s[1] / nl, rv = s[2] / nv;
        auto pcs = [&](double r) {
            const double e = L.b4 * r, om = 1.0 - e;
            return r * L.RT * (1.0 + e + e * e - e * e * e) / (om * om * om) - L.a * r * r;
        };
        double* o = out + 8 * blockIdx.x;
        o[0] = rl;
        o[1] = rv;
        o[2] = (rl - rv) / s[5];
        o[3] = pcs(rl) - pcs(rv);
        o[4] = sqrt(s[4]);
        o[5] = s[0];
        o[6] = L.geometry == 1 ? sqrt(fmax(s[0] - rv * (double)N, 0.0) / (3.14159265358979323846 * (rl - rv))) : nan("");
        o[7] = s[3];
    }
}

}  // namespace lbmk

// --------------------------------------------------------------------------------------
// Host side

struct lbm_batch {
    int n;
    std::vector<lbm_batch_lattice> spec;
    std::vector<BatchLattice> lat;       // host copy of the device table
    std::vector<int> resident_ids;       // sorted longest-first
    std::vector<BatchItem> items;        // sorted by lattice nsteps, longest first
    int max_tiled_steps;
    int resident_threads;
    size_t resident_smem;
    int strip_rows;
    char* pool;
    BatchLattice* d_lat;
    BatchItem* d_items;
    int* d_ids;
    int* d_step;
    int* d_err;
    double* d_obs;
    std::vector<double> h_obs;
    cudaStream_t s_res, s_tile;
    cudaEvent_t ev_fork, ev_join;
    cudaGraphExec_t chunk;
    bool ran;
    std::vector<std::vector<double>> rho0;  // kept for re-initialisation after autotuning trials
};

namespace {

struct TuneKey {
    int kind, a, b;
    bool operator<(const TuneKey& o) const {
        return kind != o.kind ? kind < o.kind : (a != o.a ? a < o.a : b < o.b);
    }
};
std::map<TuneKey, int> g_tune_cache;
std::mutex g_tune_mu;

int batch_init_state(lbm_batch* b) {
    BCK(cudaStreamSynchronize(b->s_res));
    BCK(cudaStreamSynchronize(b->s_tile));
    for (int i = 0; i < b->n; ++i) {
        const BatchLattice& L = b->lat[i];
        const size_t n = (size_t)L.P.nx * L.P.ny;
        BCK(cudaMemcpyAsync(L.scratch, b->rho0[i].data(), n * sizeof(double), cudaMemcpyHostToDevice, b->s_tile));
        lbmk::init_kernel<float, double><<<std::min<long long>(304, (n + 255) / 256), 256, 0, b->s_tile>>>(
            reinterpret_cast<const double*>(L.scratch), L.buf[0], LBM_PSEUDOPOTENTIAL, L.P.nx, L.P.ny, L.P.pitch,
            L.P.rest_inv);
    }
    BCK(cudaGetLastError());
    const int zero = 0;
    BCK(cudaMemcpyAsync(b->d_step, &zero, sizeof(int), cudaMemcpyHostToDevice, b->s_tile));
    BCK(cudaMemsetAsync(b->d_err, 0, sizeof(int) * 16, b->s_tile));
    BCK(cudaStreamSynchronize(b->s_tile));
    return LBM_OK;
}

int launch_resident(lbm_batch* b, int step_limit, cudaStream_t s) {
    if (b->resident_ids.empty()) return LBM_OK;
    const int nb = (int)b->resident_ids.size();
    lbmk::pp_resident_kernel<<<nb, b->resident_threads, b->resident_smem, s>>>(b->d_lat, b->d_ids, step_limit);
    BCK(cudaGetLastError());
    return LBM_OK;
}

int launch_tiled_step(lbm_batch* b, int k, cudaStream_t s) {
    if (b->items.empty()) return LBM_OK;
    lbmk::pp_batch_pair<kBPWarps, kBPStages><<<(unsigned)b->items.size(), (kBPWarps + 1) * 32, sizeof(BPSmem), s>>>(
        b->d_lat, b->d_items, b->d_step, k, b->d_err);
    BCK(cudaGetLastError());
    return LBM_OK;
}

// Strip items of every tiled lattice for a given strip height, longest lattice first.
void build_items(lbm_batch* b, int rows) {
    b->items.clear();
    std::vector<int> order;
    for (int i = 0; i < b->n; ++i)
        if (!b->lat[i].resident) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->lat[x].nsteps > b->lat[y].nsteps; });
    for (int i : order) {
        const int nx = b->lat[i].P.nx, ny = b->lat[i].P.ny;
        const int r = std::min(rows, ny);
        b->lat[i].P.rows = r;
        // pair strips: nx split into equal widths (multiples of 4, at most kBPTX columns)
        const int gx = (nx + kBPTX - 1) / kBPTX;
        const int wb = lbmk::warp_strip_width(nx, gx);
        for (int y0 = 0; y0 < ny; y0 += r)
            for (int x0 = 0; x0 < nx; x0 += wb)
                b->items.push_back(BatchItem{i, x0, std::min(wb, nx - x0), y0, std::min(y0 + r, ny)});
    }
}

int upload_tables(lbm_batch* b) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    BCK(cudaMemcpy(b->d_lat, b->lat.data(), sizeof(BatchLattice) * b->n, cudaMemcpyHostToDevice));
    if (!b->items.empty()) {
        BCK(cudaMalloc(&b->d_items, sizeof(BatchItem) * b->items.size()));
        BCK(cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchItem) * b->items.size(), cudaMemcpyHostToDevice));
    }
    return LBM_OK;
}

double time_ms(cudaStream_t s, const std::function<int()>& fn, int* rc) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    *rc = fn();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// Autotuner: resident block size (cells per thread 1/2/4) and tiled strip height.  Each
// candidate runs a short trial on the real initial state (restored afterwards); the choice is
// cached per shape class for the lifetime of the process.
int autotune(lbm_batch* b) {
    int max_res_n = 0;
    for (int id : b->resident_ids) max_res_n = std::max(max_res_n, b->lat[id].P.nx * b->lat[id].P.ny);
    if (!b->resident_ids.empty()) {
        const TuneKey key{0, max_res_n, (int)b->resident_ids.size()};
        int choice = -1;
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) choice = it->second;
        }
        if (choice < 0) {
            double best = 1e30;
            for (int threads : {256, 512, 1024}) {
                if (threads > 32 * ((max_res_n + 31) / 32) && threads > 256) continue;
                b->resident_threads = threads;
                int rc = LBM_OK;
                const double ms = time_ms(b->s_res, [&] { return launch_resident(b, 16, b->s_res); }, &rc);
                if (rc) return rc;
                if (ms < best) {
                    best = ms;
                    choice = threads;
                }
            }
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[key] = choice;
        }
        b->resident_threads = choice;
    }
    if (!b->items.empty() || b->max_tiled_steps > 0) {
        long long cells = 0;
        for (int i = 0; i < b->n; ++i)
            if (!b->lat[i].resident) cells += (long long)b->lat[i].P.nx * b->lat[i].P.ny;
        const TuneKey key{1, (int)std::min<long long>(cells >> 10, 1 << 30), b->n};
        int choice = -1;
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) choice = it->second;
        }
        if (const char* e = std::getenv("LBM_BATCH_ROWS")) choice = std::max(1, std::atoi(e));  // tuning experiments
        if (choice < 0) {
            // two passes in opposite orders, 16 steps per trial, best time per candidate:
            // a single short pass in one order favoured whichever candidate ran last
            const int cand[3] = {16, 32, 64};
            double best_ms[3] = {1e30, 1e30, 1e30};
            for (int pass = 0; pass < 2; ++pass)
                for (int j = 0; j < 3; ++j) {
                    const int c = pass == 0 ? j : 2 - j;
                    build_items(b, cand[c]);
                    int rc = upload_tables(b);
                    if (rc) return rc;
                    const double ms = time_ms(b->s_tile, [&] {
                        for (int k = 0; k < 16; ++k) {
                            int r = launch_tiled_step(b, k, b->s_tile);
                            if (r) return r;
                        }
                        return (int)LBM_OK;
                    }, &rc);
                    if (rc) return rc;
                    best_ms[c] = std::min(best_ms[c], ms);
                }
            // the trial sees every lattice active; later, only the longest lattices remain and
            // more (shorter) strips keep the GPU busy: take the shortest strips within 5% of the
            // best trial time
            double best = 1e30;
            for (int c = 0; c < 3; ++c) best = std::min(best, best_ms[c]);
            for (int c = 0; c < 3; ++c)
                if (best_ms[c] <= 1.05 * best) {
                    choice = cand[c];
                    break;
                }
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[key] = choice;
        }
        b->strip_rows = choice;
        build_items(b, choice);
        int rc = upload_tables(b);
        if (rc) return rc;
    }
    return batch_init_state(b);  // trials advanced the state: start again from f^eq(rho0)
}

}  // namespace

extern "C" const char* lbm_batch_last_error(void) { return g_batch_msg; }

extern "C" void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->s_res);
    cudaStreamSynchronize(b->s_tile);
    if (b->chunk) cudaGraphExecDestroy(b->chunk);
    if (b->d_items) cudaFree(b->d_items);
    if (b->pool) cudaFree(b->pool);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->s_res) cudaStreamDestroy(b->s_res);
    if (b->s_tile) cudaStreamDestroy(b->s_tile);
    delete b;
}

extern "C" int lbm_batch_create(int n, const lbm_batch_lattice* specs, const double* const* rho0, lbm_batch** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !specs || !rho0) return LBM_ERR_ARG;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_ARG;
    b->n = n;
    b->spec.assign(specs, specs + n);
    b->lat.resize(n);
    b->rho0.resize(n);
    // resolve parameters and validate on the host first
    size_t pool_bytes = 0;
    std::vector<size_t> offs(n);
    b->max_tiled_steps = 0;
    std::vector<lbm_params> in_p(n), res_p(n);
    std::vector<lbm_thermo> res_t(n);
    std::vector<int> res_rc(n);
    for (int i = 0; i < n; ++i) in_p[i] = specs[i].params;
    lbm_resolve_params_many(n, in_p.data(), res_p.data(), res_t.data(), res_rc.data());
    for (int i = 0; i < n; ++i) {
        const lbm_batch_lattice& s = specs[i];
        if (s.nx < 1 || s.ny < 1 || s.nsteps < 0 || s.nsteps > (1LL << 30) || (s.geometry != 0 && s.geometry != 1) ||
            !rho0[i]) {
            delete b;
            return LBM_ERR_ARG;
        }
        if (s.params.model != LBM_PSEUDOPOTENTIAL || s.params.precision != LBM_F32) {
            delete b;
            return LBM_ERR_UNSUPPORTED;
        }
        const lbm_params& rp = res_p[i];
        const lbm_thermo& th = res_t[i];
        int rc = res_rc[i];
        if (rc) {
            delete b;
            return rc;
        }
        const size_t N = (size_t)s.nx * s.ny;
        for (size_t k = 0; k < N; ++k)
            if (!(rho0[i][k] > 0.0 && rho0[i][k] < 4.0 / rp.b)) {
                delete b;
                return LBM_ERR_ARG;
            }
        b->rho0[i].assign(rho0[i], rho0[i] + N);
        BatchLattice& L = b->lat[i];
        std::memset(&L, 0, sizeof(L));
        lbmk::StepParams<float>& P = L.P;
        P.nx = s.nx;
        P.ny = s.ny;
        P.pitch = ((long long)N + 63) / 64 * 64;
        P.rows = std::min(32, s.ny);
        const double G = -1.0, C1 = 5.0 / 6.0 * (rp.kappa_P - 1.0), C2 = 0.5 * (1.0 - rp.kappa_P);
        P.RT = (float)(rp.R * th.T);
        P.a = (float)rp.a;
        P.b4 = (float)(0.25 * rp.b);
        P.kA = (float)(G * (C1 - C2 / 3.0));
        P.kB = (float)(G * (C2 + 0.5 * rp.kappa_Li));
        P.li = (float)(12.0 * rp.kappa_P * rp.sigma_Li);
        P.s_e = (float)(1.0 / rp.tau_e);
        P.s_z = (float)(1.0 / rp.tau_zeta);
        P.s_q = (float)(1.0 / rp.tau_q);
        P.s_nu = (float)(1.0 / rp.tau_nu);
        P.fx = (float)rp.body_fx;
        P.fy = (float)rp.body_fy;
        P.rest_unit = (float)lbm_host::rest_unit(rp.b);
        P.rest_inv = (float)lbm_host::rest_inv(rp.b);
        P.h_e = (float)(1.0 - 0.5 / rp.tau_e);
        P.h_z = (float)(1.0 - 0.5 / rp.tau_zeta);
        P.h_q = (float)(1.0 - 0.5 / rp.tau_q);
        P.h_nu = (float)(1.0 - 0.5 / rp.tau_nu);
        P.h6_e = (float)(6.0 * (1.0 - 0.5 / rp.tau_e));
        P.h6_z = (float)(6.0 * (1.0 - 0.5 / rp.tau_zeta));
        L.RT = rp.R * th.T;
        L.a = rp.a;
        L.b4 = 0.25 * rp.b;
        L.nsteps = (int)s.nsteps;
        L.geometry = s.geometry;
        L.resident = resident_bytes(N) <= kResidentSmemMax;
        if (!L.resident && (s.nx % 4 != 0 || s.nx < 8 || s.ny < 4)) {
            delete b;
            return LBM_ERR_UNSUPPORTED;  // tiled lattices use the TMA strip kernels
        }
        if (!L.resident) b->max_tiled_steps = std::max(b->max_tiled_steps, L.nsteps);
        offs[i] = pool_bytes;
        pool_bytes += 2 * buffer_bytes(P.pitch) + a256(2 * N * 4 + 8 * N);
    }
    const size_t tail = pool_bytes;
    pool_bytes += a256(sizeof(BatchLattice) * n) + a256(sizeof(int) * n) + 256 + 256 + a256(8 * sizeof(double) * n);
    cudaError_t e = cudaMalloc(&b->pool, pool_bytes);
    if (e != cudaSuccess) {
        delete b;
        return bfail(e, "cudaMalloc(batch pool)");
    }
    size_t smax = 0;
    for (int i = 0; i < n; ++i) {
        BatchLattice& L = b->lat[i];
        const size_t fb = buffer_bytes(L.P.pitch);
        L.buf[0] = reinterpret_cast<float*>(b->pool + offs[i]);
        L.buf[1] = reinterpret_cast<float*>(b->pool + offs[i] + fb);
        L.scratch = reinterpret_cast<float*>(b->pool + offs[i] + 2 * fb);
        if (L.resident) {
            b->resident_ids.push_back(i);
            smax = std::max(smax, resident_bytes((size_t)L.P.nx * L.P.ny));
        }
    }
    std::stable_sort(b->resident_ids.begin(), b->resident_ids.end(), [&](int x, int y) {
        return (long long)b->lat[x].nsteps * b->lat[x].P.nx * b->lat[x].P.ny >
               (long long)b->lat[y].nsteps * b->lat[y].P.nx * b->lat[y].P.ny;
    });
    b->resident_smem = smax;
    b->d_lat = reinterpret_cast<BatchLattice*>(b->pool + tail);
    b->d_ids = reinterpret_cast<int*>(b->pool + tail + a256(sizeof(BatchLattice) * n));
    b->d_step = reinterpret_cast<int*>(reinterpret_cast<char*>(b->d_ids) + a256(sizeof(int) * n));
    b->d_err = reinterpret_cast<int*>(reinterpret_cast<char*>(b->d_step) + 256);
    b->d_obs = reinterpret_cast<double*>(reinterpret_cast<char*>(b->d_err) + 256);
    b->h_obs.assign(8 * (size_t)n, 0.0);
    int rc = LBM_OK;
    auto fail = [&](int code) {
        lbm_batch_destroy(b);
        return code;
    };
    if ((e = cudaStreamCreateWithFlags(&b->s_res, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->s_tile, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return fail(bfail(e, "stream/event create"));
    if (!b->resident_ids.empty()) {
        if ((e = cudaMemcpy(b->d_ids, b->resident_ids.data(), sizeof(int) * b->resident_ids.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(bfail(e, "cudaMemcpy(ids)"));
        if ((e = cudaFuncSetAttribute(lbmk::pp_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smax)) != cudaSuccess)
            return fail(bfail(e, "cudaFuncSetAttribute(resident smem)"));
    }
    if ((e = cudaFuncSetAttribute(lbmk::pp_batch_pair<kBPWarps, kBPStages>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BPSmem))) != cudaSuccess)
        return fail(bfail(e, "cudaFuncSetAttribute(batch strip smem)"));
    build_items(b, 32);
    if ((rc = upload_tables(b))) return fail(rc);
    if ((rc = batch_init_state(b))) return fail(rc);
    if ((rc = autotune(b))) return fail(rc);
    *out = b;
    return LBM_OK;
}

extern "C" int lbm_batch_run(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    if (b->ran) {
        int rc = batch_init_state(b);
        if (rc) return rc;
    }
    b->ran = true;
    // tiled lattices: replays of a captured chunk of 64 single-step launches + step advance
    if (!b->items.empty() && !b->chunk) {
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->s_tile, cudaStreamCaptureModeThreadLocal));
        int rc = LBM_OK;
        for (int k = 0; k < kChunk && rc == LBM_OK; ++k) rc = launch_tiled_step(b, k, b->s_tile);
        if (rc == LBM_OK) lbmk::advance_step<<<1, 1, 0, b->s_tile>>>(b->d_step, kChunk);
        cudaError_t e = cudaStreamEndCapture(b->s_tile, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return bfail(e, "cudaStreamEndCapture(batch)");
        e = cudaGraphInstantiate(&b->chunk, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(e, "cudaGraphInstantiate(batch)");
    }
    // resident lattices: one persistent launch, concurrent with the tiled replays
    int rc = launch_resident(b, -1, b->s_res);
    if (rc) return rc;
    for (int s = 0; s < b->max_tiled_steps; s += kChunk) BCK(cudaGraphLaunch(b->chunk, b->s_tile));
    BCK(cudaEventRecord(b->ev_join, b->s_res));
    BCK(cudaStreamWaitEvent(b->s_tile, b->ev_join, 0));
    return LBM_OK;
}

extern "C" int lbm_batch_observables(lbm_batch* b, lbm_obs* out) {
    if (!b || !out) return LBM_ERR_ARG;
    if (!b->ran) return LBM_ERR_STATE;
    lbmk::batch_obs_kernel<<<b->n, 1024, 0, b->s_tile>>>(b->d_lat, b->d_obs);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(b->h_obs.data(), b->d_obs, sizeof(double) * 8 * b->n, cudaMemcpyDeviceToHost, b->s_tile));
    int herr = 0;
    BCK(cudaMemcpyAsync(&herr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->s_tile));
    BCK(cudaStreamSynchronize(b->s_tile));
    for (int i = 0; i < b->n; ++i) {
        const double* h = &b->h_obs[8 * (size_t)i];
        lbm_obs& o = out[i];
        o.rho_l = h[0];
        o.rho_v = h[1];
        o.width = h[2];
        o.dp = h[3];
        o.u_max = h[4];
        o.mass = h[5];
        o.radius = h[6];
        o.step = b->ran ? b->lat[i].nsteps : 0;
        o.pad_ = 0;
        o.status = herr ? LBM_ERR_TIMEOUT : ((h[7] != 0.0 || !std::isfinite(h[5])) ? LBM_ERR_DIVERGED : LBM_OK);
    }
    return LBM_OK;
}

extern "C" int lbm_batch_populations(lbm_batch* b, int i, double* f) {
    if (!b || !f || i < 0 || i >= b->n) return LBM_ERR_ARG;
    if (!b->ran) return LBM_ERR_STATE;
    BCK(cudaStreamSynchronize(b->s_tile));
    BCK(cudaStreamSynchronize(b->s_res));
    const BatchLattice& L = b->lat[i];
    const int nx = L.P.nx, ny = L.P.ny;
    const size_t n = (size_t)nx * ny;
    std::vector<float> plane(n);
    const float* src = L.buf[b->ran ? (L.nsteps & 1) : 0];
    static const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, cys[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int q = 0; q < 9; ++q) {
        BCK(cudaMemcpy(plane.data(), src + q * L.P.pitch, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int xs = (x + cxs[q] + nx) % nx, ys = (y + cys[q] + ny) % ny;  // f_i(x + c_i) = S_i(x)
                f[q * n + (size_t)ys * nx + xs] = plane[(size_t)y * nx + x];
            }
    }
    std::vector<short> ext(n);  // the rest population's extension (plane 9)
    BCK(cudaMemcpy(ext.data(), reinterpret_cast<const char*>(src + 9 * L.P.pitch), n * sizeof(short),
                   cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < n; ++k) f[k] = lbm_host::rest_decode((float)f[k], ext[k], (double)L.P.rest_unit);
    return LBM_OK;
}

extern "C" int lbm_batch_info(const lbm_batch* b, int* n_resident, int* n_items, int* resident_threads,
                              int* strip_rows) {
    if (!b) return LBM_ERR_ARG;
    if (n_resident) *n_resident = (int)b->resident_ids.size();
    if (n_items) *n_items = (int)b->items.size();
    if (resident_threads) *resident_threads = b->resident_threads;
    if (strip_rows) *strip_rows = b->strip_rows;
    return LBM_OK;
}

extern "C" void* lbm_batch_stream(const lbm_batch* b) { return b ? static_cast<void*>(b->s_tile) : nullptr; }
