// lbm_api.cu -- C ABI of the single-lattice solver (contexts, stepping, observables).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"
#include "ring.cuh"
#include "step_pair.cuh"
#include "step_ext.cuh"
#include "step_iwb_pair.cuh"
#include "rest_host.h"
#include "thermo.h"

namespace {

thread_local char g_cuda_msg[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", what, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

constexpr int kTXf = 256;  // columns per CTA of the FP32 direct-load kernels
constexpr int kTXd = 64;   // columns per CTA, FP64
constexpr int kWallBandPP = 2;  // rows next to each wall that a periodic step gets wrong
constexpr int kWallBandFE = 3;
constexpr int kGraphSteps = 64;
constexpr int kRedBlocks = 304;  // observables partial-reduction blocks (2 x 152 SMs)
// FP32 strip kernels (two cells per lane in warp windows fed by the row ring).  A consumer warp
// reads staged rows q-2 .. q+1 (pseudopotential) or q-3 .. q+1 (free energy) while the producer
// fills the next row, so the rings need at least 4 and 5 stages; fewer would leave the
// producer waiting on a stage that is never released.
#ifndef LBM_PPP_STAGES
#define LBM_PPP_STAGES 6
#endif
#ifndef LBM_FEP_STAGES
#define LBM_FEP_STAGES 8
#endif
constexpr int kPPPWarps = 4;
constexpr int kPPPStages = LBM_PPP_STAGES;
static_assert(kPPPStages >= 4, "the pseudopotential strip ring needs at least 4 stages");
using PPPSmem = lbmk::WarpStripSmem<kPPPWarps, kPPPStages, 60>;
constexpr int kPPPTX = PPPSmem::TX;
#ifndef LBM_FEP_WARPS
#define LBM_FEP_WARPS 4
#endif
constexpr int kFEPWarps = LBM_FEP_WARPS;       // consumer warps per CTA
constexpr int kFEPStages = LBM_FEP_STAGES;
static_assert(kFEPStages >= 5, "the free-energy strip ring needs at least 5 stages");
using FEPSmem = lbmk::WarpStripSmem<kFEPWarps, kFEPStages, 60>;
// Strip kernel of the full free-energy model (A != 0, buoyancy): rows q-4 .. q+1 live, 8
// stages, 3 CTAs per SM (128 registers without spills, the velocity derivatives being taken
// before the collision's populations are pulled).
constexpr int kIWBWarps = 4;
constexpr int kIWBStages = 8;
using IWBSmem = lbmk::IwbStripSmem<kIWBWarps, kIWBStages>;
constexpr int kFEPTX = FEPSmem::TX;            // widest strip (240 columns)

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

struct lbm_ctx {
    lbm_params prm;
    lbm_thermo th;
    int nx, ny, prec;
    size_t esz;
    long long pitch;
    char* ws;
    bool own_ws;
    void* f[2];
    int cur;
    void* fields;        // 4 N reals: rho, aux, ux, uy
    double* partials;    // kRedBlocks x 3
    double* d_obs;       // 8 doubles
    int* d_err;          // device error word of the TMA kernels (bounded waits)
    bool use_tma;
    bool walls;          // no-slip walls on rows 0 and ny-1 (direct wall kernels)
    bool onesided;       // free-energy walls with the one-sided normal mu gradient (LBM_BC_WALL_ZOUHE_ONESIDED)
    void* wall;          // 14 nx reals: the wall rows' J_y and solve scratch (fe_wall_solve_kernel)
    double* dmass;       // per-warp stored mass of the driven FP32 strip steps (drive_mass_slots)
    bool drive;          // droplet-collision drive configured (lbm_set_drive)
    bool grav;           // gravity configured (lbm_set_gravity; free-energy model)
    double g, rho_g, y_ref;
    double drive_lo, drive_hi, drive_split;
    long long drive_t_on;
    double* h_pinned;    // 8 doubles, pinned
    cudaStream_t stream;
    bool own_stream;
    cudaGraphExec_t graph[2][2];  // [buffer parity][drive active]
    long long step;
    int status;
    bool ready;
    int rows;
    lbmk::StepParams<float> spf;
    lbmk::StepParams<double> spd;
};

extern "C" const char* lbm_last_cuda_error(void) { return g_cuda_msg; }

extern "C" const char* lbm_strerror(int s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_UNSUPPORTED: return "unsupported feature";
        case LBM_ERR_CUDA: return "CUDA runtime error";
        case LBM_ERR_DIVERGED: return "simulation diverged (NaN/Inf or rho <= 0)";
        case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
        case LBM_ERR_NOCONVERGE: return "host solve did not converge";
        case LBM_ERR_STATE: return "call out of order";
        case LBM_ERR_IO: return "checkpoint I/O error";
        default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------------
// Self-test of the bounded device wait (failure detection without a fault): one CTA
// initialises an mbarrier and waits, with a short poll limit, for its first phase.  With
// arrive = 0 nothing ever completes that phase, so every thread gives up, records the
// timeout and the CTA exits normally; with arrive = 1 thread 0 completes the phase first.
namespace {
__device__ int g_selftest_flag;

__global__ void bounded_wait_selftest_kernel(int arrive, uint32_t polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        lbmk::mbar_init(&bar, 1);
        lbmk::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile(
            "{\n\t.reg .b64 st;\n\t"
            "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(lbmk::smem_u32(&bar))
            : "memory");
    if (!lbmk::mbar_wait_polls(&bar, 0, polls)) atomicExch(&g_selftest_flag, 1);
}
}  // namespace

extern "C" int lbm_selftest_bounded_wait(int arrive, int polls) {
    if (polls < 1 || polls > (1 << 22) || (arrive != 0 && arrive != 1)) return LBM_ERR_ARG;
    const int zero = 0;
    CK(cudaMemcpyToSymbol(g_selftest_flag, &zero, sizeof(int)));
    bounded_wait_selftest_kernel<<<1, 64>>>(arrive, (uint32_t)polls);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    int flag = 0;
    CK(cudaMemcpyFromSymbol(&flag, g_selftest_flag, sizeof(int)));
    return flag ? LBM_ERR_TIMEOUT : LBM_OK;
}

extern "C" const char* lbm_build_info(void) {
    return "gb300 D2Q9 multiphase LBM; sm_103a; fused pull collide+stream; "
           "pseudopotential (MP-LBM) and improved well-balanced free energy";
}

extern "C" int lbm_params_default(int model, lbm_params* p) {
    if (!p || (model != LBM_PSEUDOPOTENTIAL && model != LBM_FREE_ENERGY)) return LBM_ERR_ARG;
    const double nan = std::nan("");
    p->model = model;
    p->precision = LBM_F32;
    p->a = 0.5;
    p->b = 4.0;
    p->R = 1.0;
    p->Tr = 0.8;
    p->tau_nu = 1.0;
    p->tau_e = p->tau_zeta = p->tau_q = p->tau_j = 0.0;
    p->kappa_P = p->kappa_Li = p->sigma_Li = nan;
    p->match_kappa = 0.0;
    p->kappa = nan;
    p->A = 0.0;
    p->body_fx = p->body_fy = 0.0;
    return LBM_OK;
}

extern "C" int lbm_resolve_params(const lbm_params* in, lbm_params* out, lbm_thermo* th) {
    if (!in || !out || !th) return LBM_ERR_ARG;
    lbm_params p = *in;
    if (p.model != LBM_PSEUDOPOTENTIAL && p.model != LBM_FREE_ENERGY) return LBM_ERR_ARG;
    if (p.precision != LBM_F32 && p.precision != LBM_F64) return LBM_ERR_ARG;
    if (!(p.a > 0 && p.b > 0 && p.R > 0 && p.Tr > 0 && p.Tr < 1)) return LBM_ERR_ARG;
    if (!(p.tau_nu > 0.5)) return LBM_ERR_ARG;
    if (!std::isfinite(p.A)) return LBM_ERR_ARG;
    if (p.A != 0.0 && p.model == LBM_PSEUDOPOTENTIAL) return LBM_ERR_UNSUPPORTED;  // A is a FE term (Eq. 20)
    if (!(p.tau_nu - 0.5 - p.A > 0)) return LBM_ERR_ARG;  // nu = c_s^2 (tau_nu - 1/2 - A) > 0 (Eq. 23)
    if (!std::isfinite(p.body_fx) || !std::isfinite(p.body_fy)) return LBM_ERR_ARG;
    const bool pp = p.model == LBM_PSEUDOPOTENTIAL;
    if (!(p.tau_j > 0)) p.tau_j = 1.0;
    if (pp) {
        if (!(p.tau_e > 0)) p.tau_e = p.tau_nu;
        if (!(p.tau_zeta > 0)) p.tau_zeta = p.tau_nu;
        if (!(p.tau_q > 0)) p.tau_q = 1.0 / 1.99;
    } else {
        if (!(p.tau_e > 0)) p.tau_e = 0.25 + 0.5 * p.tau_nu;
        if (!(p.tau_zeta > 0)) p.tau_zeta = 1.0;
        if (!(p.tau_q > 0)) p.tau_q = 1.0;
    }
    if (!(p.tau_e > 0.5 && p.tau_zeta > 0.5 && p.tau_q > 0.5 && p.tau_j > 0.5)) return LBM_ERR_ARG;
    if (std::isnan(p.kappa)) p.kappa = 0.5;
    lbm_host::CS eos{p.a, p.b, p.R};
    lbm_thermo t;
    std::memset(&t, 0, sizeof(t));
    int rc = lbm_host::critical(eos, &t.rho_c, &t.Tc, &t.p_c);
    if (rc) return rc;
    t.T = p.Tr * t.Tc;
    rc = lbm_host::maxwell(eos, t.T, &t.rho_v, &t.rho_l, &t.p0);
    if (rc) return rc;
    if (pp) {
        if (std::isnan(p.sigma_Li)) {
            rc = lbm_host::li_epsilon(eos, t.T, t.rho_v, t.rho_l, t.p0, &t.eps);
            if (rc) return rc;
            p.sigma_Li = t.eps / 16.0;  // eps = -16 G sigma_Li, G = -1
        } else {
            t.eps = 16.0 * p.sigma_Li;
        }
        if (p.match_kappa > 0) {
            double Wfe, gfe, W1, g1;
            rc = lbm_host::fe_theory(eos, t.T, t.rho_v, t.rho_l, t.p0, p.match_kappa, &Wfe, &gfe);
            if (rc) return rc;
            rc = lbm_host::pp_theory(eos, t.T, t.rho_v, t.rho_l, t.p0, t.eps, 1.0, 0.0, &W1, &g1);
            if (rc) return rc;
            p.kappa_P = (Wfe / W1) * (Wfe / W1);  // Eq. (S44): W ~ sqrt(kappa_P)
            double Wk, gk;
            rc = lbm_host::pp_theory(eos, t.T, t.rho_v, t.rho_l, t.p0, t.eps, p.kappa_P, 0.0, &Wk, &gk);
            if (rc) return rc;
            p.kappa_Li = p.kappa_P - gfe / (gk / p.kappa_P);  // Eq. (S46) linear in (kappa_P - kappa_Li)
        }
        if (std::isnan(p.kappa_P)) p.kappa_P = 1.0;
        if (std::isnan(p.kappa_Li)) p.kappa_Li = 0.0;
        rc = lbm_host::pp_theory(eos, t.T, t.rho_v, t.rho_l, t.p0, t.eps, p.kappa_P, p.kappa_Li, &t.width, &t.gamma);
        if (rc) return rc;
        if (!(p.kappa_P > 0)) return LBM_ERR_ARG;
        // psi must exist over the coexistence range (radicand of Eq. 11 non-negative)
        for (int k = 0; k <= 64; ++k) {
            const double r = t.rho_v + (t.rho_l - t.rho_v) * k / 64.0;
            if (!(r / 3.0 - eos.p(r, t.T) >= 0.0)) return LBM_ERR_ARG;
        }
    } else {
        if (std::isnan(p.kappa_P)) p.kappa_P = 1.0;
        if (std::isnan(p.kappa_Li)) p.kappa_Li = 0.0;
        if (std::isnan(p.sigma_Li)) p.sigma_Li = 0.0;
        if (!(p.kappa > 0)) return LBM_ERR_ARG;
        t.eps = 0.0;
        rc = lbm_host::fe_theory(eos, t.T, t.rho_v, t.rho_l, t.p0, p.kappa, &t.width, &t.gamma);
        if (rc) return rc;
    }
    *out = p;
    *th = t;
    return LBM_OK;
}

extern "C" int lbm_kelvin_2d(double a, double b, double R, double T, double gamma, double radius, double* rho_v,
                             double* rho_l) {
    if (!rho_v || !rho_l || !(a > 0 && b > 0 && R > 0 && T > 0)) return LBM_ERR_ARG;
    const lbm_host::CS eos{a, b, R};
    return lbm_host::kelvin_2d(eos, T, gamma, radius, rho_v, rho_l);
}

extern "C" int lbm_resolve_params_many(int n, const lbm_params* in, lbm_params* out, lbm_thermo* th, int* status) {
    if (n < 0 || (n > 0 && (!in || !out || !th || !status))) return LBM_ERR_ARG;
    // identical inputs (byte-wise) are resolved once and copied
    std::map<std::string, int> first;
    std::vector<int> src(n), uniq;
    for (int i = 0; i < n; ++i) {
        const std::string key(reinterpret_cast<const char*>(&in[i]), sizeof(lbm_params));
        auto it = first.emplace(key, i);
        src[i] = it.first->second;
        if (it.second) uniq.push_back(i);
    }
    const int hw = (int)std::thread::hardware_concurrency();
    const int nt = std::max(1, std::min({hw > 0 ? hw : 1, (int)uniq.size(), 64}));
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int k; (k = next.fetch_add(1)) < (int)uniq.size();) {
            const int i = uniq[k];
            status[i] = lbm_resolve_params(&in[i], &out[i], &th[i]);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < n; ++i)
        if (src[i] != i) {
            status[i] = status[src[i]];
            out[i] = out[src[i]];
            th[i] = th[src[i]];
        }
    return LBM_OK;
}

static long long plane_pitch(int nx, int ny) {
    const long long n = (long long)nx * ny;
    return (n + 63) / 64 * 64;  // 256-byte aligned planes for FP32, 512 for FP64
}

// Planes of one population buffer: the 9 populations, plus for FP32 the int16 plane that
// extends the free-energy model's rest population (lbmk::rest_update).
static size_t buffer_bytes(int precision, int nx, int ny) {
    const size_t esz = precision == LBM_F64 ? 8 : 4;
    return align256((precision == LBM_F64 ? 9 : 10) * (size_t)plane_pitch(nx, ny) * esz);
}

// Slots of the driven FP32 strip steps' per-warp stored mass: one per consumer warp of every
// strip CTA of either model's strip kernel (strips of at least one row).
static size_t drive_mass_slots(int nx, int ny) {
    const size_t pp = (size_t)((nx + kPPPTX - 1) / kPPPTX) * kPPPWarps;
    const size_t fe = (size_t)((nx + kFEPTX - 1) / kFEPTX) * kFEPWarps;
    return std::max(pp, fe) * (size_t)ny;
}

extern "C" size_t lbm_workspace_bytes(int precision, int nx, int ny) {
    if (nx < 1 || ny < 1) return 0;
    const size_t esz = precision == LBM_F64 ? 8 : 4;
    const size_t n = (size_t)nx * ny;
    const size_t fbytes = buffer_bytes(precision, nx, ny);
    const size_t fields = align256(4 * n * esz);
    // ... + the one-sided walls' row solve (14 nx reals) + the drive's mass slots
    return 2 * fbytes + fields + align256(kRedBlocks * 3 * sizeof(double)) + align256(8 * sizeof(double)) + 256 +
           align256(14 * (size_t)nx * esz) + align256(drive_mass_slots(nx, ny) * sizeof(double));
}

template <typename real>
static void fill_step_params(lbmk::StepParams<real>& s, const lbm_ctx* c) {
    const lbm_params& p = c->prm;
    s.nx = c->nx;
    s.ny = c->ny;
    s.rows = c->rows;
    s.pitch = c->pitch;
    s.RT = (real)(p.R * c->th.T);
    s.a = (real)p.a;
    s.b4 = (real)(0.25 * p.b);
    const double G = -1.0;
    const double C1 = 5.0 / 6.0 * (p.kappa_P - 1.0), C2 = 0.5 * (1.0 - p.kappa_P);
    s.kA = (real)(G * (C1 - C2 / 3.0));
    s.kB = (real)(G * (C2 + 0.5 * p.kappa_Li));
    s.li = (real)(12.0 * p.kappa_P * p.sigma_Li);
    s.kappa = (real)p.kappa;
    s.rho_ref_v = (real)c->th.rho_v;
    s.rho_ref_l = (real)c->th.rho_l;
    s.rho_split = (real)(0.5 * (c->th.rho_v + c->th.rho_l));
    const lbm_host::CS eos{p.a, p.b, p.R};
    s.mu_off_l = (real)(eos.mu((double)s.rho_ref_l, c->th.T) - eos.mu((double)s.rho_ref_v, c->th.T));
    const double urv = 1.0 - 0.25 * p.b * (double)s.rho_ref_v, url = 1.0 - 0.25 * p.b * (double)s.rho_ref_l;
    s.ur_v = (real)urv;
    s.ur_l = (real)url;
    s.ur3_v = (real)(urv * urv * urv);
    s.ur3_l = (real)(url * url * url);
    s.irr_v = (real)(1.0 / (double)s.rho_ref_v);
    s.irr_l = (real)(1.0 / (double)s.rho_ref_l);
    s.s_e = (real)(1.0 / p.tau_e);
    s.s_z = (real)(1.0 / p.tau_zeta);
    s.s_q = (real)(1.0 / p.tau_q);
    s.s_nu = (real)(1.0 / p.tau_nu);
    s.fx = (real)p.body_fx;
    s.fy = (real)p.body_fy;
    s.rest_unit = (real)lbm_host::rest_unit(p.b);
    s.rest_inv = (real)lbm_host::rest_inv(p.b);
    s.h_e = (real)(1.0 - 0.5 / p.tau_e);
    s.h_z = (real)(1.0 - 0.5 / p.tau_zeta);
    s.h_q = (real)(1.0 - 0.5 / p.tau_q);
    s.h_nu = (real)(1.0 - 0.5 / p.tau_nu);
    s.h6_e = (real)(6.0 * (1.0 - 0.5 / p.tau_e));
    s.h6_z = (real)(6.0 * (1.0 - 0.5 / p.tau_zeta));
}

static int choose_rows(int nx, int ny, int tx, int strips_per_sm) {
    // Enough CTAs to fill 152 SMs several times over, but long strips so the y halo
    // (recomputed rows) stays a few percent.  LBM_ROWS overrides (tuning experiments).
    if (const char* e = std::getenv("LBM_ROWS")) {
        const int r = std::atoi(e);
        if (r >= 1) return r < ny ? r : ny;
    }
    // Measured at 4096^2 (three CTAs per SM): the pseudopotential kernel is flat from 20 to
    // 36 rows, the free-energy kernel (5 halo rows per strip) best at 36-40; below 16 rows
    // the halo dominates (2048^2).
    const long long gx = (nx + tx - 1) / tx;
    const long long target = 152LL * strips_per_sm;
    long long rows = (ny * gx + target - 1) / target;
    if (rows < 8) rows = 8;
    // at least 16 rows while that still gives a full wave of CTAs (3 per SM); small lattices
    // keep shorter strips so that they still spread over the GPU
    if (rows < 16 && gx * ((ny + 15) / 16) >= 152LL * 3) rows = 16;
    if (rows > 64) rows = 64;
    if (rows > ny) rows = ny;
    return (int)rows;
}

extern "C" int lbm_create(const lbm_params* p, int nx, int ny, int bc_x, int bc_y, void* stream, void* workspace,
                          size_t workspace_bytes, lbm_ctx** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!p || nx < 1 || ny < 1 || (long long)nx * ny > (1LL << 31)) return LBM_ERR_ARG;
    if (bc_x != LBM_BC_PERIODIC ||
        (bc_y != LBM_BC_PERIODIC && bc_y != LBM_BC_WALL_ZOUHE && bc_y != LBM_BC_WALL_ZOUHE_ONESIDED))
        return LBM_ERR_UNSUPPORTED;
    const bool walls = bc_y == LBM_BC_WALL_ZOUHE || bc_y == LBM_BC_WALL_ZOUHE_ONESIDED;
    if (walls && ny < 4) return LBM_ERR_ARG;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_ARG;
    int rc = lbm_resolve_params(p, &c->prm, &c->th);
    if (rc) {
        delete c;
        return rc;
    }
    c->nx = nx;
    c->ny = ny;
    c->prec = c->prm.precision;
    c->esz = c->prec == LBM_F64 ? 8 : 4;
    c->pitch = plane_pitch(nx, ny);
    {
        const bool ppm = p->model == LBM_PSEUDOPOTENTIAL;
        const bool fast = c->prec == LBM_F32 && nx % 4 == 0 && nx >= 8 && ny >= 2 * kWallBandFE &&
                          std::getenv("LBM_NO_TMA") == nullptr;
        const int tx = c->prec == LBM_F64 ? kTXd : (walls && !fast) ? kTXf : ppm ? kPPPTX : kFEPTX;
        c->rows = choose_rows(nx, ny, tx, ppm ? 16 : 12);
    }
    const size_t need = lbm_workspace_bytes(c->prec, nx, ny);
    if (workspace) {
        if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
            delete c;
            return LBM_ERR_ARG;
        }
        c->ws = static_cast<char*>(workspace);
        c->own_ws = false;
    } else {
        cudaError_t e = cudaMalloc(&c->ws, need);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaMalloc(workspace)");
        }
        c->own_ws = true;
    }
    const size_t fbytes = buffer_bytes(c->prec, nx, ny);
    const size_t n = (size_t)nx * ny;
    c->f[0] = c->ws;
    c->f[1] = c->ws + fbytes;
    c->fields = c->ws + 2 * fbytes;
    c->partials = reinterpret_cast<double*>(c->ws + 2 * fbytes + align256(4 * n * c->esz));
    c->d_obs = reinterpret_cast<double*>(reinterpret_cast<char*>(c->partials) + align256(kRedBlocks * 3 * sizeof(double)));
    c->d_err = reinterpret_cast<int*>(reinterpret_cast<char*>(c->d_obs) + align256(8 * sizeof(double)));
    c->wall = reinterpret_cast<char*>(c->d_err) + 256;
    c->dmass = reinterpret_cast<double*>(static_cast<char*>(c->wall) + align256(14 * (size_t)nx * c->esz));
    c->walls = walls;
    c->onesided = bc_y == LBM_BC_WALL_ZOUHE_ONESIDED && p->model == LBM_FREE_ENERGY;
    // walls: the periodic strip kernels serve the interior when both wall bands fit
    c->use_tma = (!walls || ny >= 2 * kWallBandFE) && c->prec == LBM_F32 && nx % 4 == 0 && nx >= 8 && ny >= 4 &&
                 std::getenv("LBM_NO_TMA") == nullptr;
    cudaError_t e = cudaMallocHost(&c->h_pinned, 8 * sizeof(double));
    if (e != cudaSuccess) {
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return cuda_fail(e, "cudaMallocHost");
    }
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaFreeHost(c->h_pinned);
            if (c->own_ws) cudaFree(c->ws);
            delete c;
            return cuda_fail(e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }
    c->graph[0][0] = c->graph[0][1] = c->graph[1][0] = c->graph[1][1] = nullptr;
    c->drive = false;
    c->grav = false;
    c->g = c->rho_g = c->y_ref = 0.0;
    c->cur = 0;
    c->step = 0;
    c->status = LBM_OK;
    c->ready = false;
    fill_step_params(c->spf, c);
    fill_step_params(c->spd, c);
    if (c->use_tma) {
        // the stage rings exceed the default 48 KB of dynamic shared memory
        cudaError_t e1 = cudaFuncSetAttribute(lbmk::fe_step_pair<kFEPWarps, kFEPStages>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FEPSmem));
        cudaError_t e2 = cudaFuncSetAttribute(lbmk::pp_step_pair<kPPPWarps, kPPPStages>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PPPSmem));
        if (e1 == cudaSuccess)  // the driven instantiations (Sec. 5.4 drive)
            e1 = cudaFuncSetAttribute(lbmk::fe_step_pair<kFEPWarps, kFEPStages, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FEPSmem));
        if (e2 == cudaSuccess)
            e2 = cudaFuncSetAttribute(lbmk::pp_step_pair<kPPPWarps, kPPPStages, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PPPSmem));
        if (e1 == cudaSuccess)  // the full free-energy model's strip kernel
            e1 = cudaFuncSetAttribute(lbmk::fe_iwb_pair<kIWBWarps, kIWBStages>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(IWBSmem));
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            lbm_destroy(c);
            return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaFuncSetAttribute(max dynamic smem)");
        }
    }
    *out = c;
    return LBM_OK;
}

extern "C" void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 2; ++i)
        for (int m = 0; m < 2; ++m)
            if (c->graph[i][m]) cudaGraphExecDestroy(c->graph[i][m]);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->own_ws) cudaFree(c->ws);
    delete c;
}

extern "C" void* lbm_stream(const lbm_ctx* c) { return c ? static_cast<void*>(c->stream) : nullptr; }

extern "C" int lbm_derived(const lbm_ctx* c, lbm_params* resolved, lbm_thermo* th) {
    if (!c) return LBM_ERR_ARG;
    if (resolved) *resolved = c->prm;
    if (th) *th = c->th;
    return LBM_OK;
}

// ----------------------------------------------------------------------------
// Kernel launches

constexpr int kMassBlocks = 608;  // block sums of the drive's domain mean (4 x 152 SMs; < 3 kRedBlocks)

template <typename real>
static lbmk::Drive<real> no_drive() {
    lbmk::Drive<real> d{};
    d.rho_ave = nullptr;
    return d;
}

// The drive of the state in buffer src: its mean density reduced on the context stream into
// partials[kMassBlocks] (block sums in partials[0, kMassBlocks)).
template <typename real>
static lbmk::Drive<real> launch_drive(lbm_ctx* c, int src) {
    const long long n = (long long)c->nx * c->ny;
    lbmk::mass_partials_kernel<real><<<kMassBlocks, 256, 0, c->stream>>>(static_cast<const real*>(c->f[src]),
                                                                       c->pitch, n, c->partials);
    lbmk::mass_final_kernel<<<1, 32, 0, c->stream>>>(c->partials, kMassBlocks, 1.0 / (double)n,
                                                     c->partials + kMassBlocks);
    lbmk::Drive<real> d;
    d.rho_ave = c->partials + kMassBlocks;
    d.x_split = (int)std::floor(std::min(std::max(c->drive_split, -1.0), (double)c->nx));
    d.ax_lo = (real)c->drive_lo;
    d.ax_hi = (real)c->drive_hi;
    return d;
}

// Jacobi sweeps of the one-sided walls' density solve (the oracle's fixed point reaches
// rounding level, 4e-16 relative, in 16-29 sweeps on the channels of Sec. 5.3)
constexpr int kWallIters = 32;

// One-sided free-energy walls: solve the wall rows' J_y for the state in buffer src; returns
// the J_y array the step and field kernels read (nullptr when the walls are mirrored).
template <typename real>
static const real* launch_wall_solve(lbm_ctx* c, int src, const lbmk::StepParams<real>& sp);

// The drive of a state whose mass the previous driven strip step left in c->dmass (its
// per-warp sums of the populations it stored): rho_ave = their fixed-order sum / cells.
static lbmk::Drive<float> chained_drive(lbm_ctx* c, dim3 grid, int nwarps) {
    const long long n = (long long)c->nx * c->ny;
    lbmk::mass_final_kernel<<<1, 32, 0, c->stream>>>(c->dmass, (int)(grid.x * grid.y) * nwarps, 1.0 / (double)n,
                                                     c->partials + kMassBlocks);
    lbmk::Drive<float> d;
    d.rho_ave = c->partials + kMassBlocks;
    d.x_split = (int)std::floor(std::min(std::max(c->drive_split, -1.0), (double)c->nx));
    d.ax_lo = (float)c->drive_lo;
    d.ax_hi = (float)c->drive_hi;
    return d;
}

// One step with the droplet-collision drive acting (periodic lattice).  FP32 lattices that
// run the strip kernels run their DRIVE instantiation: rho_ave of the state comes from the
// masses the previous driven step stored (chained: the step before, in the same graph) or,
// for the first step of a sequence, from the block-sum reduction; FP64 and other shapes run
// the direct kernels after the reduction.
static int launch_step_driven(lbm_ctx* c, int src, bool chained) {
    const void* fin = c->f[src];
    void* fout = c->f[src ^ 1];
    const bool pp = c->prm.model == LBM_PSEUDOPOTENTIAL;
    if (c->prec == LBM_F32 && c->use_tma) {
        const int tx = pp ? kPPPTX : kFEPTX;
        dim3 grid((c->nx + tx - 1) / tx, (c->ny + c->rows - 1) / c->rows);
        const lbmk::Drive<float> d =
            chained ? chained_drive(c, grid, pp ? kPPPWarps : kFEPWarps) : launch_drive<float>(c, src);
        if (pp)
            lbmk::pp_step_pair<kPPPWarps, kPPPStages, true>
                <<<grid, (kPPPWarps + 1) * 32, sizeof(PPPSmem), c->stream>>>((const float*)fin, (float*)fout, c->spf,
                                                                             c->d_err, d, c->dmass);
        else
            lbmk::fe_step_pair<kFEPWarps, kFEPStages, true>
                <<<grid, (kFEPWarps + 1) * 32, sizeof(FEPSmem), c->stream>>>((const float*)fin, (float*)fout, c->spf,
                                                                             c->d_err, d, c->dmass);
    } else if (c->prec == LBM_F32) {
        const lbmk::Drive<float> d = launch_drive<float>(c, src);
        dim3 grid((c->nx + kTXf - 1) / kTXf, (c->ny + c->rows - 1) / c->rows);
        if (pp)
            lbmk::pp_step_ext<float, kTXf, false>
                <<<grid, kTXf + 32, 0, c->stream>>>((const float*)fin, (float*)fout, c->spf, 0, d);
        else
            lbmk::fe_step_ext<float, kTXf, false>
                <<<grid, kTXf + 32, 0, c->stream>>>((const float*)fin, (float*)fout, c->spf, 0, d, nullptr);
    } else {
        const lbmk::Drive<double> d = launch_drive<double>(c, src);
        dim3 grid((c->nx + kTXd - 1) / kTXd, (c->ny + c->rows - 1) / c->rows);
        if (pp)
            lbmk::pp_step_ext<double, kTXd, false>
                <<<grid, kTXd + 32, 0, c->stream>>>((const double*)fin, (double*)fout, c->spd, 0, d);
        else
            lbmk::fe_step_ext<double, kTXd, false>
                <<<grid, kTXd + 32, 0, c->stream>>>((const double*)fin, (double*)fout, c->spd, 0, d, nullptr);
    }
    CK(cudaGetLastError());
    return LBM_OK;
}

// Free-energy contexts with A != 0 or gravity run the full model's kernel.
static bool uses_iwb(const lbm_ctx* c) {
    return c->prm.model == LBM_FREE_ENERGY && (c->prm.A != 0.0 || c->grav);
}

template <typename real>
static lbmk::Ext<real> ext_terms(const lbm_ctx* c) {
    lbmk::Ext<real> e;
    e.on = uses_iwb(c) ? 1 : 0;
    e.A = (real)c->prm.A;
    e.g = (real)(c->grav ? c->g : 0.0);
    e.rho_g = (real)(c->grav ? c->rho_g : 0.0);
    e.y_ref = (real)c->y_ref;
    return e;
}

template <typename real, int TX>
static void launch_iwb(lbm_ctx* c, int src, bool driven, const lbmk::StepParams<real>& sp) {
    if constexpr (std::is_same<real, float>::value) {
        // FP32 periodic lattices without the drive and with gravity's reference density 0 run the
        // strip kernel; the rest the direct kernel
        if (c->use_tma && !c->walls && !driven && (!c->grav || c->rho_g == 0.0)) {
            dim3 grid((c->nx + IWBSmem::TX - 1) / IWBSmem::TX, (c->ny + c->rows - 1) / c->rows);
            lbmk::fe_iwb_pair<kIWBWarps, kIWBStages><<<grid, (kIWBWarps + 1) * 32, sizeof(IWBSmem), c->stream>>>(
                static_cast<const float*>(c->f[src]), static_cast<float*>(c->f[src ^ 1]), sp, ext_terms<float>(c),
                c->d_err);
            return;
        }
    }
    const lbmk::Drive<real> d = driven ? launch_drive<real>(c, src) : no_drive<real>();
    dim3 grid((c->nx + TX - 1) / TX, (c->ny + c->rows - 1) / c->rows);
    const real* fin = static_cast<const real*>(c->f[src]);
    real* fout = static_cast<real*>(c->f[src ^ 1]);
    const real* wjy = launch_wall_solve<real>(c, src, sp);
    if (c->walls)
        lbmk::fe_step_iwb<real, TX, true>
            <<<grid, TX + 32, 0, c->stream>>>(fin, fout, sp, d, ext_terms<real>(c), wjy);
    else
        lbmk::fe_step_iwb<real, TX, false>
            <<<grid, TX + 32, 0, c->stream>>>(fin, fout, sp, d, ext_terms<real>(c), nullptr);
}

template <typename real>
static const real* launch_wall_solve(lbm_ctx* c, int src, const lbmk::StepParams<real>& sp) {
    if (!c->onesided) return nullptr;
    real* w = static_cast<real*>(c->wall);
    lbmk::fe_wall_solve_kernel<real>
        <<<2, 1024, 0, c->stream>>>(static_cast<const real*>(c->f[src]), sp, ext_terms<real>(c), w, kWallIters);
    return w;
}

// chained: the previous launch on the stream was a driven step of the same sequence (a graph
// replays its steps in order), so a driven strip step may take rho_ave from its stored masses.
static int launch_step(lbm_ctx* c, int src, bool driven = false, bool chained = false) {
    if (uses_iwb(c)) {
        if (c->prec == LBM_F32)
            launch_iwb<float, kTXf>(c, src, driven, c->spf);
        else
            launch_iwb<double, kTXd>(c, src, driven, c->spd);
        CK(cudaGetLastError());
        return LBM_OK;
    }
    if (driven) return launch_step_driven(c, src, chained);
    const void* fin = c->f[src];
    void* fout = c->f[src ^ 1];
    const bool pp = c->prm.model == LBM_PSEUDOPOTENTIAL;
    if (c->walls && c->use_tma) {
        // periodic fast step over the whole lattice, then the wall bands recomputed
        const int band = pp ? kWallBandPP : kWallBandFE;
        if (pp) {
            dim3 grid((c->nx + kPPPTX - 1) / kPPPTX, (c->ny + c->rows - 1) / c->rows);
            lbmk::pp_step_pair<kPPPWarps, kPPPStages><<<grid, (kPPPWarps + 1) * 32, sizeof(PPPSmem), c->stream>>>(
                (const float*)fin, (float*)fout, c->spf, c->d_err);
            lbmk::pp_step_ext<float, kTXf, true><<<dim3((c->nx + kTXf - 1) / kTXf, 2), kTXf + 32, 0, c->stream>>>(
                (const float*)fin, (float*)fout, c->spf, band, no_drive<float>());
        } else {
            dim3 grid((c->nx + kFEPTX - 1) / kFEPTX, (c->ny + c->rows - 1) / c->rows);
            const float* wjy = launch_wall_solve<float>(c, src, c->spf);
            lbmk::fe_step_pair<kFEPWarps, kFEPStages><<<grid, (kFEPWarps + 1) * 32, sizeof(FEPSmem), c->stream>>>(
                (const float*)fin, (float*)fout, c->spf, c->d_err);
            lbmk::fe_step_ext<float, kTXf, true><<<dim3((c->nx + kTXf - 1) / kTXf, 2), kTXf + 32, 0, c->stream>>>(
                (const float*)fin, (float*)fout, c->spf, band, no_drive<float>(), wjy);
        }
    } else if (c->walls) {
        if (c->prec == LBM_F32) {
            dim3 grid((c->nx + kTXf - 1) / kTXf, (c->ny + c->rows - 1) / c->rows);
            if (pp)
                lbmk::pp_step_ext<float, kTXf, true>
                    <<<grid, kTXf + 32, 0, c->stream>>>((const float*)fin, (float*)fout, c->spf, 0, no_drive<float>());
            else
                lbmk::fe_step_ext<float, kTXf, true><<<grid, kTXf + 32, 0, c->stream>>>(
                    (const float*)fin, (float*)fout, c->spf, 0, no_drive<float>(), launch_wall_solve<float>(c, src, c->spf));
        } else {
            dim3 grid((c->nx + kTXd - 1) / kTXd, (c->ny + c->rows - 1) / c->rows);
            if (pp)
                lbmk::pp_step_ext<double, kTXd, true>
                    <<<grid, kTXd + 32, 0, c->stream>>>((const double*)fin, (double*)fout, c->spd, 0, no_drive<double>());
            else
                lbmk::fe_step_ext<double, kTXd, true><<<grid, kTXd + 32, 0, c->stream>>>(
                    (const double*)fin, (double*)fout, c->spd, 0, no_drive<double>(),
                    launch_wall_solve<double>(c, src, c->spd));
        }
    } else if (c->use_tma && pp) {
        dim3 grid((c->nx + kPPPTX - 1) / kPPPTX, (c->ny + c->rows - 1) / c->rows);
        lbmk::pp_step_pair<kPPPWarps, kPPPStages><<<grid, (kPPPWarps + 1) * 32, sizeof(PPPSmem), c->stream>>>(
            (const float*)fin, (float*)fout, c->spf, c->d_err);
    } else if (c->use_tma) {
        dim3 grid((c->nx + kFEPTX - 1) / kFEPTX, (c->ny + c->rows - 1) / c->rows);
        lbmk::fe_step_pair<kFEPWarps, kFEPStages><<<grid, (kFEPWarps + 1) * 32, sizeof(FEPSmem), c->stream>>>(
            (const float*)fin, (float*)fout, c->spf, c->d_err);
    } else if (c->prec == LBM_F32) {
        dim3 grid((c->nx + kTXf - 1) / kTXf, (c->ny + c->rows - 1) / c->rows);
        if (pp)
            lbmk::pp_step_kernel<float, kTXf><<<grid, kTXf + 32, 0, c->stream>>>((const float*)fin, (float*)fout, c->spf);
        else
            lbmk::fe_step_kernel<float, kTXf><<<grid, kTXf + 32, 0, c->stream>>>((const float*)fin, (float*)fout, c->spf);
    } else {
        dim3 grid((c->nx + kTXd - 1) / kTXd, (c->ny + c->rows - 1) / c->rows);
        if (pp)
            lbmk::pp_step_kernel<double, kTXd><<<grid, kTXd + 32, 0, c->stream>>>((const double*)fin, (double*)fout, c->spd);
        else
            lbmk::fe_step_kernel<double, kTXd><<<grid, kTXd + 32, 0, c->stream>>>((const double*)fin, (double*)fout, c->spd);
    }
    CK(cudaGetLastError());
    return LBM_OK;
}

static int build_graph(lbm_ctx* c, int parity, int driven) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    int src = parity;
    for (int k = 0; k < kGraphSteps && rc == LBM_OK; ++k) {
        rc = launch_step(c, src, driven != 0, k > 0);
        src ^= 1;
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph[parity][driven], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return LBM_OK;
}

// Whether the collision of the state at time t is driven (Sec. 5.4: after t_on).
static bool driven_at(const lbm_ctx* c, long long t) { return c->drive && t > c->drive_t_on; }

extern "C" int lbm_step(lbm_ctx* c, long long nsteps) {
    if (!c || nsteps < 0) return LBM_ERR_ARG;
    if (!c->ready) return LBM_ERR_STATE;
    if (c->status) return c->status;
    while (nsteps > 0) {
        const bool driven = driven_at(c, c->step);
        // a 64-step graph replays one kind of step: the chunk must not straddle t_on
        const bool uniform = driven_at(c, c->step + kGraphSteps - 1) == driven;
        if (nsteps >= kGraphSteps && uniform) {
            cudaGraphExec_t& gx = c->graph[c->cur][driven ? 1 : 0];
            if (!gx) {
                int rc = build_graph(c, c->cur, driven ? 1 : 0);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(gx, c->stream));
            nsteps -= kGraphSteps;
            c->step += kGraphSteps;  // even count: buffer parity unchanged
        } else {
            int rc = launch_step(c, c->cur, driven);
            if (rc) return rc;
            c->cur ^= 1;
            --nsteps;
            ++c->step;
        }
    }
    return LBM_OK;
}

extern "C" int lbm_set_gravity(lbm_ctx* c, double g, double rho_ref, double y_ref) {
    if (!c || !std::isfinite(g) || !std::isfinite(rho_ref) || !std::isfinite(y_ref)) return LBM_ERR_ARG;
    if (c->prm.model != LBM_FREE_ENERGY) return LBM_ERR_UNSUPPORTED;
    if (rho_ref != 0.0 && !c->walls) return LBM_ERR_UNSUPPORTED;  // p_g would jump at the periodic wrap
    CK(cudaStreamSynchronize(c->stream));
    c->grav = g != 0.0;
    c->g = g;
    c->rho_g = rho_ref;
    c->y_ref = y_ref;
    for (int i = 0; i < 2; ++i)
        for (int m = 0; m < 2; ++m)
            if (c->graph[i][m]) {
                cudaGraphExecDestroy(c->graph[i][m]);
                c->graph[i][m] = nullptr;
            }
    return LBM_OK;
}

extern "C" int lbm_set_drive(lbm_ctx* c, double ax_lo, double ax_hi, double x_split, long long t_on) {
    if (!c || !std::isfinite(ax_lo) || !std::isfinite(ax_hi) || !std::isfinite(x_split)) return LBM_ERR_ARG;
    if (c->walls) return LBM_ERR_UNSUPPORTED;
    c->drive = true;
    c->drive_lo = ax_lo;
    c->drive_hi = ax_hi;
    c->drive_split = x_split;
    c->drive_t_on = t_on;
    // captured driven steps hold the old constants
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 2; ++i)
        if (c->graph[i][1]) {
            cudaGraphExecDestroy(c->graph[i][1]);
            c->graph[i][1] = nullptr;
        }
    return LBM_OK;
}

template <typename src_t>
static int launch_init(lbm_ctx* c, const src_t* rho0_dev) {
    const int model = c->prm.model;
    if (model == LBM_FREE_ENERGY && c->grav && c->rho_g != 0.0) {
        // equilibrium at rest with the gravitational reference pressure p_g of Eq. (20)
        const double coef = c->rho_g * c->g;
        if (c->prec == LBM_F32)
            lbmk::init_iwb_kernel<float, src_t><<<kRedBlocks, 256, 0, c->stream>>>(
                rho0_dev, (float*)c->f[0], c->nx, c->ny, c->pitch, coef, c->y_ref, c->spf.rest_inv);
        else
            lbmk::init_iwb_kernel<double, src_t><<<kRedBlocks, 256, 0, c->stream>>>(
                rho0_dev, (double*)c->f[0], c->nx, c->ny, c->pitch, coef, c->y_ref, 0.0f);
        CK(cudaGetLastError());
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        c->cur = 0;
        c->step = 0;
        c->status = LBM_OK;
        c->ready = true;
        return LBM_OK;
    }
    if (c->prec == LBM_F32)
        lbmk::init_kernel<float, src_t>
            <<<kRedBlocks, 256, 0, c->stream>>>(rho0_dev, (float*)c->f[0], model, c->nx, c->ny, c->pitch,
                                                c->spf.rest_inv);
    else
        lbmk::init_kernel<double, src_t>
            <<<kRedBlocks, 256, 0, c->stream>>>(rho0_dev, (double*)c->f[0], model, c->nx, c->ny, c->pitch, 0.0f);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    c->cur = 0;
    c->step = 0;
    c->status = LBM_OK;
    c->ready = true;
    return LBM_OK;
}

extern "C" int lbm_set_density(lbm_ctx* c, const double* rho0) {
    if (!c || !rho0) return LBM_ERR_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    const double top = 4.0 / c->prm.b;
    for (size_t k = 0; k < n; ++k)
        if (!(rho0[k] > 0.0 && rho0[k] < top)) return LBM_ERR_ARG;
    // stage the FP64 densities in the fields scratch (>= 8 N bytes), convert in the kernel
    CK(cudaMemcpyAsync(c->fields, rho0, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return launch_init(c, static_cast<const double*>(c->fields));
}

extern "C" int lbm_set_density_device(lbm_ctx* c, const void* rho0) {
    if (!c || !rho0) return LBM_ERR_ARG;
    if (c->prec == LBM_F32) return launch_init(c, static_cast<const float*>(rho0));
    return launch_init(c, static_cast<const double*>(rho0));
}

// Host view f_i(x) (state after streaming, Eq. 2 order) <-> stored S_i(y) = f_i(y + c_i).
static const int kCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int kCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static inline size_t shifted(int x, int y, int i, int nx, int ny) {
    int xs = (x + kCX[i] + nx) % nx, ys = (y + kCY[i] + ny) % ny;
    return (size_t)ys * nx + xs;
}

// FP32 buffers carry the compensated rest population (lbmk::rest_update; rest_host.h).
static bool has_rest_plane(const lbm_ctx* c) { return c->prec == LBM_F32; }

extern "C" int lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return LBM_ERR_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    std::vector<char> stage(n * c->esz);
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 9; ++i) {
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const double v = f[i * n + shifted(x, y, i, c->nx, c->ny)];
                const size_t k = (size_t)y * c->nx + x;
                if (c->prec == LBM_F32)
                    reinterpret_cast<float*>(stage.data())[k] = (float)v;
                else
                    reinterpret_cast<double*>(stage.data())[k] = v;
            }
        CK(cudaMemcpy(static_cast<char*>(c->f[0]) + (size_t)i * c->pitch * c->esz, stage.data(), n * c->esz,
                      cudaMemcpyHostToDevice));
    }
    if (c->prec == LBM_F32) {
        // rest-population extension: the part of f_0 below FP32
        std::vector<short> q(n, 0);
        for (size_t k = 0; k < n; ++k) q[k] = lbm_host::rest_encode(f[k], (float)f[k], lbm_host::rest_inv(c->prm.b));
        CK(cudaMemcpy(static_cast<char*>(c->f[0]) + (size_t)9 * c->pitch * 4, q.data(), n * sizeof(short),
                      cudaMemcpyHostToDevice));
    }
    CK(cudaMemset(c->d_err, 0, sizeof(int)));
    c->cur = 0;
    c->step = 0;
    c->status = LBM_OK;
    c->ready = true;
    return LBM_OK;
}

template <typename real>
static int compute_fields(lbm_ctx* c, const lbmk::StepParams<real>& sp);

// Walls: the stored state lacks the wall nodes' incoming populations until the fields pass
// completes them (in place, in slots no step reads).
static int complete_walls(lbm_ctx* c) {
    if (!c->walls) return LBM_OK;
    return c->prec == LBM_F32 ? compute_fields(c, c->spf) : compute_fields(c, c->spd);
}

extern "C" int lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return LBM_ERR_ARG;
    if (!c->ready) return LBM_ERR_STATE;
    if (int rc = complete_walls(c)) return rc;
    const size_t n = (size_t)c->nx * c->ny;
    std::vector<char> stage(n * c->esz);
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 9; ++i) {
        CK(cudaMemcpy(stage.data(), static_cast<char*>(c->f[c->cur]) + (size_t)i * c->pitch * c->esz, n * c->esz,
                      cudaMemcpyDeviceToHost));
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const size_t k = (size_t)y * c->nx + x;
                const double v = c->prec == LBM_F32 ? (double)reinterpret_cast<const float*>(stage.data())[k]
                                                    : reinterpret_cast<const double*>(stage.data())[k];
                f[i * n + shifted(x, y, i, c->nx, c->ny)] = v;
            }
    }
    if (has_rest_plane(c)) {
        std::vector<short> q(n);
        CK(cudaMemcpy(q.data(), static_cast<char*>(c->f[c->cur]) + (size_t)9 * c->pitch * 4, n * sizeof(short),
                      cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < n; ++k) f[k] = lbm_host::rest_decode((float)f[k], q[k], lbm_host::rest_unit(c->prm.b));
    }
    return LBM_OK;
}

extern "C" int lbm_get_populations_at(lbm_ctx* c, int n, const int* xs, const int* ys, double* out) {
    if (!c || n < 0 || (n > 0 && (!xs || !ys || !out))) return LBM_ERR_ARG;
    if (!c->ready) return LBM_ERR_STATE;
    for (int k = 0; k < n; ++k)
        if (xs[k] < 0 || xs[k] >= c->nx || ys[k] < 0 || ys[k] >= c->ny) return LBM_ERR_ARG;
    if (int rc = complete_walls(c)) return rc;
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < 9; ++i) {
            // f_i(x) = S_i(x - c_i)
            const int xs_ = (xs[k] - kCX[i] + c->nx) % c->nx, ys_ = (ys[k] - kCY[i] + c->ny) % c->ny;
            const size_t off = ((size_t)i * c->pitch + (size_t)ys_ * c->nx + xs_) * c->esz;
            if (c->prec == LBM_F32) {
                float v;
                CK(cudaMemcpy(&v, static_cast<char*>(c->f[c->cur]) + off, 4, cudaMemcpyDeviceToHost));
                out[9 * k + i] = v;
                if (i == 0 && has_rest_plane(c)) {
                    short q;
                    const size_t qoff = (size_t)9 * c->pitch * 4 + ((size_t)ys_ * c->nx + xs_) * sizeof(short);
                    CK(cudaMemcpy(&q, static_cast<char*>(c->f[c->cur]) + qoff, sizeof(short), cudaMemcpyDeviceToHost));
                    out[9 * k] = lbm_host::rest_decode(v, q, lbm_host::rest_unit(c->prm.b));
                }
            } else {
                CK(cudaMemcpy(&out[9 * k + i], static_cast<char*>(c->f[c->cur]) + off, 8, cudaMemcpyDeviceToHost));
            }
        }
    return LBM_OK;
}

extern "C" int lbm_device_populations(lbm_ctx* c, void** f, long long* pitch) {
    if (!c || !f) return LBM_ERR_ARG;
    *f = c->f[c->cur];
    if (pitch) *pitch = c->pitch;
    return LBM_OK;
}

// rho, aux, ux, uy fields of the current state into the fields scratch.
template <typename real>
static int compute_fields(lbm_ctx* c, const lbmk::StepParams<real>& sp) {
    const long long n = (long long)c->nx * c->ny;
    real* rho = static_cast<real*>(c->fields);
    real* aux = rho + n;
    real* ux = aux + n;
    real* uy = ux + n;
    const real* f = static_cast<const real*>(c->f[c->cur]);
    const int model = c->prm.model;
    if (c->walls || driven_at(c, c->step) || uses_iwb(c)) {
        real* fw = static_cast<real*>(c->f[c->cur]);
        const lbmk::Ext<real> ex = ext_terms<real>(c);
        if (c->walls) {
            const real* wjy = launch_wall_solve<real>(c, c->cur, sp);
            lbmk::rho_walls_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(fw, rho, aux, sp, model, ex, wjy);
            if (model == LBM_FREE_ENERGY) lbmk::mu_walls_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(rho, aux, sp);
            lbmk::walls_complete_kernel<real>
                <<<(2 * c->nx + 255) / 256, 256, 0, c->stream>>>(fw, rho, aux, sp, model, ex, c->onesided ? 1 : 0);
        } else {
            lbmk::rho_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(f, rho, aux, sp, model);
            if (model == LBM_FREE_ENERGY) lbmk::mu_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(rho, aux, sp);
        }
        const lbmk::Drive<real> d = driven_at(c, c->step) ? launch_drive<real>(c, c->cur) : no_drive<real>();
        lbmk::velocity_ext_kernel<real>
            <<<kRedBlocks, 256, 0, c->stream>>>(fw, rho, aux, ux, uy, sp, model, c->walls ? 1 : 0, d, ex,
                                                c->onesided ? 1 : 0);
        CK(cudaGetLastError());
        return LBM_OK;
    }
    lbmk::rho_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(f, rho, aux, sp, model);
    if (model == LBM_FREE_ENERGY) lbmk::mu_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(rho, aux, sp);
    lbmk::velocity_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(f, rho, aux, ux, uy, sp, model);
    CK(cudaGetLastError());
    return LBM_OK;
}

template <typename real>
static int observables_impl(lbm_ctx* c, const lbmk::StepParams<real>& sp, int geometry, lbm_obs* o) {
    int rc = compute_fields<real>(c, sp);
    if (rc) return rc;
    const long long n = (long long)c->nx * c->ny;
    const real* rho = static_cast<const real*>(c->fields);
    lbmk::obs_partial_kernel<real><<<kRedBlocks, 256, 0, c->stream>>>(rho, rho + 2 * n, rho + 3 * n, n, c->partials);
    lbmk::ObsConst C{c->nx, c->ny, geometry, kRedBlocks, c->prm.R * c->th.T, c->prm.a, 0.25 * c->prm.b};
    lbmk::obs_final_kernel<real><<<1, 256, 0, c->stream>>>(rho, c->partials, C, c->d_obs);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_pinned, c->d_obs, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (herr) c->status = LBM_ERR_TIMEOUT;
    const double* h = c->h_pinned;
    o->rho_l = h[0];
    o->rho_v = h[1];
    o->width = h[2];
    o->dp = h[3];
    o->u_max = h[4];
    o->mass = h[5];
    o->radius = h[6];
    o->step = c->step;
    o->pad_ = 0;
    if (c->status == LBM_OK && (h[7] != 0.0 || !std::isfinite(h[5]))) c->status = LBM_ERR_DIVERGED;
    o->status = c->status;
    return LBM_OK;
}

extern "C" int lbm_observables(lbm_ctx* c, int geometry, lbm_obs* out) {
    if (!c || !out || (geometry != 0 && geometry != 1)) return LBM_ERR_ARG;
    if (!c->ready) return LBM_ERR_STATE;
    int rc = c->prec == LBM_F32 ? observables_impl<float>(c, c->spf, geometry, out)
                                : observables_impl<double>(c, c->spd, geometry, out);
    if (rc) return rc;
    return out->status;
}

template <typename real>
static int fields_impl(lbm_ctx* c, const lbmk::StepParams<real>& sp, double* rho, double* ux, double* uy) {
    int rc = compute_fields<real>(c, sp);
    if (rc) return rc;
    const size_t n = (size_t)c->nx * c->ny;
    std::vector<real> stage(n);
    CK(cudaStreamSynchronize(c->stream));
    double* outs[3] = {rho, ux, uy};
    const int slot[3] = {0, 2, 3};
    for (int k = 0; k < 3; ++k) {
        if (!outs[k]) continue;
        CK(cudaMemcpy(stage.data(), static_cast<const real*>(c->fields) + slot[k] * n, n * sizeof(real),
                      cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) outs[k][i] = (double)stage[i];
    }
    return LBM_OK;
}

extern "C" int lbm_get_fields(lbm_ctx* c, double* rho, double* ux, double* uy) {
    if (!c) return LBM_ERR_ARG;
    if (!c->ready) return LBM_ERR_STATE;
    return c->prec == LBM_F32 ? fields_impl<float>(c, c->spf, rho, ux, uy) : fields_impl<double>(c, c->spd, rho, ux, uy);
}

// ----------------------------------------------------------------------------
// Observables of caller-owned device fields with no allocation: the partial sums of
// the reduction live in a file-scope device array instead of a context workspace.

static __device__ __align__(256) double g_static_partials[LBM_STATIC_MAX_BLOCKS * 3];

namespace {
constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {nullptr};
bool g_static_ready[kMaxDevices] = {false};
}  // namespace

// Device address of g_static_partials on the current device, looked up once per device
// (the host-side symbol is only a stand-in and must never be passed to a kernel).
static int static_partials_ptr(double** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
    if (!__atomic_load_n(&g_static_ready[dev], __ATOMIC_ACQUIRE)) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_static_partials));
        g_static_ptr[dev] = static_cast<double*>(p);
        __atomic_store_n(&g_static_ready[dev], true, __ATOMIC_RELEASE);
    }
    *out = g_static_ptr[dev];
    return LBM_OK;
}

template <typename real>
static int static_obs_impl(const real* rho, const real* ux, const real* uy, int nx, int ny, int geometry, double a,
                           double b, double R, double T, int nblocks, double* out, cudaStream_t s) {
    double* partials = nullptr;
    int rc = static_partials_ptr(&partials);
    if (rc) return rc;
    const long long n = (long long)nx * ny;
    lbmk::obs_partial_kernel<real><<<nblocks, 256, 0, s>>>(rho, ux, uy, n, partials);
    lbmk::ObsConst C{nx, ny, geometry, nblocks, R * T, a, 0.25 * b};
    lbmk::obs_final_kernel<real><<<1, 256, 0, s>>>(rho, partials, C, out);
    CK(cudaGetLastError());
    return LBM_OK;
}

extern "C" int lbm_observables_fields_static(int precision, const void* rho, const void* ux, const void* uy, int nx,
                                             int ny, int geometry, double a, double b, double R, double T,
                                             int nblocks, double* out_dev, void* stream) {
    if (!rho || !ux || !uy || !out_dev || nx < 1 || ny < 1 || (geometry != 0 && geometry != 1)) return LBM_ERR_ARG;
    if (nblocks < 1 || nblocks > LBM_STATIC_MAX_BLOCKS) return LBM_ERR_ARG;
    if (!(a > 0 && b > 0 && R > 0 && T > 0)) return LBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == LBM_F32)
        return static_obs_impl<float>(static_cast<const float*>(rho), static_cast<const float*>(ux),
                                      static_cast<const float*>(uy), nx, ny, geometry, a, b, R, T, nblocks, out_dev, s);
    if (precision == LBM_F64)
        return static_obs_impl<double>(static_cast<const double*>(rho), static_cast<const double*>(ux),
                                       static_cast<const double*>(uy), nx, ny, geometry, a, b, R, T, nblocks, out_dev,
                                       s);
    return LBM_ERR_ARG;
}

// ----------------------------------------------------------------------------
// Checkpoint: "LBMCKPT1", nx, ny, model, precision, step, params, f (FP64, Eq. 2 order).

extern "C" int lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_ERR_ARG;
    if (!c->ready) return LBM_ERR_STATE;
    const size_t n = (size_t)c->nx * c->ny;
    std::vector<double> f(9 * n);
    int rc = lbm_get_populations(c, f.data());
    if (rc) return rc;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return LBM_ERR_IO;
    const char magic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};
    int hdr[4] = {c->nx, c->ny, c->prm.model, c->prec};
    bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof(int), 4, fp) == 4 &&
              std::fwrite(&c->step, sizeof(long long), 1, fp) == 1 &&
              std::fwrite(&c->prm, sizeof(lbm_params), 1, fp) == 1 &&
              std::fwrite(f.data(), sizeof(double), f.size(), fp) == f.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : LBM_ERR_IO;
}

extern "C" int lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_ERR_ARG;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LBM_ERR_IO;
    char magic[8];
    int hdr[4];
    long long step;
    lbm_params prm;
    const size_t n = (size_t)c->nx * c->ny;
    std::vector<double> f(9 * n);
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "LBMCKPT1", 8) == 0 &&
              std::fread(hdr, sizeof(int), 4, fp) == 4 && std::fread(&step, sizeof(long long), 1, fp) == 1 &&
              std::fread(&prm, sizeof(lbm_params), 1, fp) == 1;
    // the checkpoint continues the run it was written from: same lattice, model, precision and
    // resolved parameters (a state of one temperature or EOS is not a state of another)
    const double saved[] = {prm.a, prm.b, prm.R, prm.Tr, prm.tau_nu, prm.tau_e, prm.tau_zeta, prm.tau_q,
                            prm.tau_j, prm.kappa_P, prm.kappa_Li, prm.sigma_Li, prm.kappa, prm.A,
                            prm.body_fx, prm.body_fy};
    const double mine[] = {c->prm.a, c->prm.b, c->prm.R, c->prm.Tr, c->prm.tau_nu, c->prm.tau_e,
                           c->prm.tau_zeta, c->prm.tau_q, c->prm.tau_j, c->prm.kappa_P, c->prm.kappa_Li,
                           c->prm.sigma_Li, c->prm.kappa, c->prm.A, c->prm.body_fx, c->prm.body_fy};
    bool same = true;
    for (size_t k = 0; k < sizeof(saved) / sizeof(saved[0]); ++k) same = same && saved[k] == mine[k];
    if (ok && (hdr[0] != c->nx || hdr[1] != c->ny || hdr[2] != c->prm.model || hdr[3] != c->prec || !same)) {
        std::fclose(fp);
        return LBM_ERR_ARG;
    }
    ok = ok && std::fread(f.data(), sizeof(double), f.size(), fp) == f.size();
    std::fclose(fp);
    if (!ok) return LBM_ERR_IO;
    int rc = lbm_set_populations(c, f.data());
    if (rc) return rc;
    c->step = step;
    return LBM_OK;
}
