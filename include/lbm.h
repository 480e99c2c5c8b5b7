/*
 * lbm.h -- C ABI of the GB300 D2Q9 multiphase lattice Boltzmann library.
 *
 * Implements the two models compared in "Fundamental comparison between the
 * pseudopotential and the free energy lattice Boltzmann methods" (Czelusniak,
 * Martins, Cabezas Gomez, Bulgarelli, Monte Verde, de Castro; arXiv:2403.11167):
 *
 *   LBM_PSEUDOPOTENTIAL  the modified pseudopotential model (MP-LBM, Sec. 4):
 *                        Eq. (1) MRT step with the Carnahan-Starling EOS (Eq. 28),
 *                        psi of Eq. (11), Shan-Chen force Eq. (10), width-control
 *                        source Eqs. (13), (30), (31) and forcing Eq. (32);
 *   LBM_FREE_ENERGY      the improved well-balanced free-energy model (Sec. 2.2):
 *                        Eq. (1) MRT step with chemical potential mu = mu_b - kappa
 *                        lap rho (Eq. 29, stencils of Eq. 24), equilibrium Eq. (20)
 *                        and forcing Eq. (21), including the viscosity-tuning term A
 *                        (lbm_params.A, Eqs. 20 and 23) and gravity (lbm_set_gravity:
 *                        p_g in Eq. 20, -grad p_g in Eq. 21, buoyancy).
 *
 * Units are lattice units: dx = dt = c = 1, c_s^2 = 1/3, G = -1 (Sec. 2.1).
 *
 * Conventions for every function below:
 *   - return value: LBM_OK (0) or a negative LBM_ERR_* code; no exception or
 *     abort crosses the ABI; lbm_strerror() names a code.
 *   - host pointers are owned by the caller and only read or written during the
 *     call; the library keeps no caller pointer.
 *   - device memory of a context is either allocated by the library (cudaMalloc)
 *     or supplied by the caller as one workspace (lbm_workspace_bytes); a
 *     context never frees a caller workspace.
 *   - all GPU work of a context runs on the context's stream, in call order.
 *     Functions that return host data synchronise that stream first.
 *   - populations are stored as 9 planes f_i[y][x] (structure of arrays) of the
 *     context precision; FP32 buffers have a tenth plane of int16 values that extends the
 *     free-energy model's rest population by 16 bits (f_0 = plane 0 + q 2^-16 ulp(plane
 *     0): in that model f_0 carries almost all of the mass, and FP32 rounding of it
 *     would random-walk the mass); host-side population arrays use the velocity order of
 *     Eq. (2) (0 rest, 1..4 = (1,0),(0,1),(-1,0),(0,-1), 5..8 = (1,1),(-1,1),
 *     (-1,-1),(1,-1)), shape [9][ny][nx], row-major, FP64.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_ERR_ARG (-1)          /* invalid argument (size, tau <= 1/2, Tr outside (0,1), ...) */
#define LBM_ERR_UNSUPPORTED (-2)  /* feature not built (walls in x, A != 0 or gravity with the
                                     pseudopotential model, ...) */
#define LBM_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define LBM_ERR_DIVERGED (-4)     /* NaN/Inf or rho <= 0 seen; sticky for the context */
#define LBM_ERR_TIMEOUT (-5)      /* a bounded device wait ran out */
#define LBM_ERR_NOCONVERGE (-6)   /* a host Newton/bisection solve failed */
#define LBM_ERR_STATE (-7)        /* call out of order (e.g. step before set_density) */
#define LBM_ERR_IO (-8)           /* checkpoint file could not be read or written */

typedef enum { LBM_PSEUDOPOTENTIAL = 0, LBM_FREE_ENERGY = 1 } lbm_model;
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL_ZOUHE = 1, LBM_BC_WALL_ZOUHE_ONESIDED = 2 } lbm_bc;
typedef enum { LBM_F32 = 0, LBM_F64 = 1 } lbm_precision;
typedef enum { LBM_GEOMETRY_FLAT = 0, LBM_GEOMETRY_DROPLET = 1 } lbm_geometry;

/* Model parameters (Eqs. 3, 28, 30-32, 20-21).  A NaN or non-positive entry
 * where noted means "derive / use the default"; lbm_resolve_params fills them.
 *   a, b, R     Carnahan-Starling EOS constants (Eq. 28); T = Tr * T_c(a, b, R).
 *   Tr          reduced temperature, 0 < Tr < 1.
 *   tau_nu      shear relaxation time (> 1/2).  Other taus <= 0 take the defaults
 *               (both models: tau_rho = tau_j = 1):
 *                 pseudopotential: tau_e = tau_zeta = tau_nu, tau_q = 1/1.99 (Sec. 5.1);
 *                 free energy:     tau_e = 1/4 + tau_nu/2 (same bulk viscosity as the
 *                                  pseudopotential model, Eqs. 9 and 23), tau_zeta = tau_q = 1.
 *   kappa_P     interface-width factor of Eqs. (30)-(32); NaN -> 1.
 *   kappa_Li    surface-tension factor of Eq. (30b); NaN -> 0.
 *   sigma_Li    Li's coexistence parameter of Eq. (32); NaN -> the Appendix-B theory
 *               value (eps = -16 G sigma_Li from Eq. S13 at the Maxwell densities).
 *   match_kappa > 0: derive kappa_P and kappa_Li so that the pseudopotential model
 *               has the interface width and surface tension of the free-energy model
 *               with kappa = match_kappa (Sec. 3, Appendix B, Eqs. 26, S44, S46).
 *   kappa       free-energy gradient coefficient (mu = mu_b - kappa lap rho); NaN -> 0.5.
 *   A           viscosity-tuning term of the free-energy equilibrium, Eq. (20) (the strain-
 *               rate terms); nu = c_s^2 (tau_nu - 1/2 - A) must be positive (Eq. 23).  Free
 *               energy only (A != 0 with the pseudopotential model: LBM_ERR_UNSUPPORTED).
 *               A != 0 runs the full free-energy kernel (direct loads, one more ring level).
 *   body_fx/fy  constant body force added to the total force of either model. */
typedef struct {
    int model;       /* lbm_model */
    int precision;   /* lbm_precision */
    double a, b, R, Tr;
    double tau_nu, tau_e, tau_zeta, tau_q, tau_j;
    double kappa_P, kappa_Li, sigma_Li, match_kappa;
    double kappa, A;
    double body_fx, body_fy;
} lbm_params;

/* Thermodynamic and theoretical quantities derived on the host (FP64). */
typedef struct {
    double T, Tc, rho_c, p_c;      /* temperature, critical point (dp/drho = d2p/drho2 = 0) */
    double rho_v, rho_l, p0;       /* Maxwell coexistence (equal p and mu_b; Eq. S12) */
    double eps;                    /* -16 G sigma_Li used by the pseudopotential model */
    double width, gamma;           /* planar tangent width and surface tension of the model's
                                      continuum profile (Eq. 26 / Eq. S44, Eq. 25 / Eq. S46) */
} lbm_thermo;

/* Observables of the current state (see lbm_observables). */
typedef struct {
    double rho_l, rho_v;   /* probe means, liquid and vapour */
    double width;          /* tangent interface width */
    double dp;             /* p_EOS(rho_l) - p_EOS(rho_v) */
    double u_max;          /* max |u| over the lattice (u of Eq. 6b) */
    double mass;           /* sum of rho (FP64 accumulation) */
    double radius;         /* equimolar radius (droplet), NaN for flat */
    long long step;        /* time steps taken since lbm_set_density */
    int status;            /* LBM_OK or LBM_ERR_DIVERGED */
    int pad_;
} lbm_obs;

typedef struct lbm_ctx lbm_ctx;

/* Fill *p with the defaults of a model (a = 0.5, b = 4, R = 1, Tr = 0.8, tau_nu = 1,
 * every derivable field NaN, precision FP32).  Never fails for a valid model. */
int lbm_params_default(int model, lbm_params* p);

/* Host-only (no GPU): resolve defaults and derived parameters of *in into *out and
 * fill *th (either may alias nothing; out and th must be non-NULL).  Follows
 * Sec. 3 and Appendix B: critical point, Maxwell densities, sigma_Li by Newton's
 * method with Simpson quadrature of Eqs. (S13)-(S14) from eps = 2, and the
 * optional width/surface-tension match.  Errors: LBM_ERR_ARG for invalid inputs
 * (including A with nu = c_s^2 (tau_nu - 1/2 - A) <= 0, Eq. 23), LBM_ERR_NOCONVERGE if a
 * solve fails, LBM_ERR_UNSUPPORTED for A != 0 with the pseudopotential model (A is a term
 * of the free-energy equilibrium, Eq. 20; the free-energy model accepts it). */
int lbm_resolve_params(const lbm_params* in, lbm_params* out, lbm_thermo* th);

/* Host-only: thermodynamically consistent densities of a 2-D droplet of radius `radius` and
 * surface tension `gamma` (Sec. 5.2, Fig. 5 discussion: the vapour density a droplet should
 * have): equal chemical potential in both phases (Eq. 29) and p(rho_l) - p(rho_v) =
 * gamma / radius (Laplace's law in 2-D), Carnahan-Starling EOS (Eq. 28) at temperature T.
 * *rho_v, *rho_l: in, the starting pair (normally the planar Maxwell densities); out, the
 * solution (Newton's method, steps down to the rounding level).  Errors: LBM_ERR_ARG for invalid
 * inputs, LBM_ERR_NOCONVERGE if Newton leaves 0 < rho_v < rho_l or does not converge. */
int lbm_kelvin_2d(double a, double b, double R, double T, double gamma, double radius, double* rho_v,
                  double* rho_l);

/* Host-only: lbm_resolve_params on each of in[0..n-1], spread over the host's cores
 * (std::thread); identical inputs are resolved once.  status[i] receives each item's
 * return code (out[i], th[i] are valid where it is LBM_OK).  Returns LBM_ERR_ARG for
 * n < 0 or NULL arrays with n > 0, else LBM_OK. */
int lbm_resolve_params_many(int n, const lbm_params* in, lbm_params* out, lbm_thermo* th, int* status);

/* Bytes of device workspace a context of this size and precision needs: two population
 * buffers (nine planes, plus the rest-population extension plane for FP32), four fields for
 * the observables, reduction partials, the one-sided walls' row solve (14 nx reals) and one
 * double per strip warp for the droplet-collision drive's stored mass (Sec. 5.4). */
size_t lbm_workspace_bytes(int precision, int nx, int ny);

/* Create a context for an nx x ny lattice (nx, ny >= 1).  Boundaries: bc_x must be
 * LBM_BC_PERIODIC; bc_y is LBM_BC_PERIODIC or LBM_BC_WALL_ZOUHE, no-slip walls on the
 * node rows 0 and ny-1 (needs ny >= 4), the parallel-plate channel of Sec. 5.3: Zou and
 * He's condition completes a wall node's incoming populations so that its momentum is
 * -F/2 (u = 0 including the half-force shift of Eq. 6b), and every stencil sees beyond
 * a wall the row mirrored through it.  The body force body_fx/fy drives the flow.
 * LBM_BC_WALL_ZOUHE_ONESIDED: the same walls, but the free-energy model takes the wall rows'
 * normal chemical-potential gradient one-sided (ghost mu(-1) = 2 mu(0) - mu(1)) and solves the
 * wall rows' densities self-consistently each step (the normal force then depends on them);
 * with a wall-normal force (body_fy, gravity) the mirrored reading drives the free-energy
 * model's neutral period-2 density mode from the walls, this one does not.  For the
 * pseudopotential model it equals LBM_BC_WALL_ZOUHE.  Any other bc returns
 * LBM_ERR_UNSUPPORTED.  stream: a cudaStream_t to run on, or
 * NULL for a stream the context creates and owns.  workspace: NULL to let the
 * library cudaMalloc its memory, or a device pointer (256-byte aligned) of at least
 * lbm_workspace_bytes(...) bytes that stays owned by the caller and must outlive
 * the context.  Parameters are resolved as in lbm_resolve_params.  Launches no
 * kernel.  *out is NULL on error. */
int lbm_create(const lbm_params* p, int nx, int ny, int bc_x, int bc_y, void* stream,
               void* workspace, size_t workspace_bytes, lbm_ctx** out);

/* Resolved parameters and thermodynamics of a context (host copies). */
int lbm_derived(const lbm_ctx* ctx, lbm_params* resolved, lbm_thermo* th);

/* Initialise f = f^eq(rho0, u = 0) of the model (Secs. 5.3-5.4: runs start from the
 * equilibrium).  rho0: host, ny*nx doubles, row-major, every entry > 0 and below the
 * EOS packing limit 4/b (else LBM_ERR_ARG).  Resets the step counter and status. */
int lbm_set_density(lbm_ctx* ctx, const double* rho0);

/* Same, rho0 already on the device (ny*nx values of the context precision). */
int lbm_set_density_device(lbm_ctx* ctx, const void* rho0_device);

/* Set / read the raw populations (host, FP64, [9][ny][nx], Eq. 2 order). */
int lbm_set_populations(lbm_ctx* ctx, const double* f);
int lbm_get_populations(lbm_ctx* ctx, double* f);

/* Gravity of the free-energy model (Eqs. 20, 21): acceleration g along -y, reference density
 * rho_ref, reference height y_ref.  The equilibrium carries p_g = rho_ref g (y - y_ref), the
 * forcing's second-order term -grad p_g, and the force the buoyancy -(rho - rho_ref) g.  With
 * rho_ref != 0 the lattice needs walls in y (p_g would jump at a periodic wrap); rho_ref = 0
 * is plain weight, -rho g, and works on periodic lattices.  Call before lbm_set_density (its
 * equilibrium includes p_g).  g = 0 switches gravity off.  Errors: LBM_ERR_ARG for a
 * non-finite value; LBM_ERR_UNSUPPORTED for the pseudopotential model or rho_ref != 0 without
 * walls.  Synchronises the stream. */
int lbm_set_gravity(lbm_ctx* ctx, double g, double rho_ref, double y_ref);

/* Droplet-collision drive of Sec. 5.4: from now on the collision of every state at time
 * t > t_on (t = steps taken since lbm_set_density) adds to the x force of each cell
 *   F_x += a_x |rho - rho_ave|,  a_x = ax_lo where x <= x_split, ax_hi where x > x_split,
 * rho_ave the mean density of that state.  The force is external: it enters the total force
 * (velocity, forcing moments) but not the interaction force of the sigma^Li term (Eq. 32).
 * Sec. 5.4 uses ax_lo = 5e-6, ax_hi = -5e-6, x_split = 100, t_on = 2000 on a 200 x 100 lattice.
 * FP32 lattices on the strip kernels run their driven instantiation: each step also sums the
 * populations it stores, which is the next state's mass, and the block-sum reduction runs
 * only at the first step of each captured 64-step graph and at single steps.  FP64 and other
 * shapes reduce every step and run the direct kernels.  The two differ only in the summation
 * order of rho_ave.  Errors: LBM_ERR_ARG for a non-finite value, LBM_ERR_UNSUPPORTED with walls (the
 * reduction sums the stored populations of a periodic lattice).  Synchronises the stream. */
int lbm_set_drive(lbm_ctx* ctx, double ax_lo, double ax_hi, double x_split, long long t_on);

/* Advance nsteps time steps (Eq. 1: collision and streaming).  Asynchronous: kernels
 * are enqueued (CUDA-graph replays of 64-step chunks plus single launches) and the
 * call returns.  Returns LBM_ERR_DIVERGED if a previous observables call saw a
 * diverged state, LBM_ERR_STATE before lbm_set_density. */
int lbm_step(lbm_ctx* ctx, long long nsteps);

/* Observables of the current state for a flat slab (geometry 0) or a centred droplet
 * (geometry 1).  Probes: flat -- columns {nx/2-1, nx/2} (liquid) and {0, nx-1}
 * (vapour); droplet -- the 4x4 block at (nx/2-2, ny/2-2) and the four 4x4 corner
 * blocks.  width = (rho_l - rho_v)/max |(rho[x+1]-rho[x-1])/2| along row 0 (flat) or
 * ny/2 (droplet); dp = p_EOS(rho_l) - p_EOS(rho_v); radius = sqrt(sum(rho - rho_v)/
 * (pi (rho_l - rho_v))).  Sets obs->status and the context status to
 * LBM_ERR_DIVERGED on NaN/Inf or rho <= 0.  Synchronises the stream. */
int lbm_observables(lbm_ctx* ctx, int geometry, lbm_obs* out);

/* Macroscopic fields of the current state (host, FP64, ny*nx each, row-major):
 * rho (Eq. 6a) and u including the half-force shift (Eq. 6b).  Any may be NULL. */
int lbm_get_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/* Populations f_i(x) (Eq. 2 order, FP64) of n cells (xs[k], ys[k]) into out[9 k + i]:
 * a few hundred values, for probing very large lattices without a full download. */
int lbm_get_populations_at(lbm_ctx* ctx, int n, const int* xs, const int* ys, double* out);

/* Device pointer of the current population buffer (9 planes, context precision; FP32
 * buffers also hold the int16 rest-population plane at 9 * pitch elements) and its plane
 * pitch in elements (plane p starts at p * pitch). */
int lbm_device_populations(lbm_ctx* ctx, void** f, long long* plane_pitch);

/* Maximum number of reduction blocks lbm_observables_fields_static accepts. */
#define LBM_STATIC_MAX_BLOCKS 1024

/* Observables of caller-owned device fields without allocating any memory.
 *
 * The paper has no counterpart: this is a library service for callers that cannot
 * call cudaMalloc -- for example a host process whose device memory is entirely
 * reserved by another allocator (a framework's caching pool that owns the GPU), or
 * a real-time loop that must not pay for an allocation or the implicit
 * synchronisation one can cause.  Everything else in this library allocates its
 * scratch inside a context workspace; this entry point needs no context.
 *
 * Inputs: rho, ux, uy -- device arrays of nx*ny values (row-major) of the given
 * precision (LBM_F32 or LBM_F64), e.g. the fields a caller keeps itself.  a, b, R, T
 * define the Carnahan-Starling pressure used for dp.  geometry and the probe, width,
 * pressure-jump and radius definitions are those of lbm_observables.  nblocks:
 * number of partial-reduction blocks, 1..LBM_STATIC_MAX_BLOCKS (else LBM_ERR_ARG).
 * Output: out_dev -- caller-owned device array of 8 doubles, written with
 * {rho_l, rho_v, width, dp, u_max, mass, radius, count of cells with NaN/Inf or
 * rho <= 0}.  stream: cudaStream_t (NULL = legacy default stream); the call only
 * enqueues work and returns.
 *
 * Scratch: a file-scope __device__ array of LBM_STATIC_MAX_BLOCKS * 3 doubles
 * (24 KiB), present on every GPU that loads the library until the process exits.
 * The first call on a device looks up that array's device address (with that device
 * current) and caches it; make that first call before any stream capture on the
 * device.  Every call shares the one array, which keeps the last call's partial
 * sums: each call writes every slot it later reads, so nothing needs clearing, but
 * calls that overlap on the GPU (different streams, no ordering) race and give wrong
 * results.  Calls no cudaMalloc, cudaFree or allocating library routine. */
int lbm_observables_fields_static(int precision, const void* rho, const void* ux, const void* uy, int nx,
                                  int ny, int geometry, double a, double b, double R, double T, int nblocks,
                                  double* out_dev, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Batched calibration sweep (pseudopotential model, FP32).                             */
/* The paper tunes sigma_Li, kappa_P and kappa_Li against coexistence densities, width  */
/* and surface tension (Sec. 3, App. B); the pseudopotential model's parameters are set */
/* from preliminary runs (Secs. 5.1-5.2).  A batch runs many such independent lattices  */
/* at once on one GPU.                                                                  */

typedef struct {
    int nx, ny;          /* lattice size (periodic); nx % 4 == 0 unless the lattice is resident */
    int geometry;        /* lbm_geometry used by lbm_batch_observables */
    int pad_;
    long long nsteps;    /* time steps of this lattice, 0 .. 2^30 */
    lbm_params params;   /* model LBM_PSEUDOPOTENTIAL, precision LBM_F32; resolved as lbm_create */
} lbm_batch_lattice;

typedef struct lbm_batch lbm_batch;

/* Create a batch of n lattices.  rho0[i]: host array of nx*ny densities of lattice i
 * (copied; f starts at f^eq(rho0, u = 0)).  Lattices whose populations, psi and rho fit in
 * one CTA's shared memory (11 nx ny floats and nx ny int16 <= 200 KB, up to 4452 cells) run resident: one CTA
 * each, all steps in shared memory, in one persistent launch.  The others run as strips
 * of a work table, one launch per step for all of them, replayed as 64-step CUDA graphs on
 * a second stream concurrently.  An autotuner picks the resident block size and the strip
 * height by timing short trials (cached per shape class); the state is re-initialised
 * afterwards.  The library allocates the device memory (one pooled cudaMalloc).
 * Errors: LBM_ERR_ARG (sizes, densities), LBM_ERR_UNSUPPORTED (other model or precision,
 * a tiled lattice with nx % 4 != 0 or nx < 8 or ny < 4), LBM_ERR_CUDA. */
int lbm_batch_create(int n, const lbm_batch_lattice* lattices, const double* const* rho0, lbm_batch** out);

/* Enqueue the whole sweep (every lattice its own nsteps); asynchronous.  A second call
 * starts again from rho0. */
int lbm_batch_run(lbm_batch* b);

/* Observables of every lattice's final state (definitions of lbm_observables) into
 * out[0..n-1]; synchronises.  LBM_ERR_STATE before lbm_batch_run. */
int lbm_batch_observables(lbm_batch* b, lbm_obs* out);

/* Final populations of lattice i (host FP64, [9][ny][nx], Eq. 2 order, post-streaming). */
int lbm_batch_populations(lbm_batch* b, int i, double* f);

/* Autotuner decisions: resident lattices, tiled work items, resident threads, strip rows. */
int lbm_batch_info(const lbm_batch* b, int* n_resident, int* n_items, int* resident_threads, int* strip_rows);

/* The stream the batch completes on (cudaStream_t). */
void* lbm_batch_stream(const lbm_batch* b);

void lbm_batch_destroy(lbm_batch* b);

/* Text of the last CUDA failure of a batch call on this host thread. */
const char* lbm_batch_last_error(void);

/* ---------------------------------------------------------------------------------- */
/* Learned calibration surrogate of the pseudopotential model (the paper has no network; */
/* it replaces the preliminary calibration runs of Secs. 5.1-5.2).  An MLP 4 -> 128 ->   */
/* 128 -> 128 -> 4 with GELU maps X = (Tr, a, b, kappa_P) to Y = (rho_l, rho_v, W,       */
/* sigma) as measured by calibration runs (flat interface: rho_l, rho_v, W; Laplace fit */
/* of droplets: sigma).  Domain of sigma: kappa_P >= 0.7.  At kappa_P = 0.4 the         */
/* calibration droplets carry large spurious currents and most diverge, so there are no  */
/* sigma labels and the sigma output there is an extrapolation, not a calibrated value;  */
/* rho_l, rho_v and W are trained for every kappa_P.                                    */
/* Internally X and (rho_l, ln rho_v, W, sigma) are standardised                        */
/* with stats16 = {mean X[4], std X[4], mean Y'[4], std Y'[4]} (Y' with ln rho_v).      */
/* Parameters: 34,180 FP32 values, per layer l = 0..3 the weights W_l [out][in]          */
/* (row-major) followed by the bias b_l.  Training: full-batch MSE in the standardised  */
/* space, Adam with bias correction, cosine learning-rate decay, FP32 kernels.          */
/* Inference: one fused kernel, BF16 inputs and weights, FP32 accumulation and          */
/* epilogue (see the inference modes).  Host arrays are row-major n x 4 floats.  One    */
/* surrogate owns a stream and                                                          */
/* device buffers; calls on the same surrogate must not overlap.                       */

typedef struct {
    int iterations;      /* Adam steps (full batch each) */
    float lr, lr_min;    /* cosine decay from lr to lr_min over the run */
    float beta1, beta2, eps, weight_decay;  /* Adam; decoupled weight decay */
} lbm_train_cfg;

typedef struct lbm_surrogate lbm_surrogate;

/* Number of parameters (34,180). */
int lbm_surrogate_num_params(void);

/* New surrogate with the given standardisation (std entries > 0, else LBM_ERR_ARG) and
 * seeded uniform He initialisation (zero biases). */
int lbm_surrogate_create(const float* stats16, unsigned seed, lbm_surrogate** out);
int lbm_surrogate_stats(const lbm_surrogate* m, float* stats16);
int lbm_surrogate_set_params(lbm_surrogate* m, const float* params);
int lbm_surrogate_get_params(lbm_surrogate* m, float* params);

/* MSE loss (standardised space) and its gradient w.r.t. the parameters for the n
 * samples X, Y (host) at the current parameters; either output may be NULL.  A NaN
 * entry of Y other than rho_v is a missing target (left out of the mean); every rho_v
 * must be finite and > 0, else LBM_ERR_ARG. */
int lbm_surrogate_loss_grad(lbm_surrogate* m, const float* X, const float* Y, int n, float* loss, float* grad);

/* Train on n samples (host X, Y as for lbm_surrogate_loss_grad; missing targets allowed).
 * *final_loss: loss before the last update.
 * LBM_ERR_DIVERGED if the loss became non-finite. */
int lbm_surrogate_train(lbm_surrogate* m, const float* X, const float* Y, int n, const lbm_train_cfg* cfg,
                        float* final_loss);

/* Inference modes of the fused tensor-core kernel (BF16 operands, FP32 accumulation):
 * LBM_INFER_SPLIT_BF16 carries every operand as BF16 hi + lo parts and sums three BF16
 * products per tile (result within ~2^-15 of the FP32 network); LBM_INFER_BF16 rounds
 * every operand to BF16 once (relative 2^-8 per operand). */
enum { LBM_INFER_SPLIT_BF16 = 0, LBM_INFER_BF16 = 1 };

/* Inference of n queries (host in, host out) in the given mode. */
int lbm_surrogate_predict(lbm_surrogate* m, const float* X, int n, float* Y, int mode);

/* Inference on device arrays (n x 4 floats each) enqueued on stream (NULL: the
 * surrogate's own); asynchronous. */
int lbm_surrogate_predict_device(lbm_surrogate* m, const float* X_dev, int n, float* Y_dev, int mode, void* stream);

/* The FP32 training forward pass, de-standardised (host in, host out). */
int lbm_surrogate_predict_fp32(lbm_surrogate* m, const float* X, int n, float* Y);

void lbm_surrogate_destroy(lbm_surrogate* m);

/* Text of the last CUDA failure of a surrogate call on this host thread. */
const char* lbm_surrogate_last_error(void);

/* Checkpoint: write/read the populations (FP64, the FP32 free-energy rest population with its
 * extension), step counter and resolved parameters (binary).  lbm_load returns LBM_ERR_ARG when
 * the file's lattice size, model, precision or any resolved parameter differs from the
 * context's (a state of one temperature or EOS is not a state of another), LBM_ERR_IO when the
 * file cannot be read. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/* The stream a context runs on (cudaStream_t). */
void* lbm_stream(const lbm_ctx* ctx);

void lbm_destroy(lbm_ctx* ctx);
const char* lbm_strerror(int status);

/* Self-test of the bounded device waits that guard the TMA pipelines (the paper has no
 * counterpart; failure detection of this library).  Launches one 64-thread block that
 * waits on a shared-memory mbarrier phase for at most `polls` polls (1 .. 2^22): with
 * arrive = 0 nothing completes the phase, the wait gives up and the call returns
 * LBM_ERR_TIMEOUT while the device context stays usable; with arrive = 1 the phase is
 * completed first and the call returns LBM_OK.  Synchronises the device.  LBM_ERR_ARG for
 * other arguments, LBM_ERR_CUDA on a CUDA failure. */
int lbm_selftest_bounded_wait(int arrive, int polls);

/* Library build information: "sm_103a ..." string. */
const char* lbm_build_info(void);

/* Text of the last CUDA failure behind an LBM_ERR_CUDA on this host thread. */
const char* lbm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
