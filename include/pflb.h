/*
 * pflb.h -- C ABI of the GB300 coupled phase-field lattice Boltzmann step.
 *
 * The library advances two lattice Boltzmann population sets coupled through
 * the order parameter phi, as compared in "Comparative study and critical
 * assessment of phase-field lattice Boltzmann models for laminar and turbulent
 * two-phase flow simulations" (arXiv 2511.11360):
 *   g_a (phase field; D2Q9 in 2D, D3Q7 in 3D) and f_b (hydrodynamics; D2Q9 in
 *   2D, D3Q19 in 3D), both relaxed by BGK with a source weighted by
 *   (1 - 1/(2 tau)) (Sec. II B, Eqs. fakhari_g_simplified and
 *   fakhari_f_simplified), with the equilibria and sources of one of four
 *   families (Sec. II C, II D) and the isotropic central stencils of Sec. III.
 *
 * Conventions for every entry point:
 *   - Return value: PFLB_OK (0) or a negative pflb_status. Errors are sticky
 *     per handle; pflb_last_error() gives the message.
 *   - Pointers documented "host or device" may point to pageable host memory,
 *     pinned host memory or device memory of the handle's device (unified
 *     addressing decides the copy direction). The caller owns every pointer it
 *     passes; the library never frees or retains them past the call.
 *   - The library owns its population buffers (device memory it allocates in
 *     pflb_create and frees in pflb_destroy).
 *   - Work is issued on the CUDA stream given at creation (NULL = legacy
 *     default stream). Calls that return data to the host synchronise that
 *     stream; pflb_step does not.
 *   - There is no CPU implementation: without a CUDA device every call that
 *     needs one returns PFLB_ECUDA.
 *   - Field layout: cell (x, y[, z]) has linear index x + nx*(y + ny*z), x
 *     fastest. Scalar fields are N = nx*ny*nz floats; vector fields are d
 *     consecutive scalar fields (x component first).
 *   - Units are lattice units (dx = dt = 1).
 */
#ifndef PFLB_H
#define PFLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pflb_status {
  PFLB_OK = 0,
  PFLB_EINVAL = -1,    /* invalid argument or parameter */
  PFLB_ENOMEM = -2,    /* device allocation failed */
  PFLB_ECUDA = -3,     /* CUDA runtime error or no device */
  PFLB_EUNSTABLE = -4, /* a step produced rho <= 0 or a non-finite phi or u */
  PFLB_ETIMEOUT = -5   /* a bounded device-side wait expired */
} pflb_status;

/* Phase-field model family (the four categories of Sec. II C and II D, and
 * Liang2018, the second conservative Allen-Cahn model of Sec. II C 2). */
typedef enum pflb_family {
  PFLB_CAC_FAKHARI2017 = 0, /* conservative Allen-Cahn, Sec. II C 1 */
  PFLB_NLAC_CHAI2018 = 1,   /* nonlocal Allen-Cahn, Sec. II C 3 */
  PFLB_HAC_HU2019 = 2,      /* hybrid Allen-Cahn with global weight lambda, Sec. II C 4 */
  PFLB_CH_LIANG2014 = 3,    /* Cahn-Hilliard with incompressible NS, Sec. II D 1 */
  PFLB_CAC_LIANG2018 = 4,   /* conservative Allen-Cahn with the conservative NS form:
                               first-order g_eq, pressure-based f_eq, d_t(phi u) in G,
                               Sec. II C 2 (Eqs. liang_geq, liang_feq, liang_G_final,
                               liang_F_final, liang_velocity_update, liang_p_update) */
  PFLB_CH_BAO2024 = 5,      /* Cahn-Hilliard with singular mobility M = 4 M_0 |phi - phi_H|
                               |phi - phi_L| / (phi_H - phi_L)^2 (M_0 = params.M), lattice
                               kinetic scheme and quasi-incompressible NS, Sec. II D 3
                               (Eqs. bao_g_eq, bao_f_eq, bao_Mphi, bao_v, Yang_G, Yang_F,
                               yang_update). Constant tau_phi = M_0/(c_s^2 eta) + 1/2 and
                               tau = max(nu_H, nu_L)/c_s^2 + 1/2. Periodic domains, FP32
                               storage, D2Q9 / D3Q19 + D3Q7; stepped by four passes
                               (phi, mu, u and p, collision) instead of the fused kernel */
  PFLB_HAC_LIU2023 = 6      /* hybrid Allen-Cahn with lambda(x) = 1 within 3 xi of the
                               interface and 0 elsewhere, from the log-transform predictor
                               and reinitialisation (ceil(6 xi) Godunov steps of 1/2) of a
                               signed distance; Liang2018's equilibria, forcing and updates,
                               Sec. II C 5 (Eqs. Liu_G, Liu_F); gamma over the lambda = 0
                               region. Periodic domains, FP32 storage, D2Q9 / D3Q19 + D3Q7;
                               stepped by passes (phi*, reinitialisation, lambda and gamma,
                               phi, collision) */
} pflb_family;

/* Population storage in device memory. Arithmetic is always FP32. The 16-bit
 * forms store (value - w_a c) / s_a: the deviation from the rest state (c =
 * (phi_H + phi_L)/2 for g, 0 for f; w_a = 1 where the weight is zero) scaled by
 * s_a, the power of two nearest w_a (exact both ways, so only the 16-bit
 * rounding of the deviation is lost). */
typedef enum pflb_storage {
  PFLB_FP32 = 0,
  PFLB_FP16_DEV = 1,
  PFLB_BF16_DEV = 2
} pflb_storage;

/* Nondimensional parameters of one run (lattice units). */
typedef struct pflb_params {
  int32_t dim;          /* 2 or 3 */
  int32_t nx, ny, nz;   /* cells per axis; nz must be 1 in 2D */
  int32_t family;       /* pflb_family */
  int32_t storage;      /* pflb_storage */
  int32_t bc_y;         /* 0 periodic; 1 resting walls; 2 walls moving in x
                           (2D only): halfway bounce-back at y = -1/2 and
                           y = ny - 1/2, mirrored phi ghosts */
  int32_t visc_interp;  /* 0 linear kinematic viscosity (Eq. fakhari_mu_update);
                           1 linear dynamic (Eq. mu_linear); 2 inverse-linear
                           (Eq. mu_inverse); 3 logarithmic (Eq. mu_log) */
  int32_t freeze_phi;   /* 1: the phase field is held fixed (Sec. III D) */
  int32_t obs_capacity; /* length of the per-step observables ring, >= 1 */
  double phi_H, phi_L;  /* bulk order parameters (Sec. II: 1 and 0) */
  double rho_H, rho_L;  /* bulk densities */
  double nu_H, nu_L;    /* bulk kinematic viscosities; tau = nu/c_s^2 + 1/2 */
  double sigma;         /* surface tension */
  double W;             /* interface thickness xi */
  double M;             /* mobility M_phi; tau_phi = M/c_s^2 + 1/2
                           (M/(eta c_s^2) + 1/2 for Cahn-Hilliard) */
  double lambda_hybrid; /* Hu2019 weight lambda (Sec. III: 0.9) */
  double eta_ch;        /* Liang2014 eta (paper leaves it free; 1) */
  double gravity[3];    /* body force F_b = rho * gravity */
  double force_density[3]; /* uniform force density added to F_b */
  double lundgren_A;    /* linear forcing F = A rho u (turbulence driver) */
  double wall_u[2];     /* x velocity of the bottom and top wall (bc_y = 2) */
  double grad_eps;      /* regularisation of the interface normal,
                           n = grad phi / sqrt(|grad phi|^2 + grad_eps^2)
                           (1e-4; the paper leaves n undefined at 0) */
  int32_t lattice_f;    /* 3D hydrodynamic lattice: 19 (D3Q19; 0 means 19) or 27
                           (D3Q27, the paper's 3D lattice, Sec. IV); 2D: 0 or 9 */
  int32_t collision;    /* 0 BGK (Sec. II B); 1 multiple-relaxation-time (Sec. IV,
                           D3Q27 only): raw moments sum f e_x^i e_y^j e_z^k,
                           i,j,k <= 2; conserved, first-order and traceless
                           second-order moments at 1/tau, the trace of the
                           second-order moments at mrt_s_bulk, orders >= 3 at
                           mrt_s_ho; forcing (I - S/2) in moment space */
  double mrt_s_bulk;    /* MRT rate of the second-moment trace, in (0, 2) */
  double mrt_s_ho;      /* MRT rate of the moments of order >= 3, in (0, 2) */
} pflb_params;

/* Bookkeeping of one state: sums over all cells of its macroscopic fields. */
typedef struct pflb_obs {
  int64_t step;         /* time level the fields belong to */
  double sum_phi;       /* sum of phi (FP64 accumulation of FP32 terms) */
  double vol_smooth;    /* sum (phi - phi_L)/(phi_H - phi_L), Eq. volume_continuous */
  int64_t vol_count;    /* number of cells with phi > (phi_H + phi_L)/2 (Sec. IV A) */
  double ke;            /* sum 1/2 rho |u|^2 */
  double phi_max, phi_min;
  double centroid[3];   /* sum x c / sum c with c = (phi - phi_L)/(phi_H - phi_L) */
  int32_t status;       /* PFLB_OK, PFLB_EUNSTABLE or PFLB_ETIMEOUT */
  int32_t pad;
} pflb_obs;

typedef struct pflb_handle pflb_handle;

/* Validate the parameters, allocate the populations on the current device
 * and bind the handle to `cuda_stream` (a cudaStream_t, may be NULL).
 * PFLB_EINVAL for: dim not 2/3, sizes < 1, nz != 1 in 2D, walls in 3D or with ny < 4,
 * phi_H == phi_L, W <= 0, sigma < 0, tau <= 1/2 for either phase, tau_phi <=
 * 1/2, unknown family/storage/interpolation, obs_capacity < 1. */
int pflb_create(const pflb_params* params, void* cuda_stream, pflb_handle** out);

/* Set the state to equilibrium with the given phi and u and pressure 0
 * (step count 0). phi0: N floats; u0: d*N floats or NULL for rest; host or
 * device. For Cahn-Hilliard the chemical potential of phi0 enters g_eq
 * (Eq. liang2_geq), computed with the Sec. III stencils. */
int pflb_init(pflb_handle* h, const float* phi0, const float* u0);

/* Advance nsteps >= 0 time steps, asynchronously on the handle's stream.
 * One step: the macroscopic stage (phi, rho, nu, the stencils of Sec. III,
 * chemical potential, forces, u, p), BGK collision of g and f with the
 * family's equilibria and sources, streaming (g: two-array push; f: AA-pattern
 * in place), and the observables of the pre-collision state into the
 * per-step ring. Nonlocal and hybrid families first reduce the two integrals
 * of Eq. (lagrange_multiplier) over the whole domain. Returns the sticky
 * status known so far (instability is reported once the stream is
 * synchronised). */
int pflb_step(pflb_handle* h, int64_t nsteps);

/* Wait for the handle's stream; returns PFLB_EUNSTABLE if any step flagged
 * an instability, PFLB_ETIMEOUT if a step's staging copies did not complete
 * within the kernel's bounded wait (the step's results are then invalid). */
int pflb_sync(pflb_handle* h);

/* Observables of the current state (time level pflb_step_count). Runs one
 * read-only pass, synchronises. */
int pflb_observables(pflb_handle* h, pflb_obs* out);

/* Copy the observables the last min(n, steps taken, obs_capacity) steps
 * recorded (each the pre-collision state of its step), oldest first.
 * *written receives the count. out: n pflb_obs in host memory. */
int pflb_obs_history(pflb_handle* h, pflb_obs* out, int32_t n, int32_t* written);

/* Macroscopic fields of the current state, as the next step's collision
 * would compute them: phi (N), u (d*N, the force-corrected velocity), p (N,
 * the thermodynamic pressure). Any pointer may be NULL. Host or device. */
int pflb_get_fields(pflb_handle* h, float* phi, float* u, float* p);

/* Size in floats of the canonical state: Qg*N populations g, Qf*N
 * populations f (both post-streaming, i.e. what the next step reads, in the
 * velocity order of pflb_lattice; Qf = 27 with lattice_f = 27), then for
 * Liang2014 and Liang2018 d*N values of phi*u of the previous step. */
int64_t pflb_state_floats(const pflb_handle* h);

/* Write / read the canonical FP32 state (host or device buffer of
 * pflb_state_floats floats). pflb_load keeps the step count. For FP16/BF16
 * storage the values are decoded / encoded. */
int pflb_save(pflb_handle* h, float* state);
int pflb_load(pflb_handle* h, const float* state);

/* Time levels advanced since pflb_init. */
int64_t pflb_step_count(const pflb_handle* h);

/* Algorithmic device-memory bytes per lattice update of one step (each
 * stored population read once and written once, plus the phi*u field for
 * Cahn-Hilliard and the extra read of g for the nonlocal reduction). */
double pflb_bytes_per_update(const pflb_handle* h);

/* Launch shape of the fused step: cells per block along the marching axis
 * (z in 3D, y in 2D), 0 = library default (about eight blocks per SM,
 * marches of 4 to 128 planes; TMA-staged steps march at most 32 planes on
 * even AA steps). The state after a step does not depend on it. */
int pflb_set_chunk(pflb_handle* h, int32_t chunk);

/* How the fused 3D step stages each plane's populations in shared memory.
 * TMA staging: tensor-memory-accelerator bulk copies of boxes of the
 * population arrays (a 5-D view: lane, slot, 32-cell x-block, y, z),
 * completed on shared-memory barriers whose waits are bounded; available
 * where the domain is 3D, nx is a multiple of 32, ny a multiple of the
 * tile's rows (4) and at least 8, and the family is Fakhari2017, Chai2018,
 * Hu2019 or Liang2018. cp.async staging: per-thread asynchronous copies.
 *   mode 0: cp.async staging everywhere;
 *   mode 1: TMA staging where available;
 *   mode 2 (the default): TMA staging where available and measured
 *           faster: FP32 storage on D3Q19 (both AA parities) and on the
 *           even AA steps of D3Q27; cp.async on the odd D3Q27 steps (27
 *           shifted boxes per plane at three blocks per SM measured slower)
 *           and for the 16-bit forms (bound by instruction issue, where the
 *           per-thread barrier waits cost more than the copies they
 *           replace).
 * Both stagings compute bit-identical populations. PFLB_EINVAL for another
 * mode. */
int pflb_set_staging(pflb_handle* h, int32_t mode);

/* 1 if the next step of h (its AA parity included) uses TMA staging, 0 if
 * it uses cp.async staging, PFLB_EINVAL for a NULL handle. */
int pflb_get_staging(const pflb_handle* h);

/* Failure-injection hook for tests of the bounded waits (the paper has no
 * counterpart). With polls > 0, every block of each following TMA-staged
 * step first waits on a shared-memory barrier that nothing completes, gives
 * up after `polls` polls and reports a timed-out wait in that step's status;
 * the step itself then runs unchanged. pflb_sync and pflb_observables turn
 * that status into PFLB_ETIMEOUT, which, like every error but
 * PFLB_EUNSTABLE, stays on the handle (pflb_step and pflb_init refuse
 * further work; the handle can still be read and destroyed, and other
 * handles are unaffected). polls = 0 switches the hook off; steps staged by
 * cp.async have no waits and ignore it. PFLB_EINVAL for polls outside
 * [0, 65536] or, with polls > 0, a handle whose next step is not
 * TMA-staged (pflb_get_staging). */
int pflb_inject_wait_timeout(pflb_handle* h, int32_t polls);

/* Velocity set of a lattice in canonical order. which: 0 = phase field (g),
 * 1 = hydrodynamics (f: D2Q9 / D3Q19), 2 = the D3Q27 hydrodynamic lattice
 * (dim 3 only). q receives Q; e receives 3*Q ints (ex, ey, ez per
 * velocity, ez = 0 in 2D) and w receives Q weights; either may be NULL. */
int pflb_lattice(int32_t dim, int32_t which, int32_t* q, int32_t* e, double* w);

int pflb_destroy(pflb_handle* h);
const char* pflb_last_error(const pflb_handle* h);

/* ---------------------------------------------------------------------------
 * Adjoint: gradients of a droplet objective by a reverse sweep.
 *
 * For the conservative Allen-Cahn family (Fakhari2017, Sec. II C 1) on a
 * periodic domain at density ratio 1 (rho_H = rho_L; the viscosities may
 * differ, linear interpolation), FP32 storage, 2D or 3D, pflb_adjoint runs
 * nsteps time levels from the state pflb_init made and returns the
 * objective of the final state
 *     J = w_vol V_s + sum_k w_cen[k] c_k,
 *     V_s = sum_x (1 + tanh((phi - phi_0)/eps_v))/2   (smooth volume),
 *     c_k = sum_x x_k phi / sum_x phi                 (centroid, cell-index
 *                                                      coordinates)
 * with phi = sum_a g_a of the final state, and its derivatives with respect
 * to the mobility M, the surface tension sigma, the interface width W and
 * the initial velocity field u0 given to pflb_init (through the
 * equilibrium initial populations). The reverse sweep differentiates the
 * step exactly as the library computes it (stencils of Sec. III,
 * regularised normal of the counter term), in FP32 with FP64 parameter sums.
 *
 * Checkpointing: the forward sweep keeps every checkpoint_every-th state
 * (0 = ceil(sqrt(nsteps))); the reverse sweep recomputes each segment from
 * its checkpoint and walks it backwards. Device memory: (nsteps/K + K + 3)
 * canonical states (pflb_state_floats floats each) plus small buffers,
 * allocated for the call and freed before it returns.
 *
 * The handle must be initialised and at step 0; on success it is left at
 * step nsteps with the state and observables records pflb_step(h, nsteps)
 * gives. du0: NULL or d*N floats (host or device, layout of the u0 given to
 * pflb_init) that receive dJ/du0. Synchronises the stream.
 *
 * Errors: PFLB_EINVAL for another family, walls, 16-bit storage, a density
 * contrast, a non-linear viscosity interpolation, freeze_phi, a handle not at
 * step 0, nsteps < 1 or eps_v <= 0; PFLB_ENOMEM when the checkpoints do not
 * fit; PFLB_EUNSTABLE when the final sum of phi is zero or not finite.
 *
 * Conditioning: where the counter term of Eq. (fakhari_G_modified) acts on
 * a droplet whose centre is not saturated (R/W below about 2.5 at
 * grad_eps = 1e-4), its regularised normal is anti-diffusive there and the
 * model amplifies perturbations; gradients are then dominated by that
 * amplification (finite differences of such runs are noise).
 * ------------------------------------------------------------------------- */
typedef struct pflb_obs_weights {
  double w_vol;     /* weight of V_s */
  double w_cen[3];  /* weights of the centroid components (x, y, z; z unused in 2D) */
  double eps_v;     /* width of the smooth volume indicator, > 0 (e.g. 0.05) */
} pflb_obs_weights;

typedef struct pflb_grads {
  double J;                          /* objective of the final state */
  double vol_smooth;                 /* V_s of the final state */
  double centroid[3];                /* c_k of the final state */
  double dJ_dM, dJ_dsigma, dJ_dW;    /* parameter derivatives */
  int64_t steps;
  int32_t checkpoint_every;          /* K used */
  int32_t checkpoints;               /* states kept by the forward sweep */
} pflb_grads;

int pflb_adjoint(pflb_handle* h, int64_t nsteps, int32_t checkpoint_every, const pflb_obs_weights* w,
                 pflb_grads* out, float* du0);

/* ---------------------------------------------------------------------------
 * Batched step: many independent 2D domains in one persistent launch.
 *
 * A batch owns n domains (pflb_handle each) of any size, family and
 * parameters -- a parameter sweep such as the four-family comparisons of
 * Secs. III and IV -- and advances all of them one time level per kernel launch.
 * Every (domain, tile) pair is an entry of a work list that resident blocks
 * claim from an atomic counter, so domains of uneven size share the GPU
 * without one launch per domain. Each domain's per-cell update is the one of
 * pflb_step: a domain advanced in a batch has bitwise the same state as the
 * same domain advanced alone; its observables agree up to the order of the
 * FP64 sums (the nonlocal gamma of Chai2018/Hu2019 likewise).
 *
 * Restrictions: dim = 2 and FP32 storage for every domain (PFLB_EINVAL
 * otherwise). Each domain keeps an observables ring of 2 records (the
 * obs_capacity field is overridden).
 *
 * The domains are ordinary handles: pflb_batch_domain() returns domain i,
 * on which pflb_init, pflb_get_fields, pflb_observables, pflb_save,
 * pflb_load, pflb_obs_history and even pflb_step may be called (the batch
 * notices a domain advanced on its own). The batch destroys them; never
 * call pflb_destroy on one. All work is issued on the batch's stream (given
 * at creation; every domain uses it).
 * ------------------------------------------------------------------------- */
typedef struct pflb_batch pflb_batch;

/* Launch shape of the batched step. tile_a: cells per tile (and threads per
 * block) along x, one of 64, 128, 256. chunk: rows per tile along y (>= 1).
 * blocks_per_sm: resident blocks per SM of the persistent grid (0 = as many
 * as fit). ms_per_step: the measured time of one batched step (autotuner
 * output; ignored on input). from_cache: 1 if the autotuner read the shape
 * from its cache file. */
typedef struct pflb_batch_launch {
  int32_t tile_a, chunk, blocks_per_sm, from_cache;
  double ms_per_step;
} pflb_batch_launch;

/* Create n domains from params[0..n) (host array). Each needs dim = 2,
 * storage = PFLB_FP32. On error *out may still receive a batch that carries
 * the message (read it with pflb_batch_last_error, then destroy it). */
int pflb_batch_create(const pflb_params* params, int32_t n, void* cuda_stream, pflb_batch** out);

/* Number of domains, and domain i (0 <= i < n; NULL when out of range). */
int32_t pflb_batch_size(const pflb_batch* b);
pflb_handle* pflb_batch_domain(pflb_batch* b, int32_t i);

/* Initialise domain i as pflb_init does (host or device phi0, u0). */
int pflb_batch_init(pflb_batch* b, int32_t i, const float* phi0, const float* u0);

/* Advance every domain nsteps time levels. Asynchronous on the batch's
 * stream. Every domain must have been initialised. */
int pflb_batch_step(pflb_batch* b, int64_t nsteps);

/* Replay the step through CUDA graphs (on = 1) or launch it directly (0,
 * the default). With graphs, the launches of two consecutive steps (the
 * gamma pre-pass where the batch holds nonlocal/hybrid domains, then the
 * persistent step kernel, twice) are captured once on an internal stream
 * and replayed; the batch's stream waits for the replay through events. */
int pflb_batch_set_graph(pflb_batch* b, int32_t on);

/* Set / read the launch shape (see pflb_batch_launch). */
int pflb_batch_set_launch(pflb_batch* b, const pflb_batch_launch* cfg);
int pflb_batch_get_launch(const pflb_batch* b, pflb_batch_launch* out);

/* Choose the launch shape by timing candidate shapes (tile_a in {64, 128,
 * 256}, chunk in {8, 16, 32, 64}, blocks_per_sm in {all that fit, half})
 * over steps_per_trial steps each (>= 1), then restore every domain's state
 * and observables bit for bit, so tuning does not advance the batch.
 * cache_path (may be NULL): a text file keyed by the device and the batch's
 * (size, family) list; a matching line is used without timing, a new result
 * is appended. The chosen shape is applied and written to *out (may be
 * NULL). Synchronises the stream. */
int pflb_batch_autotune(pflb_batch* b, int32_t steps_per_trial, const char* cache_path,
                        pflb_batch_launch* out);

/* The observables each domain recorded during its most recent step (as the
 * last record of pflb_obs_history), for all n domains: out is a host array
 * of n pflb_obs. Synchronises the stream. Returns PFLB_EUNSTABLE if any
 * domain's record has that status. */
int pflb_batch_observables(pflb_batch* b, pflb_obs* out);

/* Synchronise the batch's stream; PFLB_EUNSTABLE if the most recent step of
 * any domain flagged rho <= 0 or a non-finite phi or u. */
int pflb_batch_sync(pflb_batch* b);

/* Cells of all domains (one batched step performs this many lattice
 * updates), and the algorithmic device-memory bytes of one batched step
 * (the sum over domains of pflb_bytes_per_update x cells). */
int64_t pflb_batch_cells(const pflb_batch* b);
double pflb_batch_bytes_per_step(const pflb_batch* b);

int pflb_batch_destroy(pflb_batch* b);
const char* pflb_batch_last_error(const pflb_batch* b);

/* ---------------------------------------------------------------------------
 * Allocation-free phase-field sums. (The paper has no counterpart: this is a
 * service of the library for callers that cannot allocate device memory.)
 *
 * Some callers must not call cudaMalloc: an application that manages every
 * byte of device memory through its own allocator and forbids allocations
 * behind its back, or a latency-bound loop that cannot pay for the
 * device-wide synchronisation that cudaMalloc and cudaFree imply. For them,
 * pflb_phase_sums_static computes the phase-field part of pflb_observables --
 * sum_phi, vol_smooth, vol_count, phi_max, phi_min and the centroid -- of a
 * phi field the caller owns, without allocating anything: no cudaMalloc, no
 * cudaFree, no allocating library call. Its scratch space is a file-scope
 * device array of PFLB_STATIC_PARTIALS + 1 records (about 230 KB) that every
 * GPU loading the library holds until the process exits.
 *
 *   params  only dim, nx, ny, nz, phi_H, phi_L are read;
 *   phi     device pointer to N = nx*ny*nz floats (field layout as above);
 *   out     host struct; ke is 0 and step is -1 (no velocity, no handle);
 *   stream  cudaStream_t (may be NULL); the call synchronises it.
 *
 * Returns PFLB_EINVAL for a NULL argument, bad sizes, phi_H == phi_L, or
 * N > PFLB_STATIC_MAX_CELLS (2^28 cells: the scratch holds one partial record
 * per 65536 cells); PFLB_ECUDA without a device or on a CUDA error. Every
 * call looks up the scratch array's device address on the current device
 * (cudaGetSymbolAddress, no allocation), so a device reset or a new context
 * leaves no stale address behind. The call copies its result to the host
 * and synchronises the stream: it must not be called while that stream is
 * being captured into a CUDA graph. The result does not depend on the
 * previous call (every record used is written before it is read), but all
 * calls share the array: calls that overlap on the GPU (different streams or
 * host threads) race and must be serialised.
 *
 * The library cannot check phi's length or residence: a host pointer or a
 * buffer shorter than N floats is read out of bounds. The Python binding
 * refuses such buffers before the call.
 * ------------------------------------------------------------------------- */
#define PFLB_STATIC_PARTIALS 4096
#define PFLB_STATIC_CELLS_PER_BLOCK 65536LL
#define PFLB_STATIC_MAX_CELLS (PFLB_STATIC_PARTIALS * PFLB_STATIC_CELLS_PER_BLOCK)
int pflb_phase_sums_static(const pflb_params* params, const float* phi, pflb_obs* out,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PFLB_H */
