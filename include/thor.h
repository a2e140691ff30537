/*
 * thor.h -- C ABI of the GB300 resonant-line Monte Carlo library (libthor.so).
 *
 * The library implements the data-parallel hot path of the method described by
 * THOR (Byrohl & Nelson, "thor: a GPU-accelerated Monte Carlo radiative transfer
 * code for resonant lines", arXiv:2507.11603): the Lyman-alpha photon-packet loop
 * (Sec. 3.4: emission, propagation through gridless shells or a uniform grid,
 * interaction, resonant and dust scattering, peeling-off, escape) and the
 * Lyman-alpha forest optical-depth ray-march (Sec. 3.5.2, Eq. 11), on one CUDA
 * device (sm_103a).
 *
 * Conventions
 *  - Every call returns an int status: THOR_OK (0) or a negative THOR_ERR_* code;
 *    thor_last_error() then holds a one-line message.  No call aborts the process.
 *  - Pointers are plain host or device pointers; `mem_kind` says which
 *    (THOR_MEM_HOST or THOR_MEM_DEVICE).  Input arrays are only read during the
 *    call (geometry creation copies and packs them).  Output buffers are owned by
 *    the caller and must hold the sizes stated below.
 *  - 3-D fields are C-contiguous arrays of shape (nz, ny, nx): cell (ix, iy, iz)
 *    is element ix + nx * (iy + ny * iz).  Positions are in cell units.
 *  - Frequencies are lab-frame velocity offsets X = c (nu - nu0) / nu0 in km/s
 *    (positive = blue); velocities in km/s; the gas-frame dimensionless frequency
 *    is x = (X - v . k) / v_th (Sec. 2.3.1).
 *  - Results are deterministic for fixed (seed, photon ids): photon i draws from the
 *    Philox4x32-10 blocks keyed by the run seed with counter (i, event, block), and
 *    all spectrum tallies are integer counts.
 *  - Calls on one context are serialised by the caller; contexts are independent.
 */
#ifndef THOR_H
#define THOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THOR_OK 0
#define THOR_ERR_INVALID_ARG (-1) /* bad pointer, size or parameter */
#define THOR_ERR_OOM (-2)         /* device allocation failed */
#define THOR_ERR_CAPACITY (-3)    /* request exceeds a configured capacity */
#define THOR_ERR_TIMEOUT (-4)     /* a bounded wait ran out */
#define THOR_ERR_DEVICE (-5)      /* CUDA error (message in thor_last_error) */
#define THOR_ERR_CANCELLED (-6)   /* served request was cancelled */
#define THOR_ERR_NOT_FOUND (-7)   /* unknown ticket */

#define THOR_MEM_HOST 0
#define THOR_MEM_DEVICE 1

/* Phase function of resonant scattering (Sec. 2.3.1): isotropic, dipole
 * P(mu) = 3/8 (1 + mu^2), or the 1:2 isotropic:dipole mix in the line core
 * (|x_atom| < 0.2) with pure dipole in the wings. */
#define THOR_PHASE_ISOTROPIC 0
#define THOR_PHASE_DIPOLE 1
#define THOR_PHASE_MIXED 2

typedef struct thor_ctx* thor_ctx_t;
typedef struct thor_geom* thor_geom_t;
typedef struct thor_server* thor_server_t;

/* ---- context --------------------------------------------------------------------- */

/* Create a context on CUDA device `device` (Sec. 3.6.1: one compute thread drives
 * one device).  *out receives the handle.  Errors: INVALID_ARG, DEVICE. */
int thor_init(int device, thor_ctx_t* out);
/* Release the context and everything it allocated.  NULL is ignored. */
void thor_destroy(thor_ctx_t ctx);
/* Last error message of the context (never NULL; "" after success).  With ctx NULL,
 * the message of the last failed thor_init. */
const char* thor_last_error(thor_ctx_t ctx);
/* Use `cuda_stream` (a cudaStream_t, may be NULL = legacy default stream) for all
 * subsequent work of this context. */
int thor_ctx_set_stream(thor_ctx_t ctx, void* cuda_stream);
/* Launch configuration of the persistent photon loops: threads per block (multiple
 * of 32, <= 256) and resident blocks per SM (0 = occupancy maximum). */
int thor_ctx_set_launch(thor_ctx_t ctx, int block_size, int blocks_per_sm);

/* Tail compaction of the gridless photon loop: once no new photons are left, a warp
 * with fewer than spill_below (0..32; 0 = off, the default) live lanes saves its packets
 * and exits, and the next launch repacks the survivors (a few per warp, spread over all
 * schedulers), for at most max_phases launches (default 24).  Off by default: a run that
 * is bound by the latency of its longest photons finishes soonest when each of them
 * stays alone in its warp, which the single launch already gives.  Runs with fewer
 * photons than lanes spread them over all warps either way.  Results do not depend on
 * these settings. */
int thor_ctx_set_tail(thor_ctx_t ctx, int spill_below, int max_phases);
/* Pipelined events of the gridless photon loop on homologous shells.  In warps with at
 * most pipe_lanes live packets (0..32; 0 = never; default 32) each event first tries its
 * line-core form (start-point step inside the safety ball, resonant scattering at |x| <= 2,
 * u_par sample accepted within two trials), with the next event's random words, its optical depth and
 * the outgoing direction formed beside the frequency chain, and runs the general event
 * from the same words otherwise.  In warps with at most burst_lanes live packets (0..32;
 * default 1; only where events are pipelined) a packet runs up to 32 core events back to
 * back in one tight loop, for the lone lanes of a run's tail; with at most 10 such packets
 * the warp's other lanes form their next events' random words ahead (cooperative burst).  Both forms evaluate an event
 * exactly as the general event does, so results do not depend on these settings (only the
 * time to reach them does). */
int thor_ctx_set_bursts(thor_ctx_t ctx, int pipe_lanes, int burst_lanes);
/* Work sharing in the tail of a one-launch gridless run (share 1, the default; 0 = off).
 * Once no new photons are left, a warp whose packets have all finished waits (sleeping)
 * for a packet that a warp with several live packets gives away, and runs it alone, so
 * the longest histories of a run run at a lone lane's latency as soon as there is room.
 * Packets move with their complete state (as tail compaction saves them), so results do
 * not depend on this setting.  Applies when tail compaction is off (thor_ctx_set_tail) and
 * the run has more photons than the launch has warps (otherwise each photon has a warp). */
int thor_ctx_set_tail_share(thor_ctx_t ctx, int share);
/* Event-based execution of the grid photon loop (the propagate / interact split that
 * Sec. 7.2.2 proposes against divergence).  With slots > 0, thor_run on a grid keeps up to
 * `slots` packets in device memory and advances all of them one event per round, in three
 * kernels: the move to the interaction site (with emission into free slots, dust
 * interactions and escapes), the resonant scatterings of the packets that reached one,
 * and the peel-off rays that leave their first cell.  Once no new photons are left and at
 * most `handoff` packets remain in flight (the run's tail, where rounds would hold few
 * packets each), the survivors finish in the one-kernel loop.  slots = 0 (the default)
 * runs the one-kernel loop throughout.  slots in [0, 2^26], handoff in [0, slots].  Photon
 * histories, spectra, counters and per-photon records are identical either way; peel-off
 * images agree up to the order of their floating-point sums. */
int thor_ctx_set_grid_exec(thor_ctx_t ctx, int64_t slots, int64_t handoff);

/* ---- geometries (Sec. 3.3 datasets) ----------------------------------------------- */

/* Gridless spherical shell (Sec. 3.3; a sphere when R_in = 0), lengths in units of
 * R_out, a central point source in the empty cavity.
 *   profile THOR_PROFILE_HOMOLOGOUS: uniform density, homologous radial outflow
 *     v(r) = v_max r / R_out (Sec. 4 validation setups);
 *   profile THOR_PROFILE_POWER_LAW: the shell-model sweep geometry of Sec. 5.1, density
 *     n ~ r^alpha_rho normalised to the radial column (N_HI or tau0), radial outflow
 *     v ~ r^alpha_v with distance average v_max over [R_in, R_out] (R_in > 0), dust
 *     following the gas with radial optical depth tau_dust and albedo 0, and the step
 *     limiter f min(v_th / max|d(v r_hat.k)/ds|, R_in / |alpha_rho|) (Sec. 5.1). */
#define THOR_PROFILE_HOMOLOGOUS 0
#define THOR_PROFILE_POWER_LAW 1
/* Scattering species (power-law shells): HI Lyman alpha, or the Mg II doublet (Sec. 2.4:
 * K 2796.352 A and H 2803.531 A, total cross-section the sum of both, re-emission in the
 * absorbing transition; N_HI / tau0 then give the Mg II column / the K line-centre depth;
 * frequencies X are relative to the K line). */
#define THOR_SPECIES_HI 0
#define THOR_SPECIES_MGII 1
typedef struct {
  double R_in, R_out;    /* radii, 0 <= R_in < R_out */
  double N_HI;           /* HI column R_in -> R_out [cm^-2]; used when tau0 <= 0 */
  double tau0;           /* line-centre optical depth n sigma_0 (R_out - R_in); > 0 overrides N_HI */
  double T;              /* gas temperature [K] */
  double v_max;          /* outflow speed at R_out [km/s] */
  double tau_dust;       /* dust extinction optical depth R_in -> R_out (frequency independent) */
  double albedo;         /* dust albedo (Eq. 8); 0 = pure absorption */
  double g_hg;           /* Henyey-Greenstein asymmetry (Eq. 9) */
  int32_t phase;         /* THOR_PHASE_* for resonant scattering */
  int32_t core_skip;     /* 1: core-skipping, x_crit = 0.2 (a tau0)^(1/3) when a tau0 >= 1 (Sec. 3.4.2) */
  double step_dx;        /* step limiter f (Sec. 5.1): sub-step length f v_th / |dv/dr|; 0 -> 0.01 */
  int32_t profile;       /* THOR_PROFILE_* (0 = homologous) */
  int32_t species;       /* THOR_SPECIES_* (power-law shells; 0 = HI) */
  double alpha_rho;      /* power law: density index */
  double alpha_v;        /* power law: velocity index */
} thor_shell_params;

/* Checks every parameter on the host: finite values, the ranges above, and FP32
 * opacities that do not overflow; THOR_ERR_INVALID_ARG otherwise. */
int thor_shell_create(thor_ctx_t ctx, const thor_shell_params* p, thor_geom_t* out);

/* Uniform Cartesian grid (Sec. 3.3).  n_HI [cm^-3], T [K], v = 3 arrays (vx, vy, vz)
 * laid out one after another (3 * N floats) [km/s], dust = dust extinction
 * coefficient [cm^-1] (may be NULL = no dust).  dims = (nx, ny, nz).  Fields are
 * packed into one 32-byte record per cell on the device (zeroth-order cells,
 * Sec. 3.4) together with the emission CDF (emissivity proportional to n_HI^2).
 * The inputs are not referenced after the call.  Every cell needs T > 0, n_HI >= 0,
 * dust >= 0 and finite values (also after conversion to FP32 opacities); the cells are
 * checked on the device and any violation returns THOR_ERR_INVALID_ARG with the count,
 * as does n_HI = 0 everywhere. */
int thor_grid_create(thor_ctx_t ctx, const float* n_HI, const float* T, const float* v, const float* dust,
                     const int32_t dims[3], double cell_size_cm, int mem_kind, thor_geom_t* out);

/* Scattering parameters of a grid run (Sec. 2.3): phase function of resonant
 * scattering, dust albedo (Eq. 8) and Henyey-Greenstein g (Eq. 9).  Defaults:
 * dipole, 0.32, 0.73 (the paper's fiducial dust values). */
int thor_grid_set_scattering(thor_geom_t g, int phase, double albedo, double g_hg);

void thor_geom_destroy(thor_geom_t g);

/* ---- Monte Carlo run (Sec. 3.4) ----------------------------------------------------- */

/* Photon source.  kind 0: point source at the centre of a shell geometry with a
 * delta (sigma = 0) or Gaussian (sigma > 0) line at X0 in the source frame;
 * kind 1: gas emission of a grid, cells with probability proportional to n_HI^2,
 * thermal line in the cell frame (Sec. 2.1).  One source per run. */
typedef struct {
  int32_t kind;
  int32_t reserved;
  double X0, sigma;      /* km/s */
  /* kind 0 on a power-law shell only: the line has equivalent width ew [km/s] on a flat
   * continuum over [X0 - C, X0 + C] (Sec. 5.1); C = 0: line only */
  double ew, C;
} thor_source;

typedef struct {
  /* escaped spectrum: counts of escaping photons in n_bins bins of lab X over
   * [X_min, X_max), then underflow, overflow: n_bins + 2 uint64 entries */
  int32_t n_bins;
  int32_t mem_kind;      /* where the buffers below live */
  double X_min, X_max;
  uint64_t* spectrum;    /* required */
  /* peeling-off (grid only, Sec. 3.4.1): 3 observers along +x, +y, +z, images
   * img_n x img_n (img_n divides the grid size), peel_bins bins over
   * [peel_X_min, peel_X_max); cube = float[3][img_n][img_n][peel_bins] (zeroed by the call) */
  int32_t peel;
  int32_t img_n;
  int32_t peel_bins;
  int32_t reserved;
  double peel_X_min, peel_X_max;
  float* cube;
  /* optional per-photon records (shells and grids), indexed by photon id - first id (may be NULL) */
  float* raw_X;          /* final lab X [km/s] */
  uint32_t* raw_nscat;   /* resonant scatterings */
  uint8_t* raw_status;   /* 1 escaped, 2 absorbed, 3 stopped at max_scat */
  uint32_t max_scat;     /* stop a photon after this many scatterings (0 = never) */
  uint32_t reserved2;
  float* raw_X0;         /* emitted lab X [km/s] (shells) */
  float* raw_col;        /* HI column traversed, in units of the radial column (power-law shells) */
} thor_output_spec;

typedef struct {
  uint64_t n_photons, n_escaped, n_absorbed, n_capped;
  uint64_t n_scat;        /* resonant HI scatterings (the throughput unit) */
  uint64_t n_dust_scat;
  uint64_t n_upar_iters;  /* rejection iterations of the u_par sampler */
  uint64_t n_steps;       /* propagation steps (sub-steps or cells) */
  uint64_t n_peel_rays, n_peel_cells;
  double sum_scat2;       /* sum over photons of n_scat^2 */
  double elapsed_ms;      /* device time of the photon loop (CUDA events) */
  uint64_t n_launches;    /* photon-loop kernel launches made by the call (thor_run, the
                             allocation-free run); 0 from the server, whose launches are
                             shared between requests */
} thor_result;

/* Run photons first_id .. first_id + n_photons - 1 of the stream `seed` through the
 * geometry (Sec. 3.4 emission / propagation / interaction / escape; Sec. 3.4.1
 * peeling-off on grids).  One persistent launch; returns when the results are in
 * `out` and the output buffers.  Errors: INVALID_ARG, OOM, DEVICE. */
int thor_run(thor_ctx_t ctx, thor_geom_t g, const thor_source* src, uint64_t first_id, uint64_t n_photons,
             uint64_t seed, const thor_output_spec* spec, thor_result* out);

/* ---- Lyman-alpha forest (Sec. 3.5.2, Eq. 11) ---------------------------------------- */

typedef struct {
  double ds_cm;           /* proper path length per cell [cm] */
  double dv_cell;         /* Hubble-flow velocity across one cell [km/s] */
  int32_t n_bins;         /* velocity bins, n_bins * dv_bin == nz * dv_cell (periodic) */
  int32_t stage_rows;     /* host arrays: rows of sightlines per staged chunk (0 = automatic) */
  double dv_bin;          /* km/s */
  int64_t first_sightline, n_sightlines;  /* sightline s = column (s % nx, s / nx) along z */
} thor_forest_spec;

/* tau_out[s * n_bins + b] = sum over cells k of the column of
 * n_HI sigma_0(T) ds H(a(T), (v_b - v_k) / v_th(T)), v_k = (k + 1/2) dv_cell + v_los,
 * v_b = (b + 1/2) dv_bin, nearest periodic image.  Fields as for grids (v_los = the
 * z velocity); all pointers of kind mem_kind.  n_bins <= 2048 per call.  Host arrays are
 * streamed through two reused device buffers in chunks of stage_rows rows of sightlines
 * (automatic: as many rows as fit in 1 GiB per buffer), each chunk computed while the next
 * is copied in; the buffers stay with the context for later calls. */
int thor_forest(thor_ctx_t ctx, const float* n_HI, const float* T, const float* v_los, const int32_t dims[3],
                int mem_kind, const thor_forest_spec* spec, float* tau_out);

/* Device time of the last thor_forest or thor_reweight call in milliseconds (CUDA events). */
double thor_last_elapsed_ms(thor_ctx_t ctx);

/* ---- Post-processing of a shell run (Sec. 5.1) -------------------------------------- */

/* Reweight the escaped photons of a run to other intrinsic spectra and dust depths:
 * photon i (status 1) gets, for target t = {sigma, ew, C, tau_d},
 *   w_ti = p_t(X0_i) / p_s(X0_i) * exp(-tau_d col_i),
 * p(X) = pl N(X; 0, sigma^2) + (1 - pl) U(X; -C, C), pl = ew / (ew + 2C) (1 when C = 0),
 * p_s the spectrum the run sampled (sample = {sigma, ew, C}), and col_i its HI column in
 * units of the radial column (dust following the gas).  out[t * (n_bins + 2) + b] = sum of
 * the weights of the photons whose X_i falls in bin b of [X_min, X_max) (then underflow,
 * overflow), divided by n.  X0, X, col, status: n entries of kind mem_kind (the raw
 * records of thor_run); targets: host, n_targets x 4 doubles; out: host, n_targets x
 * (n_bins + 2) doubles, caller-owned.  n_bins <= 4096.  Errors: THOR_ERR_INVALID_ARG. */
int thor_reweight(thor_ctx_t ctx, int64_t n, const float* X0, const float* X, const float* col,
                  const uint8_t* status, int mem_kind, const double sample[3], int32_t n_targets,
                  const double* targets, int32_t n_bins, double X_min, double X_max, double* out);

/* ---- shell run without device allocation --------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that cannot
 * allocate device memory when they need a run -- code running under an external memory
 * pool with nothing to spare, a process whose GPU quota its own buffers already use up,
 * or a host callback in which cudaMalloc is not allowed.  It runs the same shell photon
 * loop as thor_run (identical results for identical arguments; the context defaults of
 * thor_ctx_set_bursts, no tail work sharing) on the current device and
 * `stream` (a cudaStream_t, NULL = legacy default stream), with no context and no
 * cudaMalloc / cudaFree: its scratch (model record, tallies, queue, and a staging copy of
 * a host spectrum) lives in a fixed file-scope device array that every GPU loading the
 * library keeps until the process exits.
 *  - spectrum: n_bins + 2 uint64 counts (bins, underflow, overflow), host or device
 *    memory per mem_kind.  Host spectra are staged in the fixed array, so then
 *    n_bins <= THOR_NOALLOC_MAX_BINS (THOR_ERR_CAPACITY otherwise).
 *  - The first call on a device looks up the array's device address and uploads a
 *    coefficient table; make that first call before any stream capture.
 *  - All calls share the array, and each call clears what must start at zero.  Calls
 *    that overlap on the GPU race on it: serialise them.
 *  - The set-up belongs to the device's current context: after a cudaDeviceReset of a
 *    device, do not call this entry point on that device again in the same process.
 *  - Parameters are checked as thor_shell_create and thor_run check them (homologous
 *    profile only), before the device is touched.
 *  - Errors: INVALID_ARG, CAPACITY, DEVICE; message in thor_noalloc_last_error(). */
#define THOR_NOALLOC_MAX_BINS 4096
int thor_run_shell_noalloc(const thor_shell_params* p, const thor_source* src, uint64_t first_id,
                           uint64_t n_photons, uint64_t seed, int32_t n_bins, double X_min, double X_max,
                           uint64_t* spectrum, int mem_kind, void* stream, thor_result* out);
const char* thor_noalloc_last_error(void);

/* ---- served stream of shell models (continuous batching) ---------------------------- */

typedef struct {
  int32_t max_requests;      /* requests resident at once (admission limit) */
  int32_t events_per_round;  /* events per lane per device round */
  int64_t n_slots;           /* resident packet slots (0 = one per resident thread) */
  uint64_t mem_budget_bytes; /* device bytes for per-request tables (admission limit) */
  int32_t block_size;        /* 0 = context default */
  int32_t priority;          /* age priority: 0 = on (the oldest request, and the next oldest while
                                their packets in flight fit in half of the warps, run their packets
                                one per warp), -1 = off (every packet shares warps) */
  int32_t presort;           /* frequency pre-sorting of the packets in flight between rounds, so a
                                warp's packets are of one kind: 1 = on, 0 = off (the default; on the
                                measured stream it did not pay, the pipelined core events already
                                keep core packets in step) */
  int32_t reserved;
} thor_server_config;

/* Create a server on the context: a host thread runs device rounds while work is
 * pending; requests submitted while others run are admitted as slots and memory
 * free up and share the same launches. */
int thor_server_create(thor_ctx_t ctx, const thor_server_config* cfg, thor_server_t* out);
/* Queue one shell-model request (geometry, source kind 0, spectrum binning as in
 * thor_output_spec with host buffers; spectrum must stay valid until the request
 * completes).  *ticket receives its id.  Errors: INVALID_ARG, CAPACITY (can never fit). */
int thor_server_submit(thor_server_t s, const thor_shell_params* p, const thor_source* src, uint64_t n_photons,
                       uint64_t seed, const thor_output_spec* spec, int64_t* ticket);
/* *done = 1 when the request finished (results written), else 0. */
int thor_server_poll(thor_server_t s, int64_t ticket, int* done);
/* Block until the request finished or timeout_ms passed (< 0 = no limit): fills *out
 * (elapsed_ms = submit-to-completion latency).  Errors: TIMEOUT, NOT_FOUND, CANCELLED. */
int thor_server_wait(thor_server_t s, int64_t ticket, int64_t timeout_ms, thor_result* out);
/* Cancel a request that has not finished. */
int thor_server_cancel(thor_server_t s, int64_t ticket);
/* Statistics: rounds launched, photons resident per round (average). */
int thor_server_stats(thor_server_t s, uint64_t* rounds, double* mean_resident, uint64_t* admitted);
/* Stop the server thread (after its current round), free its device state and drop the
 * requests that were not waited for.  No other thread may be inside a call on the same
 * server while it runs (a waiter would be left on a destroyed object). */
void thor_server_destroy(thor_server_t s);

/* ---- diagnostics: the device building blocks, one at a time ------------------------- */

/* H[i] = Voigt function H(a[i], x[i]) in FP32 (App. A.3); precise selects the
 * accurate exponential (forest kernel) instead of the fast one (photon loop). */
int thor_voigt_eval(thor_ctx_t ctx, const float* a, const float* x, float* H, int64_t n, int precise, int mem_kind);
/* xcw[i] = core-to-wing transition x_cw(a[i]) of the Voigt profile (App. A.2: the
 * frequency where e^{-x^2} = a / (sqrt(pi) x^2)) by the B25 polynomial in ln a with a fast
 * logarithm, as the u_par sampler uses it.  a[i] > 0 and normal; n values, host or device
 * arrays per mem_kind (same-kind in and out; host arrays are staged through the device). */
int thor_xcw_eval(thor_ctx_t ctx, const float* a, float* xcw, int64_t n, int mem_kind);
/* Measured issue rate of one instruction kind over the whole device, in warp instructions
 * per second (the denominators of the photon loops' ALU rooflines): kind 0 = FP32 FMA (the
 * issue-slot peak, four schedulers per SM), kind 1 = MUFU ex2 (the special-function pipe).
 * Eight independent dependency chains per thread, 64 warps per SM, best of five launches
 * timed with CUDA events on the context's stream. */
int thor_issue_peak(thor_ctx_t ctx, int kind, double* warp_inst_per_s);
/* Cell walk of n rays (origins 3n doubles in cell units, directions 3n floats) through
 * a grid of dims; cells[r * max_steps + j] = linear cell index, seg[...] = path length,
 * count[r] = cells visited (Sec. 3.4 face-to-face propagation). */
int thor_dda_trace(thor_ctx_t ctx, const int32_t dims[3], const double* origins, const float* dirs, int32_t n,
                   int32_t max_steps, int64_t* cells, double* seg, int32_t* count, int mem_kind);
/* n samples of u_par at fixed (x, a) (Eq. 6 by the rejection scheme of Eq. 10),
 * sample i from photon stream i of `seed`; *iters = total rejection iterations.
 * Needs finite x and finite a > 0 (THOR_ERR_INVALID_ARG otherwise). */
int thor_sample_upar(thor_ctx_t ctx, float x, float a, uint64_t seed, int64_t n, float* out, uint64_t* iters,
                     int mem_kind);
/* One resonant scattering (Eq. 5-7) of n photons moving along +z at gas-frame x in
 * static gas: x_out and mu = k_in . k_out.  Needs finite x and finite a > 0. */
int thor_scatter_once(thor_ctx_t ctx, float x, float a, int phase, uint64_t seed, int64_t n, float* x_out,
                      float* mu_out, int mem_kind);
/* Philox4x32-10 blocks: ctr 4n words, key 2n words, out 4n words. */
int thor_philox(thor_ctx_t ctx, const uint32_t* ctr, const uint32_t* key, uint32_t* out, int32_t n, int mem_kind);

/* Line parameters at T (Sec. 2.3.1): v_th [km/s], Voigt a, sigma_0 [cm^2]. */
void thor_line_params(double T, double* vth_kms, double* a, double* sigma0);

#ifdef __cplusplus
}
#endif
#endif /* THOR_H */
