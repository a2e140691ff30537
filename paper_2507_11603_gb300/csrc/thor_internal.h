// thor_internal.h -- plain structs shared by the host runtime and the kernels.
#pragma once

#include <cmath>
#include <cstdint>
#include <initializer_list>
#include <cuda_runtime.h>

namespace thor {

// Per-model tallies (device, 8-byte aligned).  Integer fields are exact and
// independent of the order in which photons finish.
struct Tally {
  unsigned long long n_escaped, n_absorbed, n_capped, n_done;
  unsigned long long n_scat, n_dust_scat, n_upar_iters, n_steps;
  double sum_scat2;
  double pad[3];
};

// Gridless model (Sec. 3.3 spherical shell / sphere) as the kernels read it.
struct ShellModel {
  double R_in, R_out;        // radii (R_out normalises lengths)
  float kap0;                // HI line-centre opacity per unit length
  float kapd;                // dust extinction per unit length
  float vth, inv_vth, a;     // km/s, s/km, Voigt parameter
  float vgrad;               // km/s per unit length (homologous v = vgrad r)
  float gam;                 // |dx/ds| = vgrad / vth
  float ds_core;             // sub-step length (step limiter, Sec. 5.1: f l_v)
  float xcrit;               // core-skipping threshold (Sec. 3.4.2), 0 = off
  float albedo, g_hg;
  int32_t phase;
  int32_t line;              // 0 delta, 1 Gaussian
  float X0, sigma;           // source line (km/s)
  float X_min, inv_dX;       // spectrum binning
  int32_t n_bins;
  uint32_t seed_lo, seed_hi;
  uint32_t max_scat;         // 0 = none
  unsigned long long* spectrum;  // n_bins + 2
  Tally* tally;
  float* raw_X;              // optional per-photon outputs (indexed by photon id - id_base)
  uint32_t* raw_nscat;
  uint8_t* raw_status;
  unsigned long long id_base;
  unsigned long long n_photons;
  int32_t cancelled;         // served requests: drop in-flight packets (set by the host)
  int32_t priority;          // served requests: packets run one per warp (set by the host per round)
  int32_t profile;           // 0 homologous uniform shell, 1 power-law shell (Sec. 5.1)
  // power law: n(r) / n(1) = r^ar, v(r) = v1 r^av (radial), opacities per unit length at r = 1
  float ar, av, v1, kapn, kapdn;
  float invF;                // HI column per unit length at r = 1, in units of the radial column
  float p_line, cont_C;      // source: probability of the line, continuum half-width (km/s; 0 = none)
  int32_t n_lines;           // power law: 2 = Mg II doublet (line 2 = H, isotropic re-emission)
  float kapn2, a2, eps2;     // line 2: opacity at r = 1, Voigt a, lambda_2 / lambda_1 - 1
  float* raw_X0;             // optional per-photon emitted X and column
  float* raw_col;
};

// Every FP32 parameter of a shell record is finite and the thermal speed and Voigt a are
// positive (a parameter set whose opacities overflow FP32 is rejected, since a photon
// with an infinite opacity would never move).
inline bool shell_record_finite(const ShellModel& m) {
  for (float q : {m.kap0, m.kapd, m.vth, m.inv_vth, m.a, m.vgrad, m.gam, m.ds_core, m.xcrit, m.ar, m.av, m.v1, m.kapn,
                  m.kapdn, m.invF, m.kapn2, m.a2, m.eps2})
    if (!std::isfinite(q)) return false;
  return m.vth > 0.0f && m.a > 0.0f && (m.n_lines < 2 || m.a2 > 0.0f);
}

// Scale from a lab frequency to a spectrum bin: bin = floor((X - X_min) * inv_dX).  Every
// path that bins photons (the single run, the served stream, the allocation-free run, the
// peel cubes) takes it from here, so identical arguments give identical bins.
inline float spectrum_inv_dX(int n_bins, double X_min, double X_max) {
  return 1.0f / (float)((X_max - X_min) / n_bins);
}

// Photon work queue: photon g in [0, total) belongs to model m with
// prefix[m] <= g < prefix[m+1] and has id first_id[m] + g - prefix[m].
struct WorkQueue {
  unsigned long long* next;          // device counter
  unsigned long long total;
  const unsigned long long* prefix;  // n_models + 1
  const unsigned long long* first_id;
  const int32_t* model;              // model table index per queue entry
  int32_t n_entries;
  // optional: {total, n_entries, event budget} read from device memory at kernel start
  // instead of the fields above (and the launch's budget), so one captured launch (CUDA
  // graph) serves every round
  const unsigned long long* hdr = nullptr;
};

// A packet saved between launches of the run-to-completion loop (tail compaction).
struct PhotonRec {
  double px, py, pz;  // FP64 anchor
  float ox, oy, oz;   // FP32 offset from the anchor (saved as is: resuming is bit-exact)
  float X0, col_hi, col_lo;  // emitted X, HI column traversed (two-level sum)
  float kx, ky, kz, x, X, safe;
  int32_t region;
  uint32_t nscat, ndust, iters, steps, event;
  unsigned long long pid;
};

// Tail compaction (optional, off by default): a launch first resumes saved packets, then
// takes fresh photons; once the queue is drained, a warp with fewer than `spill_below` live
// lanes saves them to `spill` and exits, and the next launch repacks the survivors
// `per_warp` to a warp.  Also carries per_warp for the first launch (few photons spread
// over all warps).
struct Compact {  // every field defaults to off / empty
  const PhotonRec* resume = nullptr;
  unsigned long long n_resume = 0;
  unsigned long long* resume_next = nullptr;
  PhotonRec* spill = nullptr;
  unsigned long long* n_spill = nullptr;
  int32_t spill_below = 0;  // 0: run to completion
  int32_t per_warp = 32;    // lanes per warp that take packets (1..32): few packets spread over all schedulers
  int32_t core_lanes = 32;  // warps with at most this many live packets run pipelined events (0 = never)
  int32_t burst_lanes = 1;  // ... and, with at most this many, core bursts (0 = never)
  // Work sharing in the tail of a one-launch run (pool = NULL: off).  Once the queue is
  // drained, a warp whose lanes are all done waits for a packet that a warp with several
  // live packets gives away, and runs it alone.
  PhotonRec* pool = nullptr;            // given-away packets (one entry per photon at most)
  uint32_t* ready = nullptr;            // pool entry i written (1), set after the record
  unsigned long long* share = nullptr;  // [0] entries reserved, [1] taken, [2] empty warps waiting,
                                        // [3] photons finished, [4] a taken entry never became ready
  unsigned long long n_total = 0;       // photons of the run
};

// Resident packet state for time-sliced (served) execution, SoA, one slot per thread.
struct SlotState {
  double *px, *py, *pz;              // FP64 anchor
  float *ox, *oy, *oz, *safe;        // FP32 offset, safety distance (saved as is)
  float *kx, *ky, *kz, *X, *x;
  uint32_t* event;                   // RNG position: events done
  uint32_t *nscat, *ndust, *iters, *steps;
  int32_t* model;
  unsigned long long* pid;
  uint8_t* region;
  int64_t n_slots;                   // capacity (packets)
  // [0] packets stored in this buffer from the front, [1] their append counter in the next
  // buffer; [2] priority packets stored from the back (entry j at n_slots - 1 - j), [3] their
  // append counter in the next buffer
  unsigned long long* live;
};

// Grid model (Sec. 3.3 uniform Cartesian grid), packed 32 B per cell.
struct GridCell {
  float kap0;   // n_HI sigma_0(T) L_cell: HI line-centre opacity per cell length
  float a;      // Voigt parameter
  float inv_vth;
  float vth;
  float vx, vy, vz;  // km/s
  float kd;     // dust extinction per cell length
};

struct GridModel {
  const GridCell* cells;
  const double* cdf;      // emission CDF over cells (n_HI^2), last entry = total
  int32_t nx, ny, nz;
  int32_t phase;
  float albedo, g_hg;
  float X_min, inv_dX;    // escaped spectrum
  int32_t n_bins;
  int32_t peel;           // 0/1
  int32_t img_n;          // pixels per image axis
  int32_t peel_bins;
  float pX_min, pinv_dX;
  float tau_cut;
  uint32_t max_scat;
  uint32_t seed_lo, seed_hi;
  unsigned long long* spectrum;
  float* cube;            // [3][img_n][img_n][peel_bins]
  Tally* tally;
  unsigned long long n_photons;
  unsigned long long id_base;
  unsigned long long* peel_rays;   // statistics: peel rays traced, cells visited
  unsigned long long* peel_cells;
  int32_t per_warp;       // lanes per warp that take photons (1..32): few photons spread over all schedulers
  float* raw_X;           // optional per-photon records (NULL = off), indexed by pid - id_base
  uint32_t* raw_nscat;
  uint8_t* raw_status;
};

// Event-based grid loop: packets in flight, one slot each (SoA, device memory), and the
// queues between its kernels.
struct PeelRay {  // a peel-off ray in flight: its start, frequency, weight and walk state
  double px, py, pz;
  double t;        // distance from the start to the entry face of cell i
  float Xp, w0, tau;
  int32_t ax, i;   // axis, next cell along it
  int32_t pad;
};
struct TallySlab {  // counters of one block index of the event-based loop's kernels
  unsigned long long esc, ab, cap, sc, du, it, stp, dn, pr, pc;
  double sc2;
  unsigned long long pad;
};
struct GridSlots {
  int64_t n;                   // slots
  double *px, *py, *pz;        // FP64 anchor (cell units)
  float *ox, *oy, *oz;         // FP32 offset from the anchor
  float *fx, *fy, *fz;         // distances from the anchor to the cell's + faces
  float* safe;
  float *kx, *ky, *kz, *X;
  float* xs;                   // gas-frame frequency at the interaction site (move -> interact)
  uint32_t *nscat, *ndust, *iters, *steps, *event;
  unsigned long long* pid;
  uint8_t* live;               // 1 = a packet in flight
  int32_t* rq;                 // slots awaiting a resonant scattering (n entries)
  PeelRay* rays[2];            // peel rays in flight, per round parity (kRayCap n entries each)
  // [0] packets in flight; [2] entries of the resume list (in rq) and [3] its cursor;
  // round parity r: [4 + 4r] resonant queue length, [5 + 4r] ray queue length
  unsigned long long* ctr;
  TallySlab* slab;             // one entry per block index (kGridSlabBlocks), summed at the end
};
constexpr int kGridSlabBlocks = 4096;
constexpr int kRayCap = 6;       // ray queue entries per slot and parity (3 new per round + carried)
constexpr int kRayChunk = 32;    // cells a queued ray advances per round

// ---- launchers (implemented in the .cu files) ------------------------------------
int shell_grid(int block, int blocks_per_sm, bool sliced);  // persistent grid size
int grid_grid(int block, int blocks_per_sm);
cudaError_t launch_shell_run(const ShellModel* d_models, WorkQueue q, const float* d_ktab, int grid,
                             int block, int profile, int per_warp, int core_lanes, int burst_lanes, cudaStream_t s,
                             const Compact* share = nullptr);
cudaError_t launch_shell_run_compact(const ShellModel* d_models, WorkQueue q, Compact c, const float* d_ktab,
                                     int grid, int block, int profile, cudaStream_t s);
cudaError_t launch_reweight(int64_t n, const float* X0, const float* X, const float* col, const uint8_t* status,
                            const float* d_params, int n_targets, int n_bins, double X_min, double X_max,
                            double* d_out, int n_sm, cudaStream_t s);
cudaError_t launch_slot_presort(SlotState from, SlotState to, unsigned long long* cnt, cudaStream_t s);
cudaError_t launch_shell_slice(const ShellModel* d_models, WorkQueue q, SlotState in, SlotState out,
                               uint32_t event_budget,
                               const float* d_ktab, int grid, int block, bool mixed, cudaStream_t s);
cudaError_t launch_grid_pack(const float* nHI, const float* T, const float* vx, const float* vy,
                             const float* vz, const float* dust, int64_t n, double cell_cm, GridCell* out,
                             double* w, unsigned long long* bad, cudaStream_t s);  // bad: count of unusable cells
cudaError_t launch_scan_f64(double* data, int64_t n, double* scratch, cudaStream_t s);
size_t scan_f64_scratch(int64_t n);
cudaError_t launch_grid_run(GridModel m, WorkQueue q, const float* d_ktab, int grid, int block,
                            cudaStream_t s);
// Event-based grid loop: one round (move, resonant scatterings, peel rays) with counters of
// parity `parity`; the list of packets in flight (for the hand-off); the one-kernel loop
// resuming that list first.
cudaError_t launch_grid_round(GridModel m, WorkQueue q, GridSlots S, int parity, const float* d_ktab, int block,
                              cudaStream_t s);
cudaError_t launch_grid_list_live(GridSlots S, cudaStream_t s);
cudaError_t launch_grid_slab_sum(GridModel m, GridSlots S, cudaStream_t s);
cudaError_t launch_grid_ray_drain(GridModel m, GridSlots S, int parity, const float* d_ktab, int block,
                                  cudaStream_t s);
cudaError_t launch_grid_resume(GridModel m, WorkQueue q, GridSlots S, const float* d_ktab, int grid, int block,
                               cudaStream_t s);
size_t grid_slots_bytes(int64_t n);
GridSlots grid_slots_carve(void* base, int64_t n);
cudaError_t launch_forest(const float* nHI, const float* T, const float* vlos, int nx, int ny, int nz,
                          int64_t first, int64_t count, double ds_cm, double dv_cell, int n_bins,
                          double dv_bin, float* tau, const float* d_ktab, cudaStream_t s);
cudaError_t launch_voigt_eval(const float* a, const float* x, float* H, int64_t n, const float* d_ktab,
                              cudaStream_t s, int precise);
cudaError_t launch_xcw_eval(const float* a, float* out, int64_t n, cudaStream_t s);
cudaError_t launch_issue_probe(int kind, float* sink, int grid, int block, int iters, cudaStream_t s);
cudaError_t launch_dda_trace(int nx, int ny, int nz, const double* org, const float* dir, int n, int max_steps,
                             int64_t* cells, double* seg, int32_t* count, cudaStream_t s);
cudaError_t launch_upar(float x, float a, uint64_t seed, int64_t n, float* out, unsigned long long* iters,
                        cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, cudaStream_t s);
cudaError_t launch_scatter_once(float x, float a, int phase, uint64_t seed, int64_t n, float* x_out,
                                float* mu_out, cudaStream_t s);

}  // namespace thor
