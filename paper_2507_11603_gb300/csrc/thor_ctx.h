// thor_ctx.h -- host-side objects behind the opaque handles of include/thor.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <string>

#include "../../include/thor.h"
#include "thor_internal.h"

struct thor_ctx {
  struct Buf {
    void* p = nullptr;
    size_t cap = 0;
  };
  int device = 0;
  int sm_count = 0, cc_major = 0, cc_minor = 0;
  cudaStream_t stream = nullptr;
  int block = 128;          // threads per block of the photon loops
  int blocks_per_sm = 0;    // 0 = occupancy maximum
  float* d_ktab = nullptr;  // Voigt coefficient table (device copy)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.0f;
  std::string last_error;
  // grow-only scratch buffers reused across calls
  Buf b_models, b_tally, b_queue, b_spec, b_cube, b_raw, b_raw2, b_diag, b_stats, b_spill, b_cmp;
  Buf b_stage[2];                   // host-input staging, double-buffered (forest)
  cudaStream_t copy_stream = nullptr;  // host<->device copies overlapped with kernels
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
  // tail compaction of the shell photon loop
  int spill_below = 0;      // warps with fewer live lanes hand them to the next launch (0 = off)
  int max_phases = 24;      // launches at most
  int final_below = 256;    // run to completion once this few packets are left
  int core_lanes = 32;      // warps with at most this many live packets run pipelined events (0 = never)
  int burst_lanes = 1;      // ... and, with at most this many, core bursts (0 = never)
  int share_tail = 1;       // work sharing in the tail of a one-launch shell run
  Buf b_share;
  // event-based grid loop (0 slots = the one-kernel loop throughout)
  int64_t grid_slots = 0;
  int64_t grid_handoff = 0;  // packets in flight at which the tail goes to the one-kernel loop
  Buf b_gslots;
  int64_t grid_rounds_last = 0;
  int phases_last = 0;

  int fail(int code, const char* fmt, ...);
  int cuda(cudaError_t e, const char* what);
  int select();
  void* scratch(Buf& b, size_t bytes);
  ~thor_ctx();
};

struct thor_geom {
  enum Kind { SHELL, GRID } kind = SHELL;
  thor_ctx* ctx = nullptr;
  // shell
  thor::ShellModel shell{};
  thor_shell_params shell_params{};
  // grid
  int32_t dims[3] = {0, 0, 0};
  double cell_cm = 0.0;
  int64_t n_cells = 0;
  thor::GridCell* cells = nullptr;
  double* cdf = nullptr;
  double* scan_tmp = nullptr;
  int grid_phase = THOR_PHASE_DIPOLE;
  double grid_albedo = 0.32, grid_g = 0.73;
  ~thor_geom();
};

namespace thor {
struct OutBufs {
  unsigned long long* spec = nullptr;
  float* cube = nullptr;
  float* raw_X = nullptr;
  uint32_t* raw_n = nullptr;
  uint8_t* raw_s = nullptr;
  float* raw_X0 = nullptr;
  float* raw_col = nullptr;
};
// Where the shell checks below report: fail() writes the message into buf (truncated to
// cap bytes) and returns the code.  Needs no context, so the allocation-free entry point
// runs exactly the same checks as thor_shell_create and the server.
struct ErrSink {
  char* buf;
  size_t cap;
  int fail(int code, const char* msg) const {
    if (buf && cap) std::snprintf(buf, cap, "%s", msg);
    return code;
  }
};
// Shell model record from its parameters (homologous or power-law; HI or Mg II), every
// parameter checked; and the source fields of a shell model (line, continuum), validated
// against the profile.
int shell_model_from_params(ErrSink err, const thor_shell_params* p, ShellModel* m);
int shell_source_into_model(ErrSink err, const thor_source* src, ShellModel* m);
// The same, reporting through the context's last error.
int fill_shell_source(thor_ctx* ctx, const thor_source* src, ShellModel* m);
int fill_shell_model(thor_ctx* ctx, const thor_shell_params* p, ShellModel* m);
int prepare_outputs(thor_ctx* ctx, const thor_output_spec* spec, uint64_t n_photons, bool grid, OutBufs* o);
int finish_outputs(thor_ctx* ctx, const thor_output_spec* spec, uint64_t n_photons, bool grid, const OutBufs& o);
void tally_to_result(const Tally& t, uint64_t n_photons, thor_result* r);
}  // namespace thor
