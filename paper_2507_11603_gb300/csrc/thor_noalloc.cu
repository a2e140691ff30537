// thor_noalloc.cu -- the shell photon loop without any device allocation.
//
// For callers that cannot allocate device memory at the time they need a run: code
// that runs under an external allocator or memory pool that leaves nothing to spare,
// a process whose GPU memory quota is already spent by its own buffers, or a host
// callback from which cudaMalloc is not allowed.  This entry point takes no context
// (creating one allocates), and keeps its scratch -- the model record, the tallies,
// the photon queue and, for host outputs, a staging copy of the spectrum -- in one
// file-scope device array.  Every GPU that loads the library holds that array until
// the process exits.  All calls share it, so calls that overlap on the GPU (two host
// threads, or two streams) race on it and must be serialised by the caller.
#include <cstring>
#include <mutex>

#include "../../include/thor.h"
#include "thor_ctx.h"
#include "thor_device.cuh"
#include "thor_internal.h"
#include "voigt_coeffs.h"

using namespace thor;

namespace {

// Scratch layout (bytes): [0, 512) model record, [512, 640) tallies, [640, 768) queue,
// [1024, ...) spectrum staging (host outputs), THOR_NOALLOC_MAX_BINS + 2 counters.
constexpr size_t kOffModel = 0, kOffTally = 512, kOffQueue = 640, kOffSpec = 1024;
constexpr size_t kScratchBytes = kOffSpec + (size_t)(THOR_NOALLOC_MAX_BINS + 2) * 8;
static_assert(sizeof(ShellModel) <= 512 && sizeof(Tally) <= 128, "scratch layout");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
__device__ __align__(256) float g_ktab[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices];
float* g_ktab_ptr[kMaxDevices];
char g_err[256];

int fail(int code, const char* msg) {
  std::strncpy(g_err, msg, sizeof g_err - 1);
  return code;
}

// Once per device, with that device current: device addresses of the two arrays (the
// host-side symbols are stand-ins, not device addresses) and the coefficient table.
int setup(int dev, unsigned char** scratch, float** ktab) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    unsigned char* s = nullptr;
    float* k = nullptr;
    if (cudaGetSymbolAddress((void**)&s, g_scratch) != cudaSuccess || !s)
      return fail(THOR_ERR_DEVICE, "thor_run_shell_noalloc: cudaGetSymbolAddress(scratch) failed");
    if (cudaGetSymbolAddress((void**)&k, g_ktab) != cudaSuccess || !k)
      return fail(THOR_ERR_DEVICE, "thor_run_shell_noalloc: cudaGetSymbolAddress(table) failed");
    if (cudaMemcpy(k, kVoigtK, sizeof(kVoigtK), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(THOR_ERR_DEVICE, "thor_run_shell_noalloc: table upload failed");
    g_ktab_ptr[dev] = k;
    g_scratch_ptr[dev] = s;
  }
  *scratch = g_scratch_ptr[dev];
  *ktab = g_ktab_ptr[dev];
  return THOR_OK;
}

// The shell's model record, as thor_shell_create builds it (same checks, no context).
int model_from_params(const thor_shell_params* p, ShellModel* m) {
  for (double q : {p->R_in, p->R_out, p->N_HI, p->tau0, p->T, p->v_max, p->tau_dust, p->albedo, p->g_hg, p->step_dx})
    if (!std::isfinite(q)) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: parameters must be finite");
  if (!(p->R_out > 0.0) || !(p->R_in >= 0.0) || !(p->R_in < p->R_out))
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: radii must satisfy 0 <= R_in < R_out");
  if (!(p->T > 0.0)) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: temperature must be > 0");
  if (!(p->tau_dust >= 0.0) || !(p->albedo >= 0.0 && p->albedo <= 1.0) || !(p->g_hg > -1.0 && p->g_hg < 1.0))
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: dust parameters out of range");
  if (p->phase < 0 || p->phase > 2) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: unknown phase");
  if (!(p->v_max >= 0.0)) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: v_max must be >= 0");
  if (p->profile != THOR_PROFILE_HOMOLOGOUS)
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: homologous shells only");
  double tau0 = p->tau0;
  if (!(tau0 > 0.0)) {
    if (!(p->N_HI >= 0.0)) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: N_HI must be >= 0");
    tau0 = p->N_HI * line_sigma0(p->T);
  }
  const double L = (p->R_out - p->R_in) / p->R_out;
  const double vth = line_vth_kms(p->T);
  const double f = (p->step_dx > 0.0) ? p->step_dx : 0.01;
  const double at = line_a(p->T) * tau0;
  std::memset(m, 0, sizeof(*m));
  m->R_in = p->R_in / p->R_out;
  m->R_out = 1.0;
  m->kap0 = (float)(tau0 / L);
  m->kapd = (float)(p->tau_dust / L);
  m->vth = (float)vth;
  m->inv_vth = (float)(1.0 / vth);
  m->a = (float)line_a(p->T);
  m->vgrad = (float)p->v_max;
  m->gam = (float)(p->v_max / vth);
  m->ds_core = (p->v_max > 0.0) ? (float)(f * vth / p->v_max) : 1e30f;
  m->albedo = (float)p->albedo;
  m->g_hg = (float)p->g_hg;
  m->phase = p->phase;
  m->xcrit = (p->core_skip && at >= 1.0) ? (float)(0.2 * cbrt(at)) : 0.0f;
  if (!shell_record_finite(*m))
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: opacity or line parameters overflow FP32");
  return THOR_OK;
}

}  // namespace

extern "C" const char* thor_noalloc_last_error(void) { return g_err; }

extern "C" int thor_run_shell_noalloc(const thor_shell_params* p, const thor_source* src, uint64_t first_id,
                                      uint64_t n_photons, uint64_t seed, int32_t n_bins, double X_min, double X_max,
                                      uint64_t* spectrum, int mem_kind, void* stream, thor_result* out) {
  g_err[0] = 0;
  if (!p || !src || !spectrum || !out) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: NULL argument");
  if (n_photons == 0 || first_id + n_photons < first_id)
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: bad photon range");
  if (src->kind != 0 || !(src->sigma >= 0.0) || src->C > 0.0 || !std::isfinite(src->X0) || !std::isfinite(src->sigma))
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: shells take a central point source (kind 0, no continuum)");
  if (n_bins <= 0 || !(X_max > X_min)) return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: bad binning");
  if (mem_kind != THOR_MEM_HOST && mem_kind != THOR_MEM_DEVICE)
    return fail(THOR_ERR_INVALID_ARG, "thor_run_shell_noalloc: bad mem_kind");
  if (mem_kind == THOR_MEM_HOST && n_bins > THOR_NOALLOC_MAX_BINS)
    return fail(THOR_ERR_CAPACITY, "thor_run_shell_noalloc: host spectra are staged in the fixed scratch "
                                   "array and may have at most THOR_NOALLOC_MAX_BINS bins");
  ShellModel m;  // every argument is checked before the device is touched
  if (int rc = model_from_params(p, &m)) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(THOR_ERR_DEVICE, "thor_run_shell_noalloc: no current CUDA device");
  unsigned char* scratch = nullptr;
  float* ktab = nullptr;
  if (int rc = setup(dev, &scratch, &ktab)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* spec = (mem_kind == THOR_MEM_DEVICE) ? (unsigned long long*)spectrum
                                                           : (unsigned long long*)(scratch + kOffSpec);
  Tally* tally = (Tally*)(scratch + kOffTally);
  m.line = (src->sigma > 0.0) ? 1 : 0;
  m.X0 = (float)src->X0;
  m.sigma = (float)src->sigma;
  m.p_line = 1.0f;
  m.cont_C = 0.0f;
  m.profile = THOR_PROFILE_HOMOLOGOUS;
  m.raw_X0 = nullptr;
  m.raw_col = nullptr;
  m.X_min = (float)X_min;
  m.inv_dX = (float)(n_bins / (X_max - X_min));
  m.n_bins = n_bins;
  m.seed_lo = (uint32_t)seed; m.seed_hi = (uint32_t)(seed >> 32);
  m.spectrum = spec;
  m.tally = tally;
  m.id_base = first_id;
  m.n_photons = n_photons;
  struct QHost { unsigned long long next, prefix[2], first_id; int32_t model; } qh{0, {0, n_photons}, first_id, 0};
  char* qb = (char*)(scratch + kOffQueue);
  // everything that must start at zero is cleared here: spectrum, tallies, queue counter
  cudaError_t e = cudaMemsetAsync(spec, 0, (size_t)(n_bins + 2) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tally, 0, sizeof(Tally), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + kOffModel, &m, sizeof m, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(qb, &qh, sizeof qh, cudaMemcpyHostToDevice, s);
  WorkQueue q;
  q.next = (unsigned long long*)(qb + offsetof(QHost, next));
  q.total = n_photons;
  q.prefix = (const unsigned long long*)(qb + offsetof(QHost, prefix));
  q.first_id = (const unsigned long long*)(qb + offsetof(QHost, first_id));
  q.model = (const int32_t*)(qb + offsetof(QHost, model));
  q.n_entries = 1;
  if (e == cudaSuccess)
    e = launch_shell_run((const ShellModel*)(scratch + kOffModel), q, ktab, shell_grid(128, 0, false), 128,
                         THOR_PROFILE_HOMOLOGOUS, 32, s);
  Tally t;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&t, tally, sizeof t, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && mem_kind == THOR_MEM_HOST)
    e = cudaMemcpyAsync(spectrum, spec, (size_t)(n_bins + 2) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(THOR_ERR_DEVICE, cudaGetErrorString(e));
  std::memset(out, 0, sizeof *out);
  tally_to_result(t, n_photons, out);
  out->n_launches = 1;
  if (t.n_done != n_photons) return fail(THOR_ERR_DEVICE, "thor_run_shell_noalloc: photon loop did not finish");
  return THOR_OK;
}
