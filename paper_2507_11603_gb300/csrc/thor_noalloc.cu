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
#include <cstdio>
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
  std::snprintf(g_err, sizeof g_err, "thor_run_shell_noalloc: %s", msg);
  return code;
}

// Once per device, with that device current: device addresses of the two arrays (the
// host-side symbols are stand-ins, not device addresses) and the coefficient table.  The
// cached addresses and the uploaded table belong to the device's current context; a
// cudaDeviceReset ends it, so this entry point must not be called again on a device after
// a reset (the table would be gone and the addresses stale).
int setup(int dev, unsigned char** scratch, float** ktab) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    unsigned char* s = nullptr;
    float* k = nullptr;
    if (cudaGetSymbolAddress((void**)&s, g_scratch) != cudaSuccess || !s)
      return fail(THOR_ERR_DEVICE, "cudaGetSymbolAddress(scratch) failed");
    if (cudaGetSymbolAddress((void**)&k, g_ktab) != cudaSuccess || !k)
      return fail(THOR_ERR_DEVICE, "cudaGetSymbolAddress(table) failed");
    if (cudaMemcpy(k, kVoigtK, sizeof(kVoigtK), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(THOR_ERR_DEVICE, "table upload failed");
    g_ktab_ptr[dev] = k;
    g_scratch_ptr[dev] = s;
  }
  *scratch = g_scratch_ptr[dev];
  *ktab = g_ktab_ptr[dev];
  return THOR_OK;
}

}  // namespace

extern "C" const char* thor_noalloc_last_error(void) { return g_err; }

extern "C" int thor_run_shell_noalloc(const thor_shell_params* p, const thor_source* src, uint64_t first_id,
                                      uint64_t n_photons, uint64_t seed, int32_t n_bins, double X_min, double X_max,
                                      uint64_t* spectrum, int mem_kind, void* stream, thor_result* out) {
  g_err[0] = 0;
  if (!p || !src || !spectrum || !out) return fail(THOR_ERR_INVALID_ARG, "NULL argument");
  if (n_photons == 0 || first_id + n_photons < first_id)
    return fail(THOR_ERR_INVALID_ARG, "bad photon range");
  if (n_bins <= 0 || !(X_max > X_min)) return fail(THOR_ERR_INVALID_ARG, "bad binning");
  if (mem_kind != THOR_MEM_HOST && mem_kind != THOR_MEM_DEVICE)
    return fail(THOR_ERR_INVALID_ARG, "bad mem_kind");
  if (mem_kind == THOR_MEM_HOST && n_bins > THOR_NOALLOC_MAX_BINS)
    return fail(THOR_ERR_CAPACITY, "host spectra are staged in the fixed scratch "
                                   "array and may have at most THOR_NOALLOC_MAX_BINS bins");
  // every argument is checked before the device is touched, by the same checks as
  // thor_shell_create and thor_run
  ShellModel m;
  char msg[200] = {0};
  if (int rc = shell_model_from_params(ErrSink{msg, sizeof msg}, p, &m)) return fail(rc, msg);
  if (p->profile != THOR_PROFILE_HOMOLOGOUS) return fail(THOR_ERR_INVALID_ARG, "homologous shells only");
  if (int rc = shell_source_into_model(ErrSink{msg, sizeof msg}, src, &m)) return fail(rc, msg);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(THOR_ERR_DEVICE, "no current CUDA device");
  unsigned char* scratch = nullptr;
  float* ktab = nullptr;
  if (int rc = setup(dev, &scratch, &ktab)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* spec = (mem_kind == THOR_MEM_DEVICE) ? (unsigned long long*)spectrum
                                                           : (unsigned long long*)(scratch + kOffSpec);
  Tally* tally = (Tally*)(scratch + kOffTally);
  m.raw_X0 = nullptr;
  m.raw_col = nullptr;
  m.X_min = (float)X_min;
  m.inv_dX = spectrum_inv_dX(n_bins, X_min, X_max);
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
  // launch shape of thor_run with its default block: fewer photons than lanes are spread
  // over all warps (each then runs closer to alone)
  const int block = 128, gsz = shell_grid(block, 0, false);
  const unsigned long long warps = (unsigned long long)gsz * (block / 32);
  const unsigned long long pw = (n_photons + warps - 1) / warps;
  const int per_warp = (int)(pw < 1 ? 1 : (pw > 32 ? 32 : pw));
  if (e == cudaSuccess)
    e = launch_shell_run((const ShellModel*)(scratch + kOffModel), q, ktab, gsz, block, THOR_PROFILE_HOMOLOGOUS,
                         per_warp, 32, 1, s);  // the context defaults of thor_ctx_set_bursts
  Tally t;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&t, tally, sizeof t, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && mem_kind == THOR_MEM_HOST)
    e = cudaMemcpyAsync(spectrum, spec, (size_t)(n_bins + 2) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(THOR_ERR_DEVICE, cudaGetErrorString(e));
  std::memset(out, 0, sizeof *out);
  tally_to_result(t, n_photons, out);
  out->n_launches = 1;
  if (t.n_done != n_photons) return fail(THOR_ERR_DEVICE, "photon loop did not finish");
  return THOR_OK;
}
