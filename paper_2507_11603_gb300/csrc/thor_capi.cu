// thor_capi.cu -- host runtime behind include/thor.h: contexts, geometry objects,
// the single-model run, the forest ray-march and the diagnostic entry points.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/thor.h"
#include "thor_ctx.h"
#include "thor_device.cuh"
#include "thor_internal.h"

using namespace thor;

// ------------------------------------------------------------------------------ errors
static std::string g_init_error;

int thor_ctx::fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  last_error = buf;
  return code;
}

int thor_ctx::cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return THOR_OK;
  if (e == cudaErrorMemoryAllocation) return fail(THOR_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(THOR_ERR_DEVICE, "%s: %s", what, cudaGetErrorString(e));
}

int thor_ctx::select() { return cuda(cudaSetDevice(device), "cudaSetDevice"); }

void* thor_ctx::scratch(Buf& b, size_t bytes) {
  if (b.cap >= bytes && b.p) return b.p;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t cap = bytes < 256 ? 256 : bytes;
  if (cudaMalloc(&b.p, cap) != cudaSuccess) return nullptr;
  b.cap = cap;
  return b.p;
}

thor_ctx::~thor_ctx() {
  cudaSetDevice(device);
  for (Buf* b : {&b_models, &b_tally, &b_queue, &b_spec, &b_cube, &b_raw, &b_raw2, &b_diag, &b_stats, &b_spill, &b_cmp,
                 &b_stage[0], &b_stage[1], &b_gslots, &b_share})
    if (b->p) cudaFree(b->p);
  for (cudaEvent_t e : {ev_copied[0], ev_copied[1], ev_done[0], ev_done[1]})
    if (e) cudaEventDestroy(e);
  if (copy_stream) cudaStreamDestroy(copy_stream);
  if (d_ktab) cudaFree(d_ktab);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}

// ------------------------------------------------------------------------------ context
// Target warps per SM sub-partition (scheduler) when a tail relaunch spreads survivors.
constexpr int kWarpsPerSmsp = 4;

extern "C" int thor_init(int device, thor_ctx_t* out) {
  if (!out) { g_init_error = "thor_init: out is NULL"; return THOR_ERR_INVALID_ARG; }
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    g_init_error = std::string("thor_init: no CUDA device ") + std::to_string(device) + " (" +
                   cudaGetErrorString(e) + ")";
    return THOR_ERR_DEVICE;
  }
  thor_ctx* c = new thor_ctx();
  c->device = device;
  if (c->select() != THOR_OK) { g_init_error = c->last_error; delete c; return THOR_ERR_DEVICE; }
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  c->sm_count = prop.multiProcessorCount;
  c->cc_major = prop.major;
  c->cc_minor = prop.minor;
  if (cudaMalloc(&c->d_ktab, sizeof(kVoigtK)) != cudaSuccess ||
      cudaMemcpy(c->d_ktab, kVoigtK, sizeof(kVoigtK), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
    g_init_error = "thor_init: device setup failed";
    delete c;
    return THOR_ERR_DEVICE;
  }
  *out = c;
  return THOR_OK;
}

extern "C" void thor_destroy(thor_ctx_t ctx) { delete ctx; }

extern "C" const char* thor_last_error(thor_ctx_t ctx) {
  if (!ctx) return g_init_error.c_str();
  return ctx->last_error.c_str();
}

extern "C" int thor_ctx_set_stream(thor_ctx_t ctx, void* s) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)s;
  return THOR_OK;
}

extern "C" int thor_ctx_set_tail(thor_ctx_t ctx, int spill_below, int max_phases) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (spill_below < 0 || spill_below > 32 || max_phases < 1)
    return ctx->fail(THOR_ERR_INVALID_ARG, "thor_ctx_set_tail: spill_below in [0, 32], max_phases >= 1");
  ctx->spill_below = spill_below;
  ctx->max_phases = max_phases;
  return THOR_OK;
}

extern "C" int thor_ctx_set_bursts(thor_ctx_t ctx, int pipe_lanes, int burst_lanes) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (pipe_lanes < 0 || pipe_lanes > 32 || burst_lanes < 0 || burst_lanes > 32)
    return ctx->fail(THOR_ERR_INVALID_ARG, "thor_ctx_set_bursts: pipe_lanes and burst_lanes in [0, 32]");
  ctx->core_lanes = pipe_lanes;
  ctx->burst_lanes = burst_lanes;
  return THOR_OK;
}

extern "C" int thor_ctx_set_tail_share(thor_ctx_t ctx, int share) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (share != 0 && share != 1) return ctx->fail(THOR_ERR_INVALID_ARG, "thor_ctx_set_tail_share: share must be 0 or 1");
  ctx->share_tail = share;
  return THOR_OK;
}

extern "C" int thor_ctx_set_grid_exec(thor_ctx_t ctx, int64_t slots, int64_t handoff) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (slots < 0 || slots > ((int64_t)1 << 26) || handoff < 0 || handoff > slots)
    return ctx->fail(THOR_ERR_INVALID_ARG, "thor_ctx_set_grid_exec: slots in [0, 2^26], handoff in [0, slots]");
  ctx->grid_slots = slots;
  ctx->grid_handoff = handoff;
  return THOR_OK;
}

extern "C" int thor_ctx_set_launch(thor_ctx_t ctx, int block_size, int blocks_per_sm) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (block_size <= 0 || block_size > 256 || (block_size & 31) || blocks_per_sm < 0)
    return ctx->fail(THOR_ERR_INVALID_ARG, "thor_ctx_set_launch: block_size must be a multiple of 32 in [32, 256]");
  ctx->block = block_size;
  ctx->blocks_per_sm = blocks_per_sm;
  return THOR_OK;
}

extern "C" void thor_line_params(double T, double* vth, double* a, double* sigma0) {
  if (vth) *vth = line_vth_kms(T);
  if (a) *a = line_a(T);
  if (sigma0) *sigma0 = line_sigma0(T);
}

// ------------------------------------------------------------------------------ geometry
// int_lo^hi r^alpha dr
static double pow_int(double alpha, double lo, double hi) {
  if (fabs(alpha + 1.0) < 1e-12) return log(hi / lo);
  return (pow(hi, alpha + 1.0) - pow(lo, alpha + 1.0)) / (alpha + 1.0);
}

// Power-law shell (Sec. 5.1): lengths in units of R_out, n ~ r^alpha_rho with radial
// column tau0 / sigma_0, v ~ r^alpha_v with distance average v_max, dust following the
// gas, global step limiter f min(v_th / G, r_i / |alpha_rho|) with G a bound on
// |d(v r_hat . k)/ds| = |v' mu_r^2 + v (1 - mu_r^2) / r| <= max(|v'|, v / r).
// Mg II doublet (Sec. 2.4), NIST Atomic Spectra Database: vacuum wavelengths [cm],
// oscillator strengths, Einstein A [1/s]; ion mass 24.305 u.
static const double kMgLamK = 2796.352e-8, kMgLamH = 2803.531e-8, kMgFK = 0.608, kMgFH = 0.303;
static const double kMgAK = 2.60e8, kMgAH = 2.57e8, kMgMass = 24.305 * 1.66053906660e-24;

static int fill_power_law(ErrSink err, const thor_shell_params* p, ShellModel* m) {
  using namespace thor;
  if (!(p->R_in > 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "power-law shells need R_in > 0");
  if (p->species != THOR_SPECIES_HI && p->species != THOR_SPECIES_MGII)
    return err.fail(THOR_ERR_INVALID_ARG, "unknown species");
  if (!(fabs(p->alpha_rho) <= 8.0) || !(fabs(p->alpha_v) <= 8.0))
    return err.fail(THOR_ERR_INVALID_ARG, "power-law indices out of range");
  if (p->albedo != 0.0) return err.fail(THOR_ERR_INVALID_ARG, "power-law shells take albedo 0 (dust absorbs)");
  const bool mg = p->species == THOR_SPECIES_MGII;
  // thermal speed, Voigt a and line-centre cross-section of the (first) transition
  const double vth = mg ? sqrt(2.0 * 1.380649e-16 * p->T / kMgMass) * 1e-5 : line_vth_kms(p->T);
  const double esu2_mec = 1.7724538509055159 * 4.80320471e-10 * 4.80320471e-10 / (9.1093837015e-28 * 2.99792458e10);
  const double sig_K = mg ? kMgFK * esu2_mec * kMgLamK / (vth * 1e5) : line_sigma0(p->T);
  double tau0 = p->tau0;
  if (!(tau0 > 0.0)) {
    if (!(p->N_HI >= 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "N_HI must be >= 0");
    tau0 = p->N_HI * sig_K;
  }
  const double ri = p->R_in / p->R_out;
  const double F = pow_int(p->alpha_rho, ri, 1.0);
  const double v1 = p->v_max * (1.0 - ri) / pow_int(p->alpha_v, ri, 1.0);
  double G = 0.0;
  for (int i = 0; i <= 2000; ++i) {
    const double r = ri + (1.0 - ri) * i / 2000.0;
    const double v = v1 * pow(r, p->alpha_v);
    G = fmax(G, fmax(fabs(p->alpha_v) * v / r, v / r));
  }
  const double f = (p->step_dx > 0.0) ? p->step_dx : 0.01;
  double ds = (G > 0.0) ? f * vth / (1.05 * G) : 1e30;
  if (p->alpha_rho != 0.0) ds = fmin(ds, f * ri / fabs(p->alpha_rho));
  std::memset(m, 0, sizeof(*m));
  m->profile = THOR_PROFILE_POWER_LAW;
  m->R_in = ri;
  m->R_out = 1.0;
  m->kapn = (float)(tau0 / F);
  m->kapdn = (float)(p->tau_dust / F);
  m->invF = (float)(1.0 / F);
  m->ar = (float)p->alpha_rho;
  m->av = (float)p->alpha_v;
  m->v1 = (float)v1;
  m->vth = (float)vth;
  m->inv_vth = (float)(1.0 / vth);
  m->a = mg ? (float)(kMgAK * kMgLamK / (4.0 * M_PI * vth * 1e5)) : (float)line_a(p->T);
  m->n_lines = 1;
  if (mg) {
    const double sig_H = kMgFH * esu2_mec * kMgLamH / (vth * 1e5);
    m->n_lines = 2;
    m->kapn2 = (float)(tau0 * (sig_H / sig_K) / F);
    m->a2 = (float)(kMgAH * kMgLamH / (4.0 * M_PI * vth * 1e5));
    m->eps2 = (float)(kMgLamH / kMgLamK - 1.0);
  }
  m->ds_core = (float)ds;
  m->albedo = 0.0f;
  m->g_hg = (float)p->g_hg;
  m->phase = p->phase;
  const double at = (double)m->a * tau0;
  m->xcrit = (p->core_skip && at >= 1.0) ? (float)(0.2 * cbrt(at)) : 0.0f;
  if (!shell_record_finite(*m)) return err.fail(THOR_ERR_INVALID_ARG, "shell opacity or line parameters overflow FP32");
  return THOR_OK;
}

int thor::shell_source_into_model(ErrSink err, const thor_source* src, ShellModel* m) {
  if (src->kind != 0) return err.fail(THOR_ERR_INVALID_ARG, "shells take source kind 0 (central point source)");
  for (double q : {src->X0, src->sigma, src->ew, src->C})
    if (!std::isfinite(q)) return err.fail(THOR_ERR_INVALID_ARG, "source parameters must be finite");
  if (!(src->sigma >= 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "source sigma must be >= 0");
  if (!(src->C >= 0.0) || !(src->ew >= 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "source ew and C must be >= 0");
  if (src->C > 0.0 && m->profile != THOR_PROFILE_POWER_LAW)
    return err.fail(THOR_ERR_INVALID_ARG, "a continuum source needs a power-law shell");
  if (src->C > 0.0 && !(src->sigma > 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "a continuum source needs sigma > 0");
  m->line = (src->sigma > 0.0) ? 1 : 0;
  m->X0 = (float)src->X0;
  m->sigma = (float)src->sigma;
  m->cont_C = (float)src->C;
  m->p_line = (src->C > 0.0) ? (float)(src->ew / (src->ew + 2.0 * src->C)) : 1.0f;
  return THOR_OK;
}

int thor::shell_model_from_params(ErrSink err, const thor_shell_params* p, ShellModel* m) {
  if (!p) return err.fail(THOR_ERR_INVALID_ARG, "shell parameters are NULL");
  for (double q : {p->R_in, p->R_out, p->N_HI, p->tau0, p->T, p->v_max, p->tau_dust, p->albedo, p->g_hg, p->step_dx,
                   p->alpha_rho, p->alpha_v})
    if (!std::isfinite(q)) return err.fail(THOR_ERR_INVALID_ARG, "shell parameters must be finite");
  if (!(p->R_out > 0.0) || !(p->R_in >= 0.0) || !(p->R_in < p->R_out))
    return err.fail(THOR_ERR_INVALID_ARG, "shell radii must satisfy 0 <= R_in < R_out");
  if (!(p->T > 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "temperature must be > 0");
  if (!(p->tau_dust >= 0.0) || !(p->albedo >= 0.0 && p->albedo <= 1.0) || !(p->g_hg > -1.0 && p->g_hg < 1.0))
    return err.fail(THOR_ERR_INVALID_ARG, "dust parameters out of range");
  if (p->phase < 0 || p->phase > 2) return err.fail(THOR_ERR_INVALID_ARG, "unknown phase function");
  if (!(p->v_max >= 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "v_max must be >= 0");
  if (p->profile != THOR_PROFILE_HOMOLOGOUS && p->profile != THOR_PROFILE_POWER_LAW)
    return err.fail(THOR_ERR_INVALID_ARG, "unknown density/velocity profile");
  if (p->profile == THOR_PROFILE_HOMOLOGOUS && p->species != THOR_SPECIES_HI)
    return err.fail(THOR_ERR_INVALID_ARG, "the Mg II doublet runs on power-law shells");
  if (p->profile == THOR_PROFILE_POWER_LAW) return fill_power_law(err, p, m);
  const double L = (p->R_out - p->R_in) / p->R_out;  // in units of R_out
  double tau0 = p->tau0;
  if (!(tau0 > 0.0)) {
    if (!(p->N_HI >= 0.0)) return err.fail(THOR_ERR_INVALID_ARG, "N_HI must be >= 0");
    tau0 = p->N_HI * line_sigma0(p->T);
  }
  std::memset(m, 0, sizeof(*m));
  m->R_in = p->R_in / p->R_out;
  m->R_out = 1.0;
  m->kap0 = (float)(tau0 / L);
  m->kapd = (float)(p->tau_dust / L);
  const double vth = line_vth_kms(p->T);
  m->vth = (float)vth;
  m->inv_vth = (float)(1.0 / vth);
  m->a = (float)line_a(p->T);
  m->vgrad = (float)p->v_max;  // km/s per R_out
  m->gam = (float)(p->v_max / vth);
  const double f = (p->step_dx > 0.0) ? p->step_dx : 0.01;
  m->ds_core = (p->v_max > 0.0) ? (float)(f * vth / p->v_max) : 1e30f;
  m->albedo = (float)p->albedo;
  m->g_hg = (float)p->g_hg;
  m->phase = p->phase;
  const double at = line_a(p->T) * tau0;
  m->xcrit = (p->core_skip && at >= 1.0) ? (float)(0.2 * cbrt(at)) : 0.0f;
  if (!shell_record_finite(*m)) return err.fail(THOR_ERR_INVALID_ARG, "shell opacity or line parameters overflow FP32");
  return THOR_OK;
}

int thor::fill_shell_source(thor_ctx* ctx, const thor_source* src, ShellModel* m) {
  char msg[256] = {0};
  const int rc = shell_source_into_model(ErrSink{msg, sizeof msg}, src, m);
  return rc ? ctx->fail(rc, "%s", msg) : THOR_OK;
}

int thor::fill_shell_model(thor_ctx* ctx, const thor_shell_params* p, ShellModel* m) {
  char msg[256] = {0};
  const int rc = shell_model_from_params(ErrSink{msg, sizeof msg}, p, m);
  return rc ? ctx->fail(rc, "%s", msg) : THOR_OK;
}

extern "C" int thor_shell_create(thor_ctx_t ctx, const thor_shell_params* p, thor_geom_t* out) {
  if (!ctx || !out) return THOR_ERR_INVALID_ARG;
  *out = nullptr;
  thor_geom* g = new thor_geom();
  g->ctx = ctx;
  g->kind = thor_geom::SHELL;
  int rc = fill_shell_model(ctx, p, &g->shell);
  if (rc != THOR_OK) { delete g; return rc; }
  g->shell_params = *p;
  *out = g;
  return THOR_OK;
}

static int copy_in(thor_ctx* ctx, const void* src, size_t bytes, int mem_kind, void* dst) {
  const cudaMemcpyKind k = (mem_kind == THOR_MEM_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  return ctx->cuda(cudaMemcpyAsync(dst, src, bytes, k, ctx->stream), "copy to device");
}

extern "C" int thor_grid_create(thor_ctx_t ctx, const float* n_HI, const float* T, const float* v, const float* dust,
                                const int32_t dims[3], double cell_cm, int mem_kind, thor_geom_t* out) {
  if (!ctx || !out) return THOR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!n_HI || !T || !v || !dims) return ctx->fail(THOR_ERR_INVALID_ARG, "thor_grid_create: NULL field");
  if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) return ctx->fail(THOR_ERR_INVALID_ARG, "bad dims");
  if (!(cell_cm > 0.0)) return ctx->fail(THOR_ERR_INVALID_ARG, "cell size must be > 0");
  if (mem_kind != THOR_MEM_HOST && mem_kind != THOR_MEM_DEVICE) return ctx->fail(THOR_ERR_INVALID_ARG, "mem_kind");
  if (int rc = ctx->select()) return rc;
  const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
  thor_geom* g = new thor_geom();
  g->ctx = ctx;
  g->kind = thor_geom::GRID;
  for (int a = 0; a < 3; ++a) g->dims[a] = dims[a];
  g->cell_cm = cell_cm;
  g->n_cells = n;
  const size_t fb = (size_t)n * sizeof(float);
  float* stage = nullptr;
  int rc = THOR_OK;
  if (cudaMalloc(&g->cells, (size_t)n * sizeof(GridCell)) != cudaSuccess ||
      cudaMalloc(&g->cdf, (size_t)n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&g->scan_tmp, scan_f64_scratch(n) + sizeof(unsigned long long)) != cudaSuccess) {
    delete g;
    return ctx->fail(THOR_ERR_OOM, "thor_grid_create: cannot allocate %lld cells", (long long)n);
  }
  const float *dn = n_HI, *dT = T, *dvx = v, *dvy = v + n, *dvz = v + 2 * n, *dd = dust;
  if (mem_kind == THOR_MEM_HOST) {  // stage the six fields on the device
    const int nf = dust ? 6 : 5;
    if (cudaMalloc(&stage, fb * nf) != cudaSuccess) {
      delete g;
      return ctx->fail(THOR_ERR_OOM, "thor_grid_create: cannot stage fields");
    }
    const float* srcs[6] = {n_HI, T, v, v + n, v + 2 * n, dust};
    for (int f = 0; f < nf && rc == THOR_OK; ++f) rc = copy_in(ctx, srcs[f], fb, THOR_MEM_HOST, stage + f * (size_t)n);
    dn = stage; dT = stage + n; dvx = stage + 2 * n; dvy = stage + 3 * n; dvz = stage + 4 * n;
    dd = dust ? stage + 5 * n : nullptr;
  }
  // unusable cells are counted on the device (the fields may be device-resident)
  unsigned long long* d_bad =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(g->scan_tmp) + scan_f64_scratch(n));
  if (rc == THOR_OK) rc = ctx->cuda(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), ctx->stream), "grid check");
  if (rc == THOR_OK)
    rc = ctx->cuda(launch_grid_pack(dn, dT, dvx, dvy, dvz, dd, n, cell_cm, g->cells, g->cdf, d_bad, ctx->stream),
                   "grid pack");
  if (rc == THOR_OK) rc = ctx->cuda(launch_scan_f64(g->cdf, n, g->scan_tmp, ctx->stream), "emission CDF");
  if (rc == THOR_OK) rc = ctx->cuda(cudaStreamSynchronize(ctx->stream), "grid create");
  if (stage) cudaFree(stage);
  if (rc != THOR_OK) { delete g; return rc; }
  unsigned long long bad = 0;
  double total = 0.0;
  if ((rc = ctx->cuda(cudaMemcpy(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost), "grid check")) ||
      (rc = ctx->cuda(cudaMemcpy(&total, g->cdf + (n - 1), sizeof(double), cudaMemcpyDeviceToHost), "grid CDF"))) {
    delete g;
    return rc;
  }
  if (bad) {
    delete g;
    return ctx->fail(THOR_ERR_INVALID_ARG,
                     "thor_grid_create: %llu cells out of range (need T > 0, n_HI >= 0, dust >= 0, all finite)", bad);
  }
  if (!(total > 0.0)) { delete g; return ctx->fail(THOR_ERR_INVALID_ARG, "thor_grid_create: n_HI is zero everywhere"); }
  *out = g;
  return THOR_OK;
}

thor_geom::~thor_geom() {
  if (ctx) cudaSetDevice(ctx->device);
  if (cells) cudaFree(cells);
  if (cdf) cudaFree(cdf);
  if (scan_tmp) cudaFree(scan_tmp);
}

extern "C" void thor_geom_destroy(thor_geom_t g) { delete g; }

// ------------------------------------------------------------------------------ run
int thor::prepare_outputs(thor_ctx* ctx, const thor_output_spec* spec, uint64_t n_photons, bool grid, OutBufs* o) {
  if (!spec || !spec->spectrum) return ctx->fail(THOR_ERR_INVALID_ARG, "output spec / spectrum is NULL");
  if (spec->n_bins <= 0 || !(spec->X_max > spec->X_min)) return ctx->fail(THOR_ERR_INVALID_ARG, "bad spectrum binning");
  if (spec->mem_kind != THOR_MEM_HOST && spec->mem_kind != THOR_MEM_DEVICE)
    return ctx->fail(THOR_ERR_INVALID_ARG, "bad output mem_kind");
  const bool dev = spec->mem_kind == THOR_MEM_DEVICE;
  const size_t sb = (size_t)(spec->n_bins + 2) * sizeof(uint64_t);
  o->spec = dev ? (unsigned long long*)spec->spectrum : (unsigned long long*)ctx->scratch(ctx->b_spec, sb);
  if (!o->spec) return ctx->fail(THOR_ERR_OOM, "spectrum buffer");
  if (int rc = ctx->cuda(cudaMemsetAsync(o->spec, 0, sb, ctx->stream), "clear spectrum")) return rc;
  o->cube = nullptr;
  if (grid && spec->peel) {
    if (!spec->cube || spec->img_n <= 0 || spec->peel_bins <= 0 || !(spec->peel_X_max > spec->peel_X_min))
      return ctx->fail(THOR_ERR_INVALID_ARG, "bad peeling-off spec");
    const size_t cb = (size_t)3 * spec->img_n * spec->img_n * spec->peel_bins * sizeof(float);
    o->cube = dev ? spec->cube : (float*)ctx->scratch(ctx->b_cube, cb);
    if (!o->cube) return ctx->fail(THOR_ERR_OOM, "cube buffer");
    if (int rc = ctx->cuda(cudaMemsetAsync(o->cube, 0, cb, ctx->stream), "clear cube")) return rc;
  }
  o->raw_X = nullptr; o->raw_n = nullptr; o->raw_s = nullptr; o->raw_X0 = nullptr; o->raw_col = nullptr;
  if (spec->raw_X0 || spec->raw_col) {
    if (grid) return ctx->fail(THOR_ERR_INVALID_ARG, "raw_X0 / raw_col are shell records");
    if (dev) {
      o->raw_X0 = spec->raw_X0; o->raw_col = spec->raw_col;
    } else {
      char* p = (char*)ctx->scratch(ctx->b_raw2, (size_t)n_photons * 8 + 64);
      if (!p) return ctx->fail(THOR_ERR_OOM, "raw buffers");
      if (spec->raw_X0) o->raw_X0 = (float*)p;
      if (spec->raw_col) o->raw_col = (float*)(p + 4 * n_photons);
    }
  }
  if (spec->raw_X || spec->raw_nscat || spec->raw_status) {
    if (!spec->raw_X || !spec->raw_nscat || !spec->raw_status)
      return ctx->fail(THOR_ERR_INVALID_ARG, "raw_X, raw_nscat and raw_status go together");
    if (dev) {
      o->raw_X = spec->raw_X; o->raw_n = spec->raw_nscat; o->raw_s = spec->raw_status;
    } else {
      const size_t rb = (size_t)n_photons * 9 + 64;
      char* p = (char*)ctx->scratch(ctx->b_raw, rb);
      if (!p) return ctx->fail(THOR_ERR_OOM, "raw buffers");
      o->raw_X = (float*)p;
      o->raw_n = (uint32_t*)(p + 4 * n_photons);
      o->raw_s = (uint8_t*)(p + 8 * n_photons);
    }
  }
  return THOR_OK;
}

int thor::finish_outputs(thor_ctx* ctx, const thor_output_spec* spec, uint64_t n_photons, bool grid, const OutBufs& o) {
  if (spec->mem_kind == THOR_MEM_DEVICE) return THOR_OK;
  cudaStream_t s = ctx->stream;
  int rc = ctx->cuda(cudaMemcpyAsync(spec->spectrum, o.spec, (size_t)(spec->n_bins + 2) * 8, cudaMemcpyDeviceToHost, s),
                     "copy spectrum");
  if (rc == THOR_OK && o.cube)
    rc = ctx->cuda(cudaMemcpyAsync(spec->cube, o.cube, (size_t)3 * spec->img_n * spec->img_n * spec->peel_bins * 4,
                                   cudaMemcpyDeviceToHost, s), "copy cube");
  if (rc == THOR_OK && o.raw_X) {
    rc = ctx->cuda(cudaMemcpyAsync(spec->raw_X, o.raw_X, n_photons * 4, cudaMemcpyDeviceToHost, s), "copy raw");
    if (rc == THOR_OK) rc = ctx->cuda(cudaMemcpyAsync(spec->raw_nscat, o.raw_n, n_photons * 4, cudaMemcpyDeviceToHost, s), "copy raw");
    if (rc == THOR_OK) rc = ctx->cuda(cudaMemcpyAsync(spec->raw_status, o.raw_s, n_photons, cudaMemcpyDeviceToHost, s), "copy raw");
  }
  if (rc == THOR_OK && o.raw_X0)
    rc = ctx->cuda(cudaMemcpyAsync(spec->raw_X0, o.raw_X0, n_photons * 4, cudaMemcpyDeviceToHost, s), "copy raw");
  if (rc == THOR_OK && o.raw_col)
    rc = ctx->cuda(cudaMemcpyAsync(spec->raw_col, o.raw_col, n_photons * 4, cudaMemcpyDeviceToHost, s), "copy raw");
  return rc;
}

void thor::tally_to_result(const Tally& t, uint64_t n_photons, thor_result* r) {
  r->n_photons = n_photons;
  r->n_escaped = t.n_escaped; r->n_absorbed = t.n_absorbed; r->n_capped = t.n_capped;
  r->n_scat = t.n_scat; r->n_dust_scat = t.n_dust_scat; r->n_upar_iters = t.n_upar_iters;
  r->n_steps = t.n_steps; r->sum_scat2 = t.sum_scat2;
}

// Event-based grid loop (thor_ctx_set_grid_exec): rounds of (move, resonant scatterings,
// peel rays) over the slots until no new photons are left and at most grid_handoff packets
// remain, then the one-kernel loop finishes them.  The host checks the counters every
// kCheck rounds (one small copy and a sync); between checks rounds are queued back to back.
template <class PerWarp>
static int run_grid_events(thor_ctx* ctx, thor::GridModel m, thor::WorkQueue q, int gsz,
                           PerWarp per_warp, unsigned long long* n_launch) {
  using namespace thor;
  constexpr int kCheck = 8;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->grid_slots;
  void* base = ctx->scratch(ctx->b_gslots, grid_slots_bytes(n));
  if (!base) return ctx->fail(THOR_ERR_OOM, "event-based grid loop: %lld slots", (long long)n);
  GridSlots S = grid_slots_carve(base, n);
  int rc;
  if ((rc = ctx->cuda(cudaMemsetAsync(S.live, 0, (size_t)n, s), "clear slots"))) return rc;
  if ((rc = ctx->cuda(cudaMemsetAsync(S.ctr, 0, 16 * 8, s), "clear slot counters"))) return rc;
  if ((rc = ctx->cuda(cudaMemsetAsync(S.slab, 0, (size_t)kGridSlabBlocks * sizeof(TallySlab), s), "clear slab")))
    return rc;
  cudaEventRecord(ctx->ev0, s);
  int64_t r = 0;
  unsigned long long h[2] = {0, 0};  // packets in flight, photons taken from the queue
  for (;;) {
    for (int k = 0; k < kCheck; ++k, ++r) {
      if ((rc = ctx->cuda(launch_grid_round(m, q, S, (int)(r & 1), ctx->d_ktab, ctx->block, s), "grid round")))
        return rc;
      *n_launch += 3;
    }
    if ((rc = ctx->cuda(cudaMemcpyAsync(&h[0], S.ctr, 8, cudaMemcpyDeviceToHost, s), "slot counters"))) return rc;
    if ((rc = ctx->cuda(cudaMemcpyAsync(&h[1], q.next, 8, cudaMemcpyDeviceToHost, s), "queue counter"))) return rc;
    if ((rc = ctx->cuda(cudaStreamSynchronize(s), "grid rounds"))) return rc;
    if (h[1] >= q.total && (long long)h[0] <= ctx->grid_handoff) break;
  }
  ctx->grid_rounds_last = r;
  // peel rays still walking after the last round (parity (r - 1) & 1) are in the other queue
  if ((rc = ctx->cuda(launch_grid_ray_drain(m, S, (int)(r & 1), ctx->d_ktab, ctx->block, s), "peel rays"))) return rc;
  if ((rc = ctx->cuda(launch_grid_slab_sum(m, S, s), "round counters"))) return rc;
  *n_launch += 2;
  if (h[0] > 0) {  // the tail: the one-kernel loop resumes the packets in flight
    if ((rc = ctx->cuda(cudaMemsetAsync(S.ctr + 2, 0, 16, s), "clear resume list"))) return rc;
    if ((rc = ctx->cuda(launch_grid_list_live(S, s), "list packets in flight"))) return rc;
    m.per_warp = per_warp(h[0]);
    if ((rc = ctx->cuda(launch_grid_resume(m, q, S, ctx->d_ktab, gsz, ctx->block, s), "grid photon loop (tail)")))
      return rc;
    *n_launch += 2;
  }
  cudaEventRecord(ctx->ev1, s);
  return THOR_OK;
}

extern "C" int thor_run(thor_ctx_t ctx, thor_geom_t g, const thor_source* src, uint64_t first_id, uint64_t n_photons,
                        uint64_t seed, const thor_output_spec* spec, thor_result* out) {
  if (!ctx || !g || !src || !out) return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_run: NULL argument") : THOR_ERR_INVALID_ARG;
  if (g->ctx != ctx) return ctx->fail(THOR_ERR_INVALID_ARG, "geometry belongs to another context");
  if (n_photons == 0) return ctx->fail(THOR_ERR_INVALID_ARG, "n_photons must be > 0");
  if (first_id + n_photons < first_id) return ctx->fail(THOR_ERR_INVALID_ARG, "photon id range overflows");
  const bool grid = g->kind == thor_geom::GRID;
  if (grid && src->kind != 1) return ctx->fail(THOR_ERR_INVALID_ARG, "grids take source kind 1 (gas emission)");
  if (!grid && src->kind != 0) return ctx->fail(THOR_ERR_INVALID_ARG, "shells take source kind 0 (central point source)");
  if (!grid && !(src->sigma >= 0.0)) return ctx->fail(THOR_ERR_INVALID_ARG, "source sigma must be >= 0");
  if (grid && spec && spec->peel && spec->img_n > 0 &&
      (g->dims[0] % spec->img_n || g->dims[1] % spec->img_n || g->dims[2] % spec->img_n))
    return ctx->fail(THOR_ERR_INVALID_ARG, "img_n must divide the grid dimensions");
  if (int rc = ctx->select()) return rc;
  OutBufs o;
  if (int rc = prepare_outputs(ctx, spec, n_photons, grid, &o)) return rc;
  cudaStream_t s = ctx->stream;
  // per-run device scratch: tally, queue counter + tables, model record, peel statistics
  Tally* d_tally = (Tally*)ctx->scratch(ctx->b_tally, sizeof(Tally));
  char* qb = (char*)ctx->scratch(ctx->b_queue, 256);
  unsigned long long* d_stats = (unsigned long long*)ctx->scratch(ctx->b_stats, 2 * sizeof(unsigned long long));
  if (!d_tally || !qb || !d_stats) return ctx->fail(THOR_ERR_OOM, "run scratch");
  struct QHost { unsigned long long next, prefix[2], first_id; int32_t model; } qh{0, {0, n_photons}, first_id, 0};
  if (int rc = ctx->cuda(cudaMemcpyAsync(qb, &qh, sizeof qh, cudaMemcpyHostToDevice, s), "queue upload")) return rc;
  if (int rc = ctx->cuda(cudaMemsetAsync(d_tally, 0, sizeof(Tally), s), "clear tally")) return rc;
  if (int rc = ctx->cuda(cudaMemsetAsync(d_stats, 0, 16, s), "clear stats")) return rc;
  unsigned long long n_launch = 0;
  WorkQueue q;
  q.next = (unsigned long long*)(qb + offsetof(QHost, next));
  q.total = n_photons;
  q.prefix = (const unsigned long long*)(qb + offsetof(QHost, prefix));
  q.first_id = (const unsigned long long*)(qb + offsetof(QHost, first_id));
  q.model = (const int32_t*)(qb + offsetof(QHost, model));
  q.n_entries = 1;
  int rc = THOR_OK;
  if (!grid) {
    ShellModel m = g->shell;
    if ((rc = fill_shell_source(ctx, src, &m))) return rc;
    if (o.raw_col && m.profile != THOR_PROFILE_POWER_LAW)
      return ctx->fail(THOR_ERR_INVALID_ARG, "raw_col is recorded on power-law shells");
    m.raw_X0 = o.raw_X0; m.raw_col = o.raw_col;
    m.X_min = (float)spec->X_min;
    m.inv_dX = spectrum_inv_dX(spec->n_bins, spec->X_min, spec->X_max);
    m.n_bins = spec->n_bins;
    m.seed_lo = (uint32_t)seed; m.seed_hi = (uint32_t)(seed >> 32);
    m.max_scat = spec->max_scat;
    m.spectrum = o.spec;
    m.tally = d_tally;
    m.raw_X = o.raw_X; m.raw_nscat = o.raw_n; m.raw_status = o.raw_s;
    m.id_base = first_id;
    m.n_photons = n_photons;
    ShellModel* d_m = (ShellModel*)ctx->scratch(ctx->b_models, sizeof(ShellModel));
    if (!d_m) return ctx->fail(THOR_ERR_OOM, "model table");
    if ((rc = ctx->cuda(cudaMemcpyAsync(d_m, &m, sizeof m, cudaMemcpyHostToDevice, s), "model upload"))) return rc;
    const int gsz = shell_grid(ctx->block, ctx->blocks_per_sm, false);
    // fewer photons than lanes: spread them over all warps (each runs closer to alone)
    const unsigned long long warps0 = (unsigned long long)gsz * (ctx->block / 32);
    const unsigned long long pw0 = (n_photons + warps0 - 1) / warps0;
    const int per_warp0 = (int)(pw0 < 1 ? 1 : (pw0 > 32 ? 32 : pw0));
    if (ctx->spill_below <= 0) {
      // work sharing in the tail: a pool of one record per photon, its ready flags, counters
      Compact sh{};
      const bool share = ctx->share_tail != 0 && n_photons > warps0;  // else every photon has a warp already
      if (share) {
        auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t b_pool = r256((size_t)n_photons * sizeof(PhotonRec)), b_ready = r256((size_t)n_photons * 4);
        char* sb = (char*)ctx->scratch(ctx->b_share, b_pool + b_ready + 64);
        if (!sb) return ctx->fail(THOR_ERR_OOM, "tail work-sharing pool");
        sh.pool = (PhotonRec*)sb;
        sh.ready = (uint32_t*)(sb + b_pool);
        sh.share = (unsigned long long*)(sb + b_pool + b_ready);
        sh.n_total = n_photons;
        if ((rc = ctx->cuda(cudaMemsetAsync(sh.ready, 0, b_ready + 64, s), "clear sharing pool"))) return rc;
      }
      cudaEventRecord(ctx->ev0, s);
      rc = ctx->cuda(launch_shell_run(d_m, q, ctx->d_ktab, gsz, ctx->block, m.profile, per_warp0, ctx->core_lanes,
                                      ctx->burst_lanes, s, share ? &sh : nullptr),
                     "shell photon loop");
      ++n_launch;
      if (!rc && share) {
        // packets left in the pool (every waiting warp gave up first) finish in a relaunch
        unsigned long long h[5];
        if ((rc = ctx->cuda(cudaMemcpyAsync(h, sh.share, sizeof h, cudaMemcpyDeviceToHost, s), "sharing counters")))
          return rc;
        if ((rc = ctx->cuda(cudaStreamSynchronize(s), "shell photon loop"))) return rc;
        if (h[4]) return ctx->fail(THOR_ERR_DEVICE, "tail work sharing: a packet given away was never written");
        if (h[1] < h[0]) {
          unsigned long long* ctr = (unsigned long long*)ctx->scratch(ctx->b_cmp, 4 * sizeof(unsigned long long));
          if (!ctr) return ctx->fail(THOR_ERR_OOM, "resume counters");
          if ((rc = ctx->cuda(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s), "clear counters"))) return rc;
          Compact c{};
          c.resume = sh.pool + h[1];
          c.n_resume = h[0] - h[1];
          c.resume_next = ctr;
          c.spill = nullptr;
          c.n_spill = ctr + 1;
          c.spill_below = 0;
          c.per_warp = 1;
          c.core_lanes = ctx->core_lanes;
          c.burst_lanes = ctx->burst_lanes;
          const unsigned long long want = (c.n_resume * 32 + ctx->block - 1) / ctx->block;
          const int g = (int)(want < (unsigned long long)gsz ? want : gsz);
          if ((rc = ctx->cuda(launch_shell_run_compact(d_m, q, c, ctx->d_ktab, g, ctx->block, m.profile, s),
                              "shell photon loop (pool)")))
            return rc;
          ++n_launch;
        }
      }
      cudaEventRecord(ctx->ev1, s);
    } else {
      // Tail compaction: launch, then relaunch over the saved survivors until none are
      // left (the last phase runs to completion).  A relaunch packs per_warp survivors
      // into each warp, per_warp chosen so that the survivors fill about kWarpsPerSmsp
      // warps on every scheduler: once few packets are left each one runs alone in its
      // warp, at the latency of a lone lane, instead of waiting on 31 divergent others.
      const unsigned long long lanes = (unsigned long long)gsz * ctx->block;
      const unsigned long long cap = n_photons < lanes ? n_photons : lanes;
      PhotonRec* bufs = (PhotonRec*)ctx->scratch(ctx->b_spill, 2 * cap * sizeof(PhotonRec));
      unsigned long long* ctr = (unsigned long long*)ctx->scratch(ctx->b_cmp, 4 * sizeof(unsigned long long));
      if (!bufs || !ctr) return ctx->fail(THOR_ERR_OOM, "tail compaction buffers");
      PhotonRec* in = bufs;
      PhotonRec* outb = bufs + cap;
      unsigned long long n_in = 0;
      cudaEventRecord(ctx->ev0, s);
      for (int phase = 0;; ++phase) {
        const bool last = phase + 1 >= ctx->max_phases || (phase > 0 && n_in <= (unsigned long long)ctx->final_below);
        if ((rc = ctx->cuda(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s), "clear counters"))) break;
        Compact c{};
        c.resume = in;
        c.n_resume = n_in;
        c.resume_next = ctr;
        c.spill = outb;
        c.n_spill = ctr + 1;
        c.spill_below = last ? 0 : ctx->spill_below;
        c.per_warp = per_warp0;
        c.core_lanes = ctx->core_lanes;
        c.burst_lanes = ctx->burst_lanes;
        if (per_warp0 <= 2) c.spill_below = 0;
        else if (c.spill_below > per_warp0 / 2) c.spill_below = per_warp0 / 2;
        int g = gsz;
        if (phase > 0) {
          const unsigned long long warps_target = (unsigned long long)ctx->sm_count * 4 * kWarpsPerSmsp;
          unsigned long long pw = (n_in + warps_target - 1) / warps_target;
          pw = pw < 1 ? 1 : (pw > 32 ? 32 : pw);
          c.per_warp = (int)pw;
          // a warp spills once fewer than half its resumed packets are live; one or two
          // per warp run to completion
          if (pw <= 2) c.spill_below = 0;
          else if (c.spill_below > (int)pw / 2) c.spill_below = (int)pw / 2;
          const unsigned long long warps = (n_in + pw - 1) / pw;
          const unsigned long long want = (warps * 32 + ctx->block - 1) / ctx->block;
          g = (int)(want < (unsigned long long)gsz ? want : gsz);
        }
        const bool final_phase = last || c.spill_below == 0;
        if ((rc = ctx->cuda(launch_shell_run_compact(d_m, q, c, ctx->d_ktab, g, ctx->block, m.profile, s),
                            "shell photon loop")))
          break;
        ++n_launch;
        if (final_phase) break;
        unsigned long long n_out = 0;
        if ((rc = ctx->cuda(cudaMemcpyAsync(&n_out, ctr + 1, sizeof n_out, cudaMemcpyDeviceToHost, s), "spill count")))
          break;
        if ((rc = ctx->cuda(cudaStreamSynchronize(s), "tail phase"))) break;
        if (n_out == 0) break;
        n_in = n_out;
        PhotonRec* t = in; in = outb; outb = t;
        ++ctx->phases_last;
      }
      cudaEventRecord(ctx->ev1, s);
    }
  } else {
    GridModel m;
    std::memset(&m, 0, sizeof m);
    m.cells = g->cells; m.cdf = g->cdf;
    m.nx = g->dims[0]; m.ny = g->dims[1]; m.nz = g->dims[2];
    m.phase = g->grid_phase;
    m.albedo = (float)g->grid_albedo; m.g_hg = (float)g->grid_g;
    m.X_min = (float)spec->X_min; m.inv_dX = spectrum_inv_dX(spec->n_bins, spec->X_min, spec->X_max);
    m.n_bins = spec->n_bins;
    m.peel = (spec->peel && o.cube) ? 1 : 0;
    m.img_n = spec->img_n; m.peel_bins = spec->peel_bins;
    if (m.peel) {
      m.pX_min = (float)spec->peel_X_min;
      m.pinv_dX = spectrum_inv_dX(spec->peel_bins, spec->peel_X_min, spec->peel_X_max);
    }
    m.tau_cut = 50.0f;
    m.max_scat = spec->max_scat;
    m.seed_lo = (uint32_t)seed; m.seed_hi = (uint32_t)(seed >> 32);
    m.spectrum = o.spec; m.cube = o.cube; m.tally = d_tally;
    m.n_photons = n_photons; m.id_base = first_id;
    m.peel_rays = d_stats; m.peel_cells = d_stats + 1;
    m.raw_X = o.raw_X; m.raw_nscat = o.raw_n; m.raw_status = o.raw_s;
    const int gsz = grid_grid(ctx->block, ctx->blocks_per_sm);
    // few photons: spread them so that each runs in a warp of its own where possible
    const unsigned long long warps = (unsigned long long)gsz * (ctx->block / 32);
    auto per_warp = [&](unsigned long long n) {
      const unsigned long long pw = (n + warps - 1) / warps;
      return (int)(pw < 1 ? 1 : (pw > 32 ? 32 : pw));
    };
    m.per_warp = per_warp(n_photons);
    ctx->grid_rounds_last = 0;
    if (ctx->grid_slots <= 0) {
      cudaEventRecord(ctx->ev0, s);
      rc = ctx->cuda(launch_grid_run(m, q, ctx->d_ktab, gsz, ctx->block, s), "grid photon loop");
      ++n_launch;
      cudaEventRecord(ctx->ev1, s);
    } else {
      rc = run_grid_events(ctx, m, q, gsz, per_warp, &n_launch);
    }
  }
  if (rc) return rc;
  Tally t;
  unsigned long long st[2];
  if ((rc = ctx->cuda(cudaMemcpyAsync(&t, d_tally, sizeof t, cudaMemcpyDeviceToHost, s), "copy tally"))) return rc;
  if ((rc = ctx->cuda(cudaMemcpyAsync(st, d_stats, sizeof st, cudaMemcpyDeviceToHost, s), "copy stats"))) return rc;
  if ((rc = finish_outputs(ctx, spec, n_photons, grid, o))) return rc;
  if ((rc = ctx->cuda(cudaStreamSynchronize(s), "photon loop"))) return rc;
  std::memset(out, 0, sizeof *out);
  tally_to_result(t, n_photons, out);
  out->n_peel_rays = st[0];
  out->n_peel_cells = st[1];
  out->n_launches = n_launch;
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  out->elapsed_ms = ms;
  if (t.n_done != n_photons) return ctx->fail(THOR_ERR_DEVICE, "photon loop finished %llu of %llu photons",
                                              (unsigned long long)t.n_done, (unsigned long long)n_photons);
  ctx->last_error.clear();
  return THOR_OK;
}

// Grid scattering parameters are set on the geometry (albedo, g, phase) -- exposed
// through thor_grid_set_scattering in thor_ctx.h for the Python binding.
extern "C" int thor_grid_set_scattering(thor_geom_t g, int phase, double albedo, double g_hg) {
  if (!g || g->kind != thor_geom::GRID) return THOR_ERR_INVALID_ARG;
  if (phase < 0 || phase > 2 || !(albedo >= 0.0 && albedo <= 1.0) || !(g_hg > -1.0 && g_hg < 1.0))
    return g->ctx->fail(THOR_ERR_INVALID_ARG, "bad grid scattering parameters");
  g->grid_phase = phase;
  g->grid_albedo = albedo;
  g->grid_g = g_hg;
  return THOR_OK;
}

// ------------------------------------------------------------------------------ forest
extern "C" int thor_forest(thor_ctx_t ctx, const float* n_HI, const float* T, const float* v_los, const int32_t dims[3],
                           int mem_kind, const thor_forest_spec* sp, float* tau_out) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (!n_HI || !T || !v_los || !dims || !sp || !tau_out) return ctx->fail(THOR_ERR_INVALID_ARG, "thor_forest: NULL argument");
  if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) return ctx->fail(THOR_ERR_INVALID_ARG, "bad dims");
  if (sp->n_bins <= 0 || sp->n_bins > 2048) return ctx->fail(THOR_ERR_INVALID_ARG, "n_bins must be in [1, 2048]");
  if (!(sp->ds_cm > 0.0) || !(sp->dv_cell > 0.0) || !(sp->dv_bin > 0.0))
    return ctx->fail(THOR_ERR_INVALID_ARG, "ds_cm, dv_cell, dv_bin must be > 0");
  const double V = dims[2] * sp->dv_cell;
  if (std::fabs(sp->n_bins * sp->dv_bin - V) > 1e-9 * V)
    return ctx->fail(THOR_ERR_INVALID_ARG, "n_bins * dv_bin must equal nz * dv_cell (periodic spectrum)");
  const int64_t ncol = (int64_t)dims[0] * dims[1];
  if (sp->first_sightline < 0 || sp->n_sightlines <= 0 || sp->first_sightline + sp->n_sightlines > ncol)
    return ctx->fail(THOR_ERR_INVALID_ARG, "sightline range outside the grid");
  if (mem_kind != THOR_MEM_HOST && mem_kind != THOR_MEM_DEVICE) return ctx->fail(THOR_ERR_INVALID_ARG, "mem_kind");
  if (int rc = ctx->select()) return rc;
  cudaStream_t s = ctx->stream;
  int rc = THOR_OK;
  if (mem_kind == THOR_MEM_DEVICE) {
    cudaEventRecord(ctx->ev0, s);
    rc = ctx->cuda(launch_forest(n_HI, T, v_los, dims[0], dims[1], dims[2], sp->first_sightline, sp->n_sightlines,
                                 sp->ds_cm, sp->dv_cell, sp->n_bins, sp->dv_bin, tau_out, ctx->d_ktab, s),
                   "forest kernel");
    cudaEventRecord(ctx->ev1, s);
    if (!rc) rc = ctx->cuda(cudaStreamSynchronize(s), "forest");
    if (!rc) cudaEventElapsedTime(&ctx->last_ms, ctx->ev0, ctx->ev1);
    return rc;
  }
  // Host arrays: the box is streamed through two reused staging buffers in chunks of rows
  // (all z of rows iy in [y0, y1): per field one strided copy, nz runs of (y1 - y0) nx
  // floats), each chunk's sightlines computed while the next chunk is copied in on a second
  // stream; optical depths go back row chunk by row chunk.  No allocation per call once the
  // buffers have grown to a chunk.
  const int nx = dims[0], ny = dims[1], nz = dims[2];
  constexpr size_t kStageBytes = (size_t)1 << 30;  // per buffer
  const size_t row_bytes = (size_t)nx * ((size_t)3 * nz + (size_t)sp->n_bins) * 4;
  if (sp->stage_rows < 0) return ctx->fail(THOR_ERR_INVALID_ARG, "thor_forest: stage_rows must be >= 0");
  const int rows = sp->stage_rows > 0 ? std::min(sp->stage_rows, ny)
                                      : (int)std::max<size_t>(1, std::min<size_t>((size_t)ny, kStageBytes / row_bytes));
  if (!ctx->copy_stream) {
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return ctx->fail(THOR_ERR_DEVICE, "thor_forest: copy stream");
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_done[b], cudaEventDisableTiming) != cudaSuccess)
        return ctx->fail(THOR_ERR_DEVICE, "thor_forest: events");
  }
  char* buf[2];
  for (int b = 0; b < 2; ++b) {
    buf[b] = (char*)ctx->scratch(ctx->b_stage[b], (size_t)rows * row_bytes);
    if (!buf[b]) return ctx->fail(THOR_ERR_OOM, "thor_forest: staging buffers");
  }
  const int64_t s_lo = sp->first_sightline, s_hi = sp->first_sightline + sp->n_sightlines;
  const int y_first = (int)(s_lo / nx), y_last = (int)((s_hi - 1) / nx);
  cudaStream_t cs = ctx->copy_stream;
  const size_t plane = (size_t)nx * ny * 4;
  cudaEventRecord(ctx->ev0, s);
  int chunk = 0;
  for (int y0 = y_first; y0 <= y_last && !rc; y0 += rows, ++chunk) {
    const int y1 = std::min(y0 + rows, y_last + 1), nr = y1 - y0;
    const int b = chunk & 1;
    float* f = (float*)buf[b];
    const size_t nf = (size_t)nr * nx * nz;
    float* dtau = f + 3 * nf;
    // the buffer's previous chunk must be computed and copied out before it is overwritten
    if (chunk >= 2) rc = ctx->cuda(cudaStreamWaitEvent(cs, ctx->ev_done[b], 0), "forest order");
    const float* src[3] = {n_HI, T, v_los};
    for (int k = 0; k < 3 && !rc; ++k)
      rc = ctx->cuda(cudaMemcpy2DAsync(f + k * nf, (size_t)nr * nx * 4, (const char*)src[k] + (size_t)y0 * nx * 4,
                                       plane, (size_t)nr * nx * 4, (size_t)nz, cudaMemcpyHostToDevice, cs),
                     "forest copy in");
    if (!rc) rc = ctx->cuda(cudaEventRecord(ctx->ev_copied[b], cs), "forest order");
    if (!rc) rc = ctx->cuda(cudaStreamWaitEvent(s, ctx->ev_copied[b], 0), "forest order");
    // sightlines of this chunk inside the requested range, relative to the chunk's rows
    const int64_t c_lo = std::max<int64_t>(s_lo, (int64_t)y0 * nx), c_hi = std::min<int64_t>(s_hi, (int64_t)y1 * nx);
    if (!rc)
      rc = ctx->cuda(launch_forest(f, f + nf, f + 2 * nf, nx, nr, nz, c_lo - (int64_t)y0 * nx, c_hi - c_lo, sp->ds_cm,
                                   sp->dv_cell, sp->n_bins, sp->dv_bin, dtau, ctx->d_ktab, s),
                     "forest kernel");
    if (!rc)
      rc = ctx->cuda(cudaMemcpyAsync(tau_out + (size_t)(c_lo - s_lo) * sp->n_bins, dtau,
                                     (size_t)(c_hi - c_lo) * sp->n_bins * 4, cudaMemcpyDeviceToHost, s),
                     "forest copy out");
    if (!rc) rc = ctx->cuda(cudaEventRecord(ctx->ev_done[b], s), "forest order");
  }
  cudaEventRecord(ctx->ev1, s);
  if (!rc) rc = ctx->cuda(cudaStreamSynchronize(s), "forest");
  if (!rc) cudaEventElapsedTime(&ctx->last_ms, ctx->ev0, ctx->ev1);
  return rc;
}

extern "C" double thor_last_elapsed_ms(thor_ctx_t ctx) { return ctx ? ctx->last_ms : -1.0; }

// ------------------------------------------------------------------------------ reweighting
// Spectrum parameters for the kernel: {pl / (sqrt(2 pi) sigma), 1 / (2 sigma^2), (1 - pl) / (2C), C, tau_d}.
static bool spectrum_params(const double* p, double tau_d, float* q) {
  const double sigma = p[0], ew = p[1], C = p[2];
  if (!(sigma > 0.0) || !(ew >= 0.0) || !(C >= 0.0) || !(tau_d >= 0.0)) return false;
  const double pl = (C > 0.0) ? ew / (ew + 2.0 * C) : 1.0;
  q[0] = (float)(pl / (2.5066282746310002 * sigma));
  q[1] = (float)(0.5 / (sigma * sigma));
  q[2] = (C > 0.0) ? (float)((1.0 - pl) / (2.0 * C)) : 0.0f;
  q[3] = (float)C;
  q[4] = (float)tau_d;
  return true;
}

extern "C" int thor_reweight(thor_ctx_t ctx, int64_t n, const float* X0, const float* X, const float* col,
                             const uint8_t* status, int mem_kind, const double sample[3], int32_t n_targets,
                             const double* targets, int32_t n_bins, double X_min, double X_max, double* out) {
  if (!ctx) return THOR_ERR_INVALID_ARG;
  if (n <= 0 || !X0 || !X || !col || !status || !sample || !targets || !out)
    return ctx->fail(THOR_ERR_INVALID_ARG, "thor_reweight: NULL or empty input");
  if (mem_kind != THOR_MEM_HOST && mem_kind != THOR_MEM_DEVICE) return ctx->fail(THOR_ERR_INVALID_ARG, "bad mem_kind");
  if (n_targets <= 0 || n_targets > 65535) return ctx->fail(THOR_ERR_INVALID_ARG, "n_targets in [1, 65535]");
  if (n_bins <= 0 || n_bins > 4096 || !(X_max > X_min)) return ctx->fail(THOR_ERR_INVALID_ARG, "bad binning");
  std::vector<float> prm((size_t)5 * (n_targets + 1));
  if (!spectrum_params(sample, 0.0, prm.data())) return ctx->fail(THOR_ERR_INVALID_ARG, "bad sampled spectrum");
  for (int t = 0; t < n_targets; ++t)
    if (!spectrum_params(targets + 4 * t, targets[4 * t + 3], prm.data() + 5 * (t + 1)))
      return ctx->fail(THOR_ERR_INVALID_ARG, "bad target %d", t);
  if (int rc = ctx->select()) return rc;
  cudaStream_t s = ctx->stream;
  const size_t ob = (size_t)n_targets * (n_bins + 2) * sizeof(double);
  const size_t pb = prm.size() * sizeof(float);
  const size_t ib = (mem_kind == THOR_MEM_HOST) ? (size_t)n * 13 + 64 : 0;
  char* d = (char*)ctx->scratch(ctx->b_diag, ob + pb + ib + 512);
  if (!d) return ctx->fail(THOR_ERR_OOM, "thor_reweight scratch");
  double* d_out = (double*)d;
  float* d_prm = (float*)(d + ((ob + 255) & ~(size_t)255));
  char* in = (char*)d_prm + ((pb + 255) & ~(size_t)255);
  const float *x0 = X0, *x = X, *c = col;
  const uint8_t* st = status;
  int rc = ctx->cuda(cudaMemsetAsync(d_out, 0, ob, s), "clear reweight output");
  if (!rc) rc = ctx->cuda(cudaMemcpyAsync(d_prm, prm.data(), pb, cudaMemcpyHostToDevice, s), "reweight params");
  if (!rc && mem_kind == THOR_MEM_HOST) {
    float* fx0 = (float*)in;
    float* fx = fx0 + n;
    float* fc = fx + n;
    uint8_t* fs = (uint8_t*)(fc + n);
    rc = ctx->cuda(cudaMemcpyAsync(fx0, X0, n * 4, cudaMemcpyHostToDevice, s), "reweight inputs");
    if (!rc) rc = ctx->cuda(cudaMemcpyAsync(fx, X, n * 4, cudaMemcpyHostToDevice, s), "reweight inputs");
    if (!rc) rc = ctx->cuda(cudaMemcpyAsync(fc, col, n * 4, cudaMemcpyHostToDevice, s), "reweight inputs");
    if (!rc) rc = ctx->cuda(cudaMemcpyAsync(fs, status, n, cudaMemcpyHostToDevice, s), "reweight inputs");
    x0 = fx0; x = fx; c = fc; st = fs;
  }
  if (rc) return rc;
  cudaEventRecord(ctx->ev0, s);
  rc = ctx->cuda(launch_reweight(n, x0, x, c, st, d_prm, n_targets, n_bins, X_min, X_max, d_out, ctx->sm_count, s),
                 "reweight kernel");
  cudaEventRecord(ctx->ev1, s);
  if (!rc) rc = ctx->cuda(cudaMemcpyAsync(out, d_out, ob, cudaMemcpyDeviceToHost, s), "reweight output");
  if (!rc) rc = ctx->cuda(cudaStreamSynchronize(s), "thor_reweight");
  if (rc) return rc;
  cudaEventElapsedTime(&ctx->last_ms, ctx->ev0, ctx->ev1);
  const double inv = 1.0 / (double)n;
  for (size_t i = 0; i < (size_t)n_targets * (n_bins + 2); ++i) out[i] *= inv;
  ctx->last_error.clear();
  return THOR_OK;
}

// ------------------------------------------------------------------------------ diagnostics
namespace {
// Stage small diagnostic buffers: device pointers pass through, host pointers are copied.
struct Stage {
  thor_ctx* ctx;
  int kind;
  std::vector<std::pair<void*, std::pair<void*, size_t>>> back;  // (host dst, (dev src, bytes))
  char* base = nullptr;
  size_t used = 0;
  void* in(const void* p, size_t bytes) {
    if (kind == THOR_MEM_DEVICE) return (void*)p;
    void* d = base + used;
    used += (bytes + 255) & ~(size_t)255;
    cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->stream);
    return d;
  }
  void* out(void* p, size_t bytes) {
    if (kind == THOR_MEM_DEVICE) return p;
    void* d = base + used;
    used += (bytes + 255) & ~(size_t)255;
    back.push_back({p, {d, bytes}});
    return d;
  }
  int finish() {
    for (auto& b : back) cudaMemcpyAsync(b.first, b.second.first, b.second.second, cudaMemcpyDeviceToHost, ctx->stream);
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "diagnostic kernel");
  }
};

int stage_begin(thor_ctx* ctx, int kind, size_t bytes, Stage* st) {
  st->ctx = ctx;
  st->kind = kind;
  if (kind != THOR_MEM_HOST && kind != THOR_MEM_DEVICE) return ctx->fail(THOR_ERR_INVALID_ARG, "mem_kind");
  if (int rc = ctx->select()) return rc;
  if (kind == THOR_MEM_HOST) {
    st->base = (char*)ctx->scratch(ctx->b_diag, bytes + 4096);
    if (!st->base) return ctx->fail(THOR_ERR_OOM, "diagnostic staging");
  }
  return THOR_OK;
}
}  // namespace

extern "C" int thor_voigt_eval(thor_ctx_t ctx, const float* a, const float* x, float* H, int64_t n, int precise,
                               int mem_kind) {
  if (!ctx || !a || !x || !H || n <= 0) return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_voigt_eval") : THOR_ERR_INVALID_ARG;
  Stage st;
  if (int rc = stage_begin(ctx, mem_kind, 3 * (size_t)n * 4 + 1024, &st)) return rc;
  const float* da = (const float*)st.in(a, n * 4);
  const float* dx = (const float*)st.in(x, n * 4);
  float* dH = (float*)st.out(H, n * 4);
  if (int rc = ctx->cuda(launch_voigt_eval(da, dx, dH, n, ctx->d_ktab, ctx->stream, precise), "voigt kernel")) return rc;
  return st.finish();
}

extern "C" int thor_xcw_eval(thor_ctx_t ctx, const float* a, float* xcw, int64_t n, int mem_kind) {
  if (!ctx || !a || !xcw || n <= 0) return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_xcw_eval") : THOR_ERR_INVALID_ARG;
  Stage st;
  if (int rc = stage_begin(ctx, mem_kind, 2 * (size_t)n * 4 + 1024, &st)) return rc;
  const float* da = (const float*)st.in(a, n * 4);
  float* dx = (float*)st.out(xcw, n * 4);
  if (int rc = ctx->cuda(launch_xcw_eval(da, dx, n, ctx->stream), "x_cw kernel")) return rc;
  return st.finish();
}

extern "C" int thor_issue_peak(thor_ctx_t ctx, int kind, double* warp_inst_per_s) {
  if (!ctx || !warp_inst_per_s || kind < 0 || kind > 1)
    return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_issue_peak: kind 0 (FMA) or 1 (MUFU ex2)") : THOR_ERR_INVALID_ARG;
  if (int rc = ctx->select()) return rc;
  const int block = 256, grid = ctx->sm_count * 8;  // 8 resident blocks of 256 per SM: 64 warps
  const int iters = (kind == 0) ? 8192 : 1024;
  float* sink = (float*)ctx->scratch(ctx->b_diag, (size_t)grid * block * 4);
  if (!sink) return ctx->fail(THOR_ERR_OOM, "thor_issue_peak");
  cudaStream_t s = ctx->stream;
  if (int rc = ctx->cuda(launch_issue_probe(kind, sink, grid, block, iters / 8, s), "issue probe warm-up")) return rc;
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(ctx->ev0, s);
    if (int rc = ctx->cuda(launch_issue_probe(kind, sink, grid, block, iters, s), "issue probe")) return rc;
    cudaEventRecord(ctx->ev1, s);
    if (int rc = ctx->cuda(cudaEventSynchronize(ctx->ev1), "issue probe")) return rc;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    best = fminf(best, ms);
  }
  const double warp_inst = (double)grid * (block / 32) * (double)iters * 8.0;
  *warp_inst_per_s = warp_inst / (best * 1e-3);
  return THOR_OK;
}

extern "C" int thor_dda_trace(thor_ctx_t ctx, const int32_t dims[3], const double* org, const float* dir, int32_t n,
                              int32_t max_steps, int64_t* cells, double* seg, int32_t* count, int mem_kind) {
  if (!ctx || !dims || !org || !dir || !cells || !seg || !count || n <= 0 || max_steps <= 0)
    return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_dda_trace") : THOR_ERR_INVALID_ARG;
  const size_t tb = (size_t)n * max_steps;
  Stage st;
  if (int rc = stage_begin(ctx, mem_kind, (size_t)n * 40 + tb * 16 + 4096, &st)) return rc;
  const double* dorg = (const double*)st.in(org, (size_t)n * 24);
  const float* ddir = (const float*)st.in(dir, (size_t)n * 12);
  int64_t* dc = (int64_t*)st.out(cells, tb * 8);
  double* ds = (double*)st.out(seg, tb * 8);
  int32_t* dn = (int32_t*)st.out(count, (size_t)n * 4);
  if (int rc = ctx->cuda(launch_dda_trace(dims[0], dims[1], dims[2], dorg, ddir, n, max_steps, dc, ds, dn, ctx->stream),
                         "dda kernel"))
    return rc;
  return st.finish();
}

extern "C" int thor_sample_upar(thor_ctx_t ctx, float x, float a, uint64_t seed, int64_t n, float* out, uint64_t* iters,
                                int mem_kind) {
  if (!ctx || !out || n <= 0 || !(a > 0.0f) || !std::isfinite(a) || !std::isfinite(x))
    return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_sample_upar: needs n > 0, finite x, finite a > 0")
               : THOR_ERR_INVALID_ARG;
  Stage st;
  if (int rc = stage_begin(ctx, mem_kind, (size_t)n * 4 + 4096, &st)) return rc;
  float* d = (float*)st.out(out, (size_t)n * 4);
  unsigned long long* dit = (unsigned long long*)ctx->scratch(ctx->b_stats, 16);
  if (!dit) return ctx->fail(THOR_ERR_OOM, "stats");
  cudaMemsetAsync(dit, 0, 8, ctx->stream);
  if (int rc = ctx->cuda(launch_upar(x, a, seed, n, d, dit, ctx->stream), "u_par kernel")) return rc;
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, dit, 8, cudaMemcpyDeviceToHost, ctx->stream);
  int rc = st.finish();
  if (iters) *iters = h;
  return rc;
}

extern "C" int thor_scatter_once(thor_ctx_t ctx, float x, float a, int phase, uint64_t seed, int64_t n, float* x_out,
                                 float* mu_out, int mem_kind) {
  if (!ctx || !x_out || !mu_out || n <= 0 || phase < 0 || phase > 2 || !(a > 0.0f) || !std::isfinite(a) ||
      !std::isfinite(x))
    return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_scatter_once: needs n > 0, phase 0-2, finite x, finite a > 0")
               : THOR_ERR_INVALID_ARG;
  Stage st;
  if (int rc = stage_begin(ctx, mem_kind, (size_t)n * 8 + 4096, &st)) return rc;
  float* dx = (float*)st.out(x_out, (size_t)n * 4);
  float* dm = (float*)st.out(mu_out, (size_t)n * 4);
  if (int rc = ctx->cuda(launch_scatter_once(x, a, phase, seed, n, dx, dm, ctx->stream), "scatter kernel")) return rc;
  return st.finish();
}

extern "C" int thor_philox(thor_ctx_t ctx, const uint32_t* ctr, const uint32_t* key, uint32_t* out, int32_t n,
                           int mem_kind) {
  if (!ctx || !ctr || !key || !out || n <= 0) return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_philox") : THOR_ERR_INVALID_ARG;
  Stage st;
  if (int rc = stage_begin(ctx, mem_kind, (size_t)n * 40 + 4096, &st)) return rc;
  const uint32_t* dc = (const uint32_t*)st.in(ctr, (size_t)n * 16);
  const uint32_t* dk = (const uint32_t*)st.in(key, (size_t)n * 8);
  uint32_t* dout = (uint32_t*)st.out(out, (size_t)n * 16);
  if (int rc = ctx->cuda(launch_philox(dc, dk, dout, n, ctx->stream), "philox kernel")) return rc;
  return st.finish();
}
