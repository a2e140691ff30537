// thor_grid.cu -- photon-packet loop on a uniform Cartesian grid (THOR Sec. 3.3-3.4.1):
// field packing, emission CDF, DDA propagation with zeroth-order cells, interaction,
// and peeling-off to three axis-aligned observers.
#include "thor_device.cuh"
#include "thor_internal.h"

namespace thor {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- packing: one 32-byte record per cell, plus n_HI^2 for the emission CDF -------
__global__ void grid_pack_kernel(const float* __restrict__ nHI, const float* __restrict__ T,
                                 const float* __restrict__ vx, const float* __restrict__ vy,
                                 const float* __restrict__ vz, const float* __restrict__ dust, int64_t n,
                                 double cell_cm, GridCell* __restrict__ out, double* __restrict__ w,
                                 unsigned long long* __restrict__ bad) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const double Tc = (double)T[c];
    const double rT = 1.0 / sqrt(Tc);
    const double nh = (double)nHI[c];
    GridCell g;
    g.kap0 = (float)(nh * THOR_SIG1 * rT * cell_cm);
    g.a = (float)(THOR_A1 * rT);
    g.vth = (float)(THOR_VTH1 * sqrt(Tc));
    g.inv_vth = (float)(1.0 / (THOR_VTH1 * sqrt(Tc)));
    g.vx = vx[c]; g.vy = vy[c]; g.vz = vz[c];
    g.kd = dust ? (float)((double)dust[c] * cell_cm) : 0.0f;
    // a cell the photon loop cannot use: T <= 0, negative density or dust, or anything
    // non-finite (before or after the conversion to per-cell opacities)
    const bool ok = Tc > 0.0 && nh >= 0.0 && g.kd >= 0.0f && isfinite(g.kap0) && isfinite(g.a) &&
                    isfinite(g.vth) && g.vth > 0.0f && isfinite(g.inv_vth) && isfinite(g.vx) && isfinite(g.vy) &&
                    isfinite(g.vz) && isfinite(g.kd) && isfinite(nh * nh);
    if (!ok) atomicAdd(bad, 1ull);
    out[c] = g;
    w[c] = nh * nh;
  }
}

// ---- inclusive FP64 prefix sum (three passes) -------------------------------------
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ double block_exclusive_scan(double v, double* sh, double& total) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const double warp_off = (wid > 0) ? sh[wid - 1] : 0.0;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanBlock) scan_tiles(double* data, int64_t n, double* tile_sums, int64_t off) {
  __shared__ double sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  double loc[kScanItems];
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + j;
    loc[j] = (i < n) ? data[i] : 0.0;
    s += loc[j];
  }
  double total;
  double pre = block_exclusive_scan(s, sh, total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    pre += loc[j];
    const int64_t i = base + j;
    if (i < n) data[i] = pre;
  }
  if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x + off] = total;
}

__global__ void add_offsets(double* data, int64_t n, const double* tile_pre) {
  const int64_t t = blockIdx.x;
  if (t == 0) return;
  const double o = tile_pre[t - 1];
  const int64_t base = t * kScanTile;
  for (int j = threadIdx.x; j < kScanTile; j += blockDim.x) {
    const int64_t i = base + j;
    if (i < n) data[i] += o;
  }
}

// ---- photon loop ------------------------------------------------------------------
struct GPhoton {
  double p[3];   // FP64 anchor, cell units; the position is anchor + offset
  float o[3];    // FP32 offset moved since the anchor (inside the current cell)
  float fhi[3];  // distance from the anchor to the + face of the current cell, per axis
  float safe;    // lower bound on the distance from the position to any face of the cell (0 = unknown)
  GridCell gc;   // record of the current cell (valid while safe > 0)
  float3 k;
  float X;
  uint32_t nscat, ndust, iters, steps;
  Rng rng;
  unsigned long long pid;
};

// Fold the offset into the anchor (before the position is used in FP64).
__device__ __forceinline__ void g_anchor(GPhoton& ph) {
#pragma unroll
  for (int a = 0; a < 3; ++a) { ph.p[a] += (double)ph.o[a]; ph.o[a] = 0.0f; }
}

// Cell-local distances from the anchor (which lies in cell i): + faces per axis and the
// nearest face overall, rounded down.
__device__ __forceinline__ void g_cell_frame(GPhoton& ph, const int i[3]) {
  float s = 1.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double lo = ph.p[a] - (double)i[a], hi = (double)(i[a] + 1) - ph.p[a];
    ph.fhi[a] = __double2float_rd(hi);
    s = fminf(s, fminf(__double2float_rd(lo), ph.fhi[a]));
  }
  ph.safe = fmaxf(s * 0.999999f, 0.0f);
}

__device__ __forceinline__ GridCell load_cell(const GridCell* __restrict__ cells, int64_t c) {
  const float4* q = reinterpret_cast<const float4*>(cells + c);
  const float4 a = __ldg(q), b = __ldg(q + 1);
  GridCell g;
  g.kap0 = a.x; g.a = a.y; g.inv_vth = a.z; g.vth = a.w;
  g.vx = b.x; g.vy = b.y; g.vz = b.z; g.kd = b.w;
  return g;
}

// Gas velocity along the direction, v . k (one rounding per fused step).
__device__ __forceinline__ float v_dot_k(const GridCell& g, float3 k) {
  return __fmaf_rn(g.vx, k.x, __fmaf_rn(g.vy, k.y, __fmul_rn(g.vz, k.z)));
}

__device__ __forceinline__ int64_t cell_index(const GridModel& m, int ix, int iy, int iz) {
  return (int64_t)ix + (int64_t)m.nx * ((int64_t)iy + (int64_t)m.ny * iz);
}

// Optical depth from p to the box face along +axis at lab frequency Xp (Sec. 3.4.1),
// cell by cell, stopping once tau > tau_cut.
// A peel ray's walk along +axis from cell index i (t: its entry distance from the start,
// tau: the optical depth so far), cell by cell, stopping once tau > tau_cut.  Cells are
// loaded four at a time (their addresses do not depend on the walk), so a long walk waits on
// memory once per four cells; the optical depth is summed in the same order as one at a
// time.  Walks at most max_cells cells (all when max_cells <= 0).  Returns true when the walk
// is over (tau > tau_cut, or the box face reached).
// H(a, x) for the peel-off rays, out of line: the six first-cell segments of a scattering's
// rays and the walk share one copy (the photon's own steps keep theirs inline).
__device__ __noinline__ float peel_voigt(float a, float x, const float* __restrict__ Ktab) {
  return voigt<false>(a, x, Ktab);
}
struct PeelWalk {
  int i;     // next cell along the axis
  double t;  // distance from the ray's start to that cell's entry face
  float tau;
};
struct WalkOut {
  PeelWalk w;
  uint32_t cells;  // cells walked
  bool done;
};
// Kept out of line: every peel-off site (emission, dust and resonant scatterings, the ray
// kernel) calls this one copy, which keeps the photon loop's code within the instruction
// cache.  c: the index of cell w.i; pa: the start's coordinate along the axis.
__device__ __noinline__ WalkOut peel_walk_cells(const GridCell* __restrict__ cells, int n_ax, int64_t stride,
                                                int64_t c, double pa, float Xp, int axis, float tau_cut,
                                                const float* __restrict__ Ktab, PeelWalk w, int max_cells) {
  WalkOut o;
  o.cells = 0;
  o.done = false;
  const int end = (max_cells > 0 && w.i + max_cells < n_ax) ? w.i + max_cells : n_ax;
  while (w.i < end && !o.done) {
    GridCell g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) g[k] = load_cell(cells, c + (int64_t)min(k, end - 1 - w.i) * stride);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (w.i >= end || o.done) break;
      const double tn = __dadd_rn((double)(w.i + 1), -pa);
      const float v = (axis == 0) ? g[k].vx : (axis == 1) ? g[k].vy : g[k].vz;
      const float x = (Xp - v) * g[k].inv_vth;
      w.tau = __fmaf_rn(__fmaf_rn(g[k].kap0, peel_voigt(g[k].a, x, Ktab), g[k].kd), (float)(tn - w.t), w.tau);
      ++o.cells;
      ++w.i;
      c += stride;
      if (w.tau > tau_cut) o.done = true;
      else w.t = tn;
    }
  }
  o.done = o.done || w.i >= n_ax;
  o.w = w;
  return o;
}
__device__ __forceinline__ bool peel_walk(const GridModel& m, const double p[3], int axis, float Xp,
                                          const float* Ktab, uint32_t& ncell, PeelWalk& w, int max_cells) {
  const int ix = (int)floor(p[0]), iy = (int)floor(p[1]), iz = (int)floor(p[2]);
  const int n_ax = (axis == 0) ? m.nx : (axis == 1) ? m.ny : m.nz;
  const int ia = (axis == 0) ? ix : (axis == 1) ? iy : iz;
  const double pa = (axis == 0) ? p[0] : (axis == 1) ? p[1] : p[2];
  const int64_t stride = (axis == 0) ? 1 : (axis == 1) ? (int64_t)m.nx : (int64_t)m.nx * m.ny;
  const int64_t c = cell_index(m, ix, iy, iz) + (int64_t)(w.i - ia) * stride;
  const WalkOut o = peel_walk_cells(m.cells, n_ax, stride, c, pa, Xp, axis, m.tau_cut, Ktab, w, max_cells);
  w = o.w;
  ncell += o.cells;
  return o.done;
}
// Optical depth from p to the box face along +axis at lab frequency Xp (Sec. 3.4.1); the
// first `skip` cells (0 or 1) are already in tau0.
__device__ __forceinline__ float peel_tau_from(const GridModel& m, const double p[3], int axis, float Xp,
                                               const float* Ktab, uint32_t& ncell, int skip, float tau0) {
  const int ia = (int)floor((axis == 0) ? p[0] : (axis == 1) ? p[1] : p[2]);
  const double pa = (axis == 0) ? p[0] : (axis == 1) ? p[1] : p[2];
  PeelWalk w{ia + skip, skip ? __dadd_rn((double)(ia + skip), -pa) : 0.0, tau0};
  peel_walk(m, p, axis, Xp, Ktab, ncell, w, 0);
  return w.tau;
}
__device__ __forceinline__ float peel_tau(const GridModel& m, const double p[3], int axis, float Xp, const float* Ktab,
                                          uint32_t& ncell) {
  return peel_tau_from(m, p, axis, Xp, Ktab, ncell, 0, 0.0f);
}

__device__ __forceinline__ void deposit(const GridModel& m, const double p[3], int axis, float Xp, float wgt) {
  const float f = (Xp - m.pX_min) * m.pinv_dX;
  if (!(f >= 0.0f) || f >= (float)m.peel_bins) return;
  const int b = (int)f;
  const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
  const int n1 = (a1 == 0) ? m.nx : (a1 == 1) ? m.ny : m.nz;
  const int n2 = (a2 == 0) ? m.nx : (a2 == 1) ? m.ny : m.nz;
  const int ix = (int)floor(p[a1]) / (n1 / m.img_n), iy = (int)floor(p[a2]) / (n2 / m.img_n);
  if (ix < 0 || iy < 0 || ix >= m.img_n || iy >= m.img_n) return;
  atomicAdd(&m.cube[(((size_t)axis * m.img_n + iy) * m.img_n + ix) * m.peel_bins + b], wgt);
}

// Emission (Sec. 2.1, 3.4): cell with probability n_HI^2 / sum, uniform position in it,
// isotropic direction, thermal x ~ N(0, 1/2) in the cell frame; peel at emission.
__device__ void grid_emit(const GridModel& m, GPhoton& ph, const float* Ktab, uint32_t& pr, uint32_t& pc) {
  ph.rng.init(((uint64_t)m.seed_hi << 32) | m.seed_lo, ph.pid, 2u);
  const int64_t n = (int64_t)m.nx * m.ny * m.nz;
  const double total = m.cdf[n - 1];
  const double R = (double)ph.rng.u(0) * total;
  int64_t lo = 0, hi = n - 1;  // smallest c with cdf[c] > R
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (m.cdf[mid] > R) hi = mid; else lo = mid + 1;
  }
  const int64_t c = lo;
  const int ix = (int)(c % m.nx), iy = (int)((c / m.nx) % m.ny), iz = (int)(c / ((int64_t)m.nx * m.ny));
  ph.p[0] = ix + (double)ph.rng.u(1);
  ph.p[1] = iy + (double)ph.rng.u(2);
  ph.p[2] = iz + (double)ph.rng.u(3);
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // a uniform of exactly 1.0 would land on the next cell's face
    const double lim = (a == 0 ? ix : a == 1 ? iy : iz) + 1.0;
    if (ph.p[a] >= lim) ph.p[a] = nextafter(lim, 0.0);
  }
  ph.o[0] = 0.0f; ph.o[1] = 0.0f; ph.o[2] = 0.0f;
  ph.safe = 0.0f;
  ph.k = iso_dir(ph.rng.u(4), ph.rng.u(5));
  const float R1 = ph.rng.u(6), R2 = ph.rng.u(7);
  const float xe = sqrtf(-__logf(R1)) * cospif(2.0f * R2);
  const GridCell g = load_cell(m.cells, c);
  ph.X = __fmaf_rn(xe, g.vth, v_dot_k(g, ph.k));
  ph.nscat = 0; ph.ndust = 0; ph.iters = 0; ph.steps = 0;
  if (m.peel) {
    const float vv[3] = {g.vx, g.vy, g.vz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float Xp = __fmaf_rn(xe, g.vth, vv[ax]);
      const float tau = peel_tau(m, ph.p, ax, Xp, Ktab, pc);
      ++pr;
      deposit(m, ph.p, ax, Xp, __expf(-tau) * (0.25f / kPiF));
    }
  }
}

// Peel-off from the current position towards +axis (Sec. 3.4.1): the first segment runs
// through the current cell, whose record is known (no load); only a ray that leaves it
// with tau <= tau_cut walks on.  Weights below e^-tau_cut are not deposited.
// The rest of such a ray (beyond the current cell) goes to `walk`: traced on the spot in the
// one-kernel loop (WalkHere), or queued for the ray kernel in the event-based loop.
struct WalkHere {
  const GridModel& m;
  const float* Ktab;
  uint32_t& pc;
  __device__ __forceinline__ void operator()(const double p[3], int ax, float Xp, float w0, float tau) const {
    tau = peel_tau_from(m, p, ax, Xp, Ktab, pc, 1, tau);
    if (tau <= m.tau_cut) deposit(m, p, ax, Xp, w0 * __expf(-tau));
  }
};
template <class Walk>
__device__ __forceinline__ void peel_from_cell(const GridModel& m, const GPhoton& ph, int ax, float Xp, float w0,
                                               const float* Ktab, uint32_t& pr, uint32_t& pc, const Walk& walk) {
  const GridCell& g = ph.gc;
  const float v = (ax == 0) ? g.vx : (ax == 1) ? g.vy : g.vz;
  const float x = (Xp - v) * g.inv_vth;
  const float d = (ax == 0) ? ph.fhi[0] - ph.o[0] : (ax == 1) ? ph.fhi[1] - ph.o[1] : ph.fhi[2] - ph.o[2];
  float tau = __fmaf_rn(g.kap0, peel_voigt(g.a, x, Ktab), g.kd) * fmaxf(d, 0.0f);
  ++pr;
  ++pc;
  if (tau > m.tau_cut) return;  // blocked inside the current cell: no FP64, no gather
  const double p[3] = {ph.p[0] + (double)ph.o[0], ph.p[1] + (double)ph.o[1], ph.p[2] + (double)ph.o[2]};
  walk(p, ax, Xp, w0, tau);
}

// An event is two halves: grid_move, then grid_interact.  grid_event runs them in sequence;
// the event-based loop runs them in separate kernels, with the packet in memory between them
// (bit-identical histories).
//
// The propagation half: the event's words, then the move to the interaction site.  Returns
// 1 if the packet left the box, else 0 with x (gas-frame frequency at the site) and kH
// (HI opacity there) set, and the packet's cell record in ph.gc.
// Fast path: while the photon is known to be inside a cell (safe > 0) and the sampled
// interaction lies within the safety distance, the event needs neither the cell walk nor
// any FP64 arithmetic (the common case for photons trapped in optically thick cells).
// Otherwise the cell walk runs from the current position (FP64, the bit-reproducible
// contract of Dda) and re-establishes the cell frame at the interaction point.
__device__ __forceinline__ int grid_move(const GridModel& m, GPhoton& ph, const float* Ktab, float& x_out,
                                         float& kH_out) {
  ph.rng.next_event(3u);
  float tau_rem = -__logf(ph.rng.u(W_TAU));
  float x = 0.0f, kH = 0.0f;
  bool fast = false;
  if (ph.safe > 0.0f) {
    const GridCell& g = ph.gc;
    x = (ph.X - v_dot_k(g, ph.k)) * g.inv_vth;
    kH = g.kap0 * voigt<false>(g.a, x, Ktab);
    const float kt = kH + g.kd;
    const float sdist = __fdividef(tau_rem, kt);
    if (kt > 0.0f && sdist <= ph.safe) {
      ++ph.steps;
      ph.o[0] = __fmaf_rn(sdist, ph.k.x, ph.o[0]);
      ph.o[1] = __fmaf_rn(sdist, ph.k.y, ph.o[1]);
      ph.o[2] = __fmaf_rn(sdist, ph.k.z, ph.o[2]);
      ph.safe = __fmaf_rd(-sdist, 1.000001f, ph.safe);
      fast = true;
    }
  }
  if (!fast) {
    g_anchor(ph);
    Dda w;
    w.init(ph.p[0], ph.p[1], ph.p[2], (double)ph.k.x, (double)ph.k.y, (double)ph.k.z);
    GridCell g;
    for (;;) {
      if (!w.inside(m.nx, m.ny, m.nz)) return 1;
      double tn;
      const int ax = w.next_axis(tn);
      g = load_cell(m.cells, cell_index(m, w.i[0], w.i[1], w.i[2]));
      x = (ph.X - v_dot_k(g, ph.k)) * g.inv_vth;
      kH = g.kap0 * voigt<false>(g.a, x, Ktab);
      const float kt = kH + g.kd;
      const float dt = (float)(tn - w.t);
      const float dtau = kt * dt;
      ++ph.steps;
      if (dtau >= tau_rem && kt > 0.0f) {
        const double ts = w.t + (double)(tau_rem / kt);
        const double kk[3] = {(double)ph.k.x, (double)ph.k.y, (double)ph.k.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double lo = (double)w.i[a], hi = nextafter((double)(w.i[a] + 1), lo);
          ph.p[a] = fmin(fmax(ph.p[a] + ts * kk[a], lo), hi);
        }
        break;
      }
      tau_rem -= dtau;
      w.advance(ax, tn);
    }
    ph.gc = g;
    g_cell_frame(ph, w.i);
  }
  x_out = x;
  kH_out = kH;
  return 0;
}

// The interaction channel at the site (Sec. 3.4): dust with probability kd / (kH + kd).
__device__ __forceinline__ bool grid_dust_channel(const GPhoton& ph, float kH) {
  const GridCell& g = ph.gc;
  return g.kd > 0.0f && ph.rng.u(W_CHANNEL) >= __fdividef(kH, kH + g.kd);
}
// A dust interaction: absorbed with probability 1 - albedo (returns 2), else scattered by the
// Henyey-Greenstein phase function (Eq. 8-9) with its peel-off (returns 0).
template <class Walk>
__device__ __forceinline__ int grid_dust(const GridModel& m, GPhoton& ph, const float* Ktab, uint32_t& pr,
                                         uint32_t& pc, const Walk& walk) {
  const GridCell& g = ph.gc;
  const float vv[3] = {g.vx, g.vy, g.vz};
  const float vk_in = v_dot_k(g, ph.k);
  bool scat;
  if (m.albedo <= 0.0f) scat = false;
  else if (m.albedo >= 1.0f) scat = true;
  else scat = ph.rng.u(W_ALBEDO) < m.albedo;
  if (!scat) return 2;
  if (m.peel) {
    const float kin[3] = {ph.k.x, ph.k.y, ph.k.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float Xp = ph.X + vv[ax] - vk_in;
      peel_from_cell(m, ph, ax, Xp, P_hg(kin[ax], m.g_hg) * (0.5f / kPiF), Ktab, pr, pc, walk);
    }
  }
  scatter_dust(m.g_hg, ph.k, ph.rng);
  ph.X += v_dot_k(g, ph.k) - vk_in;
  ++ph.ndust;
  return 0;
}
// A resonant scattering at gas-frame frequency x (Eq. 5-7) with its peel-off.  Returns 3
// if it reached the scattering cap, else 0.
template <class Walk>
__device__ __forceinline__ int grid_resonant(const GridModel& m, GPhoton& ph, float x, const float* Ktab,
                                             uint32_t& pr, uint32_t& pc, const Walk& walk) {
  const GridCell& g = ph.gc;
  const float vv[3] = {g.vx, g.vy, g.vz};
  const float kin[3] = {ph.k.x, ph.k.y, ph.k.z};
  AtomFrame af;
  const float xo = scatter_resonant(x, g.a, m.phase, ph.k, ph.rng, ph.iters, &af);
  if (m.peel) {
    const float e1[3] = {af.e1.x, af.e1.y, af.e1.z}, e2[3] = {af.e2.x, af.e2.y, af.e2.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float mu = kin[ax];
      const float xp = x - af.upar + __fmaf_rn(af.upar, mu, __fmaf_rn(af.u1, e1[ax], af.u2 * e2[ax]));
      const float Xp = __fmaf_rn(xp, g.vth, vv[ax]);
      float P;
      if (m.phase == PH_ISO) P = 0.5f;
      else if (m.phase == PH_DIPOLE) P = P_dipole(mu);
      else P = af.core ? (0.5f / 3.0f + 2.0f * P_dipole(mu) / 3.0f) : P_dipole(mu);
      peel_from_cell(m, ph, ax, Xp, P * (0.5f / kPiF), Ktab, pr, pc, walk);
    }
  }
  ph.X = __fmaf_rn(xo, g.vth, v_dot_k(g, ph.k));
  ++ph.nscat;
  if (m.max_scat && ph.nscat >= m.max_scat) return 3;
  return 0;
}

// The interaction half, from the words of the current event: channel, then dust or
// resonant scattering, each with its peel-off (Sec. 3.4.1).  Returns 0 continue,
// 2 absorbed, 3 capped.
template <class Walk>
__device__ __forceinline__ int grid_interact(const GridModel& m, GPhoton& ph, float x, float kH, const float* Ktab,
                                             uint32_t& pr, uint32_t& pc, const Walk& walk) {
  if (grid_dust_channel(ph, kH)) return grid_dust(m, ph, Ktab, pr, pc, walk);
  return grid_resonant(m, ph, x, Ktab, pr, pc, walk);
}

// One event; returns 0 continue, 1 escaped, 2 absorbed, 3 capped.
__device__ int grid_event(const GridModel& m, GPhoton& ph, const float* Ktab, uint32_t& pr, uint32_t& pc) {
  float x, kH;
  if (grid_move(m, ph, Ktab, x, kH)) return 1;
  return grid_interact(m, ph, x, kH, Ktab, pr, pc, WalkHere{m, Ktab, pc});
}

// ---- event-based loop: packets in device memory between its kernels -----------------
// A packet's state in its slot.  The cell record is not stored: it is re-read from the
// cell under the anchor (the anchor lies in the packet's cell whenever the record is used).
__device__ __forceinline__ void slot_save(const GridSlots& S, int64_t i, const GPhoton& ph) {
  S.px[i] = ph.p[0]; S.py[i] = ph.p[1]; S.pz[i] = ph.p[2];
  S.ox[i] = ph.o[0]; S.oy[i] = ph.o[1]; S.oz[i] = ph.o[2];
  S.fx[i] = ph.fhi[0]; S.fy[i] = ph.fhi[1]; S.fz[i] = ph.fhi[2];
  S.safe[i] = ph.safe;
  S.kx[i] = ph.k.x; S.ky[i] = ph.k.y; S.kz[i] = ph.k.z; S.X[i] = ph.X;
  S.nscat[i] = ph.nscat; S.ndust[i] = ph.ndust; S.iters[i] = ph.iters; S.steps[i] = ph.steps;
  S.event[i] = ph.rng.event;
  S.pid[i] = ph.pid;
}
// with_cell: re-read the cell record (always for the interaction half; for the move only
// where the fast path may use it, safe > 0)
__device__ __forceinline__ void slot_load(const GridModel& m, const GridSlots& S, int64_t i, GPhoton& ph,
                                          bool with_cell) {
  ph.p[0] = S.px[i]; ph.p[1] = S.py[i]; ph.p[2] = S.pz[i];
  ph.o[0] = S.ox[i]; ph.o[1] = S.oy[i]; ph.o[2] = S.oz[i];
  ph.fhi[0] = S.fx[i]; ph.fhi[1] = S.fy[i]; ph.fhi[2] = S.fz[i];
  ph.safe = S.safe[i];
  ph.k = make_float3(S.kx[i], S.ky[i], S.kz[i]);
  ph.X = S.X[i];
  ph.nscat = S.nscat[i]; ph.ndust = S.ndust[i]; ph.iters = S.iters[i]; ph.steps = S.steps[i];
  ph.pid = S.pid[i];
  ph.rng.keys(((uint64_t)m.seed_hi << 32) | m.seed_lo, ph.pid);
  ph.rng.event = S.event[i];
  if (with_cell || ph.safe > 0.0f)
    ph.gc = load_cell(m.cells, cell_index(m, (int)floor(ph.p[0]), (int)floor(ph.p[1]), (int)floor(ph.p[2])));
}
// Peel rays past their first cell go to the ray queue of the round (walked there in chunks);
// a ray that finds the queue full is walked to the end on the spot.
__device__ __forceinline__ void queue_ray(const GridModel& m, PeelRay* rays, unsigned long long* n, int64_t cap,
                                          const PeelRay& r, const float* Ktab, uint32_t& pc) {
  const unsigned long long j = atomicAdd(n, 1ull);
  if (j < (unsigned long long)cap) {
    rays[j] = r;
    return;
  }
  const double p[3] = {r.px, r.py, r.pz};
  PeelWalk w{r.i, r.t, r.tau};
  peel_walk(m, p, r.ax, r.Xp, Ktab, pc, w, 0);
  if (w.tau <= m.tau_cut) deposit(m, p, r.ax, r.Xp, r.w0 * __expf(-w.tau));
}
struct WalkQueue {
  const GridModel& m;
  PeelRay* rays;
  unsigned long long* n;
  int64_t cap;
  const float* Ktab;
  uint32_t& pc;
  __device__ __forceinline__ void operator()(const double p[3], int ax, float Xp, float w0, float tau) const {
    // the state after the first cell, as peel_tau_from(..., skip = 1, tau) starts
    const int ia = (int)floor(p[ax]);
    PeelRay r;
    r.px = p[0]; r.py = p[1]; r.pz = p[2];
    r.t = __dadd_rn((double)(ia + 1), -p[ax]);
    r.Xp = Xp; r.w0 = w0; r.tau = tau; r.ax = ax; r.i = ia + 1; r.pad = 0;
    queue_ray(m, rays, n, cap, r, Ktab, pc);
  }
};
// Counters of finished packets, per lane, flushed once per warp.
struct GTally {
  unsigned long long esc = 0, ab = 0, cap = 0, sc = 0, du = 0, it = 0, stp = 0, dn = 0;
  double sc2 = 0.0;
  uint32_t pr = 0, pc = 0;
};
__device__ __forceinline__ void grid_finish(const GridModel& m, const GPhoton& ph, int st, GTally& t) {
  if (st == 1) {
    ++t.esc;
    const float f = (ph.X - m.X_min) * m.inv_dX;
    int bin = !(f >= 0.0f) ? m.n_bins : (f >= (float)m.n_bins ? m.n_bins + 1 : (int)f);
    atomicAdd(&m.spectrum[bin], 1ull);
  } else if (st == 2) {
    ++t.ab;
  } else {
    ++t.cap;
  }
  if (m.raw_X) {
    const unsigned long long j = ph.pid - m.id_base;
    m.raw_X[j] = ph.X;
    m.raw_nscat[j] = ph.nscat;
    m.raw_status[j] = (uint8_t)st;
  }
  t.sc += ph.nscat; t.du += ph.ndust; t.it += ph.iters; t.stp += ph.steps; ++t.dn;
  t.sc2 += (double)ph.nscat * (double)ph.nscat;
}

__device__ __forceinline__ unsigned long long wsum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

// Flush per-lane counters: warp reduce, one atomic per warp and field.
__device__ __forceinline__ void flush_tally(const GridModel& m, const GTally& t) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long esc = wsum(t.esc), ab = wsum(t.ab), cap = wsum(t.cap), sc = wsum(t.sc), du = wsum(t.du),
                           it = wsum(t.it), stp = wsum(t.stp), dn = wsum(t.dn);
  const double sc2 = wsum(t.sc2);
  const unsigned long long prs = wsum((unsigned long long)t.pr), pcs = wsum((unsigned long long)t.pc);
  if (lane == 0 && (dn || prs || pcs)) {
    Tally* T = m.tally;
    atomicAdd(&T->n_escaped, esc); atomicAdd(&T->n_absorbed, ab); atomicAdd(&T->n_capped, cap);
    atomicAdd(&T->n_scat, sc); atomicAdd(&T->n_dust_scat, du); atomicAdd(&T->n_upar_iters, it);
    atomicAdd(&T->n_steps, stp); atomicAdd(&T->n_done, dn); atomicAdd(&T->sum_scat2, sc2);
    if (m.peel_rays) { atomicAdd(m.peel_rays, prs); atomicAdd(m.peel_cells, pcs); }
  }
}

// The event-based loop's kernels run thousands of times per run: their counters go to the
// block's own slab entry (warp and block reduction, then plain adds -- kernels of one stream
// never overlap, so no two blocks with the same index run at once), summed once at the end.
__device__ __forceinline__ void flush_slab(TallySlab* slab, const GTally& t) {
  __shared__ unsigned long long sh[8][10];
  __shared__ double sh2[8];
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const unsigned long long v[10] = {wsum(t.esc), wsum(t.ab), wsum(t.cap), wsum(t.sc), wsum(t.du), wsum(t.it),
                                    wsum(t.stp), wsum(t.dn), wsum((unsigned long long)t.pr),
                                    wsum((unsigned long long)t.pc)};
  const double v2 = wsum(t.sc2);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 10; ++k) sh[w][k] = v[k];
    sh2[w] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double a2 = 0.0;
    for (unsigned j = 0; j < (blockDim.x >> 5); ++j) {
#pragma unroll
      for (int k = 0; k < 10; ++k) a[k] += sh[j][k];
      a2 += sh2[j];
    }
    TallySlab& e = slab[blockIdx.x];
    e.esc += a[0]; e.ab += a[1]; e.cap += a[2]; e.sc += a[3]; e.du += a[4]; e.it += a[5]; e.stp += a[6];
    e.dn += a[7]; e.pr += a[8]; e.pc += a[9]; e.sc2 += a2;
  }
}

__global__ void grid_slab_sum_kernel(GridModel m, GridSlots S) {
  unsigned long long a[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double a2 = 0.0;
  for (int b = threadIdx.x; b < kGridSlabBlocks; b += blockDim.x) {
    const TallySlab& e = S.slab[b];
    a[0] += e.esc; a[1] += e.ab; a[2] += e.cap; a[3] += e.sc; a[4] += e.du; a[5] += e.it; a[6] += e.stp;
    a[7] += e.dn; a[8] += e.pr; a[9] += e.pc; a2 += e.sc2;
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) a[k] = wsum(a[k]);
  a2 = wsum(a2);
  if ((threadIdx.x & 31u) == 0) {
    Tally* T = m.tally;
    atomicAdd(&T->n_escaped, a[0]); atomicAdd(&T->n_absorbed, a[1]); atomicAdd(&T->n_capped, a[2]);
    atomicAdd(&T->n_scat, a[3]); atomicAdd(&T->n_dust_scat, a[4]); atomicAdd(&T->n_upar_iters, a[5]);
    atomicAdd(&T->n_steps, a[6]); atomicAdd(&T->n_done, a[7]); atomicAdd(&T->sum_scat2, a2);
    if (m.peel_rays) { atomicAdd(m.peel_rays, a[8]); atomicAdd(m.peel_cells, a[9]); }
  }
}

// The one-kernel loop: persistent warps, one event per lane per iteration, idle lanes
// refilled from the photon queue (warp-aggregated).  kResume: lanes first take the packets
// on the resume list of S (the tail handed over by the event-based loop).
template <bool kResume>
__global__ void __launch_bounds__(256) grid_run_kernel(GridModel m, WorkQueue q, const float* __restrict__ gK,
                                                       GridSlots S) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  load_ktab(sK, gK);
  const unsigned lane = threadIdx.x & 31u;
  GPhoton ph;
  bool active = false, done = (int)lane >= m.per_warp;
  GTally t;
  for (;;) {
    unsigned need = __ballot_sync(kFull, !active && !done);
    if (kResume && need) {
      const unsigned long long n_res = S.ctr[2];
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(&S.ctr[3], (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (!active && !done) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < n_res) { slot_load(m, S, S.rq[g], ph, false); active = true; }
      }
      need = __ballot_sync(kFull, !active && !done);
    }
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(q.next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (!active && !done) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < q.total) {
          ph.pid = q.first_id[0] + g;
          grid_emit(m, ph, sK, t.pr, t.pc);
          active = true;
        } else {
          done = true;
        }
      }
    }
    if (__all_sync(kFull, !active)) break;
    // events until some lane of the warp finishes its packet (one vote per event)
    bool fin;
    do {
      fin = false;
      if (active) {
        const int st = grid_event(m, ph, sK, t.pr, t.pc);
        if (st) {
          grid_finish(m, ph, st, t);
          active = false;
          fin = true;
        }
      }
    } while (!__any_sync(kFull, fin));
  }
  flush_tally(m, t);
}

// ---- event-based loop (Sec. 7.2.2): one event per packet per round, three kernels ----
// Round kernel 1: the move.  Free slots first take new photons (emission with its
// peel-off); then every packet moves to its interaction site.  Escapes finish here; dust
// interactions run here (rare, and their rays go to the ray queue); packets at a resonant
// scattering are queued for kernel 2.  Also clears the other parity's queue counters for the
// next round.
__global__ void __launch_bounds__(256) grid_move_kernel(GridModel m, WorkQueue q, GridSlots S, int parity,
                                                        const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  load_ktab(sK, gK);
  unsigned long long* cnt = S.ctr + 4 + 4 * parity;
  if (blockIdx.x == 0 && threadIdx.x < 2) S.ctr[4 + 4 * (parity ^ 1) + threadIdx.x] = 0ull;
  const unsigned lane = threadIdx.x & 31u;
  GTally t;
  const WalkQueue walk{m, S.rays[parity], cnt + 1, (int64_t)kRayCap * S.n, sK, t.pc};
  long long dlive = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < S.n; b0 += stride) {  // warp-uniform
    const int64_t i = b0 + threadIdx.x;
    const bool in = i < S.n;
    bool live = in && S.live[i];
    GPhoton ph;
    if (live) slot_load(m, S, i, ph, false);
    const unsigned need = __ballot_sync(kFull, in && !live);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader)  // once the queue is drained, free slots stop touching its counter
        base = (*(volatile const unsigned long long*)q.next < q.total)
                   ? atomicAdd(q.next, (unsigned long long)__popc(need)) : q.total;
      base = __shfl_sync(kFull, base, leader);
      if (in && !live) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < q.total) {
          ph.pid = q.first_id[0] + g;
          grid_emit(m, ph, sK, t.pr, t.pc);
          live = true;
          ++dlive;
        }
      }
    }
    if (!live) continue;
    float x, kH;
    int st = grid_move(m, ph, sK, x, kH);
    bool queued = false;
    if (st == 0) {
      if (grid_dust_channel(ph, kH)) {
        st = grid_dust(m, ph, sK, t.pr, t.pc, walk);
      } else {
        queued = true;
        S.xs[i] = x;
      }
    }
    const unsigned qb = __ballot_sync(__activemask(), queued);
    if (queued) {
      const int leader = __ffs(qb) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(cnt, (unsigned long long)__popc(qb));
      base = __shfl_sync(qb, base, leader);
      S.rq[base + __popc(qb & ((1u << lane) - 1u))] = (int32_t)i;
    }
    if (st) {
      grid_finish(m, ph, st, t);
      --dlive;
      S.live[i] = 0;
    } else {
      S.live[i] = 1;
      slot_save(S, i, ph);
    }
  }
  flush_slab(S.slab, t);
  const long long dl = (long long)wsum((unsigned long long)dlive);
  if (lane == 0 && dl) atomicAdd(&S.ctr[0], (unsigned long long)dl);
}

// Round kernel 2: the resonant scatterings queued by kernel 1, from the words of the same
// event (regenerated), with their peel-off; packets at the scattering cap finish.
__global__ void __launch_bounds__(256) grid_scatter_kernel(GridModel m, GridSlots S, int parity,
                                                           const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  load_ktab(sK, gK);
  const unsigned long long* cnt = S.ctr + 4 + 4 * parity;
  const unsigned long long n = cnt[0];
  GTally t;
  const WalkQueue walk{m, S.rays[parity], S.ctr + 5 + 4 * parity, (int64_t)kRayCap * S.n, sK, t.pc};
  long long dlive = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const int64_t i = S.rq[j];
    GPhoton ph;
    slot_load(m, S, i, ph, true);
    ph.rng.start_event(ph.rng.event, 3u);
    const int st = grid_resonant(m, ph, S.xs[i], sK, t.pr, t.pc, walk);
    if (st) {
      grid_finish(m, ph, st, t);
      --dlive;
      S.live[i] = 0;
    } else {
      S.kx[i] = ph.k.x; S.ky[i] = ph.k.y; S.kz[i] = ph.k.z; S.X[i] = ph.X;
      S.nscat[i] = ph.nscat; S.iters[i] = ph.iters;
    }
  }
  flush_slab(S.slab, t);
  const long long dl = (long long)wsum((unsigned long long)dlive);
  if ((threadIdx.x & 31u) == 0 && dl) atomicAdd(&S.ctr[0], (unsigned long long)dl);
}

// Round kernel 3: the round's peel rays advance up to kRayChunk cells each (one ray per
// thread); a ray that is done is deposited, the others go on in the next round's queue, so a
// round waits for no ray's whole walk.  drain: walk every ray to its end (after the last
// round).
__global__ void __launch_bounds__(256) grid_ray_kernel(GridModel m, GridSlots S, int parity, int drain,
                                                       const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  load_ktab(sK, gK);
  const int64_t cap = (int64_t)kRayCap * S.n;
  const unsigned long long n0 = S.ctr[5 + 4 * parity];
  const unsigned long long n = n0 < (unsigned long long)cap ? n0 : (unsigned long long)cap;
  PeelRay* next = S.rays[parity ^ 1];
  unsigned long long* n_next = S.ctr + 5 + 4 * (parity ^ 1);
  GTally t;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    PeelRay r = S.rays[parity][j];
    const double p[3] = {r.px, r.py, r.pz};
    PeelWalk w{r.i, r.t, r.tau};
    if (peel_walk(m, p, r.ax, r.Xp, sK, t.pc, w, drain ? 0 : kRayChunk)) {
      if (w.tau <= m.tau_cut) deposit(m, p, r.ax, r.Xp, r.w0 * __expf(-w.tau));
    } else {
      r.i = w.i; r.t = w.t; r.tau = w.tau;
      queue_ray(m, next, n_next, cap, r, sK, t.pc);
    }
  }
  flush_slab(S.slab, t);
}

// The packets in flight, listed (in slot order) for the hand-off to the one-kernel loop.
__global__ void grid_list_kernel(GridSlots S) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < S.n; b0 += stride) {
    const int64_t i = b0 + threadIdx.x;
    const bool live = i < S.n && S.live[i];
    const unsigned lb = __ballot_sync(kFull, live);
    if (!lb) continue;
    const int leader = __ffs(lb) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(&S.ctr[2], (unsigned long long)__popc(lb));
    base = __shfl_sync(kFull, base, leader);
    if (live) S.rq[base + __popc(lb & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

}  // namespace

cudaError_t launch_grid_pack(const float* nHI, const float* T, const float* vx, const float* vy, const float* vz,
                             const float* dust, int64_t n, double cell_cm, GridCell* out, double* w,
                             unsigned long long* bad, cudaStream_t s) {
  const int block = 256;
  const int64_t want = (n + block - 1) / block;
  const int grid = (int)(want < 152 * 32 ? want : 152 * 32);
  grid_pack_kernel<<<grid, block, 0, s>>>(nHI, T, vx, vy, vz, dust, n, cell_cm, out, w, bad);
  return cudaGetLastError();
}

size_t scan_f64_scratch(int64_t n) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  return (size_t)(tiles + 1) * sizeof(double);
}

// Inclusive prefix sum in place.  Tile sums are scanned with the same kernel, one
// tile at a time (a tile covers 8192 entries, so 8192 tiles = 67M cells per pass).
cudaError_t launch_scan_f64(double* data, int64_t n, double* scratch, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  scan_tiles<<<(unsigned)tiles, kScanBlock, 0, s>>>(data, n, scratch, 0);
  if (tiles > 1) {
    if (tiles > kScanTile) return cudaErrorInvalidValue;
    scan_tiles<<<1, kScanBlock, 0, s>>>(scratch, tiles, nullptr, 0);
    add_offsets<<<(unsigned)tiles, 256, 0, s>>>(data, n, scratch);
  }
  return cudaGetLastError();
}

int grid_grid(int block, int blocks_per_sm) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, grid_run_kernel<false>, block, 0);
  if (occ < 1) occ = 1;
  const int b = (blocks_per_sm > 0 && blocks_per_sm < occ) ? blocks_per_sm : occ;
  return sms * b;
}

cudaError_t launch_grid_run(GridModel m, WorkQueue q, const float* d_ktab, int grid, int block, cudaStream_t s) {
  grid_run_kernel<false><<<grid, block, 0, s>>>(m, q, d_ktab, GridSlots{});
  return cudaGetLastError();
}

cudaError_t launch_grid_resume(GridModel m, WorkQueue q, GridSlots S, const float* d_ktab, int grid, int block,
                               cudaStream_t s) {
  grid_run_kernel<true><<<grid, block, 0, s>>>(m, q, d_ktab, S);
  return cudaGetLastError();
}

// Kernel 1 covers every slot (grid-stride); kernels 2 and 3 read their queue lengths on the
// device, so a round needs no host round trip.
cudaError_t launch_grid_round(GridModel m, WorkQueue q, GridSlots S, int parity, const float* d_ktab, int block,
                              cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (S.n + 255) / 256;
  const int gmax = sms * 8 < kGridSlabBlocks ? sms * 8 : kGridSlabBlocks;  // one slab entry per block
  const int g1 = (int)(want < (int64_t)gmax ? want : (int64_t)gmax);
  grid_move_kernel<<<g1, 256, 0, s>>>(m, q, S, parity, d_ktab);
  grid_scatter_kernel<<<gmax, block, 0, s>>>(m, S, parity, d_ktab);
  grid_ray_kernel<<<gmax, block, 0, s>>>(m, S, parity, 0, d_ktab);
  return cudaGetLastError();
}

// After the last round: the rays still in flight (in the next parity's queue) walk to their end.
cudaError_t launch_grid_ray_drain(GridModel m, GridSlots S, int parity, const float* d_ktab, int block,
                                  cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gmax = sms * 8 < kGridSlabBlocks ? sms * 8 : kGridSlabBlocks;
  grid_ray_kernel<<<gmax, block, 0, s>>>(m, S, parity, 1, d_ktab);
  return cudaGetLastError();
}

cudaError_t launch_grid_slab_sum(GridModel m, GridSlots S, cudaStream_t s) {
  grid_slab_sum_kernel<<<1, 1024, 0, s>>>(m, S);
  return cudaGetLastError();
}

cudaError_t launch_grid_list_live(GridSlots S, cudaStream_t s) {
  const int64_t want = (S.n + 255) / 256;
  grid_list_kernel<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, s>>>(S);
  return cudaGetLastError();
}

// Layout of the slot buffer (each array 256-byte aligned), as grid_slots_carve takes it:
// 4 arrays of 8-byte entries (anchor, photon id), 18 of 4-byte entries (offsets, face
// distances, safety distance, direction, frequencies, counters, event, resonant queue), the
// live flags, two queues of kRayCap n peel rays, the counters and the tally slab.
size_t grid_slots_bytes(int64_t n) {
  auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return 4 * r((size_t)n * 8) + 18 * r((size_t)n * 4) + r((size_t)n) +
         2 * r((size_t)kRayCap * n * sizeof(PeelRay)) + r(16 * 8) + r((size_t)kGridSlabBlocks * sizeof(TallySlab));
}

GridSlots grid_slots_carve(void* base, int64_t n) {
  char* p = (char*)base;
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return (void*)q; };
  GridSlots S;
  S.n = n;
  S.px = (double*)take(n * 8); S.py = (double*)take(n * 8); S.pz = (double*)take(n * 8);
  S.ox = (float*)take(n * 4); S.oy = (float*)take(n * 4); S.oz = (float*)take(n * 4);
  S.fx = (float*)take(n * 4); S.fy = (float*)take(n * 4); S.fz = (float*)take(n * 4);
  S.safe = (float*)take(n * 4);
  S.kx = (float*)take(n * 4); S.ky = (float*)take(n * 4); S.kz = (float*)take(n * 4); S.X = (float*)take(n * 4);
  S.xs = (float*)take(n * 4);
  S.nscat = (uint32_t*)take(n * 4); S.ndust = (uint32_t*)take(n * 4); S.iters = (uint32_t*)take(n * 4);
  S.steps = (uint32_t*)take(n * 4); S.event = (uint32_t*)take(n * 4);
  S.pid = (unsigned long long*)take(n * 8);
  S.live = (uint8_t*)take(n);
  S.rq = (int32_t*)take(n * 4);
  S.rays[0] = (PeelRay*)take((size_t)kRayCap * n * sizeof(PeelRay));
  S.rays[1] = (PeelRay*)take((size_t)kRayCap * n * sizeof(PeelRay));
  S.ctr = (unsigned long long*)take(16 * 8);
  S.slab = (TallySlab*)take((size_t)kGridSlabBlocks * sizeof(TallySlab));
  return S;
}

}  // namespace thor
