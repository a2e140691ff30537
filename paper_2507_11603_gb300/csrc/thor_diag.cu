// thor_diag.cu -- unit-level kernels behind the diagnostic entry points: the same
// device functions the photon loops use, exposed one at a time so that each can be
// compared with the FP64 oracle (Voigt, cell walk, u_par sampler, one scattering,
// Philox known-answer vectors).
#include "thor_device.cuh"
#include "thor_internal.h"

namespace thor {
namespace {

__global__ void voigt_kernel(const float* __restrict__ a, const float* __restrict__ x, float* __restrict__ H,
                             int64_t n, const float* __restrict__ gK, int precise) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  load_ktab(sK, gK);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    H[i] = precise ? voigt<true>(a[i], x[i], sK) : voigt<false>(a[i], x[i], sK);
}

__global__ void dda_kernel(int nx, int ny, int nz, const double* __restrict__ org, const float* __restrict__ dir,
                           int n, int max_steps, int64_t* __restrict__ cells, double* __restrict__ seg,
                           int32_t* __restrict__ count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  Dda w;
  w.init(org[3 * r], org[3 * r + 1], org[3 * r + 2], (double)dir[3 * r], (double)dir[3 * r + 1],
         (double)dir[3 * r + 2]);
  int c = 0;
  while (c < max_steps && w.inside(nx, ny, nz)) {
    double tn;
    const int ax = w.next_axis(tn);
    cells[(int64_t)r * max_steps + c] = (int64_t)w.i[0] + (int64_t)nx * ((int64_t)w.i[1] + (int64_t)ny * w.i[2]);
    seg[(int64_t)r * max_steps + c] = __dadd_rn(tn, -w.t);
    ++c;
    w.advance(ax, tn);
  }
  count[r] = c;
  for (int j = c; j < max_steps; ++j) {  // unused entries: -1 / 0
    cells[(int64_t)r * max_steps + j] = -1;
    seg[(int64_t)r * max_steps + j] = 0.0;
  }
}

__global__ void upar_kernel(float x, float a, uint64_t seed, int64_t n, float* __restrict__ out,
                            unsigned long long* iters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t it = 0;
  if (i < n) {
    Rng rng;
    rng.init(seed, (uint64_t)i, 1u);
    out[i] = sample_upar(x, a, rng, it);
  }
  unsigned long long s = it;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(iters, s);
}

__global__ void scatter_once_kernel(float x, float a, int phase, uint64_t seed, int64_t n, float* __restrict__ xo,
                                    float* __restrict__ mu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Rng rng;
  rng.init(seed, (uint64_t)i, 3u);
  float3 k = make_float3(0.0f, 0.0f, 1.0f);
  uint32_t it = 0;
  xo[i] = scatter_resonant(x, a, phase, k, rng, it, nullptr);
  mu[i] = k.z;
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                              uint32_t* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c0 = ctr[4 * i], c1 = ctr[4 * i + 1], c2 = ctr[4 * i + 2], c3 = ctr[4 * i + 3];
  philox10(c0, c1, c2, c3, key[2 * i], key[2 * i + 1]);
  out[4 * i] = c0; out[4 * i + 1] = c1; out[4 * i + 2] = c2; out[4 * i + 3] = c3;
}

inline unsigned blocks_for(int64_t n, int b) {
  const int64_t g = (n + b - 1) / b;
  return (unsigned)(g < 152 * 64 ? (g > 0 ? g : 1) : 152 * 64);
}

// Issue-rate probe (the denominators of the ALU rooflines): every thread runs eight
// independent chains of `iters` dependent operations of one kind, so every scheduler always
// has an independent instruction to issue; kind 0 = FP32 FMA (the issue-slot peak, one warp
// instruction per scheduler per clock), kind 1 = MUFU ex2 (the special-function pipe).
// The sum is stored so nothing is optimised away.
template <int kKind>
__global__ void __launch_bounds__(256) issue_probe_kernel(float* __restrict__ sink, int iters, float seed) {
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = seed * (float)(threadIdx.x + 1) + 0.001f * (float)j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (kKind == 0) v[j] = __fmaf_rn(v[j], 0.9999999f, 1e-7f);
      else v[j] = ex2_approx(v[j]) - 1.5f;
    }
  }
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc += v[j];
  if (acc == 12345.678f) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // practically never
}

__global__ void xcw_kernel(const float* __restrict__ a, float* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = xcw_b25(a[i]);
}

}  // namespace

cudaError_t launch_issue_probe(int kind, float* sink, int grid, int block, int iters, cudaStream_t s) {
  if (kind == 0) issue_probe_kernel<0><<<grid, block, 0, s>>>(sink, iters, 1e-3f);
  else issue_probe_kernel<1><<<grid, block, 0, s>>>(sink, iters, 1e-3f);
  return cudaGetLastError();
}

cudaError_t launch_xcw_eval(const float* a, float* out, int64_t n, cudaStream_t s) {
  xcw_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, out, n);
  return cudaGetLastError();
}

cudaError_t launch_voigt_eval(const float* a, const float* x, float* H, int64_t n, const float* d_ktab,
                              cudaStream_t s, int precise) {
  voigt_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, x, H, n, d_ktab, precise);
  return cudaGetLastError();
}

cudaError_t launch_dda_trace(int nx, int ny, int nz, const double* org, const float* dir, int n, int max_steps,
                             int64_t* cells, double* seg, int32_t* count, cudaStream_t s) {
  dda_kernel<<<(n + 127) / 128, 128, 0, s>>>(nx, ny, nz, org, dir, n, max_steps, cells, seg, count);
  return cudaGetLastError();
}

cudaError_t launch_upar(float x, float a, uint64_t seed, int64_t n, float* out, unsigned long long* iters,
                        cudaStream_t s) {
  upar_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, a, seed, n, out, iters);
  return cudaGetLastError();
}

cudaError_t launch_scatter_once(float x, float a, int phase, uint64_t seed, int64_t n, float* x_out, float* mu_out,
                                cudaStream_t s) {
  scatter_once_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, a, phase, seed, n, x_out, mu_out);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, cudaStream_t s) {
  philox_kernel<<<(n + 127) / 128, 128, 0, s>>>(ctr, key, out, n);
  return cudaGetLastError();
}

}  // namespace thor
