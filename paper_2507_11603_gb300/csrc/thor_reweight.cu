// thor_reweight.cu -- post-processing of a shell run (Sec. 5.1): the escaped photons of
// one radiative-transfer run are reweighted to other intrinsic line widths, equivalent
// widths and dust optical depths, using their emitted frequency X0, escaping frequency X
// and the HI column they traversed (dust following the gas).
//
// Grid (photon blocks) x (targets): each CTA histograms its photons' weights for one
// target in shared memory (FP32, a few hundred photons per CTA) and adds the histogram
// to the FP64 output with one atomic per bin.  The inputs are read once per target
// (13 bytes per photon; coalesced).
#include "thor_internal.h"

namespace thor {
namespace {

constexpr int kRwThreads = 256;

// Intrinsic spectrum p(X) = pl N(X; 0, sigma^2) + (1 - pl) U(X; -C, C), as
// {pl / (sqrt(2 pi) sigma), 1 / (2 sigma^2), (1 - pl) / (2C), C}.
struct Spectrum { float gn, gi, cd, C; };

__device__ __forceinline__ float pdf(const Spectrum& s, float X) {
  const float g = s.gn * expf(-s.gi * X * X);
  return (fabsf(X) <= s.C) ? g + s.cd : g;
}

__global__ void __launch_bounds__(kRwThreads) reweight_kernel(int64_t n, const float* __restrict__ X0,
                                                              const float* __restrict__ X,
                                                              const float* __restrict__ col,
                                                              const uint8_t* __restrict__ status,
                                                              const float* __restrict__ params, int n_bins,
                                                              float X_min, float inv_dX, double* __restrict__ out) {
  extern __shared__ float hist[];  // n_bins + 2
  const int t = blockIdx.y;
  for (int b = threadIdx.x; b < n_bins + 2; b += blockDim.x) hist[b] = 0.0f;
  const Spectrum ps{params[0], params[1], params[2], params[3]};
  const float* q = params + 5 * (t + 1);
  const Spectrum pt{q[0], q[1], q[2], q[3]};
  const float tau_d = q[4];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (status[i] != 1) continue;
    const float x0 = X0[i];
    const float s = pdf(ps, x0);
    const float w = (s > 0.0f) ? pdf(pt, x0) / s * expf(-tau_d * col[i]) : 0.0f;
    const float f = (X[i] - X_min) * inv_dX;
    int b;
    if (!(f >= 0.0f)) b = n_bins;
    else if (f >= (float)n_bins) b = n_bins + 1;
    else b = (int)f;
    atomicAdd(&hist[b], w);
  }
  __syncthreads();
  double* o = out + (size_t)t * (n_bins + 2);
  for (int b = threadIdx.x; b < n_bins + 2; b += blockDim.x)
    if (hist[b] != 0.0f) atomicAdd(&o[b], (double)hist[b]);
}

}  // namespace

cudaError_t launch_reweight(int64_t n, const float* X0, const float* X, const float* col, const uint8_t* status,
                            const float* d_params, int n_targets, int n_bins, double X_min, double X_max,
                            double* d_out, int n_sm, cudaStream_t s) {
  int64_t want = (n + kRwThreads - 1) / kRwThreads;
  const int64_t cap = (int64_t)n_sm * 8;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  const dim3 grid((unsigned)want, (unsigned)n_targets);
  const size_t smem = (size_t)(n_bins + 2) * sizeof(float);
  reweight_kernel<<<grid, kRwThreads, smem, s>>>(n, X0, X, col, status, d_params, n_bins, (float)X_min,
                                                 (float)(n_bins / (X_max - X_min)), d_out);
  return cudaGetLastError();
}

}  // namespace thor
