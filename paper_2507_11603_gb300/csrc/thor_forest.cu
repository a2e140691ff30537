// thor_forest.cu -- synthetic Lyman-alpha forest optical depth (THOR Sec. 3.5.2, Eq. 11):
// tau(v_b) = sum_k n_k sigma_0(T_k) ds H(a_k, (v_b - v_k) / v_th,k) along periodic
// sightlines parallel to z, v_k = (k + 1/2) dv_cell + v_los,k, v_b = (b + 1/2) dv_bin,
// nearest periodic image in a box of width V = nz dv_cell = n_bins dv_bin.
//
// One CTA per sightline.  The sightline's cells are staged in shared memory (velocity,
// 1/v_th, a, a^2, amplitudes); every thread owns n_bins / blockDim bins and sweeps all
// cells, so each Voigt evaluation costs one shared-memory broadcast read and no global
// traffic.  Velocities are 32-bit fixed point with the period V mapped onto 2^32
// (unit V / 2^32, about 5e-7 km/s here): v_b - v_k wraps modulo 2^32, which is the
// nearest periodic image when read as a signed integer, exactly and without a branch.
// FP32 accumulation in two levels (blocks of 32 cells, then the running total) keeps
// the summation error below 1e-6 relative for positive terms.
#include "thor_device.cuh"
#include "thor_internal.h"

namespace thor {
namespace {

constexpr int kForestThreads = 256;
constexpr int kMaxBinsPerThread = 8;  // n_bins <= 2048 per pass
constexpr int kCellChunk = 1024;    // cells staged per pass

// Wing (|x| >= 6) without the a/sqrt(pi) factor: t g(t), t = 1/(x^2 + a^2), g the
// degree-4 fit of thor_device.cuh (one polynomial for the whole wing, no branch).  MUFU
// reciprocal (relative error ~1 ulp, well inside the 1e-5 budget).
__device__ __forceinline__ float wing_tP(float a2, float x2) {
  const float t = rcp_approx(x2 + a2);
  return t * wing_g(t);
}

// kBinsPerThread bins per thread per pass (1, 2, 4 or 8, the smallest that covers n_bins
// in one pass, so short spectra do not evaluate bins that do not exist)
template <int kBinsPerThread>
__global__ void __launch_bounds__(kForestThreads, 4) forest_kernel(
    const float* __restrict__ nHI, const float* __restrict__ T, const float* __restrict__ vlos, int nx, int ny,
    int nz, int64_t first, double ds_cm, double dv_cell, int n_bins, double dv_bin, float* __restrict__ tau,
    const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  __shared__ float4 sCell[kCellChunk];  // (v as fixed point bits, unit / v_th, a, a^2)
  __shared__ float2 sAmp[kCellChunk];   // (n sigma_0 ds, n sigma_0 ds a / sqrt(pi))
  load_ktab(sK, gK);
  const int64_t sl = first + blockIdx.x;
  const int ix = (int)(sl % nx), iy = (int)(sl / nx);
  const double V = (double)nz * dv_cell;
  const double to_fix = 4294967296.0 / V;  // fixed-point units per km/s
  const int64_t plane = (int64_t)nx * ny;

  for (int b0 = 0; b0 < n_bins; b0 += kForestThreads * kBinsPerThread) {
    // bin q of this thread sits q * blockDim bins after its first bin
    uint32_t vb[kBinsPerThread];
    float acc[kBinsPerThread], part[kBinsPerThread];
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      const double v = ((double)(b0 + threadIdx.x + q * kForestThreads) + 0.5) * dv_bin;
      vb[q] = (uint32_t)(unsigned long long)llrint(fmod(v, V) * to_fix);
      acc[q] = 0.0f;
      part[q] = 0.0f;
    }
    for (int k0 = 0; k0 < nz; k0 += kCellChunk) {
      const int nk = min(kCellChunk, nz - k0);
      __syncthreads();
      for (int j = threadIdx.x; j < nk; j += kForestThreads) {
        const int64_t c = (int64_t)(k0 + j) * plane + (int64_t)iy * nx + ix;
        const double Tc = (double)__ldg(T + c);
        const double rT = 1.0 / sqrt(Tc);
        double vk = ((double)(k0 + j) + 0.5) * dv_cell + (double)__ldg(vlos + c);
        vk -= V * floor(vk / V);  // into [0, V)
        const uint32_t vfix = (uint32_t)(unsigned long long)llrint(vk * to_fix);  // 2^32 wraps to 0
        const double amp = (double)__ldg(nHI + c) * THOR_SIG1 * rT * ds_cm;
        const double a = THOR_A1 * rT;
        sCell[j] = make_float4(__uint_as_float(vfix), (float)(rT / (THOR_VTH1 * to_fix)), (float)a, (float)(a * a));
        sAmp[j] = make_float2((float)amp, (float)(amp * a * 0.5641895835477563));
      }
      __syncthreads();
      for (int j = 0; j < nk; ++j) {
        const float4 cv = sCell[j];
        const float2 am = sAmp[j];
        const uint32_t vk = __float_as_uint(cv.x);
#pragma unroll
        for (int q = 0; q < kBinsPerThread; ++q) {
          const float x = (float)(int32_t)(vb[q] - vk) * cv.y;  // nearest image, in Doppler widths
          const float x2 = x * x;
          if (x2 >= 36.0f) part[q] = __fmaf_rn(am.y, wing_tP(cv.w, x2), part[q]);
          else part[q] = __fmaf_rn(am.x, voigt_core<true>(cv.z, fabsf(x), x2, sK), part[q]);
        }
        if ((j & 31) == 31) {
#pragma unroll
          for (int q = 0; q < kBinsPerThread; ++q) { acc[q] += part[q]; part[q] = 0.0f; }
        }
      }
#pragma unroll
      for (int q = 0; q < kBinsPerThread; ++q) { acc[q] += part[q]; part[q] = 0.0f; }
    }
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      const int b = b0 + threadIdx.x + q * kForestThreads;
      if (b < n_bins) tau[(size_t)blockIdx.x * n_bins + b] = acc[q];
    }
  }
}

}  // namespace

cudaError_t launch_forest(const float* nHI, const float* T, const float* vlos, int nx, int ny, int nz, int64_t first,
                          int64_t count, double ds_cm, double dv_cell, int n_bins, double dv_bin, float* tau,
                          const float* d_ktab, cudaStream_t s) {
  int64_t done = 0;
  while (done < count) {  // grid.x limit
    const int64_t n = count - done < (int64_t)0x7fffffff ? count - done : (int64_t)0x7fffffff;
    float* out = tau + (size_t)done * n_bins;
    const int64_t f = first + done;
    if (n_bins <= kForestThreads)
      forest_kernel<1><<<(unsigned)n, kForestThreads, 0, s>>>(nHI, T, vlos, nx, ny, nz, f, ds_cm, dv_cell, n_bins, dv_bin,
                                                               out, d_ktab);
    else if (n_bins <= 2 * kForestThreads)
      forest_kernel<2><<<(unsigned)n, kForestThreads, 0, s>>>(nHI, T, vlos, nx, ny, nz, f, ds_cm, dv_cell, n_bins, dv_bin,
                                                               out, d_ktab);
    else if (n_bins <= 4 * kForestThreads)
      forest_kernel<4><<<(unsigned)n, kForestThreads, 0, s>>>(nHI, T, vlos, nx, ny, nz, f, ds_cm, dv_cell, n_bins, dv_bin,
                                                               out, d_ktab);
    else
      forest_kernel<kMaxBinsPerThread><<<(unsigned)n, kForestThreads, 0, s>>>(nHI, T, vlos, nx, ny, nz, f, ds_cm,
                                                                              dv_cell, n_bins, dv_bin, out, d_ktab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += n;
  }
  return cudaSuccess;
}

}  // namespace thor
