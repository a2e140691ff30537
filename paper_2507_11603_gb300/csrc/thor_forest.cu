// thor_forest.cu -- synthetic Lyman-alpha forest optical depth (THOR Sec. 3.5.2, Eq. 11):
// tau(v_b) = sum_k n_k sigma_0(T_k) ds H(a_k, (v_b - v_k) / v_th,k) along periodic
// sightlines parallel to z, v_k = (k + 1/2) dv_cell + v_los,k, v_b = (b + 1/2) dv_bin,
// nearest periodic image in a box of width V = nz dv_cell = n_bins dv_bin.
//
// One CTA per sightline.  The sightline's cells are staged in shared memory (velocity
// as an FP32 hi/lo pair computed in FP64, 1/v_th, a, amplitude); every thread owns
// n_bins / blockDim bins and sweeps all cells, so each Voigt evaluation costs one
// shared-memory broadcast read and no global traffic.  FP32 accumulation in two
// levels (blocks of 32 cells, then the running total) keeps the summation error
// below 1e-6 relative for positive terms.
#include "thor_device.cuh"
#include "thor_internal.h"

namespace thor {
namespace {

constexpr int kForestThreads = 256;
constexpr int kBinsPerThread = 8;   // n_bins <= 2048 per pass
constexpr int kCellChunk = 1024;    // cells staged per pass

__global__ void __launch_bounds__(kForestThreads) forest_kernel(
    const float* __restrict__ nHI, const float* __restrict__ T, const float* __restrict__ vlos, int nx, int ny,
    int nz, int64_t first, double ds_cm, double dv_cell, int n_bins, double dv_bin, float* __restrict__ tau,
    const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  __shared__ float4 sCell[kCellChunk];  // (v_hi, v_lo, 1/v_th, a)
  __shared__ float sAmp[kCellChunk];    // n sigma_0 ds
  load_ktab(sK, gK);
  const int64_t sl = first + blockIdx.x;
  const int ix = (int)(sl % nx), iy = (int)(sl / nx);
  const double V = (double)nz * dv_cell;
  const float Vf = (float)V, hV = 0.5f * Vf;
  const int64_t plane = (int64_t)nx * ny;

  for (int b0 = 0; b0 < n_bins; b0 += kForestThreads * kBinsPerThread) {
    float vb_hi[kBinsPerThread], vb_lo[kBinsPerThread], acc[kBinsPerThread], part[kBinsPerThread];
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      const int b = b0 + threadIdx.x + j * kForestThreads;
      const double vb = ((double)b + 0.5) * dv_bin;
      vb_hi[j] = (float)vb;
      vb_lo[j] = (float)(vb - (double)vb_hi[j]);
      acc[j] = 0.0f;
      part[j] = 0.0f;
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
        const float hi = (float)vk;
        sCell[j] = make_float4(hi, (float)(vk - (double)hi), (float)(rT / THOR_VTH1), (float)(THOR_A1 * rT));
        sAmp[j] = (float)((double)__ldg(nHI + c) * THOR_SIG1 * rT * ds_cm);
      }
      __syncthreads();
      for (int j = 0; j < nk; ++j) {
        const float4 cv = sCell[j];
        const float amp = sAmp[j];
        const float a = cv.w;
#pragma unroll
        for (int q = 0; q < kBinsPerThread; ++q) {
          float dv = (vb_hi[q] - cv.x) + (vb_lo[q] - cv.y);
          dv = (dv >= hV) ? dv - Vf : ((dv < -hV) ? dv + Vf : dv);
          const float x = dv * cv.z;
          const float x2 = x * x;
          float H;
          if (x2 >= 36.0f) H = voigt_wing(a, x2);
          else H = voigt_core<true>(a, fabsf(x), x2, sK);
          part[q] = __fmaf_rn(amp, H, part[q]);
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
    forest_kernel<<<(unsigned)n, kForestThreads, 0, s>>>(nHI, T, vlos, nx, ny, nz, first + done, ds_cm, dv_cell,
                                                          n_bins, dv_bin, tau + (size_t)done * n_bins, d_ktab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += n;
  }
  return cudaSuccess;
}

}  // namespace thor
