// thor_device.cuh -- device building blocks of the resonant Lyman-alpha photon loop
// (THOR, arXiv:2507.11603, Sec. 2-3): line constants, Philox4x32-10 streams, the
// FP32 Voigt function, atom-velocity and phase-function samplers, the fused frame
// shift, and the bit-reproducible DDA cell walk.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "voigt_coeffs.h"

namespace thor {

// ------------------------------------------------------------------------------
// Physical constants (CGS; CODATA 2018 and NIST ASD values for Lyman-alpha).
// ------------------------------------------------------------------------------
constexpr double kPiD = 3.14159265358979323846;
constexpr double kC = 2.99792458e10;
constexpr double kBoltz = 1.380649e-16;
constexpr double kMassH = 1.6735575e-24;
constexpr double kLambda0 = 1215.67e-8;
constexpr double kA21 = 6.265e8;
constexpr double kF12 = 0.4164;
constexpr double kEsu = 4.80320471e-10;
constexpr double kMe = 9.1093837015e-28;
constexpr float kPiF = 3.14159265358979f;
constexpr float kInvSqrtPiF = 0.564189583547756f;

// Line parameters at temperature T (Sec. 2.3.1): v_th = sqrt(2kT/m_H) [km/s];
// a = A21 lambda0 / (4 pi v_th); sigma_0 = f12 sqrt(pi) e^2 lambda0 / (m_e c v_th) [cm^2]
// so that sigma(x) = sigma_0 H(a, x).
__host__ __device__ inline double line_vth_kms(double T) { return sqrt(2.0 * kBoltz * T / kMassH) * 1e-5; }
__host__ __device__ inline double line_a(double T) { return kA21 * kLambda0 / (4.0 * kPiD * line_vth_kms(T) * 1e5); }
__host__ __device__ inline double line_sigma0(double T) {
  return kF12 * 1.7724538509055160 * kEsu * kEsu * kLambda0 / (kMe * kC * line_vth_kms(T) * 1e5);
}
// T-scalings used by per-cell kernels: v_th = kVth1 sqrt(T), a = kA1 / sqrt(T), sigma_0 = kSig1 / sqrt(T).
#define THOR_VTH1 (1.2845065404917818e-1)     /* km/s at T = 1 K */
#define THOR_A1 (4.718354755551596e-2)        /* a at T = 1 K   */
#define THOR_SIG1 (5.900890163475877e-12)     /* cm^2 at T = 1 K */

// ------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011, SC'11), written from the published definition.
// Draw convention: key = seed (low, high).  Photon p's emission is event 0, its k-th
// interaction event is event k.  Word j of event e is component j % 4 of the block with
// counter (p low, p high, e, j / 4).  Every random quantity has a fixed word:
//   interaction event: 0 tau; 1, 2, 3 u_par rejection iteration 0 (region, angle,
//     acceptance); 4, 5 perpendicular atom velocity (Box-Muller radius, angle); 6 mu;
//     7 azimuth; 8 channel (HI or dust); 9 dust albedo test; 10 isotropic-or-dipole
//     choice of the mixed phase function; rejection iteration i >= 1 takes words 0, 1, 2
//     of block i + 2.  Dust scattering uses 6 (mu) and 7 (azimuth).
//   emission (gridless): 0 mu, 1 azimuth, 2, 3 Gaussian line;
//   emission (grid): 0 cell, 1-3 position in the cell, 4 mu, 5 azimuth, 6, 7 line.
// ------------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                         uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

enum : int { W_TAU = 0, W_UPAR0 = 1, W_BM_R = 4, W_BM_PHI = 5, W_MU = 6, W_PHI = 7, W_CHANNEL = 8, W_ALBEDO = 9,
             W_MIXED = 10 };

// PTX approximate square root, reciprocal and base-2 exponential (one MUFU instruction
// each, relative error of order 2^-22, no special-case branch; ftz).  Used in the
// samplers, whose parity with the oracle is statistical.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// e^x and ln x as one MUFU instruction and one multiply (relative error of order 2^-22;
// results below the FP32 normal range flush to zero).  On the latency chain of a core event
// these take ~20 cycles against ~42 for __expf / __logf (measured, single lane).
__device__ __forceinline__ float exp_fast(float x) { return ex2_approx(x * 1.44269504f); }
__device__ __forceinline__ float ln_fast(float x) { return lg2_approx(x) * 0.693147181f; }

// (w + 1/2) 2^-32 in FP32: in (0, 1]
__device__ __forceinline__ float uni32(uint32_t w) {
  return fminf(__fmaf_rn(__uint2float_rn(w), 2.3283064365386963e-10f, 1.1641532182693481e-10f), 1.0f);
}

// The first blocks of an event (one to three) are generated together when the event
// starts, at one uniform code point; they are read by constant index only, so they stay
// in registers.  Later blocks (extra rejection iterations) are generated on demand.
// The event index is the whole stream state between events.
struct Rng {
  uint32_t k0, k1, p0, p1;  // key, photon id
  uint32_t event;           // current event
  uint32_t v[12];           // words 0..11 of the current event (the preloaded blocks)

  __device__ __forceinline__ void block(uint32_t j, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) const {
    uint32_t c0 = p0, c1 = p1, c2 = event, c3 = j;
    philox10(c0, c1, c2, c3, k0, k1);
    a = c0; b = c1; c = c2; d = c3;
  }
  // nblk = 1, 2 or 3 blocks preloaded: 2 cover a resonant or dust event without the
  // channel, albedo and mixed-phase words
  __device__ __forceinline__ void start_event(uint32_t e, uint32_t nblk) {
    event = e;
    block(0u, v[0], v[1], v[2], v[3]);
    if (nblk > 1u) block(1u, v[4], v[5], v[6], v[7]);
    if (nblk > 2u) block(2u, v[8], v[9], v[10], v[11]);
  }
  __device__ __forceinline__ void keys(uint64_t seed, uint64_t pid) {
    k0 = (uint32_t)seed; k1 = (uint32_t)(seed >> 32);
    p0 = (uint32_t)pid; p1 = (uint32_t)(pid >> 32);
  }
  __device__ __forceinline__ void init(uint64_t seed, uint64_t pid, uint32_t nblk) {
    keys(seed, pid);
    start_event(0u, nblk);
  }
  // next interaction event of the photon
  __device__ __forceinline__ void next_event(uint32_t nblk) { start_event(event + 1u, nblk); }
  __device__ __forceinline__ float u(int j) const { return uni32(v[j]); }
};

// ------------------------------------------------------------------------------
// Work sharing in the tail of a one-launch photon loop (shell and grid): warps that ran
// dry wait for packets that crowded warps give away.  share: [0] pool entries reserved,
// [1] taken, [2] warps waiting, [3] photons finished, [4] a taken entry never became ready;
// ready[i] is set (after a fence) once entry i is written.
// Lane 0 of a warp whose lanes are all done (queue drained) takes the next pool entry
// (compare-and-swap on the taken counter), or gives up once every photon of the run has
// finished or after kPollMax polls (a packet still in the pool then is resumed by the
// host).  Between polls it sleeps, backing off to 32 us, so that a thousand waiting warps
// load the counters' cache lines little.  Returns the pool index, or -1.
constexpr uint32_t kPollMax = 1u << 24;
__device__ __forceinline__ unsigned long long vload(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}
static __device__ __noinline__ long long pool_take(unsigned long long* share, const uint32_t* ready,
                                                   unsigned long long n_total) {
  atomicAdd(&share[2], 1ull);
  long long got = -1;
  unsigned ns = 64;
  for (uint32_t it = 0; it < kPollMax; ++it) {
    const unsigned long long t = vload(&share[1]), n = vload(&share[0]);
    if (t < n) {
      if (atomicCAS(&share[1], t, t + 1ull) == t) { got = (long long)t; break; }
      continue;
    }
    if (vload(&share[3]) >= n_total) break;
    __nanosleep(ns);
    ns = ns < 32768u ? 2u * ns : 32768u;
  }
  atomicAdd(&share[2], ~0ull);  // -1
  if (got >= 0) {  // the giver writes the record, then the flag: wait for the flag (short)
    uint32_t it = 0;
    while (*(volatile const uint32_t*)&ready[got] == 0u && ++it < kPollMax) __nanosleep(32);
    if (it >= kPollMax) { atomicAdd(&share[4], 1ull); return -1; }
    __threadfence();
  }
  return got;
}
// How many packets a warp with `live` packets gives away: all but one, up to the warps
// waiting beyond the entries already in the pool.
__device__ __forceinline__ long long pool_give_count(const unsigned long long* share, int live) {
  const long long waiting = (long long)vload(&share[2]) - (long long)(vload(&share[0]) - vload(&share[1]));
  return min((long long)(live - 1), waiting);
}

// ------------------------------------------------------------------------------
// Voigt function H(a, x) in FP32 (App. A.3 defines the truth Re w(x + i a)).
//   |x| >= 6 : wing, H = (a/sqrt(pi)) t g(t), t = 1/(x^2 + a^2), g = 2 x^2 K(x) fitted by a
//              degree-4 polynomial in t (the asymptotic series sum_k ((2k+1)!!/2^k) t^k,
//              summed beyond what eight of its terms reach at x = 6);
//   |x| <  6 : Taylor series of w(x + i a) in a up to a^3, with K(x) = 2 x F(x) - 1
//              (F Dawson's integral) from a piecewise degree-11 fit (voigt_coeffs.h):
//              H = e^{-x^2} (1 + a^2 (1 - 2x^2)) + (2a/sqrt(pi)) K + (a^3/(3 sqrt(pi))) ((6 - 4x^2) K + 2).
// Relative error against the FP64 truth below 1e-6 for a <= 1e-2 (tested).
// Ktab points to the 6x12 coefficient table (shared memory in the kernels).
// ------------------------------------------------------------------------------
// Wing factor g(t), t = 1/(x^2 + a^2), |x| >= 6: degree-4 fit (voigt_coeffs.h), relative
// error 4e-8 before FP32 rounding.
__device__ __forceinline__ float wing_g(float t) {
  float s = __fmaf_rn(THOR_WING_C4, t, THOR_WING_C3);
  s = __fmaf_rn(s, t, THOR_WING_C2);
  s = __fmaf_rn(s, t, THOR_WING_C1);
  return __fmaf_rn(s, t, THOR_WING_C0);
}

template <bool kAccurate = true>
__device__ __forceinline__ float voigt_wing(float a, float x2) {
  const float t = kAccurate ? __frcp_rn(__fmaf_rn(a, a, x2)) : rcp_approx(__fmaf_rn(a, a, x2));
  return a * kInvSqrtPiF * t * wing_g(t);
}

template <bool kAccurateExp>
__device__ __forceinline__ float voigt_core(float a, float ax, float x2, const float* __restrict__ Ktab) {
  int i = min((int)ax, THOR_VOIGT_NINT - 1);
  const float u = ax - ((float)i + 0.5f);
  const float4* c4 = reinterpret_cast<const float4*>(Ktab + i * THOR_VOIGT_NCOEF);
  const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2];
  float k;
  if (kAccurateExp) {  // throughput-bound callers: Horner (fewest instructions)
    k = q2.w;
    k = __fmaf_rn(k, u, q2.z); k = __fmaf_rn(k, u, q2.y); k = __fmaf_rn(k, u, q2.x);
    k = __fmaf_rn(k, u, q1.w); k = __fmaf_rn(k, u, q1.z); k = __fmaf_rn(k, u, q1.y);
    k = __fmaf_rn(k, u, q1.x); k = __fmaf_rn(k, u, q0.w); k = __fmaf_rn(k, u, q0.z);
    k = __fmaf_rn(k, u, q0.y); k = __fmaf_rn(k, u, q0.x);
  } else {  // latency-bound callers (photon loops): Estrin, dependency depth 4 instead of 11
    const float u2 = u * u, u4 = u2 * u2;
    const float p01 = __fmaf_rn(q0.y, u, q0.x), p23 = __fmaf_rn(q0.w, u, q0.z);
    const float p45 = __fmaf_rn(q1.y, u, q1.x), p67 = __fmaf_rn(q1.w, u, q1.z);
    const float p89 = __fmaf_rn(q2.y, u, q2.x), pab = __fmaf_rn(q2.w, u, q2.z);
    const float p03 = __fmaf_rn(p23, u2, p01), p47 = __fmaf_rn(p67, u2, p45), p8b = __fmaf_rn(pab, u2, p89);
    k = __fmaf_rn(__fmaf_rn(p8b, u4, p47), u4, p03);
  }
  const float g = kAccurateExp ? expf(-x2) : __expf(-x2);
  const float a2 = a * a;
  const float gauss = g * __fmaf_rn(a2, __fmaf_rn(-2.0f, x2, 1.0f), 1.0f);
  const float c3 = a2 * a * (kInvSqrtPiF / 3.0f);
  return __fmaf_rn(2.0f * a * kInvSqrtPiF, k, gauss) + c3 * __fmaf_rn(__fmaf_rn(-4.0f, x2, 6.0f), k, 2.0f);
}

// |x| <= THOR_VCORE_X = 2 (the photon loops' fast core path): the same series in a, with
// K(x) from one polynomial in s = x^2 / 4 (voigt_coeffs.h, no table lookup, Estrin order:
// the chain is x^2, four FMA levels and the exponential beside them).  Relative error
// against the FP64 truth below 3e-6 for a <= 1e-2 before FP32 rounding (tested).
__device__ __forceinline__ float voigt_core_poly(float a, float x) {
  const float x2 = x * x;
  const float s = 0.25f * x2, s2 = s * s, s4 = s2 * s2, s8 = s4 * s4;
  const float p01 = __fmaf_rn(THOR_VCORE_P1, s, THOR_VCORE_P0), p23 = __fmaf_rn(THOR_VCORE_P3, s, THOR_VCORE_P2);
  const float p45 = __fmaf_rn(THOR_VCORE_P5, s, THOR_VCORE_P4), p67 = __fmaf_rn(THOR_VCORE_P7, s, THOR_VCORE_P6);
  const float p03 = __fmaf_rn(p23, s2, p01), p47 = __fmaf_rn(p67, s2, p45);
  const float k = __fmaf_rn(THOR_VCORE_P8, s8, __fmaf_rn(p47, s4, p03));
  const float g = exp_fast(-x2);
  const float a2 = a * a;
  const float gauss = g * __fmaf_rn(a2, __fmaf_rn(-2.0f, x2, 1.0f), 1.0f);
  const float c3 = a2 * a * (kInvSqrtPiF / 3.0f);
  return __fmaf_rn(2.0f * a * kInvSqrtPiF, k, gauss) + c3 * __fmaf_rn(__fmaf_rn(-4.0f, x2, 6.0f), k, 2.0f);
}

template <bool kAccurateExp = true>
__device__ __forceinline__ float voigt(float a, float x, const float* __restrict__ Ktab) {
  const float ax = fabsf(x);
  const float x2 = ax * ax;
  if (ax >= 6.0f) return voigt_wing<kAccurateExp>(a, x2);
  return voigt_core<kAccurateExp>(a, ax, x2, Ktab);
}

// ------------------------------------------------------------------------------
// Core-to-wing transition x_cw(a) of the Voigt profile (App. A.2), where the Gaussian core
// and the Lorentzian wing are equal (e^{-x^2} = a / (sqrt(pi) x^2)).  B25: the paper's
// fourth-order polynomial in L = ln a (coefficients as printed, within ~0.5% of the exact
// transition for Lyman alpha between 1 K and 1e7 K).  "fast": ln a from the IEEE-754
// exponent and a cubic in the mantissa, log2(1 + t) ~ t (b1 + t (b2 + t b3)) on [0, 1),
// fitted here (max error 8.1e-4 in log2, i.e. ~1e-4 in x_cw).  a > 0, normal.
// ------------------------------------------------------------------------------
__device__ __forceinline__ float fast_ln(float a) {
  const uint32_t b = __float_as_uint(a);
  const float e = (float)((int)(b >> 23) - 127);
  const float t = __uint_as_float((b & 0x007fffffu) | 0x3f800000u) - 1.0f;
  const float l2 = __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, 0.16417124f, -0.58750188f), 1.42405695f), e);
  return l2 * 0.69314718f;
}
__device__ __forceinline__ float xcw_b25(float a) {
  const float L = fast_ln(a);
  float p = __fmaf_rn(-2.76037084e-4f, L, -7.91384757e-3f);
  p = __fmaf_rn(p, L, -8.73073343e-2f);
  p = __fmaf_rn(p, L, -6.17680644e-1f);
  return __fmaf_rn(p, L, 1.03489162f);
}

// ------------------------------------------------------------------------------
// Atom velocity parallel to the photon (Eq. 6) by rejection with the comparison
// function of Eq. 10, sampled through alpha = theta + pi/2 = atan2(a, x - u):
//   region 1 (u <= u0): alpha ~ U(0, w1), accept with exp(-u^2);
//   region 2 (u >  u0): alpha ~ U(w1, pi), accept with exp(u0^2 - u^2);
//   w1 = atan2(a, x - u0), P(region 1) = w1 / (w1 + e^{-u0^2} (pi - w1)), u = x - a / tan(alpha).
// Split point u0 = x - sqrt(a/(2 pi x)) e^{x^2/2} (clamped at 0), the near-resonance
// solution of the envelope mass's stationarity u0^2 = ln(2 pi u0 (x - u0)^2 / a).  Three draws
// per iteration: region, alpha, acceptance.  For |x| > 2 a four-piece comparison function
// takes over (sample_upar_wing).
// ------------------------------------------------------------------------------
// atan2(a, d) for a, d >= 0: series when a/d <= 1/20 (relative error < 3e-9), else atan2f.
__device__ __forceinline__ float atan2_series(float a, float d) {  // for a <= d / 20
  const float t = __fdividef(a, d), t2 = __fmul_rn(t, t);
  return __fmul_rn(t, __fmaf_rn(t2, __fmaf_rn(t2, 0.2f, -1.0f / 3.0f), 1.0f));
}
__device__ __forceinline__ float atan2_pos(float a, float d) {
  if (a <= 0.05f * d) return atan2_series(a, d);
  return atan2f(a, d);
}

__device__ __forceinline__ float envelope_D(float xr, float a, float u0) {
  const float w1 = atan2_pos(a, xr - u0);
  return w1 + __expf(-u0 * u0) * (kPiF - w1);
}

// Near-resonance split point (the x <= 2 rule): u0 = x - d, d = sqrt(a/(2 pi x)) e^{x^2/2},
// clamped at 0; and q = a / d = sqrt(2 pi a x) e^{-x^2/2}, formed directly (no division).
// Where u0 > 0 and q <= 1/20, w1 = atan2(a, x - u0) = atan(q) = q (1 - q^2/3 + q^4/5) to
// 3e-9 relative.  The photon loops' core bursts use these same functions, so both evaluate
// an event identically.
__device__ __forceinline__ float u0_core(float xr, float a) {
  const float d = sqrt_approx(a * (0.5f / kPiF)) * rsqrtf(xr) * exp_fast(fminf(0.5f * xr * xr, 80.0f));
  return fmaxf(0.0f, xr - d);
}
__device__ __forceinline__ float upar_q(float xr, float a) {
  return sqrt_approx(a * (2.0f * kPiF)) * sqrt_approx(xr) * exp_fast(-(0.5f * xr * xr));
}
__device__ __forceinline__ float atan_small(float q) {
  const float q2 = __fmul_rn(q, q);
  return __fmul_rn(q, __fmaf_rn(q2, __fmaf_rn(q2, 0.2f, -1.0f / 3.0f), 1.0f));
}
// Region 1 of the two-piece comparison function is chosen with probability w1 / mass,
// mass = w1 + e^{-u0^2} (pi - w1): R1 < w1 / mass, tested as R1 mass < w1.
__device__ __forceinline__ float envelope_mass(float w1, float e0) { return __fmaf_rn(e0, kPiF - w1, w1); }
__device__ __forceinline__ bool region1(float R1, float mass, float w1) { return __fmul_rn(R1, mass) < w1; }

__device__ __forceinline__ float u0_rule(float xr, float a) {
  if (xr <= 0.0f) return 0.0f;
  const float c1 = u0_core(xr, a);
  if (xr <= 2.0f) return c1;
  float u = fminf(xr - 0.3f, 2.0f + 0.6f * __logf(xr));
  const float c2 = 2.0f * kPiF * rcp_approx(a);
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const float dx = xr - u;
    const float g = u * u - __logf(c2 * u * dx * dx);
    const float gp = 2.0f * u - rcp_approx(u) + 2.0f * rcp_approx(dx);
    u = fminf(fmaxf(u - __fdividef(g, gp), 0.5f), xr - 1e-3f);
  }
  return (envelope_D(xr, a, c1) <= envelope_D(xr, a, u)) ? c1 : u;
}

// cot(pi t) for t in (0, 1]: with s = t (t <= 1/2) or t - 1 (exact), z = pi s in
// [-pi/2, pi/2]; near the pole (|z| <= 1/4) the Laurent series
// 1/z - z (1/3 + z^2/45 + 2 z^4/945 + z^6/4725) (truncation < 1e-10 relative), elsewhere
// MUFU cosine / sine (|sin z| > 0.24, so their 2^-21 absolute error stays ~1e-6 relative).
__device__ __forceinline__ float cot_pi(float t) {
  const float s = (t > 0.5f) ? t - 1.0f : t;
  const float z = kPiF * s;
  const float z2 = z * z;
  float g = __fmaf_rn(z2, 1.0f / 4725.0f, 2.0f / 945.0f);
  g = __fmaf_rn(g, z2, 1.0f / 45.0f);
  g = __fmaf_rn(g, z2, 1.0f / 3.0f);
  const float laurent = __fmaf_rn(-z, g, rcp_approx(z));
  float sn, cs;
  __sincosf(z, &sn, &cs);
  const float trig = cs * rcp_approx(sn);
  return (fabsf(z) <= 0.25f) ? laurent : trig;  // both formed: a select instead of a branch
}

// One trial of the two-piece comparison function (R1: region, R2: angle, R3: acceptance):
// u = x - a cot(alpha) with alpha uniform on the region's part of (0, pi); accepted with
// e^{-u^2} in region 1 (u <= u0), e^{u0^2 - u^2} in region 2.  Every operation is an explicit
// intrinsic, so the photon loops' core form rounds exactly as this sampler does.
__device__ __forceinline__ bool upar_trial(float xr, float a, float w1, float w1p, float mass, float u02,
                                           float R1, float R2, float R3, float& u) {
  const bool reg1 = region1(R1, mass, w1);
  const float t = reg1 ? __fmul_rn(w1p, R2) : __fmaf_rn(__fsub_rn(1.0f, w1p), R2, w1p);
  u = __fmaf_rn(-a, cot_pi(t), xr);  // x - a cot(alpha)
  const float uu = __fmul_rn(u, u);
  const float acc = reg1 ? exp_fast(-uu) : exp_fast(__fsub_rn(u02, uu));
  return R3 <= acc;
}

// Iteration 0 takes words 1-3 of the event, iteration i >= 1 words 0-2 of block i + 2.
// Iteration 0 is peeled out of the loop so that it shares a basic block with the work
// the caller schedules around it (further iterations are rare in the core).  The loop
// stops after kMaxUparTrials trials so that a NaN input cannot keep a lane spinning.  The
// expected trial count stays below 3 at every x for a in [1e-5, 1e-2] (two pieces for
// |x| <= 2, four beyond), so a valid input never comes near the bound.
constexpr uint32_t kMaxUparTrials = 1u << 20;

// Wing side (|x| > kUparWing): a four-piece comparison function.  Eq. 10's two pieces bound
// the Gaussian factor e^{-u^2} of f(u) = e^{-u^2} / ((x-u)^2 + a^2) by a constant over all
// u <= u0, which wastes most trials once |x| passes ~2 (7-9 trials at x = 3, up to ~20 near
// x = 4 with any single split).  Here, with split points u_b < b1 < b2 < x:
//   piece G (u <= u_b): f <= e^{-u^2} / ((x-u_b)^2 + a^2) (x - u >= x - u_b there): u drawn from
//     N(0, 1/2) by its inverse CDF, u = erfinv(2R - 1), accepted with
//     ((x-u_b)^2 + a^2) / ((x-u)^2 + a^2) if u <= u_b, else rejected (the proposal is the whole
//     Gaussian, so a draw above u_b is a rejected trial);
//   pieces 1, 2, 3 (u_b, b1], (b1, b2], (b2, inf): the Lorentzian 1/((x-u)^2 + a^2) times the
//     Gaussian factor's value at the piece's lower end, alpha = atan2(a, x - u) uniform on the
//     piece, u = x - a cot(alpha), accepted with exp(lower^2 - u^2).
// Pieces are chosen in proportion to their masses (times a): a sqrt(pi) / ((x-u_b)^2 + a^2),
// e^{-u_b^2} dalpha_1, e^{-b1^2} dalpha_2, e^{-b2^2} (pi - alpha(b2)); the widths dalpha are
// atan2(a (b' - b), (x - b')(x - b) + a^2), free of the cancellation of a difference.  Any
// split points give the exact distribution; these keep the expected trials below 3 for every
// |x| > 2 and a in [1e-5, 1e-2] (computed from the masses and the Faddeeva function; tested):
// u_b = 1.05 + 0.22 ln(x/3), b1 = 2 + 0.16 ln(x/3) (kept below x and above u_b), and b2 where
// the top two pieces' mass is stationary, e^{b2^2 - b1^2} = 2 pi b2 (x - b2)^2 / a: the
// near-resonance root x - sqrt(a / (2 pi x)) e^{(x^2 - b1^2)/2} or the far root by four Newton
// steps, whichever gives the smaller mass.  Same words as the core loop (region, angle or
// Gaussian, acceptance); kept out of line, as wing scatterings are rare in thick gas
// (everything passes by value, so the caller's stream state stays in registers).
constexpr float kUparWing = 2.0f;
struct UparDraw { float u; uint32_t trials; };
struct WingSplit { float ub, b1, b2; };
__device__ __forceinline__ float top_mass(float xr, float a, float b1, float b2) {
  const float d12 = atan2f(a * (b2 - b1), __fmaf_rn(xr - b2, xr - b1, a * a));
  return __expf(-b1 * b1) * d12 + __expf(-b2 * b2) * (kPiF - atan2f(a, xr - b2));
}
__device__ __forceinline__ WingSplit wing_split(float xr, float a) {
  const float L = __logf(xr * (1.0f / 3.0f));
  const float ub = fminf(__fmaf_rn(0.22f, L, 1.05f), xr - 1.2f);
  const float b1 = fmaxf(fminf(__fmaf_rn(0.16f, L, 2.0f), xr - 0.6f), ub + 0.3f);
  const float d = sqrtf(a / (2.0f * kPiF * xr)) * __expf(fminf(0.5f * (xr * xr - b1 * b1), 80.0f));
  const float c1 = fmaxf(b1 + 1e-3f, xr - d);
  float u = fminf(xr - 0.3f, b1 + 1.0f + 0.6f * __logf(xr));
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const float dx = xr - u;
    const float g = u * u - b1 * b1 - __logf(2.0f * kPiF * u * dx * dx / a);
    const float gp = 2.0f * u - 1.0f / u + 2.0f / dx;
    u = fminf(fmaxf(u - g / gp, b1 + 0.05f), xr - 1e-3f);
  }
  const float b2 = (top_mass(xr, a, b1, c1) <= top_mass(xr, a, b1, u)) ? c1 : u;
  return WingSplit{ub, b1, b2};
}
static __device__ __noinline__ UparDraw sample_upar_wing(float xr, float a, Rng rng) {
  uint32_t iters = 0;
  const WingSplit sp = wing_split(xr, a);
  const float ub = sp.ub, b1 = sp.b1, b2 = sp.b2;
  const float a2 = a * a;
  const float dub = xr - ub;
  const float gden = __fmaf_rn(dub, dub, a2);  // (x - u_b)^2 + a^2
  const float al0 = atan2f(a, dub);
  const float d1 = atan2f(a * (b1 - ub), __fmaf_rn(xr - b1, dub, a2));
  const float d2 = atan2f(a * (b2 - b1), __fmaf_rn(xr - b2, xr - b1, a2));
  const float al1 = al0 + d1, al2 = al1 + d2;
  const float e1 = __expf(-ub * ub), e2 = __expf(-b1 * b1), e3 = __expf(-b2 * b2);
  const float mG = a * 1.7724538509f / gden, m1 = e1 * d1, m2 = e2 * d2, m3 = e3 * (kPiF - al2);
  const float c1 = mG + m1, c2 = c1 + m2, tot = c2 + m3;
  const float sub = ub * ub, sb1 = b1 * b1, sb2 = b2 * b2;
  auto trial = [&](uint32_t r1, uint32_t r2, uint32_t r3, float& u) {
    const float R1 = uni32(r1) * tot, R2 = uni32(r2), R3 = uni32(r3);
    ++iters;
    if (R1 < mG) {  // Gaussian piece
      u = erfinvf(__fmaf_rn(2.0f, R2, -1.0f));
      if (!(u <= ub)) return false;
      const float dx = xr - u;
      return R3 * __fmaf_rn(dx, dx, a2) <= gden;
    }
    float lo, w, sh;
    if (R1 < c1) { lo = al0; w = d1; sh = sub; }
    else if (R1 < c2) { lo = al1; w = d2; sh = sb1; }
    else { lo = al2; w = kPiF - al2; sh = sb2; }
    u = __fmaf_rn(-a, cot_pi(__fmaf_rn(w, R2, lo) * (1.0f / kPiF)), xr);
    return R3 <= __expf(sh - u * u);
  };
  float u;
  if (!trial(rng.v[W_UPAR0], rng.v[W_UPAR0 + 1], rng.v[W_UPAR0 + 2], u)) {
    uint32_t r1, r2, r3, spare, blk = 3u;
    do {
      rng.block(blk++, r1, r2, r3, spare);
    } while (!trial(r1, r2, r3, u) && blk < 2u + kMaxUparTrials);
  }
  return UparDraw{u, iters};
}

__device__ __forceinline__ float sample_upar(float x, float a, const Rng& rng, uint32_t& iters) {
  const float sgn = (x < 0.0f) ? -1.0f : 1.0f;
  const float xr = fabsf(x);
  if (xr > kUparWing) {
    const UparDraw d = sample_upar_wing(xr, a, rng);
    iters += d.trials;
    return sgn * d.u;
  }
  const float u0 = u0_rule(xr, a);
  float w1;
  if (xr <= 2.0f && u0 > 0.0f && upar_q(xr, a) <= 0.05f) w1 = atan_small(upar_q(xr, a));
  else w1 = atan2_pos(a, xr - u0);
  const float u02 = __fmul_rn(u0, u0);
  const float e0 = exp_fast(-u02);
  const float mass = envelope_mass(w1, e0);
  const float w1p = __fmul_rn(w1, 1.0f / kPiF);  // alpha in units of pi
  auto trial = [&](uint32_t r1, uint32_t r2, uint32_t r3, float& u) {
    ++iters;
    return upar_trial(xr, a, w1, w1p, mass, u02, uni32(r1), uni32(r2), uni32(r3), u);
  };
  float u;
  if (!trial(rng.v[W_UPAR0], rng.v[W_UPAR0 + 1], rng.v[W_UPAR0 + 2], u)) {
    uint32_t r1, r2, r3, spare, blk = 3u;
    do {
      rng.block(blk++, r1, r2, r3, spare);
    } while (!trial(r1, r2, r3, u) && blk < 2u + kMaxUparTrials);
  }
  return sgn * u;
}

// Phase functions (Sec. 2.3.1 resonant, Sec. 2.3.2 dust, Eq. 9): mu = k_in . k_out.
enum : int { PH_ISO = 0, PH_DIPOLE = 1, PH_MIXED = 2 };
__device__ __forceinline__ float mu_dipole(float R) {  // CDF (mu^3 + 3 mu + 4)/8, Cardano
  const float B = __fmaf_rn(4.0f, R, -2.0f);
  const float A = ex2_approx(__log2f(B + sqrt_approx(__fmaf_rn(B, B, 1.0f))) * (1.0f / 3.0f));  // cube root, argument in [0.23, 4.3]
  return A - rcp_approx(A);
}
__device__ __forceinline__ float mu_hg(float R, float g) {  // Eq. 9 inverse CDF
  if (fabsf(g) < 1e-6f) return __fmaf_rn(2.0f, R, -1.0f);
  const float t = (1.0f - g * g) / __fmaf_rn(2.0f * g, R, 1.0f - g);
  return (1.0f + g * g - t * t) / (2.0f * g);
}
__device__ __forceinline__ float P_dipole(float mu) { return 0.375f * __fmaf_rn(mu, mu, 1.0f); }
__device__ __forceinline__ float P_hg(float mu, float g) {
  const float d = __fmaf_rn(-2.0f * g, mu, 1.0f + g * g);
  return 0.5f * (1.0f - g * g) * rsqrtf(d * d * d);
}

// Orthonormal basis perpendicular to unit k (Duff et al. 2017, JCGT 6(1)).
__device__ __forceinline__ void basis(float kx, float ky, float kz, float3& e1, float3& e2) {
  const float s = copysignf(1.0f, kz);
  const float a = __fdividef(-1.0f, s + kz);
  const float b = kx * ky * a;
  e1 = make_float3(1.0f + s * kx * kx * a, s * b, -s * kx);
  e2 = make_float3(b, s + ky * ky * a, -ky);
}

struct AtomFrame {  // what peeling-off needs from a resonant scattering
  float upar, u1, u2;
  float3 e1, e2;
  bool core;
};

// One resonant scattering in the gas frame (Eq. 5-7, recoil ignored).  Returns
// x_out = x_in + u . (k_out - k_in) and overwrites k with k_out.
// Core-skipping (Sec. 3.4.2): for |x| < xcrit the perpendicular speed comes from the
// Gaussian left-truncated at xcrit, r = sqrt(xcrit^2 - ln R) (xcrit = 0: plain Eq. 5).
// The perpendicular velocity, mu and the outgoing direction do not depend on u_par, so
// they are formed before the rejection sampler and overlap with it; only the mixed phase
// function's isotropic branch (core scatterings, Sec. 2.3.1) needs u_par and redoes the
// direction afterwards.
__device__ __forceinline__ float3 turn(const float3& k, const float3& e1, const float3& e2, float mu, float st,
                                       float cp, float sp) {
  float3 ko;
  ko.x = mu * k.x + st * (cp * e1.x + sp * e2.x);
  ko.y = mu * k.y + st * (cp * e1.y + sp * e2.y);
  ko.z = mu * k.z + st * (cp * e1.z + sp * e2.z);
  const float inv = rsqrtf(ko.x * ko.x + ko.y * ko.y + ko.z * ko.z);
  return make_float3(ko.x * inv, ko.y * inv, ko.z * inv);
}

// Eq. 7 without recoil: x_out = x - u_par + u . k_out, u . k_out = u_par mu + st (u1 cos phi
// + u2 sin phi) (shared by scatter_resonant and the core bursts).
__device__ __forceinline__ float x_after_scatter(float x, float upar, float mu, float st, float u1, float u2,
                                                 float cp, float sp) {
  const float perp = __fmul_rn(st, __fmaf_rn(u1, cp, __fmul_rn(u2, sp)));
  return __fadd_rn(__fsub_rn(x, upar), __fmaf_rn(upar, mu, perp));
}

__device__ __forceinline__ float scatter_resonant(float x, float a, int phase, float3& k, const Rng& rng,
                                                  uint32_t& iters, AtomFrame* af, float xcrit = 0.0f) {
  const float xc = (fabsf(x) < xcrit) ? xcrit : 0.0f;
  const float r = sqrt_approx(__fmaf_rn(xc, xc, -__logf(rng.u(W_BM_R))));
  float sp1, cp1;
  __sincosf(2.0f * kPiF * rng.u(W_BM_PHI), &sp1, &cp1);
  const float u1 = __fmul_rn(r, cp1), u2 = __fmul_rn(r, sp1);
  const float Rm = rng.u(W_MU);
  float mu = (phase == PH_ISO) ? __fmaf_rn(2.0f, Rm, -1.0f) : mu_dipole(Rm);
  float sp, cp;
  __sincosf(2.0f * kPiF * rng.u(W_PHI), &sp, &cp);
  float3 e1, e2;
  basis(k.x, k.y, k.z, e1, e2);
  float st = sqrt_approx(fmaxf(0.0f, __fmaf_rn(-mu, mu, 1.0f)));
  float3 ko = turn(k, e1, e2, mu, st, cp, sp);
  const float upar = sample_upar(x, a, rng, iters);
  const bool core = fabsf(x - upar) < 0.2f;
  if (phase == PH_MIXED && core && rng.u(W_MIXED) < (1.0f / 3.0f)) {
    mu = __fmaf_rn(2.0f, Rm, -1.0f);
    st = sqrt_approx(fmaxf(0.0f, 1.0f - mu * mu));
    ko = turn(k, e1, e2, mu, st, cp, sp);
  }
  if (af) { af->upar = upar; af->u1 = u1; af->u2 = u2; af->e1 = e1; af->e2 = e2; af->core = core; }
  k = ko;
  return x_after_scatter(x, upar, mu, st, u1, u2, cp, sp);
}

__device__ __forceinline__ void scatter_dust(float g, float3& k, const Rng& rng) {
  const float mu = mu_hg(rng.u(W_MU), g);
  float sp, cp;
  __sincosf(2.0f * kPiF * rng.u(W_PHI), &sp, &cp);
  float3 e1, e2;
  basis(k.x, k.y, k.z, e1, e2);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
  float3 ko;
  ko.x = mu * k.x + st * (cp * e1.x + sp * e2.x);
  ko.y = mu * k.y + st * (cp * e1.y + sp * e2.y);
  ko.z = mu * k.z + st * (cp * e1.z + sp * e2.z);
  const float inv = rsqrtf(ko.x * ko.x + ko.y * ko.y + ko.z * ko.z);
  k = make_float3(ko.x * inv, ko.y * inv, ko.z * inv);
}

__device__ __forceinline__ float3 iso_dir(float Rmu, float Rphi) {
  const float mu = __fmaf_rn(2.0f, Rmu, -1.0f);
  float sp, cp;
  __sincosf(2.0f * kPiF * Rphi, &sp, &cp);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
  return make_float3(st * cp, st * sp, mu);
}

// ------------------------------------------------------------------------------
// DDA cell walk (Amanatides & Woo 1987) with a bit-reproducible contract: FP64
// round-to-nearest with explicit __dadd_rn/__dmul_rn and one IEEE division per axis
// (never contracted into FMA):
//   start cell floor(p), minus one where d < 0 and p lies on the face;
//   inv_ax = 1/d_ax once per ray (IEEE division);
//   next face distance per axis ((i + (d > 0)) - p) * inv_ax, +inf for d == 0;
//   step the axis with the smallest distance, ties to the lowest axis (x < y < z).
// Only the axis that stepped gets a new face distance (recomputed from the face,
// never accumulated).
// ------------------------------------------------------------------------------
struct Dda {
  int i[3];
  int step[3];
  double p[3], inv[3], tm[3];
  double t;

  __device__ __forceinline__ double face_t(int a) const {
    const double face = (double)(i[a] + (step[a] > 0 ? 1 : 0));
    return __dmul_rn(__dadd_rn(face, -p[a]), inv[a]);
  }
  __device__ __forceinline__ void init(double px, double py, double pz, double dx, double dy, double dz) {
    p[0] = px; p[1] = py; p[2] = pz;
    const double d[3] = {dx, dy, dz};
    t = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double f = floor(p[a]);
      int ii = (int)f;
      if (d[a] < 0.0 && p[a] == f) ii -= 1;
      i[a] = ii;
      step[a] = (d[a] > 0.0) ? 1 : (d[a] < 0.0 ? -1 : 0);
      inv[a] = (step[a] != 0) ? __ddiv_rn(1.0, d[a]) : 0.0;
      tm[a] = (step[a] != 0) ? face_t(a) : __longlong_as_double(0x7ff0000000000000ll);
    }
  }
  __device__ __forceinline__ int next_axis(double& tn) const {
    int ax = 0;
    double m = tm[0];
    if (tm[1] < m) { ax = 1; m = tm[1]; }
    if (tm[2] < m) { ax = 2; m = tm[2]; }
    tn = m;
    return ax;
  }
  __device__ __forceinline__ void advance(int ax, double tn) {
    t = tn;
    // constant indices only, so the walk state stays in registers
    if (ax == 0) { i[0] += step[0]; tm[0] = face_t(0); }
    else if (ax == 1) { i[1] += step[1]; tm[1] = face_t(1); }
    else { i[2] += step[2]; tm[2] = face_t(2); }
  }
  __device__ __forceinline__ bool inside(int nx, int ny, int nz) const {
    return i[0] >= 0 && i[1] >= 0 && i[2] >= 0 && i[0] < nx && i[1] < ny && i[2] < nz;
  }
};

// Kernel preamble: copy the Voigt coefficient table into shared memory.
__device__ __forceinline__ void load_ktab(float* sK, const float* __restrict__ gK) {
  for (int j = threadIdx.x; j < THOR_VOIGT_NINT * THOR_VOIGT_NCOEF; j += blockDim.x) sK[j] = gK[j];
  __syncthreads();
}

}  // namespace thor
