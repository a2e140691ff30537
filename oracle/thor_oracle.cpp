// thor_oracle.cpp -- plain FP64 CPU oracle for the resonant Lyman-alpha Monte Carlo
// hot path described by THOR (Byrohl & Nelson, arXiv:2507.11603).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline / reference arm may load or run this library.  It shares no code,
// header, table or constant generator with the CUDA path; the two sides agree only
// on the published definitions cited below (and on the random-number draw
// convention, see "Draw convention").
//
// Every function is written for clarity, in double precision, following the paper's
// order of steps:
//   * Sec. 2.2, Eq. 3-4      exponential attenuation, tau = int n sigma dl
//   * Sec. 2.3.1, Eq. 5-7    atom velocity (u_perp Gaussian, u_par conditional density),
//                            fused double Lorentz frame shift (recoil ignored)
//   * Sec. 2.3.1             dipole / isotropic / 1:2 mixed phase function
//   * Sec. 2.3.2, Eq. 8-9    dust albedo, Henyey-Greenstein phase function
//   * Sec. 3.4               MCRT emission, propagation (cell face to cell face,
//                            zeroth-order cells, interaction at the linear crossing),
//                            interaction channel chosen in proportion to tau_i,
//                            u_par by rejection with the comparison function of Eq. 10
//                            as printed (default), or with a three-piece variant that
//                            uses the random words as the device does (same-stream tests)
//   * Sec. 3.4.1             peeling-off towards observers
//   * Sec. 3.5.2, Eq. 11     synthetic Lyman-alpha forest optical depth
//   * App. A.3               Voigt profile H(a,x) = Re w(x + i a) (Faddeeva truth)
//   * Sec. 5.1               step limiter / velocity gradients: here the oracle does
//                            not sub-step; it integrates tau exactly along the path
//                            (Gauss-Legendre quadrature on analytic H) and root-finds
//                            the interaction point.
//
// Parity unpinned (no external value fixes the whole result; the building blocks are
// pinned): the spectra of outflowing shells (the paper's comparison runs are not
// available; pinned through first-flight escape and the pinned Voigt, sampler, phase
// function and geometry pieces).
//
// Build: g++ -O2 -std=c++17 -fPIC -shared -ffp-contract=off (no FMA contraction: the
// DDA cell walk must be bit-reproducible, see dda_*).

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

namespace {

// ------------------------------------------------------------------------------
// Physical constants (CGS; CODATA 2018, NIST ASD for the Lyman-alpha transition).
// The paper uses these quantities (Sec. 2.3.1, App. A.3) without printing them.
// ------------------------------------------------------------------------------
const double kPi = 3.14159265358979323846;
const double kSqrtPi = 1.77245385090551602730;
const double kC = 2.99792458e10;        // speed of light [cm/s]
const double kBoltz = 1.380649e-16;     // Boltzmann constant [erg/K]
const double kMassH = 1.6735575e-24;    // hydrogen atom mass [g]
const double kLambda0 = 1215.67e-8;     // Lyman-alpha wavelength [cm]
const double kA21 = 6.265e8;            // Einstein A coefficient [1/s]
const double kF12 = 0.4164;             // oscillator strength
const double kEsu = 4.80320471e-10;     // electron charge [esu]
const double kMe = 9.1093837015e-28;    // electron mass [g]

// Thermal velocity v_th = sqrt(2 k T / m) (Sec. 2.3.1) in km/s.
double vth_kms(double T) { return std::sqrt(2.0 * kBoltz * T / kMassH) * 1e-5; }
// Voigt parameter a = A21 / (4 pi Delta nu_D), Delta nu_D = nu0 v_th / c = v_th / lambda0.
double voigt_a(double T) { return kA21 * kLambda0 / (4.0 * kPi * vth_kms(T) * 1e5); }
// Line-centre cross-section normalisation sigma_0 with sigma(x) = sigma_0 H(a,x):
// int sigma dnu = (pi e^2 / m_e c) f12 and int H dx = sqrt(pi).
double sigma0_cm2(double T) {
  double dnuD = vth_kms(T) * 1e5 / kLambda0;
  return kF12 * kSqrtPi * kEsu * kEsu / (kMe * kC * dnuD);
}

// ------------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11,
// "Parallel random numbers: as easy as 1, 2, 3").  Written from the published
// definition: 10 rounds of two 32x32->64 multiplies, key bumped by the Weyl
// constants between rounds.
// ------------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Draw convention (shared by definition with the CUDA path, implemented separately):
// key = (seed low 32, seed high 32).  Photon p's emission is event 0 and its k-th
// interaction event (draw of tau, propagation, interaction) is event k.  Word j of
// event e is component j % 4 of the Philox block with counter (p low, p high, e, j / 4).
// Each random quantity has a fixed word (below); a uniform variate from word u is
// (u + 1/2) 2^-32.  Words that an event does not need are never looked at.
//   interaction event:
//     0 tau; 1, 2, 3 u_par rejection iteration 0 (region, angle, acceptance);
//     4, 5 perpendicular atom velocity (Box-Muller radius, angle); 6 mu; 7 azimuth;
//     8 channel (HI or dust); 9 dust albedo test; 10 isotropic-or-dipole choice of the
//     mixed phase function; u_par iteration i >= 1 takes words 0, 1, 2 of block i + 2.
//     Dust scattering uses 6 (Henyey-Greenstein mu) and 7 (azimuth).
//   emission (gridless): 0 mu, 1 azimuth, 2, 3 Gaussian line (Box-Muller);
//   emission (grid): 0 cell, 1-3 position in the cell, 4 mu, 5 azimuth, 6, 7 line.
enum Word : uint32_t {
  W_TAU = 0, W_UPAR0 = 1, W_BM_R = 4, W_BM_PHI = 5, W_MU = 6, W_PHI = 7, W_CHANNEL = 8, W_ALBEDO = 9,
  W_MIXED = 10
};

struct Stream {
  uint32_t key[2];
  uint32_t pid[2];
  uint32_t event = 0;
  std::vector<std::array<uint32_t, 4>> blocks;  // blocks of the current event generated so far
  Stream(uint64_t seed, uint64_t photon, uint32_t ev = 0) {
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    pid[0] = (uint32_t)photon; pid[1] = (uint32_t)(photon >> 32);
    event = ev;
  }
  void start_event(uint32_t e) { event = e; blocks.clear(); }
  uint32_t word(uint32_t j) {
    while (blocks.size() <= j / 4) {
      uint32_t ctr[4] = {pid[0], pid[1], event, (uint32_t)blocks.size()};
      std::array<uint32_t, 4> b;
      philox4x32_10(ctr, key, b.data());
      blocks.push_back(b);
    }
    return blocks[j / 4][j % 4];
  }
  double u(uint32_t j) { return ((double)word(j) + 0.5) * 2.3283064365386963e-10; }
};

// ------------------------------------------------------------------------------
// Dawson's integral F(x) = exp(-x^2) int_0^x exp(t^2) dt.
//   |x| < 0.2 : Maclaurin series F = sum_k (-1)^k 2^k x^(2k+1) / (2k+1)!!
//   otherwise : Rybicki's sampling-theorem formula (Rybicki 1989, Computers in
//               Physics 3, 85): F(x) = lim_{h->0} pi^{-1/2} sum_{n odd} e^{-(x-nh)^2}/n,
//               with h = 1/4 (truncation error ~ exp(-(pi/2h)^2) ~ 1e-17).
// ------------------------------------------------------------------------------
double dawson(double x) {
  double ax = std::fabs(x);
  if (ax < 0.2) {
    double x2 = x * x, term = x, sum = x;
    for (int k = 1; k < 40; ++k) {
      term *= -2.0 * x2 / (2.0 * k + 1.0);
      sum += term;
      if (std::fabs(term) < 1e-19 * std::fabs(sum)) break;
    }
    return sum;
  }
  const double h = 0.25, span = 8.0;
  long nlo = (long)std::floor((x - span) / h), nhi = (long)std::ceil((x + span) / h);
  double sum = 0.0;
  for (long n = nlo; n <= nhi; ++n) {
    if ((n & 1L) == 0) continue;  // odd n only
    double d = x - (double)n * h;
    sum += std::exp(-d * d) / (double)n;
  }
  return sum / kSqrtPi;
}

// ------------------------------------------------------------------------------
// Voigt function H(a,x) = Re w(x + i a) (App. A.3: the Faddeeva function is the
// truth the paper measures approximations against), with
//   H(a,x) = (a/pi) int exp(-y^2) / ((x-y)^2 + a^2) dy,   H(0,x) = exp(-x^2).
// Two expansions of w(z) = exp(-z^2) + (2i/sqrt(pi)) D(z), D = Dawson's function:
//   |x| >= 7 : asymptotic series D(z) ~ sum_k (2k-1)!! / (2^{k+1} z^{2k+1}); with
//              z = r e^{i theta}, Re[i z^{-n}] = sin(n theta) / r^n, so every term is
//              evaluated without cancellation against the large imaginary part.
//   |x| <  7 : Taylor series in a about the real axis,
//              w(x + i a) = sum_k (i a)^k w^(k)(x) / k!,
//              w(x) = exp(-x^2) + (2i/sqrt(pi)) F(x),
//              w'   = -2 z w + 2i/sqrt(pi),  w^(n+1) = -2 z w^(n) - 2 n w^(n-1).
// Domain: 0 <= a <= 0.5 (Lyman-alpha has a < 0.02 above 10 K).
// ------------------------------------------------------------------------------
double voigt_H(double a, double x) {
  if (!(a >= 0.0 && a <= 0.5)) return NAN;
  double ax = std::fabs(x);
  if (ax >= 7.0) {
    double r2 = ax * ax + a * a, r = std::sqrt(r2), th = std::atan2(a, ax);
    double gauss = std::exp(a * a - ax * ax) * std::cos(2.0 * a * ax);
    double sum = 0.0, ck = 1.0, rp = r, prev = HUGE_VAL;
    for (int k = 0; k < 200; ++k) {
      double mag = ck / rp;
      if (mag > prev) break;  // asymptotic series started to diverge
      sum += ck * std::sin((2.0 * k + 1.0) * th) / rp;
      if (mag < 1e-20 * std::fabs(sum) && k > 1) break;
      prev = mag;
      ck *= (2.0 * k + 1.0) * 0.5;
      rp *= r2;
    }
    return gauss + sum / kSqrtPi;
  }
  // Taylor series in a.  Complex numbers as (re, im) pairs.
  double F = dawson(ax);
  double w0r = std::exp(-ax * ax), w0i = 2.0 / kSqrtPi * F;
  double w1r = -2.0 * ax * w0r, w1i = -2.0 * ax * w0i + 2.0 / kSqrtPi;
  double H = w0r + a * (-w1i);  // k=0: Re w; k=1: Re(i w') = -Im w'
  double coef = a;              // a^k / k!
  double pr = w0r, pi_ = w0i, cr = w1r, ci = w1i;
  for (int k = 1; k < 80; ++k) {
    // w^(k+1) = -2x w^(k) - 2k w^(k-1)
    double nr = -2.0 * ax * cr - 2.0 * k * pr;
    double ni = -2.0 * ax * ci - 2.0 * k * pi_;
    pr = cr; pi_ = ci; cr = nr; ci = ni;
    coef *= a / (double)(k + 1);
    int m = (k + 1) & 3;  // Re(i^m w)
    double t = (m == 0) ? cr : (m == 1) ? -ci : (m == 2) ? -cr : ci;
    H += coef * t;
    if (coef * (std::fabs(cr) + std::fabs(ci)) < 1e-20 * std::fabs(H) && k > 2) break;
    if (coef == 0.0) break;
  }
  return H;
}

// ------------------------------------------------------------------------------
// Gauss-Legendre nodes/weights on [-1,1] (Newton on P_n; weights 2/((1-x^2) P_n'^2)).
// ------------------------------------------------------------------------------
struct GaussLegendre {
  static const int N = 16;
  double x[N], w[N];
  GaussLegendre() {
    for (int i = 0; i < N; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (N + 0.5)), pp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= N; ++j) {
          double p3 = p2; p2 = p1;
          p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = N * (z * p1 - p2) / (z * z - 1.0);
        double dz = p1 / pp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
  }
};
const GaussLegendre& gl() { static GaussLegendre g; return g; }

// Opacity model along one straight segment of gas with constant properties except
// for a frequency that drifts linearly, x(s) = x0 - gam * s (homologous flow):
//   dtau/ds = kap0 * H(a, x(s)) + kapd   (Eq. 4 with sigma = sigma_0 H).
struct Segment {
  double x0, gam, kap0, kapd, a;
  double kappa(double s) const { return kap0 * voigt_H(a, x0 - gam * s) + kapd; }
  // tau over [s0, s1] by Gauss-Legendre on one piece
  double tau_piece(double s0, double s1) const {
    const GaussLegendre& g = gl();
    double hm = 0.5 * (s1 - s0), c = 0.5 * (s1 + s0), sum = 0.0;
    for (int i = 0; i < GaussLegendre::N; ++i) sum += g.w[i] * kappa(c + hm * g.x[i]);
    return sum * hm;
  }
  // piece length such that |dx| stays small relative to the scale on which H varies
  double piece_len(double s) const {
    double x = std::fabs(x0 - gam * s);
    double dx = (x < 10.0) ? 0.1 : 0.01 * x;
    return dx / gam;
  }
};

// Walk the segment [0, S]; if the cumulative tau reaches tau_rem, return true and
// the crossing point s_star (found by safeguarded Newton on the exact integral);
// otherwise return false and the segment's total tau.
bool segment_walk(const Segment& sg, double S, double tau_rem, double* s_star, double* tau_tot) {
  if (sg.gam == 0.0) {
    double k = sg.kappa(0.0);
    double t = k * S;
    if (t >= tau_rem && k > 0.0) { *s_star = tau_rem / k; return true; }
    *tau_tot = t;
    return false;
  }
  double s = 0.0, acc = 0.0;
  while (s < S) {
    double s1 = std::min(S, s + sg.piece_len(s));
    double tp = sg.tau_piece(s, s1);
    if (acc + tp >= tau_rem) {
      double need = tau_rem - acc, lo = s, hi = s1;
      double t = s + (s1 - s) * (need / tp);  // linear first guess
      for (int it = 0; it < 100; ++it) {
        double f = sg.tau_piece(s, t) - need;
        if (f > 0) hi = t; else lo = t;
        double k = sg.kappa(t);
        double tn = (k > 0) ? t - f / k : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (std::fabs(tn - t) <= 1e-14 * std::max(1.0, std::fabs(t)) || hi - lo < 1e-15) { t = tn; break; }
        t = tn;
      }
      *s_star = t;
      return true;
    }
    acc += tp;
    s = s1;
  }
  *tau_tot = acc;
  return false;
}

// ------------------------------------------------------------------------------
// Atom-velocity sampling (Sec. 2.3.1 Eq. 5-6, Sec. 3.4 Eq. 10).
// ------------------------------------------------------------------------------

// Width in alpha = theta + pi/2 of region 1 (u <= u0) of the comparison function,
// theta = atan((u - x)/a): atan2(a, x - u0).  D(u0) is the envelope mass times a.
double envelope_D(double xr, double a, double u0) {
  double w1 = std::atan2(a, xr - u0);
  return w1 + std::exp(-u0 * u0) * (kPi - w1);
}

// Choice of the split point u0 of Eq. 10 (the paper notes it only changes speed).
// Two candidates from the stationarity condition of the envelope mass,
//   u0^2 = ln(2 pi u0 (x - u0)^2 / a):
//   near-resonance root u0 = x - sqrt(a/(2 pi x)) exp(x^2/2) (small-offset solution),
//   far root by three Newton steps; keep the candidate with the smaller envelope.
double u0_rule(double xr, double a) {
  if (xr <= 0.0) return 0.0;
  double d = std::sqrt(a / (2.0 * kPi * xr)) * std::exp(std::min(0.5 * xr * xr, 80.0));
  double c1 = std::max(0.0, xr - d);
  if (xr <= 2.0) return c1;
  double u = std::min(xr - 0.3, 2.0 + 0.6 * std::log(xr));
  for (int it = 0; it < 3; ++it) {
    double g = u * u - std::log(2.0 * kPi * u * (xr - u) * (xr - u) / a);
    double gp = 2.0 * u - 1.0 / u + 2.0 / (xr - u);
    u -= g / gp;
    u = std::min(std::max(u, 0.5), xr - 1e-3);
  }
  return (envelope_D(xr, a, c1) <= envelope_D(xr, a, u)) ? c1 : u;
}

// The inverse CDF of N(0, 1/2) at R: u with (1 + erf(u)) / 2 = R, i.e. erfc(-u) = 2R
// (u <= 0) or erfc(u) = 2 (1 - R) (u > 0), by Newton's method on erfc from the closed-form
// start of Winitzki (2008, "A handy approximation for the error function and its inverse",
// constant 0.147); erfc keeps the relative precision in both tails.
double gauss_half_inv(double R) {
  if (!(R > 0.0)) return -HUGE_VAL;
  if (!(R < 1.0)) return HUGE_VAL;
  const double y = 2.0 * R - 1.0;
  const double al = 0.147;
  const double w = std::log((1.0 - y) * (1.0 + y));
  const double t = 2.0 / (kPi * al) + 0.5 * w;
  double u = std::fabs(std::sqrt(std::sqrt(t * t - w / al) - t));  // |u|
  const double c = (R > 0.5) ? 2.0 * (1.0 - R) : 2.0 * R;           // erfc(|u|) = c
  for (int i = 0; i < 8; ++i) {
    const double f = std::erfc(u) - c;
    const double fp = -2.0 / kSqrtPi * std::exp(-u * u);
    const double du = f / fp;
    u -= du;
    if (std::fabs(du) <= 1e-15 * std::fabs(u) + 1e-300) break;
  }
  return (R > 0.5) ? u : -u;
}

// Split points of the four-piece comparison function for |x| > 2 (the device's rule, in
// FP64): u_b = 1.05 + 0.22 ln(x/3), b1 = 2 + 0.16 ln(x/3) (kept below x and above u_b), and
// b2 where the top two pieces' envelope mass is stationary, e^{b2^2 - b1^2} = 2 pi b2 (x-b2)^2/a:
// the near-resonance root or four Newton steps towards the far root, whichever gives the
// smaller mass.  Any split points give the exact distribution.
double top_mass(double xr, double a, double b1, double b2) {
  return std::exp(-b1 * b1) * (std::atan2(a, xr - b2) - std::atan2(a, xr - b1)) +
         std::exp(-b2 * b2) * (kPi - std::atan2(a, xr - b2));
}
void wing_split(double xr, double a, double* ub, double* b1, double* b2) {
  const double L = std::log(xr / 3.0);
  *ub = std::min(1.05 + 0.22 * L, xr - 1.2);
  *b1 = std::max(std::min(2.0 + 0.16 * L, xr - 0.6), *ub + 0.3);
  const double d = std::sqrt(a / (2.0 * kPi * xr)) * std::exp(std::min(0.5 * (xr * xr - *b1 * *b1), 80.0));
  const double c1 = std::max(*b1 + 1e-3, xr - d);
  double u = std::min(xr - 0.3, *b1 + 1.0 + 0.6 * std::log(xr));
  for (int it = 0; it < 4; ++it) {
    const double dx = xr - u;
    const double g = u * u - *b1 * *b1 - std::log(2.0 * kPi * u * dx * dx / a);
    const double gp = 2.0 * u - 1.0 / u + 2.0 / dx;
    u = std::min(std::max(u - g / gp, *b1 + 0.05), xr - 1e-3);
  }
  *b2 = (top_mass(xr, a, *b1, c1) <= top_mass(xr, a, *b1, u)) ? c1 : u;
}

// u_par from f(u) ~ exp(-u^2) / ((x-u)^2 + a^2) (Eq. 6) by rejection, reading the random
// words as the device's sampler does (for the same-stream tests; the oracle's default is the
// Eq. 10 sampler below).  The Lorentzian part is sampled through alpha = atan2(a, x - u),
// uniform on its interval, u = x - a/tan(alpha).
//   |x| <= 2, Eq. 10's two pieces: region 1 (u <= u0): alpha in (0, w1), envelope 1, accept
//     with exp(-u^2); region 2 (u > u0): alpha in (w1, pi), envelope e^{-u0^2}, accept with
//     exp(u0^2 - u^2); u0 = max(0, x - sqrt(a/(2 pi x)) e^{x^2/2}).
//   |x| > 2, four pieces: below u_b the Gaussian bound e^{-u^2} / ((x-u_b)^2 + a^2), u drawn
//     from N(0, 1/2) by its inverse CDF and accepted with ((x-u_b)^2 + a^2) / ((x-u)^2 + a^2)
//     if u <= u_b; on (u_b, b1], (b1, b2], (b2, inf) the Lorentzian times e^{-lower^2},
//     accepted with exp(lower^2 - u^2).
// Pieces are chosen in proportion to their envelope masses.  Negative x by symmetry.
// Three draws per trial: region, angle (or Gaussian), acceptance.
double sample_upar_envelope(double x, double a, Stream& rng, uint64_t* iters) {
  // iteration 0 uses words 1-3, iteration i >= 1 words 0-2 of block i + 2
  const double sgn = (x < 0.0) ? -1.0 : 1.0, xr = std::fabs(x);
  if (xr <= 2.0) {  // two pieces (Eq. 10)
    const double u0 = u0_rule(xr, a);
    const double w1 = std::atan2(a, xr - u0);
    const double e0 = std::exp(-u0 * u0);
    const double p1 = w1 / (w1 + e0 * (kPi - w1));
    for (uint64_t it = 1;; ++it) {
      const uint32_t w = (it == 1) ? (uint32_t)W_UPAR0 : 4u * (uint32_t)(it + 1);
      const double R1 = rng.u(w), R2 = rng.u(w + 1), R3 = rng.u(w + 2);
      double alpha, shift;
      if (R1 < p1) { alpha = w1 * R2; shift = 0.0; }
      else { alpha = w1 + (kPi - w1) * R2; shift = u0 * u0; }
      const double u = xr - a / std::tan(alpha);
      if (R3 <= std::exp(shift - u * u)) {
        if (iters) *iters += it;
        return sgn * u;
      }
    }
  }
  // four pieces: Gaussian below u_b, Lorentzians on (u_b, b1], (b1, b2], (b2, inf)
  double ub, b1, b2;
  wing_split(xr, a, &ub, &b1, &b2);
  const double gden = (xr - ub) * (xr - ub) + a * a;
  const double al0 = std::atan2(a, xr - ub), al1 = std::atan2(a, xr - b1), al2 = std::atan2(a, xr - b2);
  const double mG = a * kSqrtPi / gden, m1 = std::exp(-ub * ub) * (al1 - al0);
  const double m2 = std::exp(-b1 * b1) * (al2 - al1), m3 = std::exp(-b2 * b2) * (kPi - al2);
  const double tot = mG + m1 + m2 + m3;
  for (uint64_t it = 1;; ++it) {
    const uint32_t w = (it == 1) ? (uint32_t)W_UPAR0 : 4u * (uint32_t)(it + 1);
    const double R1 = rng.u(w) * tot, R2 = rng.u(w + 1), R3 = rng.u(w + 2);
    double u;
    bool acc;
    if (R1 < mG) {
      u = gauss_half_inv(R2);
      acc = (u <= ub) && (R3 * ((xr - u) * (xr - u) + a * a) <= gden);
    } else {
      double lo, hi, b;
      if (R1 < mG + m1) { lo = al0; hi = al1; b = ub; }
      else if (R1 < mG + m1 + m2) { lo = al1; hi = al2; b = b1; }
      else { lo = al2; hi = kPi; b = b2; }
      u = xr - a / std::tan(lo + (hi - lo) * R2);
      acc = R3 <= std::exp(b * b - u * u);
    }
    if (acc) {
      if (iters) *iters += it;
      return sgn * u;
    }
  }
}

// u_par by Eq. 10 exactly as printed: two pieces and nothing else.  This is the oracle's
// default sampler; it shares no design choice with the three-piece envelope above (no
// third piece, no stationarity approximation, a different parameterisation), so spectra
// computed with it check the device's sampler instead of mirroring it.
//   theta = atan((u - x)/a) maps the Lorentzian 1/(a^2 + (x - u)^2) onto a uniform density
//   on (-pi/2, pi/2) of total mass pi/a.  With th0 = theta(u0), 0 <= u0 <= x:
//     piece 1 (u <= u0): envelope g1 = 1/(a^2 + (x-u)^2),          mass (th0 + pi/2)/a;
//     piece 2 (u >  u0): envelope g2 = e^{-u0^2}/(a^2 + (x-u)^2), mass e^{-u0^2}(pi/2 - th0)/a.
//   Both bound f(u) = e^{-u^2}/(a^2 + (x-u)^2) because e^{-u^2} <= 1 everywhere and
//   e^{-u^2} <= e^{-u0^2} for u > u0 >= 0.  A trial picks a piece in proportion to its mass,
//   theta uniformly on the piece's interval, u = x + a tan(theta), and accepts with
//   f/g = e^{-u^2} (piece 1) or e^{u0^2 - u^2} (piece 2).
// The paper leaves u0 to the implementation (the choice only sets the rejection rate); here
// it is the point of [0, x] that minimises the envelope mass itself, found by a scan and a
// golden-section refinement of the exact mass (no fitted or approximated rule).  The
// expected number of trials is (envelope mass) / (pi H(a,x) / a).  Negative x by symmetry
// (f(u; -x) = f(-u; x)).  Draws: words region, angle, acceptance of the trial (as above).
double eq10_mass(double xr, double a, double u0) {  // envelope mass times a
  const double th0 = std::atan((u0 - xr) / a);
  return (th0 + 0.5 * kPi) + std::exp(-u0 * u0) * (0.5 * kPi - th0);
}

double eq10_u0(double xr, double a) {
  if (!(xr > 0.0)) return 0.0;
  // candidates: a fine grid (step 0.1) over [0, min(x, 6)], where the optimum lies for
  // resonant and wing photons, and a coarse grid (step x/32) over the whole interval;
  // the best candidate is no worse than its neighbours on its own grid, so a local
  // minimum lies within one step of it, where golden-section search refines it
  double ub = 0.0, mb = eq10_mass(xr, a, 0.0), h = 0.1;
  for (int i = 1; i <= 60 && 0.1 * i <= xr; ++i) {
    const double m = eq10_mass(xr, a, 0.1 * i);
    if (m < mb) { mb = m; ub = 0.1 * i; h = 0.1; }
  }
  for (int j = 1; j <= 32; ++j) {
    const double m = eq10_mass(xr, a, xr * j / 32.0);
    if (m < mb) { mb = m; ub = xr * j / 32.0; h = xr / 32.0; }
  }
  double lo = std::max(0.0, ub - h), hi = std::min(xr, ub + h);
  const double r = 0.6180339887498949;  // golden ratio conjugate
  double p = hi - r * (hi - lo), q = lo + r * (hi - lo);
  double fp = eq10_mass(xr, a, p), fq = eq10_mass(xr, a, q);
  for (int it = 0; it < 32; ++it) {
    if (fp < fq) { hi = q; q = p; fq = fp; p = hi - r * (hi - lo); fp = eq10_mass(xr, a, p); }
    else { lo = p; p = q; fp = fq; q = lo + r * (hi - lo); fq = eq10_mass(xr, a, q); }
  }
  const double u = 0.5 * (lo + hi);
  return (eq10_mass(xr, a, u) <= mb) ? u : ub;
}

double sample_upar_eq10(double x, double a, Stream& rng, uint64_t* iters) {
  const double sgn = (x < 0.0) ? -1.0 : 1.0, xr = std::fabs(x);
  if (!(a > 0.0)) {  // a -> 0: the Lorentzian is a delta at u = x
    if (iters) *iters += 1;
    return x;
  }
  const double u0 = eq10_u0(xr, a);
  const double th0 = std::atan((u0 - xr) / a);
  const double e0 = std::exp(-u0 * u0);
  const double m1 = th0 + 0.5 * kPi, m2 = e0 * (0.5 * kPi - th0);
  const double p1 = m1 / (m1 + m2);
  for (uint64_t it = 1;; ++it) {
    const uint32_t w = (it == 1) ? (uint32_t)W_UPAR0 : 4u * (uint32_t)(it + 1);
    const double Rp = rng.u(w), Ra = rng.u(w + 1), Racc = rng.u(w + 2);
    double th, bound;
    if (Rp < p1) { th = -0.5 * kPi + m1 * Ra; bound = 1.0; }
    else { th = th0 + (0.5 * kPi - th0) * Ra; bound = e0; }
    const double u = xr + a * std::tan(th);
    if (Racc * bound <= std::exp(-u * u)) {
      if (iters) *iters += it;
      return sgn * u;
    }
  }
}

// Which exact sampler the oracle uses (set by orc_set_upar_method before a run):
// 1 = Eq. 10 as printed (default), 0 = the three-piece envelope, which consumes the same
// words the same way as the device's sampler (for photon-by-photon same-stream tests).
int g_upar_method = 1;

double sample_upar(double x, double a, Stream& rng, uint64_t* iters) {
  return (g_upar_method == 0) ? sample_upar_envelope(x, a, rng, iters) : sample_upar_eq10(x, a, rng, iters);
}

// Core-to-wing transition of the Voigt profile (App. A.2): the frequency x_cw > 1 where the
// Gaussian core and the Lorentzian wing are equal, e^{-x^2} = a / (sqrt(pi) x^2).  With
// y = x^2 this is y - ln y = ln(sqrt(pi) / a), whose root above 1 (the lower branch of
// Lambert's W, x_cw^2 = -W_{-1}(-a / sqrt(pi))) Newton's method reaches monotonically from
// any start above it (the function is convex).  Domain: 0 < a < sqrt(pi)/e.
double xcw_exact(double a) {
  const double c = std::log(kSqrtPi / a);
  double y = c + std::log(c) + 1.0;
  for (int it = 0; it < 60; ++it) {
    const double dy = (y - std::log(y) - c) / (1.0 - 1.0 / y);
    y -= dy;
    if (std::fabs(dy) <= 1e-15 * y) break;
  }
  return std::sqrt(y);
}

// Phase functions: mu = cos(angle between incoming and outgoing direction).
enum Phase { PH_ISO = 0, PH_DIPOLE = 1, PH_MIXED = 2 };
double mu_isotropic(double R) { return 2.0 * R - 1.0; }
// Dipole P(mu) = 3/8 (1 + mu^2): CDF (mu^3 + 3 mu + 4)/8 = R, Cardano's real root.
double mu_dipole(double R) {
  double B = 4.0 * R - 2.0;
  double A = std::cbrt(B + std::sqrt(B * B + 1.0));
  return A - 1.0 / A;
}
// Henyey-Greenstein (Eq. 9) closed-form inverse CDF.
double mu_hg(double R, double g) {
  if (std::fabs(g) < 1e-12) return 2.0 * R - 1.0;
  double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * R);
  return (1.0 + g * g - t * t) / (2.0 * g);
}
// Phase-function densities per unit mu (normalised on [-1,1]).
double P_iso(double) { return 0.5; }
double P_dipole(double mu) { return 0.375 * (1.0 + mu * mu); }
double P_hg(double mu, double g) { return 0.5 * (1.0 - g * g) / std::pow(1.0 + g * g - 2.0 * g * mu, 1.5); }

// Orthonormal basis (e1, e2) perpendicular to unit k (Duff et al. 2017, JCGT 6(1)).
void basis(const double k[3], double e1[3], double e2[3]) {
  double sgn = std::copysign(1.0, k[2]);
  double a = -1.0 / (sgn + k[2]);
  double b = k[0] * k[1] * a;
  e1[0] = 1.0 + sgn * k[0] * k[0] * a; e1[1] = sgn * b; e1[2] = -sgn * k[0];
  e2[0] = b; e2[1] = sgn + k[1] * k[1] * a; e2[2] = -k[1];
}

double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// One resonant scattering in the gas frame (Eq. 5-7): returns the new gas-frame
// frequency, writes the new direction.  Also reports u_par and the perpendicular
// components for peeling-off.
struct AtomVel { double upar, u1, u2; double e1[3], e2[3]; bool core; };

double scatter_HI(double x, double a, int phase, const double kin[3], Stream& rng,
                  double kout[3], AtomVel* av, uint64_t* iters, double xcrit = 0.0) {
  double upar = sample_upar(x, a, rng, iters);
  // u_perp: two N(0, 1/2) variates by Box-Muller (Eq. 5: f = exp(-u^2)).  Core-skipping
  // (Sec. 3.4.2): for |x| < x_crit the perpendicular speed is drawn from the Gaussian
  // left-truncated at x_crit, r = sqrt(x_crit^2 - ln R).
  double xc = (std::fabs(x) < xcrit) ? xcrit : 0.0;
  double r = std::sqrt(xc * xc - std::log(rng.u(W_BM_R)));
  double ph = 2.0 * kPi * rng.u(W_BM_PHI);
  double u1 = r * std::cos(ph), u2 = r * std::sin(ph);
  bool core = std::fabs(x - upar) < 0.2;  // atom-frame frequency (Sec. 2.3.1)
  double mu;
  if (phase == PH_ISO) {
    mu = mu_isotropic(rng.u(W_MU));
  } else if (phase == PH_DIPOLE) {
    mu = mu_dipole(rng.u(W_MU));
  } else {
    double Rc = rng.u(W_MIXED);
    double Rm = rng.u(W_MU);
    mu = (core && Rc < 1.0 / 3.0) ? mu_isotropic(Rm) : mu_dipole(Rm);
  }
  double phi = 2.0 * kPi * rng.u(W_PHI);
  double e1[3], e2[3];
  basis(kin, e1, e2);
  double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  double cp = std::cos(phi), sp = std::sin(phi);
  for (int i = 0; i < 3; ++i) kout[i] = mu * kin[i] + st * (cp * e1[i] + sp * e2[i]);
  double nrm = std::sqrt(dot(kout, kout));
  for (int i = 0; i < 3; ++i) kout[i] /= nrm;
  if (av) {
    av->upar = upar; av->u1 = u1; av->u2 = u2; av->core = core;
    for (int i = 0; i < 3; ++i) { av->e1[i] = e1[i]; av->e2[i] = e2[i]; }
  }
  // Eq. 7 without recoil: x_out = x_in + u . (k_out - k_in), u = upar k_in + u1 e1 + u2 e2
  double u_dot_kout = upar * mu + st * (u1 * cp + u2 * sp);
  return x - upar + u_dot_kout;
}

// Scattering angle sampled for a dust interaction (Eq. 9), new direction.
void scatter_dust(double g, const double kin[3], Stream& rng, double kout[3]) {
  double mu = mu_hg(rng.u(W_MU), g);
  double phi = 2.0 * kPi * rng.u(W_PHI);
  double e1[3], e2[3];
  basis(kin, e1, e2);
  double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  for (int i = 0; i < 3; ++i) kout[i] = mu * kin[i] + st * (std::cos(phi) * e1[i] + std::sin(phi) * e2[i]);
  double nrm = std::sqrt(dot(kout, kout));
  for (int i = 0; i < 3; ++i) kout[i] /= nrm;
}

}  // namespace

// ==============================================================================
// C interface (ctypes)
// ==============================================================================
struct orc_line {   // per-temperature line parameters (reported for tests)
  double vth_kms, a, sigma0;
};

extern "C" void orc_line_params(double T, orc_line* out) {
  out->vth_kms = vth_kms(T);
  out->a = voigt_a(T);
  out->sigma0 = sigma0_cm2(T);
}

extern "C" void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

extern "C" void orc_stream_words(uint64_t seed, uint64_t photon, uint64_t n, uint32_t* out) {
  Stream s(seed, photon);
  for (uint64_t i = 0; i < n; ++i) out[i] = s.word((uint32_t)i);
}

extern "C" double orc_dawson(double x) { return dawson(x); }
extern "C" double orc_voigt(double a, double x) { return voigt_H(a, x); }

extern "C" void orc_voigt_batch(const double* a, const double* x, double* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = voigt_H(a[i], x[i]);
}

extern "C" double orc_u0(double x, double a) { return u0_rule(std::fabs(x), a); }
extern "C" double orc_u0_eq10(double x, double a) { return eq10_u0(std::fabs(x), a); }
extern "C" double orc_xcw(double a) { return (a > 0.0 && a < 0.65) ? xcw_exact(a) : NAN; }
extern "C" double orc_eq10_mass(double x, double a, double u0) { return eq10_mass(std::fabs(x), a, u0); }
// 1: Eq. 10 as printed (default); 0: three-piece envelope with the device's word use.
extern "C" void orc_set_upar_method(int m) { g_upar_method = (m == 0) ? 0 : 1; }
extern "C" int orc_get_upar_method(void) { return g_upar_method; }

// tau along a linear-drift segment (exposed to pin the quadrature): returns the total
// tau over [0,S] and, if tau_rem < total, *s_star.
extern "C" double orc_segment_tau(double x0, double gam, double kap0, double kapd, double a, double S,
                       double tau_rem, double* s_star) {
  Segment sg{x0, gam, kap0, kapd, a};
  double tt = 0.0, ss = -1.0;
  if (segment_walk(sg, S, tau_rem, &ss, &tt)) { *s_star = ss; return -1.0; }
  *s_star = -1.0;
  return tt;
}

// n samples of u_par at fixed (x, a), photon ids 0..n-1 of stream `seed`.
extern "C" void orc_sample_upar(double x, double a, uint64_t seed, int64_t n, double* out, uint64_t* iters) {
  uint64_t it = 0;
  for (int64_t i = 0; i < n; ++i) {
    Stream s(seed, (uint64_t)i);
    out[i] = sample_upar(x, a, s, &it);
  }
  if (iters) *iters = it;
}

extern "C" void orc_sample_mu(int kind, double g, uint64_t seed, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    Stream s(seed, (uint64_t)i);
    double R = s.u(0);
    out[i] = (kind == 0) ? mu_isotropic(R) : (kind == 1) ? mu_dipole(R) : mu_hg(R, g);
  }
}

// One resonant scattering of a photon travelling along +z at gas-frame frequency x_in
// in static gas: outputs x_out and mu = k_in . k_out.
extern "C" void orc_scatter_once(double x_in, double a, int phase, uint64_t seed, int64_t n, double* x_out,
                      double* mu_out) {
  const double kin[3] = {0.0, 0.0, 1.0};
  for (int64_t i = 0; i < n; ++i) {
    Stream s(seed, (uint64_t)i);
    double kout[3];
    x_out[i] = scatter_HI(x_in, a, phase, kin, s, kout, nullptr, nullptr);
    mu_out[i] = kout[2];
  }
}

// ------------------------------------------------------------------------------
// Gridless geometries (Sec. 3.3): spherical shell (sphere when R_in = 0) and
// infinite slab.  Lengths in units of R_out; tau0 is the line-centre HI optical
// depth n sigma_0 (R_out - R_in) across the gas (slab: centre to face).
// ------------------------------------------------------------------------------
struct orc_shell {
  int32_t geometry;  // 0 shell/sphere, 1 slab
  int32_t phase;     // 0 isotropic, 1 dipole, 2 mixed core/wing
  int32_t core_skip; // 1: core-skipping with x_crit = 0.2 (a tau0)^(1/3) when a tau0 >= 1 (Sec. 3.4.2)
  int32_t pad;
  double R_in, R_out;
  double tau0;       // line-centre HI optical depth across the gas
  double T;          // K
  double v_max;      // km/s at R_out (shell: v = v_max r/R_out radial; slab: v_z = v_max z/R_out)
  double tau_dust;   // dust extinction optical depth across the gas (frequency independent)
  double albedo, g_hg;
};

struct orc_source {
  int32_t line;     // 0: delta at X0; 1: Gaussian N(X0, sigma^2)
  int32_t pad;
  double X0, sigma; // km/s, lab frame
};

struct orc_result {
  uint64_t n_escaped, n_absorbed, n_capped;
  uint64_t sum_scat;      // resonant HI scatterings
  double sum_scat2;
  uint64_t sum_dust_scat;
  uint64_t sum_upar_iters;
  double cpu_seconds_unused;
};

namespace {

struct ShellModel {
  int geometry, phase;
  double R_in, R_out, kap0, kapd, vth, a, gam, vgrad, albedo, g, xcrit;
};

ShellModel make_shell(const orc_shell& p) {
  ShellModel m;
  m.geometry = p.geometry; m.phase = p.phase;
  m.R_in = (p.geometry == 0) ? p.R_in : 0.0;
  m.R_out = p.R_out;
  double L = (p.geometry == 0) ? (p.R_out - p.R_in) : p.R_out;
  m.kap0 = p.tau0 / L;
  m.kapd = p.tau_dust / L;
  m.vth = vth_kms(p.T);
  m.a = voigt_a(p.T);
  m.vgrad = p.v_max / p.R_out;      // km/s per unit length
  m.gam = m.vgrad / m.vth;          // |dx/ds| along a ray (shell); slab: times k_z^2
  m.albedo = p.albedo; m.g = p.g_hg;
  const double at = m.a * p.tau0;
  m.xcrit = (p.core_skip && at >= 1.0) ? 0.2 * std::cbrt(at) : 0.0;
  return m;
}

// gas velocity vector at p
void gas_vel(const ShellModel& m, const double p[3], double v[3]) {
  if (m.geometry == 0) { for (int i = 0; i < 3; ++i) v[i] = m.vgrad * p[i]; }
  else { v[0] = 0.0; v[1] = 0.0; v[2] = m.vgrad * p[2]; }
}

// distance along k from p (|p| <= R) to the sphere of radius R
double exit_sphere(const double p[3], const double k[3], double R) {
  double b = dot(p, k), c = dot(p, p) - R * R;
  double disc = b * b - c;
  if (disc < 0.0) disc = 0.0;
  return -b + std::sqrt(disc);
}

struct PhotonOut { double X; uint64_t nscat; uint32_t ndust; uint8_t status; uint64_t iters; };

// One photon packet, emission to escape/absorption (Sec. 3.4).
void run_photon_shell(const ShellModel& m, const orc_source& src, uint64_t seed, uint64_t pid,
                      uint64_t cap, PhotonOut& out) {
  Stream rng(seed, pid);
  out.nscat = 0; out.ndust = 0; out.status = 0; out.iters = 0;
  // Emission: isotropic direction, line profile in the (static) source frame.
  double p[3] = {0.0, 0.0, 0.0}, k[3];
  {
    double mu = mu_isotropic(rng.u(0));
    double phi = 2.0 * kPi * rng.u(1);
    double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    k[0] = st * std::cos(phi); k[1] = st * std::sin(phi); k[2] = mu;
  }
  double X = src.X0;
  if (src.line == 1) {
    double R1 = rng.u(2), R2 = rng.u(3);
    X += src.sigma * std::sqrt(-2.0 * std::log(R1)) * std::cos(2.0 * kPi * R2);
  }
  bool in_cavity = (m.geometry == 0 && m.R_in > 0.0);
  for (uint32_t ev = 1;; ++ev) {
    rng.start_event(ev);
    // draw the optical depth to the next interaction (Eq. 3): tau = -ln R
    double tau_rem = -std::log(rng.u(W_TAU));
    bool interact = false;
    while (!interact) {
      if (in_cavity) {
        double s = exit_sphere(p, k, m.R_in);
        for (int i = 0; i < 3; ++i) p[i] += s * k[i];
        in_cavity = false;
        continue;
      }
      // gas segment: to the outer boundary, or to the inner sphere if the ray hits it
      double S; int next;  // next: 0 escape, 1 cavity
      double v_dot_k;      // gas velocity along k at p (km/s)
      double gam;
      if (m.geometry == 0) {
        S = exit_sphere(p, k, m.R_out); next = 0;
        if (m.R_in > 0.0) {
          double b = dot(p, k), c = dot(p, p) - m.R_in * m.R_in, disc = b * b - c;
          if (b < 0.0 && disc > 0.0) {
            double s_in = -b - std::sqrt(disc);
            if (s_in < S) { S = std::max(0.0, s_in); next = 1; }
          }
        }
        v_dot_k = m.vgrad * dot(p, k);
        gam = m.gam;
      } else {
        double Z = m.R_out;
        if (k[2] > 0.0) S = (Z - p[2]) / k[2];
        else if (k[2] < 0.0) S = (-Z - p[2]) / k[2];
        else S = HUGE_VAL;
        next = 0;
        v_dot_k = m.vgrad * p[2] * k[2];
        gam = m.gam * k[2] * k[2];
      }
      Segment sg{(X - v_dot_k) / m.vth, gam, m.kap0, m.kapd, m.a};
      double s_star = 0.0, tseg = 0.0;
      if (segment_walk(sg, S, tau_rem, &s_star, &tseg)) {
        for (int i = 0; i < 3; ++i) p[i] += s_star * k[i];
        interact = true;
      } else {
        tau_rem -= tseg;
        for (int i = 0; i < 3; ++i) p[i] += S * k[i];
        if (next == 0) { out.X = X; out.status = 1; return; }
        in_cavity = true;
      }
    }
    // Interaction (Sec. 3.4): channel i with probability tau_i / sum tau.
    double v[3];
    gas_vel(m, p, v);
    double x = (X - dot(v, k)) / m.vth;
    double kHI = m.kap0 * voigt_H(m.a, x);
    bool dust = false;
    if (m.kapd > 0.0) dust = rng.u(W_CHANNEL) >= kHI / (kHI + m.kapd);
    double kout[3];
    if (dust) {
      bool scat;
      if (m.albedo <= 0.0) scat = false;
      else if (m.albedo >= 1.0) scat = true;
      else scat = rng.u(W_ALBEDO) < m.albedo;
      if (!scat) { out.X = X; out.status = 2; return; }
      scatter_dust(m.g, k, rng, kout);
      X = X + dot(v, kout) - dot(v, k);  // frequency unchanged in the gas (grain) frame
      out.ndust++;
    } else {
      double xo = scatter_HI(x, m.a, m.phase, k, rng, kout, nullptr, &out.iters, m.xcrit);
      X = xo * m.vth + dot(v, kout);
      out.nscat++;
      if (out.nscat >= cap) { out.X = X; out.status = 3; return; }
    }
    for (int i = 0; i < 3; ++i) k[i] = kout[i];
  }
}

struct SpecAcc {
  int nb; double lo, hi;
  std::vector<uint64_t> counts;  // nb + 2 (underflow, overflow)
  void init(int n, double l, double h) { nb = n; lo = l; hi = h; counts.assign(n + 2, 0); }
  void add(double X) {
    if (nb <= 0) return;
    if (X < lo) { counts[nb]++; return; }
    if (X >= hi) { counts[nb + 1]++; return; }
    int b = (int)std::floor((X - lo) / (hi - lo) * nb);
    if (b >= nb) b = nb - 1;
    counts[b]++;
  }
};

template <class F>
void parallel_photons(uint64_t n, int n_threads, F&& work) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  std::atomic<uint64_t> next{0};
  const uint64_t chunk = 16;
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t) {
    th.emplace_back([&, t]() {
      for (;;) {
        uint64_t i0 = next.fetch_add(chunk);
        if (i0 >= n) break;
        uint64_t i1 = std::min(n, i0 + chunk);
        for (uint64_t i = i0; i < i1; ++i) work(t, i);
      }
    });
  }
  for (auto& x : th) x.join();
}

}  // namespace

// Run n photons (ids first_id .. first_id+n-1).  Spectrum: escaped lab frequency X
// (km/s) in n_bins over [X_min, X_max) plus underflow/overflow (counts has n_bins+2).
// raw_X / raw_nscat / raw_status may be null.
extern "C" int orc_run_shell(const orc_shell* geo, const orc_source* src, uint64_t first_id, uint64_t n,
                  uint64_t seed, int32_t n_bins, double X_min, double X_max, uint64_t max_scat,
                  int32_t n_threads, uint64_t* counts, orc_result* res, double* raw_X,
                  uint64_t* raw_nscat, uint8_t* raw_status, uint32_t* raw_ndust) {
  if (!geo || !src || !res) return -1;
  ShellModel m = make_shell(*geo);
  if (!(m.vth > 0.0) || geo->R_out <= geo->R_in) return -1;
  int nt = (n_threads <= 0) ? (int)std::max(1u, std::thread::hardware_concurrency()) : n_threads;
  std::vector<SpecAcc> spec(nt);
  std::vector<orc_result> acc(nt);
  for (int t = 0; t < nt; ++t) { spec[t].init(n_bins, X_min, X_max); std::memset(&acc[t], 0, sizeof(orc_result)); }
  uint64_t cap = max_scat ? max_scat : ~0ull;
  parallel_photons(n, nt, [&](int t, uint64_t i) {
    PhotonOut po;
    run_photon_shell(m, *src, seed, first_id + i, cap, po);
    orc_result& r = acc[t];
    if (po.status == 1) { r.n_escaped++; spec[t].add(po.X); }
    else if (po.status == 2) r.n_absorbed++;
    else r.n_capped++;
    r.sum_scat += po.nscat;
    r.sum_scat2 += (double)po.nscat * (double)po.nscat;
    r.sum_dust_scat += po.ndust;
    r.sum_upar_iters += po.iters;
    if (raw_X) raw_X[i] = po.X;
    if (raw_nscat) raw_nscat[i] = po.nscat;
    if (raw_status) raw_status[i] = po.status;
    if (raw_ndust) raw_ndust[i] = po.ndust;
  });
  std::memset(res, 0, sizeof(orc_result));
  if (counts) std::memset(counts, 0, sizeof(uint64_t) * (size_t)(n_bins + 2));
  for (int t = 0; t < nt; ++t) {
    res->n_escaped += acc[t].n_escaped; res->n_absorbed += acc[t].n_absorbed;
    res->n_capped += acc[t].n_capped; res->sum_scat += acc[t].sum_scat;
    res->sum_scat2 += acc[t].sum_scat2; res->sum_dust_scat += acc[t].sum_dust_scat;
    res->sum_upar_iters += acc[t].sum_upar_iters;
    if (counts) for (int b = 0; b < n_bins + 2; ++b) counts[b] += spec[t].counts[b];
  }
  return 0;
}

// ------------------------------------------------------------------------------
// Power-law shells for the shell-model parameter sweep (Sec. 5.1).
// Outer radius 1, inner radius 1/dv_ratio (the ratio of the shell radii, >= 1); number
// density n(r) ~ r^alpha_rho normalised so that the radial column between the radii is
// N_HI; radial outflow v(r) ~ r^alpha_v normalised so that its distance average over
// [r_i, 1] is v_avg; uniform T; optional dust with the same radial profile as the gas
// (tau_dust = its radial optical depth).  Lengths in units of the outer radius, so the
// HI opacity per unit length is kappa(r) = tau0 f(r) / F with f = r^alpha_rho,
// F = int_{r_i}^1 f dr and tau0 = N_HI sigma_0 (line-centre column optical depth).
// Transport integrates tau exactly along each straight path (adaptive Gauss-Legendre
// pieces, Newton for the crossing), with x(s) = (X - v(r) (p + s k).k / r) / v_th.
// Each photon records its emitted and escaping lab frequencies and the HI column it
// traversed (in units of N_HI), from which the emergent spectrum is reweighted to other
// intrinsic widths, equivalent widths and dust depths (the post-processing of Sec. 5.1).
// ------------------------------------------------------------------------------
struct orc_plshell {
  double dv_ratio;          // r_o / r_i (> 1)
  double N_HI;              // cm^-2, radial column between the radii
  double T;                 // K
  double v_avg;             // km/s, distance-averaged outflow speed
  double alpha_rho, alpha_v;
  double tau_dust;          // radial dust optical depth (dust follows the gas), 0 = none
  int32_t phase;            // 0 isotropic, 1 dipole, 2 mixed
  int32_t species;          // 0: HI Lyman alpha; 1: Mg II doublet (N_HI is then the Mg II column)
};

// Intrinsic spectrum sampled at emission: a Gaussian line of width sigma (km/s) with
// equivalent width ew (km/s) on a flat continuum over [-C, C] (C = 0: line only).
struct orc_plsource {
  double sigma, ew, C;
  double X0;                // centre of the line and of the continuum (km/s)
};

namespace {

// int_{lo}^{hi} r^alpha dr
double pow_integral(double alpha, double lo, double hi) {
  if (std::fabs(alpha + 1.0) < 1e-12) return std::log(hi / lo);
  return (std::pow(hi, alpha + 1.0) - std::pow(lo, alpha + 1.0)) / (alpha + 1.0);
}

// Mg II doublet (Sec. 2.4): K = 2S1/2-2P3/2 at 2796.352 A (f 0.608, A 2.60e8 /s) and
// H = 2S1/2-2P1/2 at 2803.531 A (f 0.303, A 2.57e8 /s), vacuum wavelengths and atomic
// data of the NIST Atomic Spectra Database; ion mass 24.305 u.  Both transitions are
// resonant (the upper levels decay only to the ground state), so a scattering re-emits
// in the transition that absorbed.  The frequency variable is X = c (nu - nu_K) / nu_K;
// for transition l with r_l = lambda_l / lambda_K its own offset is
// X_l = c (nu - nu_l) / nu_l = X + (r_l - 1)(c + X).  The K line scatters with the
// configured phase function, H (J = 1/2 upper level) isotropically.
const double kC_kms = 2.99792458e5;
const double kLamMgK = 2796.352e-8, kLamMgH = 2803.531e-8;
const double kFMgK = 0.608, kFMgH = 0.303, kAMgK = 2.60e8, kAMgH = 2.57e8;
const double kMassMg = 24.305 * 1.66053906660e-24;
double vth_mg(double T) { return std::sqrt(2.0 * kBoltz * T / kMassMg) * 1e-5; }
double a_line(double A, double lam, double vth) { return A * lam / (4.0 * kPi * vth * 1e5); }
double sigma0_line(double f, double lam, double vth) {
  return f * kSqrtPi * kEsu * kEsu / (kMe * kC * (vth * 1e5 / lam));
}

struct PLShell {
  double ri, F, kap_n, kap_d, vth, a, v1, ar, av, G;  // v(r) = v1 r^av; G bounds |d(v mu_r)/ds|
  int phase;
  int n_lines = 1;                 // 2: Mg II doublet, line 2 = H
  double kap_n2 = 0.0, a2 = 0.0, eps2 = 0.0;  // line 2: opacity at r = 1, Voigt a, r_2 - 1
  double X2(double X) const { return X + eps2 * (kC_kms + X); }
  double X_from2(double X2v) const { return X2v - eps2 / (1.0 + eps2) * (kC_kms + X2v); }
  double n_rel(double r) const { return std::pow(r, ar); }
  double vel(double r) const { return v1 * std::pow(r, av); }
};

PLShell make_plshell(const orc_plshell& p) {
  PLShell m;
  m.ri = 1.0 / p.dv_ratio;
  const double F = pow_integral(p.alpha_rho, m.ri, 1.0);
  m.F = F;
  m.kap_d = p.tau_dust / F;
  if (p.species == 1) {
    m.vth = vth_mg(p.T);
    m.a = a_line(kAMgK, kLamMgK, m.vth);
    m.kap_n = p.N_HI * sigma0_line(kFMgK, kLamMgK, m.vth) / F;
    m.n_lines = 2;
    m.a2 = a_line(kAMgH, kLamMgH, m.vth);
    m.kap_n2 = p.N_HI * sigma0_line(kFMgH, kLamMgH, m.vth) / F;
    m.eps2 = kLamMgH / kLamMgK - 1.0;
  } else {
    m.vth = vth_kms(p.T);
    m.a = voigt_a(p.T);
    m.kap_n = p.N_HI * sigma0_cm2(p.T) / F;
  }
  m.ar = p.alpha_rho; m.av = p.alpha_v;
  m.v1 = p.v_avg * (1.0 - m.ri) / pow_integral(p.alpha_v, m.ri, 1.0);
  // |d(v(r) mu_r)/ds| = |v'(r) mu_r^2 + v(r) (1 - mu_r^2) / r| <= max(|v'|, v / r)
  double G = 0.0;
  for (int i = 0; i <= 2000; ++i) {
    double r = m.ri + (1.0 - m.ri) * i / 2000.0;
    G = std::max(G, std::max(std::fabs(p.alpha_v) * m.vel(r) / r, m.vel(r) / r));
  }
  m.G = 1.05 * G;
  m.phase = p.phase;
  return m;
}

// Opacity along the ray p + s k inside the gas: HI line plus dust, and the HI column
// density rate (in units of N_HI per unit length).
struct PLRay {
  const PLShell* m;
  double p[3], k[3], X;
  void at(double s, double& kap, double& col_rate, double& x) const {
    double q[3] = {p[0] + s * k[0], p[1] + s * k[1], p[2] + s * k[2]};
    double r = std::sqrt(dot(q, q));
    double mur = dot(q, k) / r;
    double nr = m->n_rel(r);
    x = (X - m->vel(r) * mur) / m->vth;
    kap = nr * (m->kap_n * voigt_H(m->a, x) + m->kap_d);
    if (m->n_lines == 2) {
      const double x2 = (m->X2(X) - m->vel(r) * mur) / m->vth;
      kap += nr * m->kap_n2 * voigt_H(m->a2, x2);
      if (std::fabs(x2) < std::fabs(x)) x = x2;  // the nearer line sets the quadrature pieces
    }
    col_rate = nr / m->F;  // column per unit length in units of the radial column
  }
  double kappa(double s) const { double k0, c, x; at(s, k0, c, x); return k0; }
  // tau and column over [s0, s1] on one Gauss-Legendre piece
  void piece(double s0, double s1, double& tau, double& col) const {
    const GaussLegendre& g = gl();
    double hm = 0.5 * (s1 - s0), c = 0.5 * (s1 + s0), st = 0.0, sc = 0.0;
    for (int i = 0; i < GaussLegendre::N; ++i) {
      double k0, cr, x;
      at(c + hm * g.x[i], k0, cr, x);
      st += g.w[i] * k0; sc += g.w[i] * cr;
    }
    tau = st * hm; col = sc * hm;
  }
  // piece length: x moves by at most 0.1 (0.01 |x| in the wings), the density by ~1%
  double piece_len(double s) const {
    double k0, cr, x;
    at(s, k0, cr, x);
    double dx = (std::fabs(x) < 10.0) ? 0.1 : 0.01 * std::fabs(x);
    double ls = dx * m->vth / m->G;
    double q[3] = {p[0] + s * k[0], p[1] + s * k[1], p[2] + s * k[2]};
    double r = std::sqrt(dot(q, q));
    if (m->ar != 0.0) ls = std::min(ls, 0.01 * r / std::fabs(m->ar));
    return ls;
  }
};

// Walk [0, S]: true and s_star when tau reaches tau_rem, else false and the total tau;
// col accumulates the HI column (units of N_HI) up to the stop.
bool plray_walk(const PLRay& ry, double S, double tau_rem, double* s_star, double* tau_tot, double* col) {
  double s = 0.0, acc = 0.0;
  while (s < S) {
    double s1 = std::min(S, s + ry.piece_len(s));
    double tp, cp;
    ry.piece(s, s1, tp, cp);
    if (acc + tp >= tau_rem && tp > 0.0) {
      double need = tau_rem - acc, lo = s, hi = s1;
      double t = s + (s1 - s) * (need / tp);
      for (int it = 0; it < 100; ++it) {
        double ft, fc;
        ry.piece(s, t, ft, fc);
        double f = ft - need;
        if (f > 0) hi = t; else lo = t;
        double k = ry.kappa(t);
        double tn = (k > 0) ? t - f / k : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (std::fabs(tn - t) <= 1e-14 * std::max(1.0, std::fabs(t)) || hi - lo < 1e-15) { t = tn; break; }
        t = tn;
      }
      double ft, fc;
      ry.piece(s, t, ft, fc);
      *col += fc;
      *s_star = t;
      return true;
    }
    acc += tp;
    *col += cp;
    s = s1;
  }
  *tau_tot = acc;
  return false;
}

struct PLOut { double X0, X, col; uint64_t nscat, iters; uint32_t ndust; uint8_t status; };

// One photon: central point source, isotropic, intrinsic spectrum of orc_plsource
// (emission words: 0 mu, 1 azimuth, 2-3 Gaussian, 4 line or continuum, 5 continuum
// position); then the event loop of the shell (Sec. 3.4) on the power-law profiles.
void run_photon_plshell(const PLShell& m, const orc_plsource& src, uint64_t seed, uint64_t pid, uint64_t cap,
                        PLOut& out) {
  Stream rng(seed, pid);
  out.nscat = 0; out.ndust = 0; out.iters = 0; out.status = 0; out.col = 0.0;
  double p[3] = {0.0, 0.0, 0.0}, k[3];
  {
    double mu = mu_isotropic(rng.u(0));
    double phi = 2.0 * kPi * rng.u(1);
    double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    k[0] = st * std::cos(phi); k[1] = st * std::sin(phi); k[2] = mu;
  }
  const double p_line = (src.C > 0.0) ? src.ew / (src.ew + 2.0 * src.C) : 1.0;
  double X;
  if (rng.u(4) <= p_line) {
    double R1 = rng.u(2), R2 = rng.u(3);
    X = src.X0 + src.sigma * std::sqrt(-2.0 * std::log(R1)) * std::cos(2.0 * kPi * R2);
  } else {
    X = src.X0 + src.C * (2.0 * rng.u(5) - 1.0);
  }
  out.X0 = X;
  bool in_cavity = true;
  for (uint32_t ev = 1;; ++ev) {
    rng.start_event(ev);
    double tau_rem = -std::log(rng.u(W_TAU));
    bool interact = false;
    while (!interact) {
      if (in_cavity) {  // empty: straight to the inner sphere
        double s = exit_sphere(p, k, m.ri);
        for (int i = 0; i < 3; ++i) p[i] += s * k[i];
        in_cavity = false;
        continue;
      }
      double S = exit_sphere(p, k, 1.0); int next = 0;
      {
        double b = dot(p, k), c = dot(p, p) - m.ri * m.ri, disc = b * b - c;
        if (b < 0.0 && disc > 0.0) {
          double s_in = -b - std::sqrt(disc);
          if (s_in < S) { S = std::max(0.0, s_in); next = 1; }
        }
      }
      PLRay ry{&m, {p[0], p[1], p[2]}, {k[0], k[1], k[2]}, X};
      double s_star = 0.0, tseg = 0.0;
      if (plray_walk(ry, S, tau_rem, &s_star, &tseg, &out.col)) {
        for (int i = 0; i < 3; ++i) p[i] += s_star * k[i];
        interact = true;
      } else {
        tau_rem -= tseg;
        for (int i = 0; i < 3; ++i) p[i] += S * k[i];
        if (next == 0) { out.X = X; out.status = 1; return; }
        in_cavity = true;
      }
    }
    // interaction at p: gas velocity v(r) r_hat
    double r = std::sqrt(dot(p, p));
    double vr = m.vel(r);
    double v[3] = {vr * p[0] / r, vr * p[1] / r, vr * p[2] / r};
    double x = (X - dot(v, k)) / m.vth;
    double k1 = m.kap_n * m.n_rel(r) * voigt_H(m.a, x);
    double kd = m.kap_d * m.n_rel(r);
    double x2 = 0.0, k2 = 0.0;
    if (m.n_lines == 2) {
      x2 = (m.X2(X) - dot(v, k)) / m.vth;
      k2 = m.kap_n2 * m.n_rel(r) * voigt_H(m.a2, x2);
    }
    // channel in proportion to the opacities: line 1, line 2, dust (one uniform)
    int ch = 0;
    if (kd > 0.0 || m.n_lines == 2) {
      const double u = rng.u(W_CHANNEL), kt = k1 + k2 + kd;
      ch = (u < k1 / kt) ? 0 : ((u < (k1 + k2) / kt) ? 1 : 2);
    }
    if (ch == 2) { out.X = X; out.status = 2; return; }  // dust absorbs (albedo 0 in the sweep)
    double kout[3];
    if (ch == 0) {
      double xo = scatter_HI(x, m.a, m.phase, k, rng, kout, nullptr, &out.iters);
      X = xo * m.vth + dot(v, kout);
    } else {
      double xo = scatter_HI(x2, m.a2, PH_ISO, k, rng, kout, nullptr, &out.iters);
      X = m.X_from2(xo * m.vth + dot(v, kout));
    }
    out.nscat++;
    if (out.nscat >= cap) { out.X = X; out.status = 3; return; }
    for (int i = 0; i < 3; ++i) k[i] = kout[i];
  }
}

// Intrinsic spectrum density (per km/s) of the line-plus-continuum model.
double intrinsic_pdf(double X, double sigma, double ew, double C) {
  const double pl = (C > 0.0) ? ew / (ew + 2.0 * C) : 1.0;
  double g = std::exp(-0.5 * X * X / (sigma * sigma)) / (std::sqrt(2.0 * kPi) * sigma);
  double c = (C > 0.0 && std::fabs(X) <= C) ? 1.0 / (2.0 * C) : 0.0;
  return pl * g + (1.0 - pl) * c;
}

}  // namespace

// Mg II line data at temperature T: v_th [km/s], a_K, sigma0_K [cm^2], a_H, sigma0_H, and the
// H line centre on the K-relative scale X [km/s].
extern "C" void orc_mgii_params(double T, double* out) {
  const double vth = vth_mg(T);
  out[0] = vth;
  out[1] = a_line(kAMgK, kLamMgK, vth);
  out[2] = sigma0_line(kFMgK, kLamMgK, vth);
  out[3] = a_line(kAMgH, kLamMgH, vth);
  out[4] = sigma0_line(kFMgH, kLamMgH, vth);
  out[5] = kC_kms * (kLamMgK / kLamMgH - 1.0);
}

extern "C" void orc_plshell_profile(const orc_plshell* geo, double r, double* n_rel_kappa, double* v) {
  PLShell m = make_plshell(*geo);
  *n_rel_kappa = m.kap_n * m.n_rel(r);
  *v = m.vel(r);
}

extern "C" int orc_run_plshell(const orc_plshell* geo, const orc_plsource* src, uint64_t first_id, uint64_t n,
                               uint64_t seed, int32_t n_bins, double X_min, double X_max, uint64_t max_scat,
                               int32_t n_threads, uint64_t* counts, orc_result* res, double* raw_X0,
                               double* raw_X, double* raw_col, uint64_t* raw_nscat, uint8_t* raw_status) {
  if (!geo || !src || !res || !(geo->dv_ratio > 1.0) || !(geo->T > 0.0)) return -1;
  PLShell m = make_plshell(*geo);
  int nt = (n_threads <= 0) ? (int)std::max(1u, std::thread::hardware_concurrency()) : n_threads;
  std::vector<SpecAcc> spec(nt);
  std::vector<orc_result> acc(nt);
  for (int t = 0; t < nt; ++t) { spec[t].init(n_bins, X_min, X_max); std::memset(&acc[t], 0, sizeof(orc_result)); }
  uint64_t cap = max_scat ? max_scat : ~0ull;
  parallel_photons(n, nt, [&](int t, uint64_t i) {
    PLOut po;
    run_photon_plshell(m, *src, seed, first_id + i, cap, po);
    orc_result& r = acc[t];
    if (po.status == 1) { r.n_escaped++; spec[t].add(po.X); }
    else if (po.status == 2) r.n_absorbed++;
    else r.n_capped++;
    r.sum_scat += po.nscat;
    r.sum_scat2 += (double)po.nscat * (double)po.nscat;
    r.sum_upar_iters += po.iters;
    if (raw_X0) raw_X0[i] = po.X0;
    if (raw_X) raw_X[i] = po.X;
    if (raw_col) raw_col[i] = po.col;
    if (raw_nscat) raw_nscat[i] = po.nscat;
    if (raw_status) raw_status[i] = po.status;
  });
  std::memset(res, 0, sizeof(orc_result));
  if (counts) std::memset(counts, 0, sizeof(uint64_t) * (size_t)(n_bins + 2));
  for (int t = 0; t < nt; ++t) {
    res->n_escaped += acc[t].n_escaped; res->n_absorbed += acc[t].n_absorbed;
    res->n_capped += acc[t].n_capped; res->sum_scat += acc[t].sum_scat;
    res->sum_scat2 += acc[t].sum_scat2; res->sum_upar_iters += acc[t].sum_upar_iters;
    if (counts) for (int b = 0; b < n_bins + 2; ++b) counts[b] += spec[t].counts[b];
  }
  return 0;
}

// Post-processing of a run's escaped photons (Sec. 5.1): weight
//   w = p_target(X0) / p_sampled(X0) * exp(-tau_d * col)
// for a target intrinsic spectrum (sigma, ew, C) and dust depth tau_d (dust following
// the gas, so its optical depth along a path is tau_d times the HI column in units of
// N_HI); out[b] = sum of weights per bin / n (n_bins + underflow, overflow).
extern "C" void orc_reweight(int64_t n, const double* X0, const double* X, const double* col,
                             const uint8_t* status, double s_sigma, double s_ew, double s_C, double t_sigma,
                             double t_ew, double t_C, double tau_d, int32_t n_bins, double X_min, double X_max,
                             double* out) {
  for (int b = 0; b < n_bins + 2; ++b) out[b] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (status[i] != 1) continue;
    const double ps = intrinsic_pdf(X0[i], s_sigma, s_ew, s_C);
    const double w = (ps > 0.0) ? intrinsic_pdf(X0[i], t_sigma, t_ew, t_C) / ps * std::exp(-tau_d * col[i]) : 0.0;
    int b;
    if (X[i] < X_min) b = n_bins;
    else if (X[i] >= X_max) b = n_bins + 1;
    else { b = (int)std::floor((X[i] - X_min) / (X_max - X_min) * n_bins); if (b >= n_bins) b = n_bins - 1; }
    out[b] += w;
  }
  for (int b = 0; b < n_bins + 2; ++b) out[b] /= (double)n;
}

// ------------------------------------------------------------------------------
// Uniform Cartesian grid (Sec. 3.3), positions in cell units, domain [0,n)^3.
// Cell walk: Amanatides & Woo (1987) with the following bit-reproducible contract,
// shared by definition with the CUDA path: FP64 round-to-nearest, no fused
// multiply-add, operations exactly as written.
//   start cell i = floor(p); if d < 0 and p == i then i - 1 (a ray starting on a face
//     and leaving through it starts in the lower cell);
//   inv_ax = 1 / d_ax once per ray (IEEE division), +inf marker when d == 0;
//   distance to the next face along each axis t_ax = ((i + (d > 0)) - p) * inv_ax;
//   step along the axis with the smallest t, ties to the lowest axis (x < y < z);
//   segment length = t_next - t_current.
// ------------------------------------------------------------------------------
namespace {

struct DDA {
  int i[3], step[3];
  double p[3], d[3], inv[3];
  double t;  // distance already travelled from p
  void init(const double pin[3], const double din[3]) {
    t = 0.0;
    for (int a = 0; a < 3; ++a) {
      p[a] = pin[a]; d[a] = din[a];
      double f = std::floor(p[a]);
      int ii = (int)f;
      if (d[a] < 0.0 && p[a] == f) ii -= 1;
      i[a] = ii;
      step[a] = (d[a] > 0.0) ? 1 : (d[a] < 0.0 ? -1 : 0);
      inv[a] = (step[a] != 0) ? 1.0 / d[a] : 0.0;
    }
  }
  double tface(int a) const {
    if (step[a] == 0) return HUGE_VAL;
    double face = (double)(i[a] + (step[a] > 0 ? 1 : 0));
    return (face - p[a]) * inv[a];
  }
  // returns the axis of the next face and its distance
  int next_axis(double* tn) const {
    double t0 = tface(0), t1 = tface(1), t2 = tface(2);
    int ax = 0; double tm = t0;
    if (t1 < tm) { ax = 1; tm = t1; }
    if (t2 < tm) { ax = 2; tm = t2; }
    *tn = tm;
    return ax;
  }
};

bool inside(const int i[3], const int n[3]) {
  return i[0] >= 0 && i[1] >= 0 && i[2] >= 0 && i[0] < n[0] && i[1] < n[1] && i[2] < n[2];
}

}  // namespace

// Trace n rays; cells[r*max_steps + s] = linear cell index (ix + nx*(iy + ny*iz)),
// seg[...] = path length in that cell (cell units); count[r] = number of cells.
// Origins FP64 (3 per ray), directions FP32 (3 per ray, as the packet state stores them).
extern "C" int orc_dda_trace(const int32_t* dims, const double* origins, const float* dirs, int32_t n,
                  int32_t max_steps, int64_t* cells, double* seg, int32_t* count) {
  int nd[3] = {dims[0], dims[1], dims[2]};
  for (int r = 0; r < n; ++r) {
    double p[3] = {origins[3 * r], origins[3 * r + 1], origins[3 * r + 2]};
    double d[3] = {(double)dirs[3 * r], (double)dirs[3 * r + 1], (double)dirs[3 * r + 2]};
    DDA w; w.init(p, d);
    int c = 0;
    while (c < max_steps && inside(w.i, nd)) {
      double tn; int ax = w.next_axis(&tn);
      cells[(int64_t)r * max_steps + c] = (int64_t)w.i[0] + (int64_t)nd[0] * ((int64_t)w.i[1] + (int64_t)nd[1] * w.i[2]);
      seg[(int64_t)r * max_steps + c] = tn - w.t;
      ++c;
      w.t = tn;
      w.i[ax] += w.step[ax];
    }
    count[r] = c;
  }
  return 0;
}

// ------------------------------------------------------------------------------
// Grid MCRT with peeling-off (Sec. 3.4, 3.4.1).
// Fields per cell (arrays of nx*ny*nz, x fastest): n_HI [cm^-3], T [K],
// v [km/s] (3 arrays), kd = dust extinction coefficient [cm^-1].
// Emission: cell chosen with probability proportional to n_HI^2 (cumulative sum +
// search), uniform position inside it, isotropic direction, thermal Gaussian
// x ~ N(0, 1/2) in the cell frame (Sec. 2.1), lab X = x v_th + v.k.
// Peeling-off at emission and at every scattering towards the three observers
// along +x, +y, +z: weight p_Omega(mu) exp(-tau_obs) with p_Omega = P(mu)/(2 pi)
// (isotropic emission: 1/(4 pi)), tau_obs integrated cell by cell to the box face
// at the frequency the photon would have towards the observer; the ray stops
// once tau_obs > 50 (weight < 2e-22).  Image pixel from the position projected on
// the two other axes (in cyclic order), spectral bin from the peel frequency.
// ------------------------------------------------------------------------------
struct orc_grid_run {
  int32_t dims[3];
  int32_t phase;
  double cell_cm;
  double albedo, g_hg;
  int32_t n_bins; int32_t img_nx;     // image pixels along each image axis
  double X_min, X_max;                // spectral range (km/s) for spectra and cubes
  int32_t peel;                       // 0/1
  int32_t pad;
  uint64_t max_scat;
};

namespace {

struct GridModel {
  int n[3];
  std::vector<double> kap0, a, vth, vx, vy, vz, kd;  // per cell, kap0 and kd per cell length
  std::vector<double> cdf;
  double total;
};

void peel_tau(const GridModel& g, const double p[3], int axis, double Xp, double* tau_out) {
  double d[3] = {0.0, 0.0, 0.0};
  d[axis] = 1.0;
  DDA w; w.init(p, d);
  double tau = 0.0;
  while (inside(w.i, g.n)) {
    double tn; int ax = w.next_axis(&tn);
    int64_t c = (int64_t)w.i[0] + (int64_t)g.n[0] * ((int64_t)w.i[1] + (int64_t)g.n[1] * w.i[2]);
    double vk = (axis == 0) ? g.vx[c] : (axis == 1) ? g.vy[c] : g.vz[c];
    double x = (Xp - vk) / g.vth[c];
    tau += (g.kap0[c] * voigt_H(g.a[c], x) + g.kd[c]) * (tn - w.t);
    if (tau > 50.0) break;
    w.t = tn;
    w.i[ax] += w.step[ax];
  }
  *tau_out = tau;
}

}  // namespace

extern "C" int orc_run_grid(const float* nHI, const float* T, const float* vx, const float* vy, const float* vz,
                 const float* kd, const orc_grid_run* run, uint64_t first_id, uint64_t n, uint64_t seed,
                 int32_t n_threads, uint64_t* spec_counts, double* cube, orc_result* res, double* raw_X,
                 uint64_t* raw_nscat, uint8_t* raw_status, double* raw_k, uint32_t* raw_ndust) {
  GridModel g;
  for (int a = 0; a < 3; ++a) g.n[a] = run->dims[a];
  int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
  g.kap0.resize(nc); g.a.resize(nc); g.vth.resize(nc); g.vx.resize(nc); g.vy.resize(nc); g.vz.resize(nc);
  g.kd.resize(nc); g.cdf.resize(nc);
  double acc = 0.0;
  for (int64_t c = 0; c < nc; ++c) {
    double Tc = T[c];
    g.kap0[c] = (double)nHI[c] * sigma0_cm2(Tc) * run->cell_cm;
    g.a[c] = voigt_a(Tc);
    g.vth[c] = vth_kms(Tc);
    g.vx[c] = vx[c]; g.vy[c] = vy[c]; g.vz[c] = vz[c];
    g.kd[c] = (double)kd[c] * run->cell_cm;
    acc += (double)nHI[c] * (double)nHI[c];
    g.cdf[c] = acc;
  }
  g.total = acc;
  const int nb = run->n_bins, ni = run->img_nx;
  const int pix[3] = {g.n[0] / ni, g.n[1] / ni, g.n[2] / ni};
  const double lo = run->X_min, hi = run->X_max;
  const uint64_t cap = run->max_scat ? run->max_scat : ~0ull;
  int nt = (n_threads <= 0) ? (int)std::max(1u, std::thread::hardware_concurrency()) : n_threads;
  std::vector<SpecAcc> spec(nt);
  std::vector<orc_result> racc(nt);
  std::vector<std::vector<double>> cubes(nt);
  const size_t cube_n = (size_t)3 * ni * ni * nb;
  for (int t = 0; t < nt; ++t) {
    spec[t].init(nb, lo, hi);
    std::memset(&racc[t], 0, sizeof(orc_result));
    if (run->peel && cube) cubes[t].assign(cube_n, 0.0);
  }
  auto deposit = [&](std::vector<double>& cb, const double p[3], int axis, double X, double wgt) {
    if (X < lo || X >= hi) return;
    int b = (int)std::floor((X - lo) / (hi - lo) * nb);
    if (b >= nb) b = nb - 1;
    int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
    int ix = (int)std::floor(p[a1]) / pix[a1], iy = (int)std::floor(p[a2]) / pix[a2];
    if (ix < 0 || iy < 0 || ix >= ni || iy >= ni) return;
    cb[(((size_t)axis * ni + iy) * ni + ix) * nb + b] += wgt;
  };
  parallel_photons(n, nt, [&](int t, uint64_t i) {
    uint64_t pid = first_id + i;
    Stream rng(seed, pid);
    orc_result& r = racc[t];
    std::vector<double>& cb = cubes[t];
    bool peel = run->peel && cube;
    // emission
    double R = rng.u(0) * g.total;
    int64_t c = std::upper_bound(g.cdf.begin(), g.cdf.end(), R) - g.cdf.begin();
    if (c >= nc) c = nc - 1;
    int ci[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((int64_t)g.n[0] * g.n[1]))};
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = (double)ci[a] + rng.u(1 + a);
    double k[3];
    {
      double mu = mu_isotropic(rng.u(4));
      double phi = 2.0 * kPi * rng.u(5);
      double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
      k[0] = st * std::cos(phi); k[1] = st * std::sin(phi); k[2] = mu;
    }
    double xe;
    {
      double R1 = rng.u(6), R2 = rng.u(7);
      xe = std::sqrt(-std::log(R1)) * std::cos(2.0 * kPi * R2);  // N(0, 1/2)
    }
    double vc[3] = {g.vx[c], g.vy[c], g.vz[c]};
    double X = xe * g.vth[c] + dot(vc, k);
    if (peel) {
      for (int ax = 0; ax < 3; ++ax) {
        double Xp = xe * g.vth[c] + vc[ax];
        double tau; peel_tau(g, p, ax, Xp, &tau);
        deposit(cb, p, ax, Xp, std::exp(-tau) / (4.0 * kPi));
      }
    }
    uint64_t nscat = 0, ndust = 0, iters = 0;
    int status = 0;
    uint32_t ev = 0;
    while (status == 0) {
      rng.start_event(++ev);
      double tau_rem = -std::log(rng.u(W_TAU));
      DDA w; w.init(p, k);
      bool hit = false;
      int64_t cc = 0;
      double xcell = 0.0, kH = 0.0, kD = 0.0;
      while (!hit) {
        if (!inside(w.i, g.n)) { status = 1; break; }
        double tn; int ax = w.next_axis(&tn);
        cc = (int64_t)w.i[0] + (int64_t)g.n[0] * ((int64_t)w.i[1] + (int64_t)g.n[1] * w.i[2]);
        double vk = g.vx[cc] * k[0] + g.vy[cc] * k[1] + g.vz[cc] * k[2];
        xcell = (X - vk) / g.vth[cc];
        kH = g.kap0[cc] * voigt_H(g.a[cc], xcell);
        kD = g.kd[cc];
        double kt = kH + kD;
        double dt = tn - w.t;
        if (kt * dt >= tau_rem && kt > 0.0) {
          double ts = w.t + tau_rem / kt;
          for (int a = 0; a < 3; ++a) p[a] = p[a] + ts * k[a];
          // keep the interaction point inside the current cell
          for (int a = 0; a < 3; ++a) {
            double lo_ = (double)w.i[a], hi_ = std::nextafter((double)(w.i[a] + 1), lo_);
            p[a] = std::min(std::max(p[a], lo_), hi_);
          }
          hit = true;
        } else {
          tau_rem -= kt * dt;
          w.t = tn;
          w.i[ax] += w.step[ax];
        }
      }
      if (status == 1) {
        r.n_escaped++;
        spec[t].add(X);
        break;
      }
      double v[3] = {g.vx[cc], g.vy[cc], g.vz[cc]};
      bool dust = false;
      if (kD > 0.0) dust = rng.u(W_CHANNEL) >= kH / (kH + kD);
      double kout[3];
      if (dust) {
        bool scat;
        if (run->albedo <= 0.0) scat = false;
        else if (run->albedo >= 1.0) scat = true;
        else scat = rng.u(W_ALBEDO) < run->albedo;
        if (!scat) { status = 2; r.n_absorbed++; break; }
        if (peel) {
          for (int ax = 0; ax < 3; ++ax) {
            double mu_o = k[ax];
            double Xp = X + v[ax] - dot(v, k);
            double tau; peel_tau(g, p, ax, Xp, &tau);
            deposit(cb, p, ax, Xp, P_hg(mu_o, run->g_hg) / (2.0 * kPi) * std::exp(-tau));
          }
        }
        scatter_dust(run->g_hg, k, rng, kout);
        X = X + dot(v, kout) - dot(v, k);
        ndust++;
      } else {
        AtomVel av;
        double xo = scatter_HI(xcell, g.a[cc], run->phase, k, rng, kout, &av, &iters);
        if (peel) {
          for (int ax = 0; ax < 3; ++ax) {
            double ko[3] = {0.0, 0.0, 0.0}; ko[ax] = 1.0;
            double mu_o = k[ax];
            double u_dot_ko = av.upar * mu_o + av.u1 * av.e1[ax] + av.u2 * av.e2[ax];
            double xp = xcell - av.upar + u_dot_ko;
            double Xp = xp * g.vth[cc] + v[ax];
            double P;
            if (run->phase == PH_ISO) P = P_iso(mu_o);
            else if (run->phase == PH_DIPOLE) P = P_dipole(mu_o);
            else P = av.core ? (P_iso(mu_o) / 3.0 + 2.0 * P_dipole(mu_o) / 3.0) : P_dipole(mu_o);
            double tau; peel_tau(g, p, ax, Xp, &tau);
            deposit(cb, p, ax, Xp, P / (2.0 * kPi) * std::exp(-tau));
            (void)ko;
          }
        }
        X = xo * g.vth[cc] + dot(v, kout);
        nscat++;
        if (nscat >= cap) { status = 3; r.n_capped++; break; }
      }
      for (int a = 0; a < 3; ++a) k[a] = kout[a];
    }
    r.sum_scat += nscat;
    r.sum_scat2 += (double)nscat * (double)nscat;
    r.sum_dust_scat += ndust;
    r.sum_upar_iters += iters;
    if (raw_X) {  // optional per-photon record: final lab X, scatterings, 1/2/3 = escaped/absorbed/capped
      raw_X[i] = X;
      raw_nscat[i] = nscat;
      raw_status[i] = (uint8_t)status;
    }
    if (raw_k)  // optional: final direction (the escape direction of escaped photons)
      for (int a = 0; a < 3; ++a) raw_k[3 * i + a] = k[a];
    if (raw_ndust) raw_ndust[i] = (uint32_t)ndust;  // optional: dust scatterings
  });
  std::memset(res, 0, sizeof(orc_result));
  if (spec_counts) std::memset(spec_counts, 0, sizeof(uint64_t) * (size_t)(nb + 2));
  if (cube && run->peel) std::memset(cube, 0, sizeof(double) * cube_n);
  for (int t = 0; t < nt; ++t) {
    res->n_escaped += racc[t].n_escaped; res->n_absorbed += racc[t].n_absorbed;
    res->n_capped += racc[t].n_capped; res->sum_scat += racc[t].sum_scat;
    res->sum_scat2 += racc[t].sum_scat2; res->sum_dust_scat += racc[t].sum_dust_scat;
    res->sum_upar_iters += racc[t].sum_upar_iters;
    if (spec_counts) for (int b = 0; b < nb + 2; ++b) spec_counts[b] += spec[t].counts[b];
    if (cube && run->peel) for (size_t j = 0; j < cube_n; ++j) cube[j] += cubes[t][j];
  }
  return 0;
}

// ------------------------------------------------------------------------------
// Lyman-alpha forest (Sec. 3.5.2, Eq. 11): for sightlines along z through cell
// columns (ix, iy), tau(v_b) = sum_k n_k sigma_0(T_k) ds H(a_k, (v_b - v_k)/v_th,k),
// v_k = (k + 1/2) dv_cell + v_los,k (Hubble flow + peculiar), v_b = (b + 1/2) dv_bin.
// Periodic: the velocity offset is taken to the nearest image in a box of width
// nz dv_cell.  tau_out[s * n_bins + b].
// ------------------------------------------------------------------------------
extern "C" int orc_forest(const float* nHI, const float* T, const float* vlos, int32_t nx, int32_t ny, int32_t nz,
               const int32_t* sel_ix, const int32_t* sel_iy, int32_t n_sel, double ds_cm, double dv_cell,
               int32_t n_bins, double dv_bin, int32_t n_threads, double* tau_out) {
  const double V = nz * dv_cell;
  int nt = (n_threads <= 0) ? (int)std::max(1u, std::thread::hardware_concurrency()) : n_threads;
  parallel_photons((uint64_t)n_sel, nt, [&](int, uint64_t s) {
    double* out = tau_out + (size_t)s * n_bins;
    for (int b = 0; b < n_bins; ++b) out[b] = 0.0;
    for (int k = 0; k < nz; ++k) {
      int64_t c = (int64_t)sel_ix[s] + (int64_t)nx * ((int64_t)sel_iy[s] + (int64_t)ny * k);
      double Tk = T[c];
      double amp = (double)nHI[c] * sigma0_cm2(Tk) * ds_cm;
      double ak = voigt_a(Tk), bk = vth_kms(Tk);
      double vk = (k + 0.5) * dv_cell + (double)vlos[c];
      for (int b = 0; b < n_bins; ++b) {
        double dv = (b + 0.5) * dv_bin - vk;
        dv -= V * std::floor(dv / V + 0.5);
        out[b] += amp * voigt_H(ak, dv / bk);
      }
    }
  });
  return 0;
}

