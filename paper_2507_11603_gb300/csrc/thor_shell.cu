// thor_shell.cu -- photon-packet loop through gridless spherical shells (THOR
// Sec. 3.3-3.4): emission, propagation with the velocity-gradient step limiter
// (Sec. 5.1), interaction channel choice, resonant / dust scattering, escape tally.
//
// Execution model: persistent warps.  Every loop iteration is one event (draw tau,
// propagate to the interaction or the boundary, interact) for every live lane;
// lanes whose packet finished are refilled from the photon work queue with one
// warp-aggregated atomic (ballot of the idle lanes), so a warp stays full until the
// queue drains (runs with fewer photons than lanes fill per_warp lanes of every warp).
// The packet state lives in registers; the time-sliced variant (serving) resumes its
// packets from a list spread over all warps and appends the survivors to the next one.
#include "thor_device.cuh"
#include "thor_internal.h"

namespace thor {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kServedPipeLanes = 32;  // served rounds: pipelined events in every warp
constexpr int kServedBurstLanes = 1;  // served rounds: core bursts for lone packets
constexpr uint32_t kLongLived = 1u << 14;
constexpr uint32_t kPriBudget = 16;  // served rounds: budget multiple of a priority warp (one packet)  // served rounds: packets past this many events run one per warp

struct Photon {
  double px, py, pz;  // FP64 anchor; the position is anchor + offset
  float ox, oy, oz;   // FP32 offset moved since the anchor (inside the safety ball)
  float3 k;
  float x;     // gas-frame frequency at p (in gas)
  float X;     // lab frequency (in the cavity, and at escape)
  float safe;  // lower bound on the distance from p to any shell boundary (0 = unknown)
  int region;  // 1 = inside the empty cavity
  uint32_t nscat, ndust, iters, steps;
  float X0;              // emitted lab frequency
  float col_hi, col_lo;  // HI column traversed (power-law shells), two-level FP32 sum
  Rng rng;
  int model;
  unsigned long long pid;
};

__device__ __forceinline__ int find_entry(const WorkQueue& q, unsigned long long g) {
  int lo = 0, hi = q.n_entries - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (q.prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Emission (Sec. 3.4): central point source, isotropic, line profile in the source frame;
// with a continuum (Sec. 5.1) word 4 picks the line (probability p_line) or the flat
// continuum, whose position is word 5.
__device__ __forceinline__ void shell_emit(const ShellModel& m, Photon& ph) {
  ph.rng.init(((uint64_t)m.seed_hi << 32) | m.seed_lo, ph.pid, m.cont_C > 0.0f ? 2u : 1u);
  ph.px = 0.0; ph.py = 0.0; ph.pz = 0.0;
  ph.ox = 0.0f; ph.oy = 0.0f; ph.oz = 0.0f;
  ph.k = iso_dir(ph.rng.u(0), ph.rng.u(1));
  float X = m.X0;
  if (m.cont_C > 0.0f && ph.rng.u(4) > m.p_line) {
    X = __fmaf_rn(m.cont_C, __fmaf_rn(2.0f, ph.rng.u(5), -1.0f), X);
  } else if (m.line == 1) {
    const float R1 = ph.rng.u(2), R2 = ph.rng.u(3);
    X = __fmaf_rn(m.sigma * sqrtf(-2.0f * __logf(R1)), cospif(2.0f * R2), X);
  }
  ph.X = X;
  ph.X0 = X;
  ph.col_hi = 0.0f; ph.col_lo = 0.0f;
  ph.x = X * m.inv_vth;  // gas at rest at the centre
  ph.region = (m.R_in > 0.0) ? 1 : 0;
  ph.safe = (float)m.R_out;
  ph.nscat = 0; ph.ndust = 0; ph.iters = 0; ph.steps = 0;
}

// Move by s along k inside the safety ball: FP32 offset only.  The moves since the last
// anchor sum to at most the safety distance (< R_out - R_in), and the offset of a packet
// trapped in the core stays tiny, so FP32 keeps it far below the step size.
__device__ __forceinline__ void advance(Photon& ph, float s) {
  ph.ox = __fmaf_rn(s, ph.k.x, ph.ox);
  ph.oy = __fmaf_rn(s, ph.k.y, ph.oy);
  ph.oz = __fmaf_rn(s, ph.k.z, ph.oz);
}
// Fold the offset into the FP64 anchor (before any use of the absolute position).
__device__ __forceinline__ void anchor(Photon& ph) {
  ph.px += (double)ph.ox; ph.py += (double)ph.oy; ph.pz += (double)ph.oz;
  ph.ox = 0.0f; ph.oy = 0.0f; ph.oz = 0.0f;
}

// Exact distance from p to the nearest boundary, rounded down (conservative).
__device__ __forceinline__ float safe_distance(const ShellModel& m, const Photon& ph) {
  const double r = sqrt(ph.px * ph.px + ph.py * ph.py + ph.pz * ph.pz);
  double d = m.R_out - r;
  if (m.R_in > 0.0) d = fmin(d, r - m.R_in);
  return fmaxf(__double2float_rd(d) * 0.999999f, 0.0f);
}

// The start of a step, shared by shell_event's fast paths and the core bursts (one
// definition, so both evaluate an event bit for bit alike): H(a, x) from the table-free
// polynomial in the core (|x| <= 2), else from the table; kH = kap0 H; the crossing at the
// start-point rate s = tau / (kH + kapd); dust is chosen when R (kH + kapd) >= kH (the
// channel of Sec. 3.4, probability kapd / (kH + kapd)).
struct StartStep { float kH, s; };
__device__ __forceinline__ float voigt_start(float a, float x, const float* __restrict__ Ktab) {
  return (fabsf(x) <= THOR_VCORE_X) ? voigt_core_poly(a, x) : voigt<false>(a, x, Ktab);
}
__device__ __forceinline__ StartStep start_step(const ShellModel& m, float H, float tau) {
  const float kH = __fmul_rn(m.kap0, H);
  return StartStep{kH, __fmul_rn(tau, rcp_approx(__fadd_rn(kH, m.kapd)))};
}
// The optical depth to the next interaction, tau = -ln R (Eq. 3), shared likewise.
__device__ __forceinline__ float draw_tau(const Rng& r) { return -ln_fast(r.u(W_TAU)); }
__device__ __forceinline__ bool dust_channel(const ShellModel& m, float kH, float R) {
  return __fmul_rn(R, __fadd_rn(kH, m.kapd)) >= kH;
}

// One event.  Returns 0 = continues, 1 = escaped, 2 = absorbed by dust, 3 = capped.
// The gas-frame frequency x is carried along the ray: in the homologous flow it drifts
// as x(s) = x0 - gam s in every direction, and a scattering leaves it at x_out at the
// same point.  A conservative safety distance to the shell boundaries lets events whose
// interaction lies inside the safety ball skip the FP64 ray-sphere geometry (the common
// case for photons trapped in the line core).
__device__ __forceinline__ uint32_t shell_blocks(const ShellModel& m) {
  return (m.kapd > 0.0f || m.phase == PH_MIXED) ? 3u : 2u;
}

// The event whose words ph.rng holds, with the optical depth tau_rem drawn from them.
__device__ int shell_event_words(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab, float tau_rem) {
  float x_site, kH;
  for (;;) {
    if (ph.region) {  // empty cavity: straight to the inner sphere, lab X conserved
      anchor(ph);
      const double kx = ph.k.x, ky = ph.k.y, kz = ph.k.z;
      const double b = ph.px * kx + ph.py * ky + ph.pz * kz;
      const double c = ph.px * ph.px + ph.py * ph.py + ph.pz * ph.pz - m.R_in * m.R_in;
      const double s = -b + sqrt(fmax(b * b - c, 0.0));
      ph.px += s * kx; ph.py += s * ky; ph.pz += s * kz;
      ph.region = 0;
      ph.x = (ph.X - m.vgrad * (float)(b + s)) * m.inv_vth;
      ph.safe = 0.0f;
    }
    // ---- fast path: the next (sub-)step lies inside the safety ball
    if (m.gam == 0.0f) {
      const StartStep st0 = start_step(m, voigt_start(m.a, ph.x, Ktab), tau_rem);
      kH = st0.kH;
      const float s = st0.s;
      ++ph.steps;
      if (s <= ph.safe) {
        advance(ph, s);
        ph.safe = __fmaf_rd(-s, 1.000001f, ph.safe);
        x_site = ph.x;
        break;
      }
    } else if (ph.safe >= m.ds_core) {
      // Rate at the start of the step: a crossing within ds_core / 16 of the start is a
      // sub-step of its own, integrated with that rate (the common case in the core).
      const StartStep st0 = start_step(m, voigt_start(m.a, ph.x, Ktab), tau_rem);
      const float s0 = st0.s;
      if (s0 <= 0.0625f * m.ds_core) {
        ++ph.steps;
        advance(ph, s0);
        ph.safe = __fmaf_rd(-s0, 1.000001f, ph.safe);
        x_site = __fmaf_rn(-m.gam, s0, ph.x);
        kH = st0.kH;
        break;
      }
      const float ds = m.ds_core;
      const float xm = ph.x - m.gam * 0.5f * ds;
      const float kap = __fmaf_rn(m.kap0, voigt<false>(m.a, xm, Ktab), m.kapd);
      const float dtau = kap * ds;
      ++ph.steps;
      if (dtau >= tau_rem) {
        const float s = __fdividef(tau_rem, kap);
        advance(ph, s);
        ph.safe = __fmaf_rd(-s, 1.000001f, ph.safe);
        x_site = ph.x - m.gam * s;
        kH = m.kap0 * voigt<false>(m.a, x_site, Ktab);
        break;
      }
      tau_rem -= dtau;
      advance(ph, ds);
      ph.safe = __fmaf_rd(-ds, 1.000001f, ph.safe);
      ph.x -= m.gam * ds;
      continue;
    }
    // ---- general path: exact segment to the next boundary (FP64), then sub-steps
    anchor(ph);
    const double kx = ph.k.x, ky = ph.k.y, kz = ph.k.z;
    const double b = ph.px * kx + ph.py * ky + ph.pz * kz;
    const double pp = ph.px * ph.px + ph.py * ph.py + ph.pz * ph.pz;
    double S = -b + sqrt(fmax(b * b - (pp - m.R_out * m.R_out), 0.0));
    int next = 1;  // 1 escape, 2 cavity
    if (m.R_in > 0.0 && b < 0.0) {
      const double disc = b * b - (pp - m.R_in * m.R_in);
      if (disc > 0.0) {
        const double s_in = -b - sqrt(disc);
        if (s_in < S) { S = s_in; next = 2; }
      }
    }
    S = fmax(S, 0.0);
    const float Sf = (float)S;
    const float x0 = ph.x;
    float s_star = -1.0f;
    if (m.gam == 0.0f) {
      const float kap = kH + m.kapd;
      if (kap * Sf >= tau_rem) s_star = fminf(tau_rem / kap, Sf);
      else tau_rem -= kap * Sf;
    } else {
      float s = 0.0f;
      while (s < Sf) {
        const float s1 = fminf(Sf, s + m.ds_core);
        const float xm = x0 - m.gam * 0.5f * (s + s1);
        const float kap = __fmaf_rn(m.kap0, voigt<false>(m.a, xm, Ktab), m.kapd);
        const float dtau = kap * (s1 - s);
        ++ph.steps;
        if (dtau >= tau_rem) { s_star = fminf(s + tau_rem / kap, Sf); break; }
        tau_rem -= dtau;
        s = s1;
      }
    }
    if (s_star >= 0.0f) {
      const double sd = s_star;
      ph.px += sd * kx; ph.py += sd * ky; ph.pz += sd * kz;
      x_site = x0 - m.gam * s_star;
      if (m.gam != 0.0f) kH = m.kap0 * voigt<false>(m.a, x_site, Ktab);
      ph.safe = safe_distance(m, ph);
      break;
    }
    ph.px += S * kx; ph.py += S * ky; ph.pz += S * kz;
    const float x_end = x0 - m.gam * Sf;
    ph.X = __fmaf_rn(x_end, m.vth, m.vgrad * (float)(b + S));  // lab frequency at the boundary
    if (next == 1) return 1;
    ph.region = 1;
  }
  ph.x = x_site;
  // Interaction (Sec. 3.4): channel i with probability tau_i / sum_i tau_i.
  bool dust = false;
  if (m.kapd > 0.0f) dust = dust_channel(m, kH, ph.rng.u(W_CHANNEL));
  if (dust) {
    bool scat;
    if (m.albedo <= 0.0f) scat = false;
    else if (m.albedo >= 1.0f) scat = true;
    else scat = ph.rng.u(W_ALBEDO) < m.albedo;
    if (!scat) return 2;
    scatter_dust(m.g_hg, ph.k, ph.rng);  // gas-frame frequency unchanged
    ++ph.ndust;
    return 0;
  }
  // Eq. 7: the gas-frame frequency after the scattering, at the same point
  ph.x = scatter_resonant(x_site, m.a, m.phase, ph.k, ph.rng, ph.iters, nullptr, m.xcrit);
  ++ph.nscat;
  if (m.max_scat && ph.nscat >= m.max_scat) {
    anchor(ph);
    const float b = (float)(ph.px * ph.k.x + ph.py * ph.k.y + ph.pz * ph.k.z);
    ph.X = __fmaf_rn(ph.x, m.vth, m.vgrad * b);
    return 3;
  }
  return 0;
}

__device__ int shell_event(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab) {
  ph.rng.next_event(shell_blocks(m));
  return shell_event_words(m, ph, Ktab, draw_tau(ph.rng));  // Eq. 3: tau ~ Exp(1)
}

// ---- pipelined events (homologous shells) -------------------------------------------
// A packet trapped in the line core spends its life in one kind of event: the crossing lies
// within ds/16 of the start (start-point rate, Sec. 5.1 step limiter) inside the safety
// ball, the interaction is a resonant scattering at |x| <= 2 (Sec. 3.4), and the u_par
// sampler (Eq. 10) accepts within two trials.  In such an event only the frequency
// chain x -> H(a,x) -> s -> x_site -> u_par -> x_out depends on the packet's state; the next
// event's Philox blocks and optical depth, the perpendicular atom velocity (Eq. 5), mu and
// the outgoing direction depend only on random words and the incoming direction.
// shell_event_pipe evaluates that kind of event in one basic block, with the next event's
// words formed beside the chain (a lone lane issues in order and would otherwise wait on
// each link), and commits it only if the event is of that kind; otherwise it runs the
// general event from the same words.  The general event evaluates these events with the
// same helpers (voigt_start, start_step, dust_channel, u0_core, upar_q / atan_small,
// region1, x_after_scatter), so both paths give bit-identical results.
// In this mode ph.rng holds the words of the event about to run ("prepared"), and
// tau_next its optical depth; pipe_prepare / pipe_unprepare switch between the modes.
__device__ __forceinline__ void pipe_prepare(const ShellModel& m, Photon& ph, float& tau_next) {
  ph.rng.next_event(shell_blocks(m));
  tau_next = draw_tau(ph.rng);
}
__device__ __forceinline__ void pipe_unprepare(Photon& ph) { ph.rng.event -= 1u; }

// The line-core form of the prepared event.  Always forms the next event's words and
// optical depth (r2, tau2).  Returns 0 if the event is not of the core kind (the packet is
// unchanged), 1 if it was committed, 3 if committed and the scattering cap was reached (the
// packet is then finished as shell_event_words finishes it).  On commit the packet is
// prepared for the next event.
__device__ __forceinline__ int core_event_with(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab,
                                               float& tau_next, const Rng& r2, float tau2);
__device__ __forceinline__ int core_event(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab,
                                          float& tau_next, Rng& r2, float& tau2) {
  r2 = ph.rng;
  r2.next_event(shell_blocks(m));
  tau2 = draw_tau(r2);
  return core_event_with(m, ph, Ktab, tau_next, r2, tau2);
}
// The core form of the prepared event, evaluated (nothing committed): the frequency chain,
// the u_par sampler's first trial (and its second, when the first is rejected) and, beside
// them, the perpendicular velocity, mu and the outgoing direction.  ok: the event is of the
// core kind.
struct CoreEval {
  float s0, xs, upar, mu, st, u1, u2, cp, sp;
  float3 ko;
  uint32_t trials;  // u_par trials (one or two)
  bool ok;
};
// live = false: a lane of a cooperative burst without a packet in it; it evaluates at line
// centre and skips the rare second trial, so that it takes the owners' branches.
__device__ __forceinline__ CoreEval core_eval(const ShellModel& m, const Photon& ph, const float* __restrict__ Ktab,
                                              float tau, bool live = true) {
  const Rng& r = ph.rng;
  CoreEval e;
  // ---- the frequency chain: rate at the start, crossing, gas-frame frequency at the site
  const float x0 = live ? ph.x : 0.0f;
  const StartStep st0 = start_step(m, voigt_start(m.a, x0, Ktab), tau);
  const float s0 = st0.s;
  const bool in_ball = (m.gam == 0.0f) ? (s0 <= ph.safe) : (ph.safe >= m.ds_core && s0 <= 0.0625f * m.ds_core);
  const float xs = (m.gam == 0.0f) ? x0 : __fmaf_rn(-m.gam, s0, x0);
  const bool dust = (m.kapd > 0.0f) && dust_channel(m, st0.kH, r.u(W_CHANNEL));
  // ---- u_par, first trial of the two-piece comparison function (as sample_upar)
  const float sgn = (xs < 0.0f) ? -1.0f : 1.0f;
  const float xr = fabsf(xs);
  const float u0 = u0_core(xr, m.a);
  const float q = upar_q(xr, m.a);
  // w1 = atan2(a, x - u0) as sample_upar forms it: the q form where u0 > 0, else (u0 = 0,
  // within ~0.04 of line centre) the series in a / x
  const bool split = u0 > 0.0f;
  const float w1 = split ? atan_small(q) : atan2_series(m.a, xr);
  const float u02 = __fmul_rn(u0, u0);
  const float mass = envelope_mass(w1, exp_fast(-u02));
  const float w1p = __fmul_rn(w1, 1.0f / kPiF);
  float u;
  bool accepted = upar_trial(xr, m.a, w1, w1p, mass, u02, r.u(W_UPAR0), r.u(W_UPAR0 + 1), r.u(W_UPAR0 + 2), u);
  e.trials = 1u;
  if (!accepted && live) {  // rare: the second trial, from block 3 of the event as sample_upar takes it
    uint32_t b0, b1, b2, b3;
    r.block(3u, b0, b1, b2, b3);
    accepted = upar_trial(xr, m.a, w1, w1p, mass, u02, uni32(b0), uni32(b1), uni32(b2), u);
    e.trials = 2u;
  }
  // ---- beside the chain: perpendicular velocity, mu, outgoing direction (as scatter_resonant)
  const float xc = (xr < m.xcrit) ? m.xcrit : 0.0f;
  const float rr = sqrt_approx(__fmaf_rn(xc, xc, -__logf(r.u(W_BM_R))));
  float sp1, cp1;
  __sincosf(2.0f * kPiF * r.u(W_BM_PHI), &sp1, &cp1);
  e.u1 = __fmul_rn(rr, cp1);
  e.u2 = __fmul_rn(rr, sp1);
  const float Rm = r.u(W_MU);
  e.mu = (m.phase == PH_ISO) ? __fmaf_rn(2.0f, Rm, -1.0f) : mu_dipole(Rm);
  __sincosf(2.0f * kPiF * r.u(W_PHI), &e.sp, &e.cp);
  float3 e1, e2;
  basis(ph.k.x, ph.k.y, ph.k.z, e1, e2);
  e.st = sqrt_approx(fmaxf(0.0f, __fmaf_rn(-e.mu, e.mu, 1.0f)));
  e.ko = turn(ph.k, e1, e2, e.mu, e.st, e.cp, e.sp);
  e.s0 = s0;
  e.xs = xs;
  e.upar = sgn * u;
  e.ok = !ph.region && m.phase != PH_MIXED && in_ball && !dust && xr <= 2.0f &&
         (split ? q <= 0.05f : m.a <= 0.05f * xr) && accepted;
  return e;
}
// Commit an evaluated core event where `ok` (selects, no branch), as shell_event_words and
// scatter_resonant do: the packet is then prepared with the next event's words r2 and
// optical depth tau2.
__device__ __forceinline__ void core_commit(Photon& ph, const CoreEval& e, bool ok, const Rng& r2, float tau2,
                                            float& tau_next) {
  ph.steps += ok ? 1u : 0u;
  ph.ox = ok ? __fmaf_rn(e.s0, ph.k.x, ph.ox) : ph.ox;  // advance(ph, s0)
  ph.oy = ok ? __fmaf_rn(e.s0, ph.k.y, ph.oy) : ph.oy;
  ph.oz = ok ? __fmaf_rn(e.s0, ph.k.z, ph.oz) : ph.oz;
  ph.safe = ok ? __fmaf_rd(-e.s0, 1.000001f, ph.safe) : ph.safe;
  ph.x = ok ? x_after_scatter(e.xs, e.upar, e.mu, e.st, e.u1, e.u2, e.cp, e.sp) : ph.x;
  ph.k.x = ok ? e.ko.x : ph.k.x;
  ph.k.y = ok ? e.ko.y : ph.k.y;
  ph.k.z = ok ? e.ko.z : ph.k.z;
  ph.iters += ok ? e.trials : 0u;
  ph.nscat += ok ? 1u : 0u;
  ph.rng.event = ok ? r2.event : ph.rng.event;
#pragma unroll
  for (int j = 0; j < 12; ++j) ph.rng.v[j] = ok ? r2.v[j] : ph.rng.v[j];
  tau_next = ok ? tau2 : tau_next;
}
// The same event with the next event's words (r2) and optical depth (tau2) given.
__device__ __forceinline__ int core_event_with(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab,
                                               float& tau_next, const Rng& r2, float tau2) {
  const CoreEval e = core_eval(m, ph, Ktab, tau_next);
  if (!e.ok) return 0;
  core_commit(ph, e, true, r2, tau2, tau_next);
  if (m.max_scat && ph.nscat >= m.max_scat) {
    anchor(ph);
    const float b = (float)(ph.px * ph.k.x + ph.py * ph.k.y + ph.pz * ph.k.z);
    ph.X = __fmaf_rn(ph.x, m.vth, m.vgrad * b);
    return 3;
  }
  return 1;
}

// One prepared event: its core form if it is of that kind, else the general event from the
// same words; the packet is then prepared for the next event.  Returns as shell_event.
__device__ __forceinline__ int shell_event_pipe(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab,
                                                float& tau_next) {
  Rng r2;
  float tau2;
  const int c = core_event(m, ph, Ktab, tau_next, r2, tau2);
  if (c == 1) return 0;
  if (c == 3) return 3;
  const int status = shell_event_words(m, ph, Ktab, tau_next);
  ph.rng = r2;
  tau_next = tau2;
  return status;
}

// A burst: core events of a prepared packet back to back, in one loop whose body is one
// basic block (no vote or exchange between events), until an event is not of the core kind
// (it is left prepared, for shell_event_pipe) or kCoreBurst events are done.  For warps with
// few live packets, where a lone lane's latency is what counts.  Returns 3 if the cap was
// reached, else 0.
constexpr uint32_t kCoreBurst = 32;
__device__ __forceinline__ int core_burst(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab,
                                          float& tau_next) {
  for (uint32_t n = 0; n < kCoreBurst; ++n) {
    Rng r2;
    float tau2;
    const int c = core_event(m, ph, Ktab, tau_next, r2, tau2);
    if (c != 1) return c;  // 0: not a core event (still prepared); 3: capped
  }
  return 0;
}

// A cooperative burst, for warps with at most kCoopOwners packets in bursts.  Called by all
// 32 lanes, converged; `mine` marks the lanes whose (prepared) packets burst.  In a core
// event the next event's three Philox blocks are about half a lone lane's instructions, and
// they depend on nothing but the key, the photon id and the event number.  So every lane
// computes one block ahead -- for owner o, event d ahead, block b: D = 32 / (3 owners)
// events deep -- and the owners take their words by shuffle, D events per round of blocks.
// The words are the ones Rng::start_event forms, so the packets' histories are those of
// core_burst, bit for bit.  Returns 0: a packet leaves the burst prepared, before its first
// event that is not of the core kind, or one scattering short of the cap.
constexpr int kCoopOwners = 10;
__device__ __forceinline__ int core_burst_coop(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab,
                                               float& tau_next, bool mine) {
  const int lane = (int)(threadIdx.x & 31u);
  const unsigned owners = __ballot_sync(kFull, mine);
  const int n_own = __popc(owners);
  if (n_own == 0) return 0;
  if (n_own > kCoopOwners) return mine ? core_burst(m, ph, Ktab, tau_next) : 0;
  const int D = 32 / (3 * n_own);  // >= 1
  const int span = 3 * D;
  // as a block computer: owner rank oi (its lane src), event offset d, block b
  const int oi = lane / span, rem = lane - oi * span;
  const int d = rem / 3, b = rem - 3 * d;
  unsigned o = owners;
#pragma unroll
  for (int k = 0; k < kCoopOwners - 1; ++k)
    if (k < oi) o &= o - 1u;
  const int src = o ? __ffs(o) - 1 : 0;  // lanes past the owners' spans compute a spare block
  // as an owner: the first lane of its span
  const int base = mine ? __popc(owners & ((1u << lane) - 1u)) * span : 0;
  const bool b3 = shell_blocks(m) > 2u;  // else words 8..11 stay as start_event leaves them
  // a burst stops one scattering short of the cap: the event that reaches it runs as
  // shell_event_pipe (which finishes the packet)
  const uint32_t room = m.max_scat ? (m.max_scat > ph.nscat + 1u ? m.max_scat - ph.nscat - 1u : 0u) : kCoreBurst;
  bool go = mine && room > 0u;
  for (uint32_t n = 0; n < kCoreBurst; n += (uint32_t)D) {
    // a round of blocks: events e+1 .. e+D of each owner (e = its prepared event now)
    const uint32_t k0 = __shfl_sync(kFull, ph.rng.k0, src), k1 = __shfl_sync(kFull, ph.rng.k1, src);
    uint32_t h0 = __shfl_sync(kFull, ph.rng.p0, src), h1 = __shfl_sync(kFull, ph.rng.p1, src);
    uint32_t h2 = __shfl_sync(kFull, ph.rng.event, src) + 1u + (uint32_t)d, h3 = (uint32_t)b;
    philox10(h0, h1, h2, h3, k0, k1);
    for (int i = 0; i < D && n + (uint32_t)i < kCoreBurst; ++i) {
      const int s0 = base + 3 * i;
      Rng r2 = ph.rng;
      r2.event = ph.rng.event + 1u;
      r2.v[0] = __shfl_sync(kFull, h0, s0); r2.v[1] = __shfl_sync(kFull, h1, s0);
      r2.v[2] = __shfl_sync(kFull, h2, s0); r2.v[3] = __shfl_sync(kFull, h3, s0);
      r2.v[4] = __shfl_sync(kFull, h0, s0 + 1); r2.v[5] = __shfl_sync(kFull, h1, s0 + 1);
      r2.v[6] = __shfl_sync(kFull, h2, s0 + 1); r2.v[7] = __shfl_sync(kFull, h3, s0 + 1);
      const uint32_t w8 = __shfl_sync(kFull, h0, s0 + 2), w9 = __shfl_sync(kFull, h1, s0 + 2);
      const uint32_t w10 = __shfl_sync(kFull, h2, s0 + 2), w11 = __shfl_sync(kFull, h3, s0 + 2);
      if (b3) { r2.v[8] = w8; r2.v[9] = w9; r2.v[10] = w10; r2.v[11] = w11; }
      // every lane evaluates (the owners' events; garbage elsewhere, never committed) and
      // commits by select: the loop body is one basic block
      const CoreEval e = core_eval(m, ph, Ktab, tau_next, go);
      go = go && e.ok && n + (uint32_t)i < room;
      core_commit(ph, e, go, r2, draw_tau(r2), tau_next);
      if (!__any_sync(kFull, go)) return 0;
    }
  }
  return 0;
}

// ---- power-law shells (Sec. 5.1) ---------------------------------------------------
// Gas state at a point q (FP32, |q| <= 1) for direction k: radius, r_hat . k, density
// relative to r = 1 and outflow speed.
struct PLState { float r, mur, nr, v; };
__device__ __forceinline__ PLState pl_state(const ShellModel& m, float qx, float qy, float qz, float3 k) {
  const float r2 = __fmaf_rn(qx, qx, __fmaf_rn(qy, qy, qz * qz));
  const float ir = rsqrtf(r2);
  PLState st;
  st.r = r2 * ir;
  st.mur = __fmaf_rn(qx, k.x, __fmaf_rn(qy, k.y, qz * k.z)) * ir;
  const float lr = __log2f(st.r);
  st.nr = ex2_approx(m.ar * lr);
  st.v = m.v1 * ex2_approx(m.av * lr);
  return st;
}
__device__ __forceinline__ void col_add(Photon& ph, float d) {
  ph.col_lo += d;
  if (ph.col_lo >= 0.00390625f) { ph.col_hi += ph.col_lo; ph.col_lo = 0.0f; }
}

// One event on a power-law shell; returns as shell_event.  The lab frequency X is the
// photon's frequency variable (the flow is not homologous, so x is evaluated from the
// local state).  A crossing predicted from the rate at the current point within
// min(safety distance, ds / 16) is taken with that rate (one Voigt evaluation, no FP64);
// otherwise sub-steps of at most ds (the global step limiter) use the midpoint state.
// Dust follows the gas and absorbs.
// Second transition of a doublet (Mg II H): its own offset X_2 = X + eps2 (c + X) on the
// scale of the first, and back.
constexpr float kCkms = 299792.458f;
__device__ __forceinline__ float to_line2(const ShellModel& m, float X) { return __fmaf_rn(m.eps2, kCkms + X, X); }
__device__ __forceinline__ float from_line2(const ShellModel& m, float X2) {
  return __fmaf_rn(-__fdividef(m.eps2, 1.0f + m.eps2), kCkms + X2, X2);
}

__device__ int shell_event_pl(const ShellModel& m, Photon& ph, const float* __restrict__ Ktab) {
  ph.rng.next_event((m.kapdn > 0.0f || m.phase == PH_MIXED || m.n_lines == 2) ? 3u : 2u);
  float tau_rem = -__logf(ph.rng.u(W_TAU));  // Eq. 3
  float kH, kH2 = 0.0f, kD;
  PLState site;
  for (;;) {
    if (ph.region) {  // empty cavity: straight to the inner sphere, lab X conserved
      anchor(ph);
      const double kx = ph.k.x, ky = ph.k.y, kz = ph.k.z;
      const double b = ph.px * kx + ph.py * ky + ph.pz * kz;
      const double c = ph.px * ph.px + ph.py * ph.py + ph.pz * ph.pz - m.R_in * m.R_in;
      const double s = -b + sqrt(fmax(b * b - c, 0.0));
      ph.px += s * kx; ph.py += s * ky; ph.pz += s * kz;
      ph.region = 0;
      ph.safe = 0.0f;
    }
    {  // short step with the rate at the current point
      const PLState st = pl_state(m, (float)ph.px + ph.ox, (float)ph.py + ph.oy, (float)ph.pz + ph.oz, ph.k);
      const float x = (ph.X - st.v * st.mur) * m.inv_vth;
      const float H = voigt<false>(m.a, x, Ktab);
      const float H2 = (m.n_lines == 2) ? voigt<false>(m.a2, (to_line2(m, ph.X) - st.v * st.mur) * m.inv_vth, Ktab)
                                         : 0.0f;
      const float kap = st.nr * __fmaf_rn(m.kapn, H, __fmaf_rn(m.kapn2, H2, m.kapdn));
      const float s0 = __fdividef(tau_rem, kap);
      ++ph.steps;
      if (s0 <= ph.safe && s0 <= 0.0625f * m.ds_core) {
        advance(ph, s0);
        ph.safe = __fmaf_rd(-s0, 1.000001f, ph.safe);
        col_add(ph, st.nr * m.invF * s0);
        kH = m.kapn * st.nr * H;
        kH2 = m.kapn2 * st.nr * H2;
        kD = m.kapdn * st.nr;
        site = pl_state(m, (float)ph.px + ph.ox, (float)ph.py + ph.oy, (float)ph.pz + ph.oz, ph.k);
        break;
      }
    }
    // general path: exact segment to the next boundary (FP64), sub-steps of <= ds
    anchor(ph);
    const double kx = ph.k.x, ky = ph.k.y, kz = ph.k.z;
    const double b = ph.px * kx + ph.py * ky + ph.pz * kz;
    const double pp = ph.px * ph.px + ph.py * ph.py + ph.pz * ph.pz;
    double S = -b + sqrt(fmax(b * b - (pp - m.R_out * m.R_out), 0.0));
    int next = 1;  // 1 escape, 2 cavity
    if (b < 0.0) {
      const double disc = b * b - (pp - m.R_in * m.R_in);
      if (disc > 0.0) {
        const double s_in = -b - sqrt(disc);
        if (s_in < S) { S = s_in; next = 2; }
      }
    }
    S = fmax(S, 0.0);
    const float Sf = (float)S;
    const float p0x = (float)ph.px, p0y = (float)ph.py, p0z = (float)ph.pz;
    float s = 0.0f, s_star = -1.0f;
    while (s < Sf) {
      const float s1 = fminf(Sf, s + m.ds_core);
      const float sm = 0.5f * (s + s1);
      const PLState st = pl_state(m, __fmaf_rn(sm, ph.k.x, p0x), __fmaf_rn(sm, ph.k.y, p0y),
                                  __fmaf_rn(sm, ph.k.z, p0z), ph.k);
      const float x = (ph.X - st.v * st.mur) * m.inv_vth;
      const float H = voigt<false>(m.a, x, Ktab);
      const float H2 = (m.n_lines == 2) ? voigt<false>(m.a2, (to_line2(m, ph.X) - st.v * st.mur) * m.inv_vth, Ktab)
                                         : 0.0f;
      const float kap = st.nr * __fmaf_rn(m.kapn, H, __fmaf_rn(m.kapn2, H2, m.kapdn));
      const float dtau = kap * (s1 - s);
      ++ph.steps;
      if (dtau >= tau_rem) {
        s_star = fminf(s + __fdividef(tau_rem, kap), Sf);
        col_add(ph, st.nr * m.invF * (s_star - s));
        kH = m.kapn * st.nr * H;
        kH2 = m.kapn2 * st.nr * H2;
        kD = m.kapdn * st.nr;
        break;
      }
      col_add(ph, st.nr * m.invF * (s1 - s));
      tau_rem -= dtau;
      s = s1;
    }
    if (s_star >= 0.0f) {
      const double sd = s_star;
      ph.px += sd * kx; ph.py += sd * ky; ph.pz += sd * kz;
      ph.safe = safe_distance(m, ph);
      site = pl_state(m, (float)ph.px, (float)ph.py, (float)ph.pz, ph.k);
      break;
    }
    ph.px += S * kx; ph.py += S * ky; ph.pz += S * kz;
    if (next == 1) return 1;  // escapes with its lab X
    ph.region = 1;
  }
  // Interaction (Sec. 3.4): transition 1, transition 2 or dust in proportion to their
  // opacities (one uniform); dust absorbs.
  int ch = 0;
  if (kD > 0.0f || m.n_lines == 2) {
    const float u = ph.rng.u(W_CHANNEL), kt = kH + kH2 + kD;
    ch = (u < __fdividef(kH, kt)) ? 0 : ((u < __fdividef(kH + kH2, kt)) ? 1 : 2);
  }
  if (ch == 2) return 2;
  const float qx = (float)ph.px + ph.ox, qy = (float)ph.py + ph.oy, qz = (float)ph.pz + ph.oz;
  float xo;
  if (ch == 0) {
    xo = scatter_resonant((ph.X - site.v * site.mur) * m.inv_vth, m.a, m.phase, ph.k, ph.rng, ph.iters, nullptr,
                          m.xcrit);
  } else {  // second transition: J = 1/2 upper level, isotropic
    xo = scatter_resonant((to_line2(m, ph.X) - site.v * site.mur) * m.inv_vth, m.a2, PH_ISO, ph.k, ph.rng,
                          ph.iters, nullptr, 0.0f);
  }
  // back to the lab frame with the new direction: X = x v_th + v(r) r_hat . k_out
  const float mur = __fmaf_rn(qx, ph.k.x, __fmaf_rn(qy, ph.k.y, qz * ph.k.z)) / site.r;
  const float Xl = __fmaf_rn(xo, m.vth, site.v * mur);
  ph.X = (ch == 0) ? Xl : from_line2(m, Xl);
  ++ph.nscat;
  if (m.max_scat && ph.nscat >= m.max_scat) return 3;
  return 0;
}

__device__ __forceinline__ void tally_spectrum(const ShellModel& m, float X) {
  int bin;
  const float f = (X - m.X_min) * m.inv_dX;
  if (!(f >= 0.0f)) bin = m.n_bins;
  else if (f >= (float)m.n_bins) bin = m.n_bins + 1;
  else bin = (int)f;
  atomicAdd(&m.spectrum[bin], 1ull);
}

__device__ __forceinline__ void write_raw(const ShellModel& m, const Photon& ph, int status) {
  const unsigned long long j = ph.pid - m.id_base;
  if (m.raw_X) {
    m.raw_X[j] = ph.X;
    m.raw_nscat[j] = ph.nscat;
    m.raw_status[j] = (uint8_t)status;
  }
  if (m.raw_X0) m.raw_X0[j] = ph.X0;
  if (m.raw_col) m.raw_col[j] = ph.col_hi + ph.col_lo;
}

// Per-photon tally with global atomics (used where lanes may belong to different models).
__device__ __forceinline__ void finish_global(const ShellModel& m, const Photon& ph, int status) {
  Tally* T = m.tally;
  if (status == 1) { atomicAdd(&T->n_escaped, 1ull); tally_spectrum(m, ph.X); }
  else if (status == 2) atomicAdd(&T->n_absorbed, 1ull);
  else atomicAdd(&T->n_capped, 1ull);
  atomicAdd(&T->n_scat, (unsigned long long)ph.nscat);
  atomicAdd(&T->n_dust_scat, (unsigned long long)ph.ndust);
  atomicAdd(&T->n_upar_iters, (unsigned long long)ph.iters);
  atomicAdd(&T->n_steps, (unsigned long long)ph.steps);
  atomicAdd(&T->sum_scat2, (double)ph.nscat * (double)ph.nscat);
  atomicAdd(&T->n_done, 1ull);
  write_raw(m, ph, status);
}

struct LaneTally {
  unsigned long long esc = 0, abs = 0, cap = 0, scat = 0, dust = 0, iters = 0, steps = 0, done = 0;
  double scat2 = 0.0;
};

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ void save_rec(const Photon& ph, PhotonRec& r) {
  r.px = ph.px; r.py = ph.py; r.pz = ph.pz;
  r.ox = ph.ox; r.oy = ph.oy; r.oz = ph.oz;
  r.X0 = ph.X0; r.col_hi = ph.col_hi; r.col_lo = ph.col_lo;
  r.kx = ph.k.x; r.ky = ph.k.y; r.kz = ph.k.z;
  r.x = ph.x; r.X = ph.X; r.safe = ph.safe;
  r.region = ph.region;
  r.nscat = ph.nscat; r.ndust = ph.ndust; r.iters = ph.iters; r.steps = ph.steps;
  r.event = ph.rng.event;
  r.pid = ph.pid;
}

__device__ __forceinline__ void load_rec(const ShellModel& m, const PhotonRec& r, Photon& ph) {
  ph.px = r.px; ph.py = r.py; ph.pz = r.pz;
  ph.ox = r.ox; ph.oy = r.oy; ph.oz = r.oz;
  ph.X0 = r.X0; ph.col_hi = r.col_hi; ph.col_lo = r.col_lo;
  ph.k = make_float3(r.kx, r.ky, r.kz);
  ph.x = r.x; ph.X = r.X; ph.safe = r.safe;
  ph.region = r.region;
  ph.nscat = r.nscat; ph.ndust = r.ndust; ph.iters = r.iters; ph.steps = r.steps;
  ph.pid = r.pid;
  ph.rng.keys(((uint64_t)m.seed_hi << 32) | m.seed_lo, ph.pid);
  ph.rng.event = r.event;
}

// ---- work sharing in the tail of a one-launch run (pool_take in thor_device.cuh) ----------
constexpr uint32_t kShareEvents = 512;  // a warp with several live packets checks for waiting warps this often
__device__ __forceinline__ long long share_take(const Compact& c) { return pool_take(c.share, c.ready, c.n_total); }

// Run-to-completion: all queue entries belong to one model (thor_run).  With kCompact,
// lanes first resume saved packets, and a warp whose sources are empty and whose live
// lanes drop below c.spill_below saves them and exits (tail compaction across launches).
template <bool kCompact, int kProfile>
__global__ void __launch_bounds__(256, 1) shell_run_kernel(const ShellModel* __restrict__ models, WorkQueue q,
                                                        Compact c, const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  __shared__ ShellModel sm;
  load_ktab(sK, gK);
  if (threadIdx.x == 0) sm = models[q.model[0]];
  __syncthreads();
  const ShellModel m = sm;  // by value: the fields the event loop reads stay in registers
  const unsigned lane = threadIdx.x & 31u;
  Photon ph;
  bool active = false, done = (int)lane >= c.per_warp;  // lanes above per_warp stay idle
  bool drained = false;  // warp-uniform: a refill found the photon queue exhausted
  bool prepared = false;  // ph.rng holds the words of the next event (pipelined mode)
  float tau_next = 0.0f;
  LaneTally lt;
  for (;;) {
    unsigned need = __ballot_sync(kFull, !active && !done);
    if (kCompact && need && c.n_resume) {  // saved packets first
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(c.resume_next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (!active && !done) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < c.n_resume) { load_rec(m, c.resume[g], ph); active = true; prepared = false; }
      }
      need = __ballot_sync(kFull, !active && !done);
    }
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(q.next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (base + __popc(need) > q.total) drained = true;
      if (!active && !done) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < q.total) {
          ph.model = q.model[0];
          ph.pid = q.first_id[0] + g;
          shell_emit(m, ph);
          active = true;
          prepared = false;
        } else {
          done = true;
        }
      }
    }
    if (kCompact && c.spill_below > 0) {
      const unsigned live = __ballot_sync(kFull, active);
      if (drained && __popc(live) < c.spill_below) {
        if (live) {
          const int leader = __ffs(live) - 1;
          unsigned long long base = 0;
          if ((int)lane == leader) base = atomicAdd(c.n_spill, (unsigned long long)__popc(live));
          base = __shfl_sync(kFull, base, leader);
          if (active && prepared) pipe_unprepare(ph);
          if (active) save_rec(ph, c.spill[base + __popc(live & ((1u << lane) - 1u))]);
        }
        active = false;
        break;
      }
    }
    if (c.pool && drained) {
      const unsigned live = __ballot_sync(kFull, active);
      if (live == 0u) {  // an empty warp: take a packet that a crowded warp gives away
        long long got = -1;
        if (lane == 0) got = share_take(c);
        got = __shfl_sync(kFull, got, 0);
        if (got < 0) break;
        if (lane == 0) { load_rec(m, c.pool[got], ph); active = true; prepared = false; }
        continue;
      }
      if (__popc(live) >= 2) {  // give packets away while empty warps wait, keeping the lowest lane's
        const int leader = __ffs(live) - 1;
        long long give = 0;
        if ((int)lane == leader) give = pool_give_count(c.share, __popc(live));
        give = __shfl_sync(kFull, give, leader);
        if (give > 0) {
          // the `give` highest live lanes: their rank from the top
          const int from_top = __popc(live & ~((2u << lane) - 1u));
          const bool giver = active && from_top < (int)give;
          unsigned long long base = 0;
          if ((int)lane == leader) base = atomicAdd(&c.share[0], (unsigned long long)give);
          base = __shfl_sync(kFull, base, leader);
          if (giver) {
            const unsigned long long j = base + (unsigned long long)from_top;
            if (prepared) { pipe_unprepare(ph); prepared = false; }
            save_rec(ph, c.pool[j]);
            __threadfence();
            *(volatile uint32_t*)&c.ready[j] = 1u;
            active = false;
          }
        }
      }
    }
    if (__all_sync(kFull, !active)) break;
    // pipelined events in warps with at most core_lanes live packets (homologous shells),
    // and core bursts in warps with at most burst_lanes
    const int n_live = __popc(__ballot_sync(kFull, active));
    const bool check_share = c.pool && drained && n_live >= 2;
    uint32_t n_ev = 0;
    const bool pipe = kProfile == 0 && n_live <= c.core_lanes;
    const bool burst = pipe && n_live <= c.burst_lanes;
    // events until some lane of the warp finishes its packet: one vote per event, the
    // refill and spill checks above run only when the set of live lanes changed
    // (bursts are cooperative up to kCoopOwners live packets: all lanes, converged)
    bool fin;
    do {
      fin = false;
      int st = 0;
      if (burst) {
        if (active && !prepared) { pipe_prepare(m, ph, tau_next); prepared = true; }
        st = core_burst_coop(m, ph, sK, tau_next, active);
      }
      if (active) {
        if (pipe) {
          if (!prepared) { pipe_prepare(m, ph, tau_next); prepared = true; }
          if (!st) st = shell_event_pipe(m, ph, sK, tau_next);
        } else {
          if (prepared) { pipe_unprepare(ph); prepared = false; }
          st = kProfile ? shell_event_pl(m, ph, sK) : shell_event(m, ph, sK);
        }
        if (st) {
          if (st == 1) { ++lt.esc; tally_spectrum(m, ph.X); }
          else if (st == 2) ++lt.abs;
          else ++lt.cap;
          lt.scat += ph.nscat; lt.dust += ph.ndust; lt.iters += ph.iters; lt.steps += ph.steps; ++lt.done;
          lt.scat2 += (double)ph.nscat * (double)ph.nscat;
          write_raw(m, ph, st);
          if (c.pool) atomicAdd(&c.share[3], 1ull);
          active = false;
          fin = true;
        }
      }
    } while (!__any_sync(kFull, fin) && !(check_share && ++n_ev >= kShareEvents));
  }
  // flush lane tallies: warp reduce, one atomic per warp and field
  const unsigned long long e = warp_sum(lt.esc), a = warp_sum(lt.abs), cp = warp_sum(lt.cap),
                           s = warp_sum(lt.scat), d = warp_sum(lt.dust), it = warp_sum(lt.iters),
                           sp = warp_sum(lt.steps), dn = warp_sum(lt.done);
  const double s2 = warp_sum(lt.scat2);
  if (lane == 0 && dn) {
    Tally* T = m.tally;
    atomicAdd(&T->n_escaped, e); atomicAdd(&T->n_absorbed, a); atomicAdd(&T->n_capped, cp);
    atomicAdd(&T->n_scat, s); atomicAdd(&T->n_dust_scat, d); atomicAdd(&T->n_upar_iters, it);
    atomicAdd(&T->n_steps, sp); atomicAdd(&T->n_done, dn); atomicAdd(&T->sum_scat2, s2);
  }
}

// Time-sliced execution (serving): packets in flight live in a list (`in`): in.live[0]
// entries from the front, and in.live[2] priority entries from the back (packets of the
// requests the host marked as priority, the oldest ones).  The first priority packets, up
// to half of the warps, each run alone in a warp of their own (one packet per warp, so
// the longest histories of the oldest requests advance at the latency of a lone lane
// instead of behind divergent packets of other requests).  The remaining entries spread
// over the other warps: lane l of warp w resumes entry w + l * (their count).  Each lane
// runs at most `budget` events, finished lanes take new photons from the queue of admitted
// requests while the warp has fewer live packets than its limit (1 for a priority warp,
// per_warp otherwise), and what is still in flight is appended to `out`: priority packets
// from the back (out.live[3]), the others from the front (out.live[1]).
// kMixed: the round holds power-law models too (the event function is chosen per lane);
// otherwise only homologous shells, compiled without the power-law event.
template <bool kMixed>
__global__ void __launch_bounds__(256, 1) shell_slice_kernel(const ShellModel* __restrict__ models, WorkQueue q,
                                                          SlotState in, SlotState out, uint32_t budget,
                                                          const float* __restrict__ gK) {
  __shared__ __align__(16) float sK[THOR_VOIGT_NINT * THOR_VOIGT_NCOEF];
  load_ktab(sK, gK);
  int per_warp = 32;  // at most this many live packets per warp after a refill
  if (q.hdr) {
    q.total = q.hdr[0]; q.n_entries = (int32_t)q.hdr[1]; budget = (uint32_t)q.hdr[2];
    per_warp = (int)q.hdr[3];
  }
  const unsigned lane = threadIdx.x & 31u;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_in = in.live[0], n_pri = in.live[2];
  // priority warps: [0, n_pw), one priority packet each; the rest of the priority list and
  // the front list spread over warps [n_pw, n_warps), at most 32 per warp.  Every stored
  // packet must find a lane: n_in + n_pri - n_pw <= 32 (n_warps - n_pw), i.e.
  // n_pw <= (32 n_warps - n_in - n_pri) / 31 (none when the list is full), and at most half
  // of the warps.
  const unsigned long long lanes = 32ull * (unsigned long long)n_warps;
  const unsigned long long fit = (lanes > n_in + n_pri) ? (lanes - n_in - n_pri) / 31ull : 0ull;
  const int64_t n_pw = (int64_t)min(min(n_pri, (unsigned long long)(n_warps / 2)), fit);
  const unsigned long long rest = n_in + (n_pri - (unsigned long long)n_pw);
  const int64_t n_rest_warps = n_warps - n_pw;
  const bool pri_warp = warp < n_pw;
  if (pri_warp) per_warp = 1;
  // A priority warp holds one packet and runs at a lone lane's latency, several times the
  // events a crowded warp runs in the same time: past the round's budget it goes on, up to
  // kPriBudget times the budget, while other warps of the round are still running (live[4]
  // counts those that finished), so the round lasts no longer for it.
  const int64_t n_regular = n_warps - n_pw;
  const uint32_t base_budget = budget;
  if (pri_warp) budget *= kPriBudget;
  int64_t slot = -1;
  if (pri_warp) {
    if (lane == 0) slot = in.n_slots - 1 - warp;
  } else {
    // contiguous entries per warp, counts differing by at most one: [w rest / W, (w+1) rest / W)
    // (the list arrives sorted by frequency bucket, so a warp's packets are of one kind)
    const unsigned long long wi = (unsigned long long)(warp - n_pw), W = (unsigned long long)n_rest_warps;
    const unsigned long long e = wi * rest / W + lane, e1 = (wi + 1) * rest / W;
    if (e < e1) slot = (e < n_in) ? (int64_t)e : in.n_slots - 1 - (int64_t)(n_pw + (e - n_in));
  }
  Photon ph;
  bool active = false, done = false;
  bool prepared = false;  // ph.rng holds the words of the next event (pipelined mode)
  float tau_next = 0.0f;
  const SlotState& st = in;
  if (slot >= 0) {
    ph.model = st.model[slot];
    const ShellModel& m = models[ph.model];
    ph.pid = st.pid[slot];
    ph.rng.keys(((uint64_t)m.seed_hi << 32) | m.seed_lo, ph.pid);
    ph.rng.event = st.event[slot];
    ph.px = st.px[slot]; ph.py = st.py[slot]; ph.pz = st.pz[slot];
    ph.ox = st.ox[slot]; ph.oy = st.oy[slot]; ph.oz = st.oz[slot];
    ph.k = make_float3(st.kx[slot], st.ky[slot], st.kz[slot]);
    ph.X = st.X[slot];
    ph.x = st.x[slot];
    ph.safe = st.safe[slot];
    ph.X0 = 0.0f; ph.col_hi = 0.0f; ph.col_lo = 0.0f;  // raw records are not served
    ph.region = st.region[slot];
    ph.nscat = st.nscat[slot]; ph.ndust = st.ndust[slot]; ph.iters = st.iters[slot]; ph.steps = st.steps[slot];
    active = true;
  }
  uint32_t ev = 0;  // event iterations of this launch (warp-uniform)
  auto others_done = [&]() { return pri_warp && ev >= base_budget && (int64_t)vload(&in.live[4]) >= n_regular; };
  while (ev < budget && !others_done()) {
    const unsigned idle = __ballot_sync(kFull, !active && !done);
    const int room = per_warp - __popc(__ballot_sync(kFull, active));
    const bool take = ((idle >> lane) & 1u) && (int)__popc(idle & ((1u << lane) - 1u)) < room;
    const unsigned need = __ballot_sync(kFull, take);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(q.next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (take) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < q.total) {
          const int e = find_entry(q, g);
          ph.model = q.model[e];
          ph.pid = q.first_id[e] + (g - q.prefix[e]);
          shell_emit(models[ph.model], ph);
          active = true;
          prepared = false;
        } else {
          done = true;
        }
      }
    }
    if (__all_sync(kFull, !active)) break;
    // The lane's model record, and the cancel flag, once per run of events: a request
    // cancelled on the host drops its packets here (the flag is set between launches).
    const ShellModel* mp = models + (active ? ph.model : 0);
    bool dropped = false;
    if (active && *(volatile const int32_t*)&mp->cancelled) {
      atomicAdd(&mp->tally->n_done, 1ull);
      active = false;
      dropped = true;
    }
    if (__any_sync(kFull, dropped)) { ++ev; continue; }  // refill the dropped lanes first
    const ShellModel mr = *mp;  // by value: the fields the event loop reads stay in registers
    // events until some lane finishes its packet or the budget is used: one vote per event;
    // homologous shells run pipelined events in warps with at most kServedPipeLanes live
    // packets
    const int n_live = __popc(__ballot_sync(kFull, active));
    const bool pipe = n_live <= kServedPipeLanes;
    const bool burst = n_live <= kServedBurstLanes;
    bool fin;
    do {
      fin = false;
      uint32_t nb = 0;
      int r = 0;
      const bool pl = pipe && !(kMixed && mr.profile);  // this lane's packet runs pipelined events
      if (burst && budget - ev > kCoreBurst) {  // cooperative burst: all lanes, converged
        if (active && pl && !prepared) { pipe_prepare(mr, ph, tau_next); prepared = true; }
        const uint32_t before = ph.nscat;
        r = core_burst_coop(mr, ph, sK, tau_next, active && pl);
        if (active && pl) nb = ph.nscat - before;
      }
      if (active) {
        if (pl) {
          if (!prepared) { pipe_prepare(mr, ph, tau_next); prepared = true; }
          if (!r) r = shell_event_pipe(mr, ph, sK, tau_next);
        } else {
          if (prepared) { pipe_unprepare(ph); prepared = false; }
          r = (kMixed && mr.profile) ? shell_event_pl(mr, ph, sK) : shell_event(mr, ph, sK);
        }
        if (r) { finish_global(mr, ph, r); active = false; fin = true; }
      }
      ev += 1u + __reduce_max_sync(kFull, nb);  // a burst is charged its events
    } while (ev < budget && !__any_sync(kFull, fin) && !others_done());
  }
  if (!pri_warp && lane == 0) atomicAdd(&in.live[4], 1ull);  // this regular warp's round is over
  if (active && prepared) pipe_unprepare(ph);  // saved packets hold their last completed event
  // append the packets still in flight to the next list (one atomic per warp and list):
  // priority packets from the back, the others from the front.  Priority: packets of the
  // requests the host marked (the oldest), and long-lived packets (more than kLongLived
  // events: photons trapped in the line core, whose histories set the requests' latency)
  const bool pri = active && ((ph.nscat + ph.ndust) >= kLongLived ||
                              *(volatile const int32_t*)&models[ph.model].priority);
  const unsigned live_f = __ballot_sync(kFull, active && !pri), live_b = __ballot_sync(kFull, pri);
  if (live_f | live_b) {
    const int lead_f = live_f ? __ffs(live_f) - 1 : 0, lead_b = live_b ? __ffs(live_b) - 1 : 0;
    unsigned long long base_f = 0, base_b = 0;
    if (live_f && (int)lane == lead_f) base_f = atomicAdd(&out.live[1], (unsigned long long)__popc(live_f));
    if (live_b && (int)lane == lead_b) base_b = atomicAdd(&out.live[3], (unsigned long long)__popc(live_b));
    base_f = __shfl_sync(kFull, base_f, lead_f);
    base_b = __shfl_sync(kFull, base_b, lead_b);
    if (active) {
      const unsigned mine = pri ? live_b : live_f;
      const unsigned long long r = (pri ? base_b : base_f) + __popc(mine & ((1u << lane) - 1u));
      const unsigned long long j = pri ? (unsigned long long)(out.n_slots - 1) - r : r;
      SlotState& o = out;
      o.model[j] = ph.model; o.pid[j] = ph.pid;
      o.event[j] = ph.rng.event;
      o.px[j] = ph.px; o.py[j] = ph.py; o.pz[j] = ph.pz;
      o.ox[j] = ph.ox; o.oy[j] = ph.oy; o.oz[j] = ph.oz; o.safe[j] = ph.safe;
      o.kx[j] = ph.k.x; o.ky[j] = ph.k.y; o.kz[j] = ph.k.z;
      o.X[j] = ph.X; o.x[j] = ph.x; o.region[j] = (uint8_t)ph.region;
      o.nscat[j] = ph.nscat; o.ndust[j] = ph.ndust; o.iters[j] = ph.iters; o.steps[j] = ph.steps;
    }
  }
}

// ---- frequency pre-sorting of resident packets between served rounds ----------------
// Sorting packets by frequency before they are handed to warps groups those that take the
// same branches (the paper's pre-sorting, App. A.1 and Sec. 7.1): here, between rounds, the
// front list of `from` (from.live[1] packets) is copied into `to` by bucket -- line core
// (|x| <= 2), near wing (|x| <= 5), far wing, empty cavity -- and the resume hands each warp
// contiguous entries, so a warp's packets are of one kind (core packets then run the
// pipelined core events in step, wing packets the general event).  The back (priority)
// list is copied in place.  cnt[0..3]: bucket sizes, cnt[4..7]: cursors, zero on entry.
// The order inside a bucket does not matter: a packet's history does not depend on its
// warp or lane.
__device__ __forceinline__ int slot_bucket(const SlotState& s, int64_t i) {
  if (s.region[i]) return 3;
  const float ax = fabsf(s.x[i]);
  return ax <= 2.0f ? 0 : (ax <= 5.0f ? 1 : 2);
}
__device__ __forceinline__ void copy_slot(const SlotState& a, int64_t i, const SlotState& b, int64_t j) {
  b.px[j] = a.px[i]; b.py[j] = a.py[i]; b.pz[j] = a.pz[i];
  b.ox[j] = a.ox[i]; b.oy[j] = a.oy[i]; b.oz[j] = a.oz[i]; b.safe[j] = a.safe[i];
  b.kx[j] = a.kx[i]; b.ky[j] = a.ky[i]; b.kz[j] = a.kz[i]; b.X[j] = a.X[i]; b.x[j] = a.x[i];
  b.event[j] = a.event[i];
  b.nscat[j] = a.nscat[i]; b.ndust[j] = a.ndust[i]; b.iters[j] = a.iters[i]; b.steps[j] = a.steps[i];
  b.model[j] = a.model[i]; b.pid[j] = a.pid[i]; b.region[j] = a.region[i];
}
__global__ void slot_hist_kernel(SlotState from, unsigned long long* __restrict__ cnt) {
  const unsigned long long n = from.live[1];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool mine = (unsigned long long)i < n;
  const int key = mine ? slot_bucket(from, i) : 4;
  const unsigned peers = __match_any_sync(kFull, key);
  if (mine && (int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd(&cnt[key], (unsigned long long)__popc(peers));
}
__global__ void slot_sort_kernel(SlotState from, SlotState to, unsigned long long* __restrict__ cnt) {
  const unsigned long long n = from.live[1], nb = from.live[3];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const bool mine = (unsigned long long)i < n;
  const int key = mine ? slot_bucket(from, i) : 4;
  const unsigned peers = __match_any_sync(kFull, key);
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (mine && (int)lane == leader) base = atomicAdd(&cnt[4 + key], (unsigned long long)__popc(peers));
  base = __shfl_sync(kFull, base, leader);
  if (mine) {
    unsigned long long off = 0;
    for (int k = 0; k < key; ++k) off += cnt[k];
    copy_slot(from, i, to, (int64_t)(off + base + __popc(peers & ((1u << lane) - 1u))));
  }
  if ((unsigned long long)i < nb) copy_slot(from, from.n_slots - 1 - i, to, to.n_slots - 1 - i);
}

}  // namespace

cudaError_t launch_slot_presort(SlotState from, SlotState to, unsigned long long* cnt, cudaStream_t s) {
  const unsigned grid = (unsigned)((from.n_slots + 255) / 256);
  cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s);
  slot_hist_kernel<<<grid, 256, 0, s>>>(from, cnt);
  slot_sort_kernel<<<grid, 256, 0, s>>>(from, to, cnt);
  return cudaGetLastError();
}

int shell_grid(int block, int blocks_per_sm, bool sliced) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sliced) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, shell_slice_kernel<true>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, shell_run_kernel<true, 0>, block, 0);
  if (occ < 1) occ = 1;
  const int b = (blocks_per_sm > 0 && blocks_per_sm < occ) ? blocks_per_sm : occ;
  return sms * b;
}

cudaError_t launch_shell_run(const ShellModel* d_models, WorkQueue q, const float* d_ktab, int grid, int block,
                             int profile, int per_warp, int core_lanes, int burst_lanes, cudaStream_t s,
                             const Compact* share) {
  Compact none{};
  if (share) {  // the work-sharing fields
    none.pool = share->pool;
    none.ready = share->ready;
    none.share = share->share;
    none.n_total = share->n_total;
  }
  none.per_warp = per_warp;
  none.core_lanes = core_lanes;
  none.burst_lanes = burst_lanes;
  if (profile) shell_run_kernel<false, 1><<<grid, block, 0, s>>>(d_models, q, none, d_ktab);
  else shell_run_kernel<false, 0><<<grid, block, 0, s>>>(d_models, q, none, d_ktab);
  return cudaGetLastError();
}

cudaError_t launch_shell_run_compact(const ShellModel* d_models, WorkQueue q, Compact c, const float* d_ktab,
                                     int grid, int block, int profile, cudaStream_t s) {
  if (profile) shell_run_kernel<true, 1><<<grid, block, 0, s>>>(d_models, q, c, d_ktab);
  else shell_run_kernel<true, 0><<<grid, block, 0, s>>>(d_models, q, c, d_ktab);
  return cudaGetLastError();
}

cudaError_t launch_shell_slice(const ShellModel* d_models, WorkQueue q, SlotState in, SlotState out, uint32_t budget,
                               const float* d_ktab, int grid, int block, bool mixed, cudaStream_t s) {
  if (mixed) shell_slice_kernel<true><<<grid, block, 0, s>>>(d_models, q, in, out, budget, d_ktab);
  else shell_slice_kernel<false><<<grid, block, 0, s>>>(d_models, q, in, out, budget, d_ktab);
  return cudaGetLastError();
}

}  // namespace thor
