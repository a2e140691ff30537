// thor_server.cu -- continuous batching of shell-model requests on one device.
//
// A host worker thread runs device rounds while work exists.  A round is one launch
// of the time-sliced photon loop over the resident packet slots: every lane resumes
// its packet, runs at most `events_per_round` events, refills from the queue of
// admitted requests when its packet finishes, and saves what is still in flight.
// Between rounds the worker admits pending requests (free model slot and memory
// for their tables within the budget), rebuilds the queue from the photons each
// admitted request still has to issue, and retires requests whose photons all
// finished (their spectrum and tallies are copied to the caller's buffers).
// Packet state and tallies stay on the device across rounds; the per-round host
// traffic is the queue table (a few hundred bytes) and the tallies of the active
// requests.  A round (queue upload, photon-loop launch, counter and tally download) is
// one CUDA graph captured when the server is created and replayed every round: the
// kernel reads the queue size from the uploaded table, and the host side of both copies
// is a fixed pinned buffer.  Each photon's stream depends only on (request seed, photon id), and
// tallies are integers, so a request's result does not depend on what else ran.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/thor.h"
#include "thor_ctx.h"
#include "thor_internal.h"

using namespace thor;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  int64_t ticket = 0;
  ShellModel model{};
  uint64_t n_photons = 0, issued = 0;
  int32_t n_bins = 0;
  uint64_t* user_spectrum = nullptr;
  size_t table_bytes = 0;
  int slot = -1;           // model-table index while admitted
  int state = 0;           // 0 pending, 1 active, 2 done, 3 cancelled
  bool cancel = false;
  bool cancel_sent = false;
  bool priority = false;       // wanted this round: packets one per warp
  bool priority_sent = false;  // as last set on the device
  uint64_t done_seen = 0;      // photons finished, as of the last round's tallies
  Clock::time_point t_submit, t_done;
  thor_result result{};
};

}  // namespace

struct thor_server {
  thor_ctx* ctx = nullptr;
  thor_server_config cfg{};
  int grid = 0, block = 128;
  int64_t n_slots = 0;
  int max_bins = 0;
  // device memory
  ShellModel* d_models = nullptr;
  Tally* d_tally = nullptr;
  unsigned long long* d_spec = nullptr;  // max_requests x (max_bins + 2)
  char* d_queue = nullptr;               // counter, total, n_entries, prefix, first_id, model
  void* d_slots = nullptr;               // two packet lists (in, out) of n_slots entries + counters
  size_t slot_bytes = 0;
  SlotState st_in{}, st_out{};
  cudaStream_t stream = nullptr;
  // one round as a graph: h_queue (pinned, layout of d_queue) -> d_queue, slice kernel,
  // d_queue counter and the tallies -> h_out (pinned)
  char* h_queue = nullptr;
  char* h_out = nullptr;
  // [0]: homologous shells only; [1]: power-law models among them (event chosen per lane)
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // host state
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> active;  // indexed by model slot
  std::map<int64_t, Request*> all;
  int64_t next_ticket = 1;
  uint64_t mem_used = 0;
  bool stop = false;
  bool device_error = false;
  std::string error;
  uint64_t rounds = 0, admitted = 0;
  uint64_t last_resident = 0;  // packets in flight after the last round
  double resident_sum = 0.0;
  std::thread worker;

  void run();
};

namespace {

// d_queue / h_queue layout: next counter, total, n_entries, event budget, lanes per warp
// that take new packets (u64 each), prefix[R + 1], first_id[R] (u64), model[R] (i32)
struct QLayout {
  size_t next = 0, total = 8, n_entries = 16, budget = 24, per_warp = 32, prefix = 40, first, model, bytes;
  explicit QLayout(int R) {
    first = prefix + (size_t)(R + 1) * 8;
    model = first + (size_t)R * 8;
    bytes = model + (size_t)R * 4;
  }
};
size_t queue_bytes(int max_req) { return QLayout(max_req).bytes; }

constexpr uint64_t kIdleRounds = 4;

}  // namespace

void thor_server::run() {
  cudaSetDevice(ctx->device);
  const int R = cfg.max_requests;
  const QLayout L(R);
  unsigned long long* h_prefix = (unsigned long long*)(h_queue + L.prefix);
  unsigned long long* h_first = (unsigned long long*)(h_queue + L.first);
  int32_t* h_model = (int32_t*)(h_queue + L.model);
  std::vector<int> h_entry_req(R);
  std::vector<Tally> h_tally(R);
  std::vector<uint64_t> h_spec;
  for (;;) {
    std::vector<Request*> fresh;
    int n_entries = 0;
    uint64_t budget = 0, per_warp = 32;
    unsigned long long total = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) return;
        // admission: free model slot and table memory within the budget
        while (!pending.empty()) {
          Request* r = pending.front();
          if (r->cancel) { pending.pop_front(); r->state = 3; cv_done.notify_all(); continue; }
          int slot = -1;
          for (int i = 0; i < R; ++i) if (!active[i]) { slot = i; break; }
          if (slot < 0 || mem_used + r->table_bytes > cfg.mem_budget_bytes) break;
          pending.pop_front();
          r->slot = slot;
          r->state = 1;
          active[slot] = r;
          mem_used += r->table_bytes;
          ++admitted;
          fresh.push_back(r);
        }
        bool any = false;
        for (int i = 0; i < R; ++i) if (active[i]) { any = true; break; }
        if (any) break;
        cv_work.wait(lk);
      }
      // queue entries oldest request first: free lanes go to the photons that waited longest
      std::vector<std::pair<int64_t, int>> order;
      for (int i = 0; i < R; ++i)
        if (active[i] && !active[i]->cancel && active[i]->issued < active[i]->n_photons)
          order.emplace_back(active[i]->ticket, i);
      std::sort(order.begin(), order.end());
      for (const auto& oi : order) {
        const int i = oi.second;
        Request* r = active[i];
        h_prefix[n_entries] = total;
        h_first[n_entries] = r->issued;
        h_model[n_entries] = i;
        h_entry_req[n_entries] = i;
        total += r->n_photons - r->issued;
        ++n_entries;
      }
      h_prefix[n_entries] = total;
      // priority: the oldest request, and the next oldest while their packets in flight fit
      // in half of the warps, run their packets one per warp, so the longest histories of the
      // requests that have waited longest advance at the latency of a lone lane (the slice
      // kernel gives each such packet a warp of its own, up to half of the warps, and spreads
      // the rest with the other packets)
      {
        std::vector<std::pair<int64_t, int>> by_age;
        for (int i = 0; i < R; ++i)
          if (active[i] && !active[i]->cancel) by_age.emplace_back(active[i]->ticket, i);
        std::sort(by_age.begin(), by_age.end());
        const uint64_t cap = (uint64_t)(n_slots / 32) / 2;
        uint64_t cum = 0;
        bool open = cfg.priority >= 0;
        for (const auto& oi : by_age) {
          Request* r = active[oi.second];
          const uint64_t resident = r->issued - std::min(r->issued, r->done_seen);
          r->priority = open && (cum == 0 || cum + resident <= cap);
          if (r->priority) cum += resident + 1;
          else open = false;
        }
      }
      // rounds run kIdleRounds x longer while nobody waits for admission: fewer launches
      // and host round trips for the tails of admitted requests
      budget = pending.empty() ? (uint64_t)cfg.events_per_round * kIdleRounds : (uint64_t)cfg.events_per_round;
      // few packets in flight: new ones spread over the warps (each runs closer to alone,
      // not behind the divergent packets of other requests); many: full warps
      const uint64_t n_warps = (uint64_t)(n_slots / 32);
      const uint64_t load = last_resident + total;
      uint64_t pw = n_warps ? (load + n_warps - 1) / n_warps : 32;
      per_warp = pw < 1 ? 1 : (pw > 32 ? 32 : pw);
    }
    cudaStream_t s = stream;
    bool ok = true;
    for (Request* r : fresh) {
      ShellModel m = r->model;
      m.spectrum = d_spec + (size_t)r->slot * (max_bins + 2);
      m.tally = d_tally + r->slot;
      m.priority = 0;
      r->priority_sent = false;
      ok &= cudaMemcpyAsync(d_models + r->slot, &m, sizeof m, cudaMemcpyHostToDevice, s) == cudaSuccess;
      ok &= cudaMemsetAsync(m.spectrum, 0, (size_t)(max_bins + 2) * 8, s) == cudaSuccess;
      ok &= cudaMemsetAsync(m.tally, 0, sizeof(Tally), s) == cudaSuccess;
    }
    {
      // tell the device which admitted requests were cancelled (their packets are dropped);
      // after the model uploads of this round, which would otherwise overwrite the flag
      std::lock_guard<std::mutex> lk(mu);
      for (int i = 0; i < R; ++i) {
        Request* r = active[i];
        if (r && r->cancel && !r->cancel_sent) {
          static const int32_t one = 1;
          ok &= cudaMemcpyAsync(&d_models[i].cancelled, &one, sizeof one, cudaMemcpyHostToDevice, s) == cudaSuccess;
          r->cancel_sent = true;
        }
      }
    }
    {
      // priority flags that changed since the last round
      static const int32_t kOne = 1, kZero = 0;
      std::lock_guard<std::mutex> lk(mu);
      for (int i = 0; i < R; ++i) {
        Request* r = active[i];
        if (r && r->priority != r->priority_sent) {
          ok &= cudaMemcpyAsync(&d_models[i].priority, r->priority ? &kOne : &kZero, sizeof(int32_t),
                                cudaMemcpyHostToDevice, s) == cudaSuccess;
          r->priority_sent = r->priority;
        }
      }
    }
    // queue header (the tables were filled in place above), then the captured round
    ((unsigned long long*)(h_queue + L.next))[0] = 0;
    ((unsigned long long*)(h_queue + L.total))[0] = total;
    ((unsigned long long*)(h_queue + L.n_entries))[0] = (unsigned long long)n_entries;
    ((unsigned long long*)(h_queue + L.budget))[0] = (unsigned long long)budget;
    ((unsigned long long*)(h_queue + L.per_warp))[0] = (unsigned long long)per_warp;
    bool mixed = false;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (int i = 0; i < R; ++i) if (active[i] && active[i]->model.profile != 0) mixed = true;
    }
    ok &= cudaGraphLaunch(gexec[mixed ? 1 : 0], s) == cudaSuccess;
    ok &= cudaStreamSynchronize(s) == cudaSuccess;
    const unsigned long long h_next = ((const unsigned long long*)h_out)[0];
    std::memcpy(h_tally.data(), h_out + 8, sizeof(Tally) * R);
    if (!ok) {
      std::lock_guard<std::mutex> lk(mu);
      device_error = true;
      error = cudaGetErrorString(cudaGetLastError());
      for (int i = 0; i < R; ++i) if (active[i]) { active[i]->state = 3; active[i] = nullptr; }
      for (Request* r : pending) r->state = 3;
      pending.clear();
      cv_done.notify_all();
      return;
    }
    ++rounds;
    // photons handed out this round, entry by entry in prefix order
    const unsigned long long handed = std::min<unsigned long long>(h_next, total);
    std::vector<Request*> finished;
    {
      std::lock_guard<std::mutex> lk(mu);
      uint64_t resident = 0;
      for (int e = 0; e < n_entries; ++e) {
        Request* r = active[h_entry_req[e]];
        if (!r) continue;
        const unsigned long long lo = h_prefix[e], hi = h_prefix[e + 1];
        const unsigned long long got = handed <= lo ? 0 : std::min(handed, hi) - lo;
        r->issued += got;
      }
      for (int i = 0; i < R; ++i) {
        Request* r = active[i];
        if (!r) continue;
        resident += r->issued - h_tally[i].n_done;
        r->done_seen = h_tally[i].n_done;
        const bool all_done = h_tally[i].n_done >= r->n_photons;
        const bool cancelled_drained = r->cancel && h_tally[i].n_done >= r->issued;
        if (all_done || cancelled_drained) finished.push_back(r);
      }
      resident_sum += (double)resident;
      last_resident = resident;
    }
    for (Request* r : finished) {
      const size_t nb = (size_t)r->n_bins + 2;
      h_spec.resize((size_t)max_bins + 2);
      cudaMemcpyAsync(h_spec.data(), d_spec + (size_t)r->slot * (max_bins + 2), (size_t)(max_bins + 2) * 8,
                      cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      // the device row holds n_bins bins followed by underflow, overflow
      if (!r->cancel) std::memcpy(r->user_spectrum, h_spec.data(), nb * 8);
      std::lock_guard<std::mutex> lk(mu);
      tally_to_result(h_tally[r->slot], r->n_photons, &r->result);
      r->t_done = Clock::now();
      r->result.elapsed_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
      r->state = r->cancel ? 3 : 2;
      active[r->slot] = nullptr;
      mem_used -= r->table_bytes;
      cv_done.notify_all();
    }
  }
}

extern "C" int thor_server_create(thor_ctx_t ctx, const thor_server_config* cfg, thor_server_t* out) {
  if (!ctx || !cfg || !out) return ctx ? ctx->fail(THOR_ERR_INVALID_ARG, "thor_server_create: NULL") : THOR_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->max_requests <= 0 || cfg->max_requests > 4096 || cfg->events_per_round <= 0)
    return ctx->fail(THOR_ERR_INVALID_ARG, "max_requests in [1, 4096], events_per_round > 0");
  if (cfg->block_size && (cfg->block_size & 31 || cfg->block_size > 256))
    return ctx->fail(THOR_ERR_INVALID_ARG, "block_size must be a multiple of 32 <= 256");
  if (int rc = ctx->select()) return rc;
  thor_server* s = new thor_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  if (s->cfg.mem_budget_bytes == 0) s->cfg.mem_budget_bytes = 1ull << 30;
  s->block = cfg->block_size ? cfg->block_size : ctx->block;
  s->grid = shell_grid(s->block, ctx->blocks_per_sm, true);
  const int64_t resident = (int64_t)s->grid * s->block;
  if (cfg->n_slots > 0 && cfg->n_slots < resident) s->grid = (int)((cfg->n_slots + s->block - 1) / s->block);
  s->n_slots = (int64_t)s->grid * s->block;
  s->max_bins = 4096;
  const int R = cfg->max_requests;
  s->active.assign(R, nullptr);
  const size_t spec_bytes = (size_t)R * (s->max_bins + 2) * 8;
  const int64_t n = s->n_slots;
  const size_t slot_bytes = (size_t)n * (3 * 8 + 4 * 4 + 5 * 4 + 4 + 4 * 4 + 4 + 8 + 1) + 24 * 256;
  s->slot_bytes = slot_bytes;
  bool ok = cudaMallocHost(&s->h_queue, queue_bytes(R)) == cudaSuccess &&
            cudaMallocHost(&s->h_out, 8 + sizeof(Tally) * R) == cudaSuccess &&
            cudaMalloc(&s->d_models, sizeof(ShellModel) * R) == cudaSuccess &&
            cudaMalloc(&s->d_tally, sizeof(Tally) * R) == cudaSuccess &&
            cudaMalloc(&s->d_spec, spec_bytes) == cudaSuccess &&
            cudaMalloc(&s->d_queue, queue_bytes(R)) == cudaSuccess &&
            cudaMalloc(&s->d_slots, 2 * slot_bytes + 256) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    thor_server_destroy(s);
    return ctx->fail(THOR_ERR_OOM, "thor_server_create: device allocation failed");
  }
  // carve the two packet lists (256-byte aligned SoA arrays, identical layouts) and the
  // counters {packets in the in list from the front, their append counter in the out list,
  // priority packets in the in list from the back, their append counter}
  auto carve = [&](char* p, SlotState& st) {
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return (void*)q; };
    st.px = (double*)take(n * 8); st.py = (double*)take(n * 8); st.pz = (double*)take(n * 8);
    st.ox = (float*)take(n * 4); st.oy = (float*)take(n * 4); st.oz = (float*)take(n * 4);
    st.safe = (float*)take(n * 4);
    st.kx = (float*)take(n * 4); st.ky = (float*)take(n * 4); st.kz = (float*)take(n * 4); st.X = (float*)take(n * 4);
    st.x = (float*)take(n * 4);
    st.event = (uint32_t*)take(n * 4);
    st.nscat = (uint32_t*)take(n * 4); st.ndust = (uint32_t*)take(n * 4); st.iters = (uint32_t*)take(n * 4);
    st.steps = (uint32_t*)take(n * 4);
    st.model = (int32_t*)take(n * 4);
    st.pid = (unsigned long long*)take(n * 8);
    st.region = (uint8_t*)take(n);
    st.n_slots = n;
  };
  char* base = (char*)s->d_slots;
  carve(base, s->st_in);
  carve(base + slot_bytes, s->st_out);
  unsigned long long* live = (unsigned long long*)(base + 2 * slot_bytes);
  s->st_in.live = live;
  s->st_out.live = live;
  cudaMemsetAsync(live, 0, 32, s->stream);  // no packets in flight
  cudaStreamSynchronize(s->stream);
  // capture one round (thread-local capture mode: other host threads are unaffected)
  {
    const QLayout L(R);
    WorkQueue wq;
    wq.next = (unsigned long long*)(s->d_queue + L.next);
    wq.total = 0;
    wq.prefix = (const unsigned long long*)(s->d_queue + L.prefix);
    wq.first_id = (const unsigned long long*)(s->d_queue + L.first);
    wq.model = (const int32_t*)(s->d_queue + L.model);
    wq.n_entries = 0;
    wq.hdr = (const unsigned long long*)(s->d_queue + L.total);
    cudaStream_t cs = s->stream;
    bool cap = true;
    for (int v = 0; v < 2 && cap; ++v) {
      cap = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (!cap) break;
      cudaMemcpyAsync(s->d_queue, s->h_queue, L.bytes, cudaMemcpyHostToDevice, cs);
      cudaMemsetAsync(&s->st_in.live[4], 0, 8, cs);  // regular warps done this round
      launch_shell_slice(s->d_models, wq, s->st_in, s->st_out, (uint32_t)s->cfg.events_per_round, ctx->d_ktab,
                         s->grid, s->block, v == 1, cs);
      // the survivors become the next round's list: sorted by frequency bucket (pre-sorting),
      // or copied as they are
      if (s->cfg.presort > 0) launch_slot_presort(s->st_out, s->st_in, s->st_in.live + 8, cs);
      else cudaMemcpyAsync(s->d_slots, (char*)s->d_slots + s->slot_bytes, s->slot_bytes, cudaMemcpyDeviceToDevice, cs);
      cudaMemcpyAsync(&s->st_in.live[0], &s->st_in.live[1], 8, cudaMemcpyDeviceToDevice, cs);
      cudaMemsetAsync(&s->st_in.live[1], 0, 8, cs);
      cudaMemcpyAsync(&s->st_in.live[2], &s->st_in.live[3], 8, cudaMemcpyDeviceToDevice, cs);
      cudaMemsetAsync(&s->st_in.live[3], 0, 8, cs);
      cudaMemcpyAsync(s->h_out, s->d_queue + L.next, 8, cudaMemcpyDeviceToHost, cs);
      cudaMemcpyAsync(s->h_out + 8, s->d_tally, sizeof(Tally) * R, cudaMemcpyDeviceToHost, cs);
      cap = cudaStreamEndCapture(cs, &s->graph[v]) == cudaSuccess &&
            cudaGraphInstantiate(&s->gexec[v], s->graph[v], 0) == cudaSuccess;
    }
    if (!cap) {
      cudaGetLastError();
      thor_server_destroy(s);
      return ctx->fail(THOR_ERR_DEVICE, "thor_server_create: capturing the round graph failed");
    }
  }
  s->worker = std::thread([s]() { s->run(); });
  *out = s;
  return THOR_OK;
}

extern "C" int thor_server_submit(thor_server_t s, const thor_shell_params* p, const thor_source* src,
                                  uint64_t n_photons, uint64_t seed, const thor_output_spec* spec, int64_t* ticket) {
  if (!s || !p || !src || !spec || !ticket) return s ? s->ctx->fail(THOR_ERR_INVALID_ARG, "thor_server_submit: NULL") : THOR_ERR_INVALID_ARG;
  thor_ctx* ctx = s->ctx;
  if (n_photons == 0 || n_photons > (1ull << 40)) return ctx->fail(THOR_ERR_INVALID_ARG, "n_photons out of range");
  if (src->kind != 0) return ctx->fail(THOR_ERR_INVALID_ARG, "served requests take a point source");
  if (!spec->spectrum || spec->mem_kind != THOR_MEM_HOST || spec->n_bins <= 0 || !(spec->X_max > spec->X_min))
    return ctx->fail(THOR_ERR_INVALID_ARG, "served requests need a host spectrum buffer and a valid binning");
  if (spec->n_bins > s->max_bins) return ctx->fail(THOR_ERR_CAPACITY, "n_bins exceeds %d", s->max_bins);
  Request* r = new Request();
  if (int rc = fill_shell_model(ctx, p, &r->model)) { delete r; return rc; }
  ShellModel& m = r->model;
  if (int rc = fill_shell_source(ctx, src, &m)) { delete r; return rc; }
  m.X_min = (float)spec->X_min;
  m.inv_dX = spectrum_inv_dX(spec->n_bins, spec->X_min, spec->X_max);
  m.n_bins = spec->n_bins;
  m.seed_lo = (uint32_t)seed; m.seed_hi = (uint32_t)(seed >> 32);
  m.max_scat = spec->max_scat;
  m.id_base = 0;
  m.n_photons = n_photons;
  r->n_photons = n_photons;
  r->n_bins = spec->n_bins;
  r->user_spectrum = spec->spectrum;
  r->table_bytes = sizeof(ShellModel) + sizeof(Tally) + (size_t)(spec->n_bins + 2) * 8;
  if (r->table_bytes > s->cfg.mem_budget_bytes) { delete r; return ctx->fail(THOR_ERR_CAPACITY, "request never fits the memory budget"); }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->device_error) { delete r; return ctx->fail(THOR_ERR_DEVICE, "server stopped after a device error: %s", s->error.c_str()); }
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_all();
  *ticket = r->ticket;
  return THOR_OK;
}

extern "C" int thor_server_poll(thor_server_t s, int64_t ticket, int* done) {
  if (!s || !done) return THOR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return THOR_ERR_NOT_FOUND;
  *done = it->second->state >= 2 ? 1 : 0;
  return THOR_OK;
}

extern "C" int thor_server_wait(thor_server_t s, int64_t ticket, int64_t timeout_ms, thor_result* out) {
  if (!s || !out) return THOR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return THOR_ERR_NOT_FOUND;
  Request* r = it->second;
  auto pred = [r]() { return r->state >= 2; };
  if (timeout_ms < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return THOR_ERR_TIMEOUT;
  if (r->state == 3) {
    s->all.erase(it);
    delete r;
    return s->device_error ? THOR_ERR_DEVICE : THOR_ERR_CANCELLED;
  }
  *out = r->result;
  s->all.erase(it);
  delete r;
  return THOR_OK;
}

extern "C" int thor_server_cancel(thor_server_t s, int64_t ticket) {
  if (!s) return THOR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return THOR_ERR_NOT_FOUND;
  it->second->cancel = true;
  s->cv_work.notify_all();
  return THOR_OK;
}

extern "C" int thor_server_stats(thor_server_t s, uint64_t* rounds, double* mean_resident, uint64_t* admitted) {
  if (!s) return THOR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (rounds) *rounds = s->rounds;
  if (mean_resident) *mean_resident = s->rounds ? s->resident_sum / (double)s->rounds : 0.0;
  if (admitted) *admitted = s->admitted;
  return THOR_OK;
}

extern "C" void thor_server_destroy(thor_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (int v = 0; v < 2; ++v) {
    if (s->gexec[v]) cudaGraphExecDestroy(s->gexec[v]);
    if (s->graph[v]) cudaGraphDestroy(s->graph[v]);
  }
  for (void* p : {(void*)s->d_models, (void*)s->d_tally, (void*)s->d_spec, (void*)s->d_queue, s->d_slots})
    if (p) cudaFree(p);
  if (s->h_queue) cudaFreeHost(s->h_queue);
  if (s->h_out) cudaFreeHost(s->h_out);
  if (s->stream) cudaStreamDestroy(s->stream);
  for (auto& kv : s->all) delete kv.second;
  delete s;
}
