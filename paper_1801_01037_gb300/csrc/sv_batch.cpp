// Batched circuits (many independent states, passes interleaved in shared launches) and the serving loop
// (continuous batching under an HBM budget).  Both drive the batched fused-pass kernel: one launch per round
// applies the next pass of every circuit in the round.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "sv_state.h"

using namespace svi;

namespace {

int default_mode(sv_dtype dt) { return dt == SV_C64 ? MODE_C64_F32 : MODE_C128_DF32; }

int validate_circuit(int n, const sv_gate *g, size_t ng, std::string &why) {
  if (n < 1 || n > kMaxQubits) { why = "n out of range"; return SV_ERR_ARG; }
  if (!g && ng) { why = "gates is NULL"; return SV_ERR_ARG; }
  std::string w;
  size_t bad = 0;
  const int rc = validate_records(g, ng, n, w, bad);
  if (rc != SV_OK) { why = "gate " + std::to_string(bad) + ": " + w; return rc; }
  return SV_OK;
}

// Plan a circuit whose first pass synthesises |0...0>; every step is a fused pass.
void plan_fresh(sv_state *s, const sv_gate *g, size_t ng, Plan &P) {
  PlanConfig cfg = plan_config(s);
  cfg.init_first = true;
  cfg.init_x = 0;
  cfg.single_as_sweep = false;
  cfg.fusion = true;
  make_plan(s->n, cfg, s->perm, g, ng, P);
}

// Grow-only device buffer.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes, cudaStream_t st) {
    if (bytes <= cap) return SV_OK;
    if (p) { cudaStreamSynchronize(st); cudaFree(p); p = nullptr; cap = 0; }
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return SV_ERR_OOM; }
    cap = bytes;
    return SV_OK;
  }
  ~DevBuf() { if (p) cudaFree(p); }
};

} // namespace

extern "C" sv_status sv_run_batch(int count, const int *n, sv_dtype dtype, const sv_gate *const *gates,
                                  const size_t *ngates, void *stream, sv_state **out) {
  return sv_run_batch_k(count, n, dtype, gates, ngates, nullptr, stream, out);
}

extern "C" sv_status sv_run_batch_k(int count, const int *n, sv_dtype dtype, const sv_gate *const *gates,
                                    const size_t *ngates, const int *chunk_k, void *stream, sv_state **out) {
  if (count < 0 || (count > 0 && (!n || !gates || !ngates || !out))) return set_error(SV_ERR_ARG, "NULL argument");
  if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "bad dtype");
  if (count == 0) return SV_OK;
  if (chunk_k)
    for (int i = 0; i < count; ++i)
      if (chunk_k[i] != 0 && (chunk_k[i] < 6 || chunk_k[i] > kMaxChunkQubits))
        return set_error(SV_ERR_ARG, "circuit " + std::to_string(i) + ": chunk qubits must be 0 or 6..13");
  int rc = check_device();
  if (rc != SV_OK) return rc;
  for (int i = 0; i < count; ++i) {
    std::string why;
    if ((rc = validate_circuit(n[i], gates[i], ngates[i], why)) != SV_OK)
      return set_error(rc, "circuit " + std::to_string(i) + ": " + why);
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<sv_state *> states(count, nullptr);
  std::vector<Plan> plans(count);
  auto cleanup = [&](int code) {
    for (sv_state *s : states) if (s) sv_destroy(s);
    return code;
  };
  // One device allocation holds every state of the batch (256-byte aligned slices); each state keeps a
  // reference, so the memory is freed when the last of them is destroyed.  Their small scratch buffers are
  // made on first use.
  std::vector<size_t> off(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    off[i] = total;
    total += ((amp_bytes(dtype) << n[i]) + 255) & ~(size_t)255;
  }
  if (std::getenv("SV_FAULT_ALLOC")) return set_error(SV_ERR_OOM, "allocation failure injected (SV_FAULT_ALLOC)");
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
  if (total > free_b) return set_error(SV_ERR_OOM, "batch states of " + std::to_string(total) + " bytes exceed free device memory");
  void *base = nullptr;
  if ((e = cudaMalloc(&base, total)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(SV_ERR_OOM, "cudaMalloc of the batch states failed");
  }
  std::shared_ptr<void> arena(base, [](void *p) { cudaFree(p); });
  for (int i = 0; i < count; ++i) {
    sv_state *s = new sv_state();
    s->n = n[i];
    s->dtype = dtype;
    s->stream = st;
    s->perm.resize(n[i]);
    for (int t = 0; t < n[i]; ++t) s->perm[t] = t;
    s->psi = (char *)base + off[i];
    s->owned = false;
    s->arena = arena;
    s->chunk_k = chunk_k ? chunk_k[i] : 0;
    states[i] = s;
  }
  // Plans are independent: several host threads make them.
  const int nthreads = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), std::min(16, (count + 31) / 32)));
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&, t] {
      for (int i = t; i < count; i += nthreads) plan_fresh(states[i], gates[i], ngates[i], plans[i]);
    });
  for (std::thread &th : pool) th.join();
  size_t max_rounds = 0;
  for (int i = 0; i < count; ++i) max_rounds = std::max(max_rounds, plans[i].passes.size());
  // Gates of every circuit in one device blob; per round, the pass descriptors and chunk prefix sums.
  std::vector<size_t> blob_off(count);
  size_t blob_bytes = 0;
  for (int i = 0; i < count; ++i) {
    blob_off[i] = blob_bytes;
    blob_bytes += (plan_blob_bytes(plans[i]) + 15) & ~(size_t)15;
  }
  std::vector<unsigned char> blob(std::max<size_t>(blob_bytes, 16));
  for (int i = 0; i < count; ++i) plan_blob_fill(plans[i], blob.data() + blob_off[i]);
  std::vector<PassDesc> descs;
  std::vector<uint64_t> starts;
  struct Round { size_t desc_off, start_off; int npass; uint64_t total; int kmax; };
  std::vector<Round> rounds;
  for (size_t r = 0; r < max_rounds; ++r) {
    Round R{descs.size(), starts.size(), 0, 0, 0};
    for (int i = 0; i < count; ++i) {
      if (r >= plans[i].passes.size()) continue;
      PassDesc d = plans[i].passes[r];
      d.psi = states[i]->psi;
      d.init_x = (uint64_t)i;  // circuit index; replaced by the real fields below
      descs.push_back(d);
      starts.push_back(R.total);
      R.total += 1ull << (d.n - d.k);
      R.kmax = std::max(R.kmax, d.k);
      ++R.npass;
    }
    starts.push_back(R.total);
    rounds.push_back(R);
  }
  DevBuf dg, dd, ds, dsched;
  if (dsched.ensure(sizeof(FusedSched), st) != SV_OK || dg.ensure(blob.size(), st) != SV_OK ||
      dd.ensure(std::max<size_t>(1, descs.size()) * sizeof(PassDesc), st) != SV_OK ||
      ds.ensure(std::max<size_t>(1, starts.size()) * sizeof(uint64_t), st) != SV_OK)
    return cleanup(set_error(SV_ERR_OOM, "batch descriptor allocation failed"));
  for (size_t r = 0, di = 0; r < rounds.size(); ++r)
    for (int i = 0; i < count; ++i) {
      if (r >= plans[i].passes.size()) continue;
      PassDesc &d = descs[di++];
      plan_pass_pointers(plans[i], (int)r, (const unsigned char *)dg.p + blob_off[i], d);
      d.init_x = plans[i].passes[r].init_x;
    }
  e = cudaMemcpyAsync(dg.p, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(PassDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds.p, starts.data(), starts.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  const int mode = default_mode(dtype);
  for (size_t r = 0; r < rounds.size() && e == cudaSuccess; ++r) {
    const Round &R = rounds[r];
    e = launch_fused_batch((const PassDesc *)dd.p + R.desc_off, (const uint64_t *)ds.p + R.start_off, R.npass, R.total,
                           mode, R.kmax, st, kDefaultF64Share, (FusedSched *)dsched.p);
  }
  // The descriptor buffers are freed on return, so wait for the launches that read them.
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "batched passes"));
  for (int i = 0; i < count; ++i) {
    states[i]->st_passes = (int)plans[i].passes.size();
    states[i]->st_fused = plans[i].n_fused_gates;
    states[i]->st_relabels = plans[i].n_relabels;
    out[i] = states[i];
  }
  return SV_OK;
}

// =========================================================================================================
// Serving loop
// =========================================================================================================
struct sv_server {
  struct Request {
    uint64_t ticket;
    int n;
    sv_dtype dtype;
    std::vector<sv_gate> gates;
  };
  struct Active {
    uint64_t ticket;
    sv_state *st;
    Plan plan;
    void *d_gates;   // device blob: the plan's gates
    size_t next;
    size_t bytes;
  };
  size_t budget = 0, used = 0;
  int max_active = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> pending;
  std::vector<Active> active;
  std::unordered_map<uint64_t, std::pair<sv_state *, size_t>> done;
  std::unordered_map<uint64_t, std::pair<int, std::string>> failed;
  std::unordered_set<uint64_t> live;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  cudaStream_t stream = nullptr;
  DevBuf d_desc, d_start, d_sched;
  PassDesc *h_desc = nullptr;
  uint64_t *h_start = nullptr;
  size_t h_cap = 0;

  void fail_request(uint64_t ticket, int code, const std::string &msg) {
    failed[ticket] = {code, msg};
  }

  // Move admissible pending requests into the active set (called with mu held).
  void admit() {
    while (!pending.empty() && (int)active.size() < max_active) {
      Request &r = pending.front();
      const size_t bytes = amp_bytes(r.dtype) << r.n;
      if (used + bytes > budget) break;
      Active a{r.ticket, nullptr, Plan(), nullptr, 0, bytes};
      int rc = alloc_state(r.n, r.dtype, stream, &a.st, false);
      if (rc != SV_OK) {
        if (rc == SV_ERR_OOM && !active.empty()) break;  // wait for memory to free up
        fail_request(r.ticket, rc, sv_last_error());
        pending.pop_front();
        continue;
      }
      plan_fresh(a.st, r.gates.data(), r.gates.size(), a.plan);
      if (plan_blob_bytes(a.plan) > 0) {
        const size_t gb = plan_blob_bytes(a.plan);
        std::vector<unsigned char> blob(gb);
        plan_blob_fill(a.plan, blob.data());
        if (cudaMalloc(&a.d_gates, gb) != cudaSuccess ||
            cudaMemcpyAsync(a.d_gates, blob.data(), gb, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
          cudaGetLastError();
          if (a.d_gates) cudaFree(a.d_gates);
          sv_destroy(a.st);
          fail_request(r.ticket, SV_ERR_OOM, "gate buffer allocation failed");
          pending.pop_front();
          continue;
        }
      }
      used += bytes;
      active.push_back(std::move(a));
      pending.pop_front();
    }
  }

  int ensure_host(size_t m) {
    if (m <= h_cap) return SV_OK;
    if (h_desc) cudaFreeHost(h_desc);
    if (h_start) cudaFreeHost(h_start);
    h_desc = nullptr;
    h_start = nullptr;
    h_cap = 0;
    if (cudaMallocHost(&h_desc, m * sizeof(PassDesc)) != cudaSuccess ||
        cudaMallocHost(&h_start, (m + 1) * sizeof(uint64_t)) != cudaSuccess)
      return SV_ERR_OOM;
    h_cap = m;
    return SV_OK;
  }

  void loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      admit();
      if (active.empty()) {
        if (stop) break;
        cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      // One round: the next pass of every active request of one dtype, in one launch.
      const int mode = default_mode(active[0].st->dtype);
      std::vector<size_t> in_round;
      for (size_t i = 0; i < active.size(); ++i)
        if (default_mode(active[i].st->dtype) == mode) in_round.push_back(i);
      const size_t m = active.size();
      const size_t used_m = in_round.size();
      if (ensure_host(used_m) != SV_OK || d_desc.ensure(used_m * sizeof(PassDesc), stream) != SV_OK ||
          d_start.ensure((used_m + 1) * sizeof(uint64_t), stream) != SV_OK ||
          d_sched.ensure(sizeof(FusedSched), stream) != SV_OK) {
        for (Active &a : active) {
          fail_request(a.ticket, SV_ERR_OOM, "round descriptor allocation failed");
          if (a.d_gates) cudaFree(a.d_gates);
          sv_destroy(a.st);
          used -= a.bytes;
        }
        active.clear();
        continue;
      }
      uint64_t total = 0;
      int kmax = 0;
      for (size_t j = 0; j < used_m; ++j) {
        Active &a = active[in_round[j]];
        PassDesc d = a.plan.passes[a.next];
        d.psi = a.st->psi;
        plan_pass_pointers(a.plan, (int)a.next, a.d_gates, d);
        h_desc[j] = d;
        h_start[j] = total;
        total += 1ull << (d.n - d.k);
        kmax = std::max(kmax, d.k);
      }
      h_start[used_m] = total;
      lk.unlock();
      cudaError_t e = cudaMemcpyAsync(d_desc.p, h_desc, used_m * sizeof(PassDesc), cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_start.p, h_start, (used_m + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = launch_fused_batch((const PassDesc *)d_desc.p, (const uint64_t *)d_start.p, (int)used_m, total, mode, kmax, stream,
                               kDefaultF64Share, (FusedSched *)d_sched.p);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      lk.lock();
      std::vector<Active> keep;
      std::vector<char> in(m, 0);
      for (size_t i : in_round) in[i] = 1;
      for (size_t i = 0; i < m; ++i) {
        Active &a = active[i];
        if (!in[i]) { keep.push_back(std::move(a)); continue; }
        if (e != cudaSuccess) {
          fail_request(a.ticket, SV_ERR_CUDA, std::string("serving round: ") + cudaGetErrorString(e));
          if (a.d_gates) cudaFree(a.d_gates);
          sv_destroy(a.st);
          used -= a.bytes;
          continue;
        }
        ++a.next;
        if (a.next >= a.plan.passes.size()) {
          if (a.d_gates) cudaFree(a.d_gates);
          a.st->st_passes = (int)a.plan.passes.size();
          done[a.ticket] = {a.st, a.bytes};
        } else {
          keep.push_back(std::move(a));
        }
      }
      active.swap(keep);
    }
  }
};

extern "C" {

sv_status sv_server_create(size_t hbm_budget_bytes, int max_active, sv_server **out) {
  if (!out || hbm_budget_bytes == 0 || max_active < 1) return set_error(SV_ERR_ARG, "bad server arguments");
  int rc = check_device();
  if (rc != SV_OK) return rc;
  sv_server *s = new sv_server();
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return set_error(SV_ERR_CUDA, "server stream creation failed");
  }
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return SV_OK;
}

sv_status sv_server_destroy(sv_server *s) {
  if (!s) return SV_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->pending.clear();
  }
  s->cv.notify_all();
  s->th.join();
  for (auto &kv : s->done) sv_destroy(kv.second.first);
  for (auto &a : s->active) { if (a.d_gates) cudaFree(a.d_gates); sv_destroy(a.st); }
  if (s->h_desc) cudaFreeHost(s->h_desc);
  if (s->h_start) cudaFreeHost(s->h_start);
  cudaStreamDestroy(s->stream);
  delete s;
  return SV_OK;
}

sv_status sv_submit(sv_server *s, int n, sv_dtype dtype, const sv_gate *gates, size_t ngates, uint64_t *ticket) {
  if (!s || !ticket) return set_error(SV_ERR_ARG, "NULL argument");
  if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "bad dtype");
  std::string why;
  int rc = validate_circuit(n, gates, ngates, why);
  if (rc != SV_OK) return set_error(rc, why);
  const size_t bytes = amp_bytes(dtype) << n;
  if (bytes > s->budget) return set_error(SV_ERR_OOM, "state exceeds the server's HBM budget");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->pending.size() >= 65536) return set_error(SV_ERR_BUSY, "pending queue is full");
    sv_server::Request r{s->next_ticket++, n, dtype, std::vector<sv_gate>(gates, gates + ngates)};
    *ticket = r.ticket;
    s->live.insert(r.ticket);
    s->pending.push_back(std::move(r));
  }
  s->cv.notify_all();
  return SV_OK;
}

sv_status sv_poll(sv_server *s, uint64_t ticket, int *done, sv_state **result) {
  if (!s || !done || !result) return set_error(SV_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *done = 1;
    *result = it->second.first;
    s->used -= it->second.second;
    s->done.erase(it);
    s->live.erase(ticket);
    s->cv.notify_all();
    return SV_OK;
  }
  auto f = s->failed.find(ticket);
  if (f != s->failed.end()) {
    const int code = f->second.first;
    const std::string msg = f->second.second;
    s->failed.erase(f);
    s->live.erase(ticket);
    *done = 1;
    *result = nullptr;
    return set_error(code, msg);
  }
  if (s->live.count(ticket)) {
    *done = 0;
    *result = nullptr;
    return SV_OK;
  }
  return set_error(SV_ERR_NOT_FOUND, "unknown ticket");
}

} // extern "C"
