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

// Plan a circuit whose first pass synthesises |0...0>; every step is a fused pass.  Dense tensor-core blocks
// (tensor_blocks as SV_OPT_TENSOR_BLOCKS) only for complex128 double-float circuits with chunks of 2^kBatchTcK
// amplitudes, the one chunk size the batched tensor-core kernel takes; other passes apply gates one by one.
void plan_fresh(sv_state *s, const sv_gate *g, size_t ng, Plan &P, int tensor_blocks = 0) {
  PlanConfig cfg = plan_config(s);
  cfg.init_first = true;
  cfg.init_x = 0;
  cfg.single_as_sweep = false;
  cfg.fusion = true;
  cfg.block_mode = -1;
  if (tensor_blocks > 0 && mode_of(s) == MODE_C128_DF32 && cfg.k == kBatchTcK && s->n >= kBatchTcK) {
    cfg.block_mode = MODE_C128_DF32;
    if (tensor_blocks >= 2) cfg.block_min_cost = (double)tensor_blocks;
  }
  make_plan(s->n, cfg, s->perm, g, ng, P);
}

thread_local sv_batch_stats t_batch_stats{};
thread_local int t_batch_tensor_blocks = 0;

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

extern "C" sv_status sv_batch_set_option(int option, int value) {
  if (option != SV_OPT_TENSOR_BLOCKS) return set_error(SV_ERR_ARG, "only SV_OPT_TENSOR_BLOCKS applies to batches");
  if (value < 0 || value > 64) return set_error(SV_ERR_ARG, "SV_OPT_TENSOR_BLOCKS must be in 0..64");
  t_batch_tensor_blocks = value;
  return SV_OK;
}

extern "C" sv_status sv_last_batch_stats(sv_batch_stats *out) {
  if (!out) return set_error(SV_ERR_ARG, "NULL argument");
  *out = t_batch_stats;
  return SV_OK;
}

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
  const int tensor_blocks = t_batch_tensor_blocks;
  const int nthreads = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), std::min(16, (count + 31) / 32)));
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&, t] {
      for (int i = t; i < count; i += nthreads) plan_fresh(states[i], gates[i], ngates[i], plans[i], tensor_blocks);
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
  // Per round two launches: the passes that apply their gates one by one, and the passes with dense blocks
  // (tensor-core kernel); each has its own descriptor list and chunk prefix sums.
  std::vector<PassDesc> descs;
  std::vector<std::pair<int, int>> desc_src;  // (circuit, pass) of each descriptor
  std::vector<uint64_t> starts;
  struct Round {
    size_t desc_off, start_off; int npass; uint64_t total; int kmax;
    size_t tc_desc_off, tc_start_off; int tc_npass; uint64_t tc_total;
  };
  std::vector<Round> rounds;
  bool any_tc = false;
  for (size_t r = 0; r < max_rounds; ++r) {
    Round R{descs.size(), starts.size(), 0, 0, 0, 0, 0, 0, 0};
    for (int tc = 0; tc < 2; ++tc) {
      if (tc) { starts.push_back(R.total); R.tc_desc_off = descs.size(); R.tc_start_off = starts.size(); }
      for (int i = 0; i < count; ++i) {
        // (plan_fresh forms blocks only in passes of 2^kBatchTcK-amplitude chunks)
        if (r >= plans[i].passes.size() || (plans[i].passes[r].nblocks > 0) != (tc == 1)) continue;
        PassDesc d = plans[i].passes[r];
        d.psi = states[i]->psi;
        descs.push_back(d);
        desc_src.emplace_back(i, (int)r);
        if (tc) {
          starts.push_back(R.tc_total);
          R.tc_total += 1ull << (d.n - d.k);
          ++R.tc_npass;
        } else {
          starts.push_back(R.total);
          R.total += 1ull << (d.n - d.k);
          R.kmax = std::max(R.kmax, d.k);
          ++R.npass;
        }
      }
    }
    starts.push_back(R.tc_total);
    any_tc |= R.tc_npass > 0;
    rounds.push_back(R);
  }
  DevBuf dg, dd, ds, dsched;
  if (dsched.ensure(sizeof(FusedSched), st) != SV_OK || dg.ensure(blob.size(), st) != SV_OK ||
      dd.ensure(std::max<size_t>(1, descs.size()) * sizeof(PassDesc), st) != SV_OK ||
      ds.ensure(std::max<size_t>(1, starts.size()) * sizeof(uint64_t), st) != SV_OK)
    return cleanup(set_error(SV_ERR_OOM, "batch descriptor allocation failed"));
  for (size_t di = 0; di < descs.size(); ++di) {
    const int i = desc_src[di].first, r = desc_src[di].second;
    plan_pass_pointers(plans[i], r, (const unsigned char *)dg.p + blob_off[i], descs[di]);
  }
  // the tensor-core kernel's error word (and the split kernel's counters, which it resets itself) start at 0
  e = cudaMemsetAsync(dsched.p, 0, sizeof(FusedSched), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg.p, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd.p, descs.data(), descs.size() * sizeof(PassDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds.p, starts.data(), starts.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  const int mode = default_mode(dtype);
  sv_batch_stats bs{};
  // Every round's launch is queued without a host wait in between (each round's passes depend only on the
  // previous round, which the stream orders).  With more than one round the launches are captured once into
  // a CUDA graph on a private stream and the graph is launched on `st`; if capture is not possible the
  // rounds are launched directly.
  auto enqueue_rounds = [&](cudaStream_t q) {
    cudaError_t err = cudaSuccess;
    bs = sv_batch_stats{};
    for (size_t r = 0; r < rounds.size() && err == cudaSuccess; ++r) {
      const Round &R = rounds[r];
      int mixed = 0;
      if (R.npass > 0)
        err = launch_fused_batch((const PassDesc *)dd.p + R.desc_off, (const uint64_t *)ds.p + R.start_off, R.npass,
                                 R.total, mode, R.kmax, q, kDefaultF64Share, (FusedSched *)dsched.p, &mixed);
      if (err == cudaSuccess && R.tc_npass > 0) {
        err = launch_fused_batch_tc((const PassDesc *)dd.p + R.tc_desc_off, (const uint64_t *)ds.p + R.tc_start_off,
                                    R.tc_npass, R.tc_total, q, (FusedSched *)dsched.p);
        ++bs.tc_rounds;
      }
      ++bs.rounds;
      bs.mixed_rounds += (uint64_t)mixed;
      bs.max_round_chunks = std::max<uint64_t>(bs.max_round_chunks, R.total + R.tc_total);
      bs.total_chunks += R.total + R.tc_total;
    }
    return err;
  };
  bool launched = false;
  if (e == cudaSuccess && rounds.size() > 1) {
    // Shared-memory grants are raised outside the capture.
    for (const Round &R : rounds)
      if (R.npass > 0 && (e = prepare_fused_batch(mode, R.kmax)) != cudaSuccess) break;
    if (e == cudaSuccess && any_tc) e = prepare_fused_batch_tc();
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess) {
      if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const cudaError_t le = enqueue_rounds(cap);
        const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        if (le == cudaSuccess && ce == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          // the uploads above were queued on `st`; the graph runs after them on the same stream
          e = cudaGraphLaunch(exec, st);
          launched = true;
        }
      }
      cudaGetLastError();  // a failed capture leaves its error here; the direct path below reports its own
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
    }
    // The descriptor buffers are freed on return, so wait for the launches that read them (a graph exec may be
    // destroyed as soon as it is launched).
    if (launched && e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
  }
  if (!launched && e == cudaSuccess) {
    e = enqueue_rounds(st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  t_batch_stats = bs;
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "batched passes"));
  if (any_tc) {
    unsigned tc_err = 0;
    e = cudaMemcpy(&tc_err, &((FusedSched *)dsched.p)->tc_err, sizeof tc_err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "tensor-core error word"));
    if (tc_err) return cleanup(set_error(SV_ERR_TIMEOUT, "a wait for the tensor cores ran out in a batched pass"));
  }
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
namespace {

// Host-side check of a pass descriptor before it is handed to the batched kernel: every field the kernel
// indexes with must lie in range.  A descriptor that fails is never launched.
bool pass_is_sane(const PassDesc &d, int n) {
  if (!d.psi || d.n != n || d.k < 1 || d.k > kMaxChunkQubits || d.k > n || d.c < 0 || d.c > d.k) return false;
  if (d.ngates < 0 || (d.ngates > 0 && !d.gates)) return false;
  uint64_t mask = 0;
  for (int j = 0; j < d.k; ++j) {
    const int q = d.qpos[j];
    if (q < 0 || q >= n || (j > 0 && q <= d.qpos[j - 1]) || (j < d.c && q != j)) return false;
    mask |= 1ull << q;
  }
  return mask == d.qmask;
}

// Test hooks (host only; the GPU never sees the bad data): the ticket named by SV_FAULT_POISON_TICKET has its
// gate records overwritten in the queue before admission, the one named by SV_FAULT_CORRUPT_DESC_TICKET has
// its first pass descriptor corrupted before its first round.
uint64_t env_ticket(const char *name) {
  const char *v = std::getenv(name);
  return v ? (uint64_t)std::strtoull(v, nullptr, 10) : 0;
}

} // namespace

struct sv_server {
  struct Request {
    uint64_t ticket;
    int n;
    sv_dtype dtype;
    std::vector<sv_gate> gates;
  };
  struct Active {
    uint64_t ticket = 0;
    sv_state *st = nullptr;
    Plan plan;
    std::vector<unsigned char> blob;  // host copy of the gate blob (the source of its upload)
    void *d_gates = nullptr;          // device blob (stream-ordered allocation on the server stream)
    size_t launched = 0;              // passes queued so far
    int inflight = 0;                 // queued rounds not yet retired that hold one of its passes
    size_t bytes = 0;
    int mode = 0;
    int err = SV_OK;                  // set when the request failed; it leaves once `inflight` is 0
    std::string why;
  };
  // One queued round: host/device descriptor buffers, the event that marks its end, its members.
  struct Slot {
    PassDesc *h_desc = nullptr;
    uint64_t *h_start = nullptr;
    size_t cap = 0;
    DevBuf d_desc, d_start;
    cudaEvent_t ev = nullptr;
    std::vector<Active *> members;
    bool busy = false;
  };
  static constexpr int kSlots = 4;

  size_t budget = 0, used = 0;
  int max_active = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, std::pair<sv_state *, size_t>> done;
  std::unordered_map<uint64_t, std::pair<int, std::string>> failed;
  std::unordered_set<uint64_t> live;
  uint64_t next_ticket = 1;
  bool stop = false, paused = false;
  sv_server_stats stats{};
  std::thread th;
  cudaStream_t stream = nullptr;
  // loop-thread state (no lock needed)
  std::vector<Active *> active;
  Slot slots[kSlots];
  std::deque<int> queued;  // slot indices in launch order
  DevBuf d_sched;
  uint64_t poison = 0, corrupt = 0;

  ~sv_server() {
    for (Slot &sl : slots) {
      if (sl.h_desc) cudaFreeHost(sl.h_desc);
      if (sl.h_start) cudaFreeHost(sl.h_start);
      if (sl.ev) cudaEventDestroy(sl.ev);
    }
  }

  // Called with mu held.
  void record_failure(uint64_t ticket, int code, const std::string &msg) {
    failed[ticket] = {code, msg};
    ++stats.failed;
  }

  // Release an Active that left (finished or failed); its state goes to `done` or is destroyed.
  void retire_active(Active *a) {
    if (a->d_gates) cudaFreeAsync(a->d_gates, stream);
    a->d_gates = nullptr;
    if (a->err != SV_OK) {
      sv_destroy(a->st);  // waits for the server stream: outside the lock
      a->st = nullptr;
    } else {
      a->st->st_passes = (int)a->plan.passes.size();
    }
    std::lock_guard<std::mutex> lk(mu);
    if (a->err == SV_OK) {
      done[a->ticket] = {a->st, a->bytes};
      ++stats.completed;
    } else {
      record_failure(a->ticket, a->err, a->why);
      used -= a->bytes;
    }
    --stats.active;
    delete a;
  }

  // Admission of one popped request, outside the lock: state allocation, planning, gate upload.
  // Returns false if it must wait for memory (the request is put back in front of the queue).
  bool admit_one(Request &r) {
    const size_t bytes = amp_bytes(r.dtype) << r.n;
    std::string why;
    size_t bad = 0;
    int rc = validate_records(r.gates.data(), r.gates.size(), r.n, why, bad);
    if (rc != SV_OK) {
      std::lock_guard<std::mutex> lk(mu);
      used -= bytes;
      record_failure(r.ticket, rc, "gate " + std::to_string(bad) + " failed validation at admission: " + why);
      return true;
    }
    Active *a = new Active();
    a->ticket = r.ticket;
    a->bytes = bytes;
    a->mode = default_mode(r.dtype);
    rc = alloc_state(r.n, r.dtype, stream, &a->st, false);
    if (rc != SV_OK) {
      const std::string msg = sv_last_error();
      delete a;
      std::lock_guard<std::mutex> lk(mu);
      used -= bytes;
      if (rc == SV_ERR_OOM && !active.empty()) {  // wait for running requests to free memory
        pending.push_front(std::move(r));
        return false;
      }
      record_failure(r.ticket, rc, msg);
      return true;
    }
    plan_fresh(a->st, r.gates.data(), r.gates.size(), a->plan);
    const size_t gb = plan_blob_bytes(a->plan);
    cudaError_t e = cudaSuccess;
    if (gb > 0) {
      a->blob.resize(gb);
      plan_blob_fill(a->plan, a->blob.data());
      e = cudaMallocAsync(&a->d_gates, gb, stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(a->d_gates, a->blob.data(), gb, cudaMemcpyHostToDevice, stream);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (a->d_gates) cudaFreeAsync(a->d_gates, stream);
      sv_destroy(a->st);
      delete a;
      std::lock_guard<std::mutex> lk(mu);
      used -= bytes;
      record_failure(r.ticket, SV_ERR_OOM, "gate buffer allocation failed");
      return true;
    }
    if (r.ticket == corrupt && !a->plan.passes.empty()) a->plan.passes[0].k = 40;  // test hook (host only)
    active.push_back(a);
    std::lock_guard<std::mutex> lk(mu);
    ++stats.admitted;
    ++stats.active;
    return true;
  }

  int ensure_slot(Slot &sl, size_t m) {
    if (!sl.ev && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) return SV_ERR_CUDA;
    if (m > sl.cap) {
      if (sl.h_desc) cudaFreeHost(sl.h_desc);
      if (sl.h_start) cudaFreeHost(sl.h_start);
      sl.h_desc = nullptr;
      sl.h_start = nullptr;
      sl.cap = 0;
      const size_t c = std::max<size_t>(m, 64);
      if (cudaMallocHost(&sl.h_desc, c * sizeof(PassDesc)) != cudaSuccess ||
          cudaMallocHost(&sl.h_start, (c + 1) * sizeof(uint64_t)) != cudaSuccess)
        return SV_ERR_OOM;
      sl.cap = c;
    }
    if (sl.d_desc.ensure(sl.cap * sizeof(PassDesc), stream) != SV_OK ||
        sl.d_start.ensure((sl.cap + 1) * sizeof(uint64_t), stream) != SV_OK)
      return SV_ERR_OOM;
    return SV_OK;
  }

  // Queue one round of `mode`: the next pass of every active request of that mode with passes left.
  // Returns true if a round was queued.
  bool launch_round(int mode) {
    int si = -1;
    for (int i = 0; i < kSlots; ++i)
      if (!slots[i].busy) { si = i; break; }
    if (si < 0) return false;
    Slot &sl = slots[si];
    std::vector<Active *> members;
    for (Active *a : active)
      if (a->mode == mode && a->err == SV_OK && a->launched < a->plan.passes.size()) members.push_back(a);
    if (members.empty()) return false;
    if (ensure_slot(sl, members.size()) != SV_OK || d_sched.ensure(sizeof(FusedSched), stream) != SV_OK) {
      for (Active *a : members) { a->err = SV_ERR_OOM; a->why = "round descriptor allocation failed"; }
      return false;
    }
    uint64_t total = 0;
    int kmax = 0;
    size_t m = 0;
    sl.members.clear();
    for (Active *a : members) {
      PassDesc d = a->plan.passes[a->launched];
      d.psi = a->st->psi;
      plan_pass_pointers(a->plan, (int)a->launched, a->d_gates, d);
      if (!pass_is_sane(d, a->st->n)) {
        a->err = SV_ERR_ARG;
        a->why = "pass " + std::to_string(a->launched) + " failed the host's descriptor check; not launched";
        continue;
      }
      sl.h_desc[m] = d;
      sl.h_start[m] = total;
      total += 1ull << (d.n - d.k);
      kmax = std::max(kmax, d.k);
      sl.members.push_back(a);
      ++m;
    }
    if (m == 0) return false;
    sl.h_start[m] = total;
    cudaError_t e = cudaMemcpyAsync(sl.d_desc.p, sl.h_desc, m * sizeof(PassDesc), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sl.d_start.p, sl.h_start, (m + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, stream);
    int mixed = 0;
    if (e == cudaSuccess)
      e = launch_fused_batch((const PassDesc *)sl.d_desc.p, (const uint64_t *)sl.d_start.p, (int)m, total, mode, kmax,
                             stream, kDefaultF64Share, (FusedSched *)d_sched.p, &mixed);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      const std::string msg = std::string("serving round: ") + cudaGetErrorString(e);
      for (Active *a : sl.members) { a->err = SV_ERR_CUDA; a->why = msg; }
      sl.members.clear();
      return false;
    }
    for (Active *a : sl.members) {
      ++a->launched;
      ++a->inflight;
    }
    sl.busy = true;
    queued.push_back(si);
    std::lock_guard<std::mutex> lk(mu);
    ++stats.rounds;
    stats.mixed_rounds += (uint64_t)mixed;
    stats.max_round_chunks = std::max<uint64_t>(stats.max_round_chunks, total);
    return true;
  }

  // Wait for the oldest queued round and retire the requests whose last pass it held.
  void retire_oldest() {
    const int si = queued.front();
    queued.pop_front();
    Slot &sl = slots[si];
    const cudaError_t e = cudaEventSynchronize(sl.ev);
    for (Active *a : sl.members) {
      --a->inflight;
      if (e != cudaSuccess && a->err == SV_OK) {
        a->err = SV_ERR_CUDA;
        a->why = std::string("serving round: ") + cudaGetErrorString(e);
      }
    }
    sl.members.clear();
    sl.busy = false;
  }

  // Requests that finished (all passes queued and retired) or failed (nothing of theirs still queued) leave.
  void sweep_finished() {
    std::vector<Active *> keep;
    for (Active *a : active) {
      const bool finished = a->err == SV_OK && a->launched == a->plan.passes.size() && a->inflight == 0;
      const bool dead = a->err != SV_OK && a->inflight == 0;
      if (finished || dead) retire_active(a);
      else keep.push_back(a);
    }
    active.swap(keep);
  }

  void loop() {
    poison = env_ticket("SV_FAULT_POISON_TICKET");
    corrupt = env_ticket("SV_FAULT_CORRUPT_DESC_TICKET");
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      // Admission: pick requests under the lock (reserving their budget), do the work outside it.
      std::vector<Request> take;
      while (!paused && !pending.empty() && active.size() + take.size() < (size_t)max_active) {
        Request &r = pending.front();
        const size_t bytes = amp_bytes(r.dtype) << r.n;
        if (used + bytes > budget) break;
        used += bytes;
        if (r.ticket == poison && !r.gates.empty()) r.gates[0].target = 1000;  // test hook (host only)
        take.push_back(std::move(r));
        pending.pop_front();
      }
      stats.pending = pending.size();
      const bool stopping = stop;
      lk.unlock();
      for (size_t i = 0; i < take.size(); ++i)
        if (!admit_one(take[i])) {
          // put the rest back in order, behind the one admit_one returned to the front
          std::lock_guard<std::mutex> g(mu);
          for (size_t j = take.size(); j-- > i + 1;) {
            used -= amp_bytes(take[j].dtype) << take[j].n;
            pending.insert(pending.begin() + 1, std::move(take[j]));
          }
          break;
        }
      sweep_finished();
      // One round per dtype with work, while queue slots are free: complex64 and complex128 advance together.
      bool any = false;
      for (int mode : {(int)MODE_C64_F32, (int)MODE_C128_DF32})
        if (queued.size() < (size_t)kSlots) any |= launch_round(mode);
      // Keep at most two rounds ahead of the host; wait for the oldest when full or when nothing new was queued.
      if (!queued.empty() && (queued.size() >= 2 || !any)) retire_oldest();
      sweep_finished();
      lk.lock();
      if (active.empty() && queued.empty()) {
        if (stopping && pending.empty()) break;
        if (pending.empty() || paused) cv.wait_for(lk, std::chrono::milliseconds(2));
      }
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
    s->paused = false;
    for (const auto &r : s->pending) s->live.erase(r.ticket);
    s->pending.clear();
  }
  s->cv.notify_all();
  s->th.join();
  cudaStreamSynchronize(s->stream);
  for (auto &kv : s->done) sv_destroy(kv.second.first);
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
    ++s->stats.submitted;
    s->stats.pending = s->pending.size();
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

sv_status sv_server_pause(sv_server *s, int paused) {
  if (!s) return set_error(SV_ERR_ARG, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
  }
  s->cv.notify_all();
  return SV_OK;
}

sv_status sv_server_get_stats(sv_server *s, sv_server_stats *out) {
  if (!s || !out) return set_error(SV_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->pending = s->pending.size();
  out->budget_used = s->used;
  return SV_OK;
}

} // extern "C"
