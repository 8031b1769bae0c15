// C ABI: read-out in logical order, checkpoint write, norm, renormalisation and the CUDA-graph apply path.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "sv_state.h"

using namespace svi;

namespace {

constexpr uint64_t kReadChunk = 1ull << 22;  // amplitudes per gather round trip

bool identity_layout(const sv_state *s) {
  for (int t = 0; t < s->n; ++t)
    if (s->perm[t] != t) return false;
  return true;
}

int ensure_read_buffer(sv_state *s, size_t bytes) {
  if (bytes <= s->d_read_cap) return SV_OK;
  cudaError_t e;
  if (s->d_read) {
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "stream sync");
    cudaFree(s->d_read);
    s->d_read = nullptr;
    s->d_read_cap = 0;
  }
  if ((e = cudaMalloc(&s->d_read, bytes)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(SV_ERR_OOM, "read-out staging allocation failed");
  }
  s->d_read_cap = bytes;
  return SV_OK;
}

int check_range(const sv_state *s, uint64_t first, uint64_t count) {
  const uint64_t dim = 1ull << s->n;
  if (first > dim || count > dim - first) return set_error(SV_ERR_ARG, "index range exceeds 2^n");
  return SV_OK;
}

void free_entry(GraphEntry &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.d_gates) cudaFree(g.d_gates);
  for (cudaEvent_t ev : g.evs) cudaEventDestroy(ev);
  g.exec = nullptr;
  g.d_gates = nullptr;
  g.evs.clear();
}

uint64_t hash_bytes(const void *p, size_t n, uint64_t h) {
  const unsigned char *b = (const unsigned char *)p;
  for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  return h;
}

} // namespace

extern "C" {

sv_status sv_read_amplitudes(sv_state *s, uint64_t first, uint64_t count, void *host_out) {
  if (!s || (!host_out && count)) return set_error(SV_ERR_ARG, "NULL argument");
  int rc = check_range(s, first, count);
  if (rc != SV_OK) return rc;
  if (count == 0) return SV_OK;
  const size_t ab = amp_bytes(s->dtype);
  cudaError_t e;
  if (identity_layout(s)) {
    e = cudaMemcpyAsync(host_out, (const char *)s->psi + first * ab, count * ab, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? check_tc_error(s) : cuda_fail(e, "read amplitudes");
  }
  const uint64_t chunk = std::min<uint64_t>(count, kReadChunk);
  if ((rc = ensure_read_buffer(s, chunk * ab)) != SV_OK) return rc;
  for (uint64_t off = 0; off < count; off += chunk) {
    const uint64_t m = std::min(chunk, count - off);
    e = launch_gather(s->psi, s->n, mode_of(s), s->perm.data(), first + off, m, nullptr, s->d_read, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)host_out + off * ab, s->d_read, m * ab, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gather amplitudes");
  }
  return check_tc_error(s);
}

sv_status sv_read_amplitudes_at(sv_state *s, const uint64_t *idx, uint64_t count, void *host_out) {
  if (!s || ((!idx || !host_out) && count)) return set_error(SV_ERR_ARG, "NULL argument");
  const uint64_t dim = 1ull << s->n;
  for (uint64_t i = 0; i < count; ++i)
    if (idx[i] >= dim) return set_error(SV_ERR_ARG, "index " + std::to_string(i) + " out of range");
  if (count == 0) return SV_OK;
  const size_t ab = amp_bytes(s->dtype);
  const uint64_t chunk = std::min<uint64_t>(count, kReadChunk);
  int rc = ensure_read_buffer(s, chunk * (ab + sizeof(uint64_t)));
  if (rc != SV_OK) return rc;
  uint64_t *d_idx = (uint64_t *)((char *)s->d_read + chunk * ab);
  for (uint64_t off = 0; off < count; off += chunk) {
    const uint64_t m = std::min(chunk, count - off);
    cudaError_t e = cudaMemcpyAsync(d_idx, idx + off, m * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = launch_gather(s->psi, s->n, mode_of(s), s->perm.data(), 0, m, d_idx, s->d_read, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)host_out + off * ab, s->d_read, m * ab, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gather amplitudes");
  }
  return SV_OK;
}

sv_status sv_read_probabilities(sv_state *s, uint64_t first, uint64_t count, double *host_out) {
  if (!s || (!host_out && count)) return set_error(SV_ERR_ARG, "NULL argument");
  int rc = check_range(s, first, count);
  if (rc != SV_OK) return rc;
  if (count == 0) return SV_OK;
  const uint64_t chunk = std::min<uint64_t>(count, kReadChunk);
  if ((rc = ensure_read_buffer(s, chunk * sizeof(double))) != SV_OK) return rc;
  for (uint64_t off = 0; off < count; off += chunk) {
    const uint64_t m = std::min(chunk, count - off);
    cudaError_t e = launch_probs(s->psi, s->n, mode_of(s), s->perm.data(), first + off, m, (double *)s->d_read, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host_out + off, s->d_read, m * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "probabilities");
  }
  return SV_OK;
}

sv_status sv_write_amplitudes(sv_state *s, uint64_t first, uint64_t count, const void *host_in) {
  if (!s || (!host_in && count)) return set_error(SV_ERR_ARG, "NULL argument");
  int rc = check_range(s, first, count);
  if (rc != SV_OK) return rc;
  // Every component must be finite; complex128 components must also lie below 2^126 in magnitude, the range
  // in which the double-float working form (float exponents) and the sums of a pair update cannot overflow.
  if (s->dtype == SV_C128) {
    const double *v = (const double *)host_in;
    for (uint64_t i = 0; i < 2 * count; ++i)
      if (!std::isfinite(v[i]) || std::fabs(v[i]) >= 0x1p126)
        return set_error(SV_ERR_ARG, "amplitude " + std::to_string(first + i / 2) +
                                         " is not finite or has a component of magnitude >= 2^126");
  } else {
    const float *v = (const float *)host_in;
    for (uint64_t i = 0; i < 2 * count; ++i)
      if (!std::isfinite(v[i])) return set_error(SV_ERR_ARG, "amplitude " + std::to_string(first + i / 2) + " is not finite");
  }
  if (!identity_layout(s) && (rc = canonicalize_now(s)) != SV_OK) return rc;
  s->product = false;
  const size_t ab = amp_bytes(s->dtype);
  cudaError_t e = cudaMemcpyAsync((char *)s->psi + first * ab, host_in, count * ab, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "write amplitudes");
}

sv_status sv_norm(sv_state *s, double *out) {
  if (!s || !out) return set_error(SV_ERR_ARG, "NULL argument");
  const int src = ensure_scratch(s);
  if (src != SV_OK) return src;
  double *d_out = s->d_scalars + norm_parts();
  cudaError_t e = launch_norm(s->psi, s->n, mode_of(s), s->d_scalars, d_out, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? check_tc_error(s) : cuda_fail(e, "norm");
}

sv_status sv_expect_z(sv_state *s, uint64_t mask, double *out) {
  if (!s || !out) return set_error(SV_ERR_ARG, "NULL argument");
  if (s->n < 64 && (mask >> s->n) != 0) return set_error(SV_ERR_ARG, "mask names qubits >= n");
  uint64_t pmask = 0;  // the same qubits, as physical index bits
  for (int t = 0; t < s->n; ++t)
    if (mask >> t & 1ull) pmask |= 1ull << s->perm[t];
  const int src = ensure_scratch(s);
  if (src != SV_OK) return src;
  double *d_out = s->d_scalars + norm_parts();
  cudaError_t e = launch_norm(s->psi, s->n, mode_of(s), s->d_scalars, d_out, s->stream, pmask);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "expectation");
}

sv_status sv_sample(sv_state *s, const double *u, uint64_t count, uint64_t *out) {
  if (!s || ((!u || !out) && count)) return set_error(SV_ERR_ARG, "NULL argument");
  for (uint64_t i = 0; i < count; ++i)
    if (!(u[i] >= 0.0 && u[i] < 1.0)) return set_error(SV_ERR_ARG, "u[" + std::to_string(i) + "] is not in [0, 1)");
  if (count == 0) return SV_OK;
  const int b = s->n < 10 ? s->n : 10;
  const uint64_t nblocks = 1ull << (s->n - b);
  double *d_blocks = nullptr;
  cudaError_t e = cudaMalloc(&d_blocks, nblocks * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(SV_ERR_OOM, "sampling scratch allocation failed");
  }
  std::vector<double> blocks(nblocks);
  e = launch_block_probs(s->psi, s->n, mode_of(s), s->perm.data(), b, d_blocks, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(blocks.data(), d_blocks, nblocks * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(d_blocks);
  if (e != cudaSuccess) return cuda_fail(e, "block probabilities");
  // Inclusive prefix sums over the blocks (FP64, logical order) and one binary search per shot.
  for (uint64_t j = 1; j < nblocks; ++j) blocks[j] += blocks[j - 1];
  const double total = blocks[nblocks - 1];
  if (!(total > 0.0)) return set_error(SV_ERR_ARG, "the state has zero norm");
  const uint64_t chunk = std::min<uint64_t>(count, kReadChunk);
  int rc = ensure_read_buffer(s, chunk * 3 * sizeof(uint64_t));
  if (rc != SV_OK) return rc;
  uint64_t *d_blk = (uint64_t *)s->d_read;
  double *d_res = (double *)(d_blk + chunk);
  uint64_t *d_out = (uint64_t *)(d_res + chunk);
  std::vector<uint64_t> blk(chunk);
  std::vector<double> res(chunk);
  for (uint64_t off = 0; off < count; off += chunk) {
    const uint64_t m = std::min(chunk, count - off);
    for (uint64_t i = 0; i < m; ++i) {
      const double target = u[off + i] * total;
      const uint64_t j = (uint64_t)(std::upper_bound(blocks.begin(), blocks.end(), target) - blocks.begin());
      const uint64_t jj = j < nblocks ? j : nblocks - 1;
      blk[i] = jj;
      res[i] = target - (jj > 0 ? blocks[jj - 1] : 0.0);
    }
    e = cudaMemcpyAsync(d_blk, blk.data(), m * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_res, res.data(), m * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = launch_sample_block(s->psi, s->n, mode_of(s), s->perm.data(), b, d_blk, d_res, m, d_out, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + off, d_out, m * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sampling");
  }
  return SV_OK;
}

sv_status sv_renormalize(sv_state *s) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  s->product = false;
  const int src = ensure_scratch(s);
  if (src != SV_OK) return src;
  double *d_out = s->d_scalars + norm_parts();
  cudaError_t e = launch_norm(s->psi, s->n, mode_of(s), s->d_scalars, d_out, s->stream);
  if (e == cudaSuccess) e = launch_scale(s->psi, s->n, mode_of(s), d_out, s->stream);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "renormalise");
}

// Capture the planned launches once per (gates, layout, state, options) and replay the graph afterwards.
sv_status sv_apply_circuit_graph(sv_state *s, const sv_gate *gates, size_t ngates) {
  if (!s || (!gates && ngates)) return set_error(SV_ERR_ARG, "NULL argument");
  {
    std::string why;
    size_t bad = 0;
    const int rc = validate_records(gates, ngates, s->n, why, bad);
    if (rc != SV_OK) return set_error(rc, "gate " + std::to_string(bad) + ": " + why);
  }
  int src = ensure_scratch(s);
  if (src != SV_OK) return src;
  std::vector<sv_gate> rest;
  const int prc = product_prologue(s, gates, ngates, rest);
  if (prc != SV_OK) return prc;
  if (ngates == 0 && s->st_absorbed > 0) {  // everything folded into a product state: nothing to capture
    s->st_passes = s->st_fused = s->st_sweeps = s->st_relabels = s->st_remaps = 0;
    s->last_evs = nullptr;
    s->last_kind.clear();
    return SV_OK;
  }
  const PlanConfig cfg = plan_config(s);
  // The key material: gate records, layout, options and the state's address, hashed (FNV-1a) to find the
  // entry and compared byte for byte before a replay.
  const int opts[8] = {s->n, mode_of(s), cfg.k, cfg.c, (int)cfg.fusion, s->canonical, f64_share_of(s), (int)cfg.cubes};
  std::vector<unsigned char> kb(ngates * sizeof(sv_gate) + s->perm.size() * sizeof(int) + sizeof opts + sizeof s->psi);
  {
    unsigned char *q = kb.data();
    if (ngates) std::memcpy(q, gates, ngates * sizeof(sv_gate));
    q += ngates * sizeof(sv_gate);
    std::memcpy(q, s->perm.data(), s->perm.size() * sizeof(int));
    q += s->perm.size() * sizeof(int);
    std::memcpy(q, opts, sizeof opts);
    q += sizeof opts;
    std::memcpy(q, &s->psi, sizeof s->psi);
  }
  uint64_t key = hash_bytes(kb.data(), kb.size(), 1469598103934665603ull);
  // Test hook: with SV_TEST_GRAPH_KEY_COLLIDE set every circuit gets the same key, as a hash collision would.
  if (std::getenv("SV_TEST_GRAPH_KEY_COLLIDE")) key = 42;
  auto it = s->graphs.find(key);
  cudaError_t e;
  if (it != s->graphs.end() && it->second.key_bytes == kb && (it->second.evs.empty() != (s->profile != 0))) {
    if ((e = cudaGraphLaunch(it->second.exec, s->stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
    s->perm = it->second.perm_after;
    s->last_evs = it->second.evs.empty() ? nullptr : it->second.evs.data();
    s->last_kind = it->second.ev_kind;
    return SV_OK;
  }
  if (it != s->graphs.end()) {  // same key with other contents (a collision) or profiling setting: replace it
    cudaStreamSynchronize(s->stream);
    free_entry(it->second);
    s->graphs.erase(it);
  }
  if (s->graphs.size() >= 64) {
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->graphs) free_entry(kv.second);
    s->graphs.clear();
  }
  GraphEntry ent;
  ent.perm_before = s->perm;
  ent.key_bytes = std::move(kb);
  std::vector<int> perm = s->perm;
  Plan P;
  make_plan(s->n, cfg, perm, gates, ngates, P);
  if (plan_blob_bytes(P) > 0) {
    if ((e = cudaMalloc(&ent.d_gates, plan_blob_bytes(P))) != cudaSuccess)
      return set_error(SV_ERR_OOM, "graph gate buffer allocation failed");
    std::vector<unsigned char> blob(plan_blob_bytes(P));
    plan_blob_fill(P, blob.data());
    if ((e = cudaMemcpy(ent.d_gates, blob.data(), blob.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
      cudaFree(ent.d_gates);
      return cuda_fail(e, "graph gate upload");
    }
  }
  if (s->profile) {
    for (size_t i = 0; i < 2 * P.steps.size(); ++i) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
        for (cudaEvent_t x : ent.evs) cudaEventDestroy(x);
        cudaFree(ent.d_gates);
        return cuda_fail(e, "profiling event");
      }
      ent.evs.push_back(ev);
    }
    ent.ev_kind = step_kinds(P);
  }
  cudaStream_t cap = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
    free_entry(ent);
    return cuda_fail(e, "capture stream");
  }
  // Renormalisation is not part of a captured graph.
  const int64_t saved_period = s->renorm_period;
  s->renorm_period = 0;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  int rc = SV_OK;
  if (e == cudaSuccess) {
    rc = run_plan(s, P, ent.d_gates, cap, ent.evs.empty() ? nullptr : ent.evs.data(), true);
    if (rc == SV_OK && s->canonical) rc = canonicalize_on(s, perm, cap, nullptr);
    e = cudaStreamEndCapture(cap, &graph);
  }
  s->renorm_period = saved_period;
  cudaStreamDestroy(cap);
  if (rc != SV_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    free_entry(ent);
    return rc != SV_OK ? rc : cuda_fail(e, "stream capture");
  }
  e = cudaGraphInstantiate(&ent.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    free_entry(ent);
    return cuda_fail(e, "graph instantiate");
  }
  ent.perm_after = perm;
  if ((e = cudaGraphLaunch(ent.exec, s->stream)) != cudaSuccess) {
    free_entry(ent);
    return cuda_fail(e, "graph launch");
  }
  s->perm = perm;
  s->st_passes = (int)P.passes.size();
  s->st_fused = P.n_fused_gates;
  s->st_sweeps = P.n_sweep_gates;
  s->st_relabels = P.n_relabels;
  s->st_blocks = P.n_blocks;
  s->st_block_gates = P.n_block_gates;
  auto ins = s->graphs.emplace(key, std::move(ent));
  s->last_evs = ins.first->second.evs.empty() ? nullptr : ins.first->second.evs.data();
  s->last_kind = ins.first->second.ev_kind;
  return SV_OK;
}

} // extern "C"
