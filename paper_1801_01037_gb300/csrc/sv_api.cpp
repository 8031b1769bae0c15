// C ABI: handles, host-side validation, planning and launch of the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sv_state.h"

using namespace svi;

namespace svi {

static thread_local std::string g_err;

int set_error(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return set_error(SV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t amp_bytes(sv_dtype dt) { return dt == SV_C64 ? 8 : 16; }

int mode_of(const sv_state *s) {
  if (s->dtype == SV_C64) return MODE_C64_F32;
  return s->arith == SV_ARITH_F64 ? MODE_C128_F64 : MODE_C128_DF32;
}

int check_device() {
  static std::once_flag once;
  static int status = SV_OK;
  static std::string why;
  std::call_once(once, [] {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
      status = SV_ERR_NO_DEVICE;
      why = std::string("no CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "count = 0");
      return;
    }
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
      status = SV_ERR_NO_DEVICE;
      why = "the kernels are built for sm_103a only; device is sm_" + std::to_string(major * 10 + minor);
    }
  });
  if (status != SV_OK) return set_error(status, why);
  return SV_OK;
}

PlanConfig plan_config(const sv_state *s) {
  PlanConfig c;
  // Measured defaults (20 random layers, GB300): c128 k = 12 at every n; c64 k = 13 from n = 23 on, but
  // k = 12 below (n = 20: 0.57 vs 0.69 ms; with fewer amplitudes the smaller chunks keep more CTAs busy).
  if (s->dtype == SV_C64) { c.k = s->n <= 22 ? 12 : 13; c.c = 5; }
  else { c.k = 12; c.c = 4; }
  if (s->chunk_k > 0) c.k = s->chunk_k;
  c.fusion = s->fusion != 0;
  c.cubes = s->dtype == SV_C64 && s->cubes != 0;
  // Dense tensor-core blocks: complex64, and complex128 in double-float arithmetic with chunks of at most 2^12
  // amplitudes (the digit planes of larger chunks do not fit in shared memory).
  if (s->tensor_blocks && s->dtype == SV_C64) c.block_mode = MODE_C64_F32;
  if (s->tensor_blocks && mode_of(s) == MODE_C128_DF32 && c.k <= 12) c.block_mode = MODE_C128_DF32;
  if (s->tensor_blocks >= 2) c.block_min_cost = (double)s->tensor_blocks;
  return c;
}

int check_tc_error(sv_state *s) {
  if (!s->tc_used || !s->d_sched) return SV_OK;
  unsigned err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, &s->d_sched->tc_err, sizeof err, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core error word");
  if (err == 0) return SV_OK;
  cudaMemsetAsync(&s->d_sched->tc_err, 0, sizeof err, s->stream);
  return set_error(SV_ERR_TIMEOUT, "a tensor-core pass gave up waiting for its MMAs; the state is not valid");
}

int upload_plan(sv_state *s, const Plan &P, void **d_blob) {
  const size_t total = plan_blob_bytes(P);
  *d_blob = nullptr;
  if (total == 0) return SV_OK;
  cudaError_t e;
  if (s->stage_pending) {
    if ((e = cudaEventSynchronize(s->stage_ev)) != cudaSuccess) return cuda_fail(e, "gate staging wait");
    s->stage_pending = false;
  }
  if (total > s->d_gates_cap) {
    if (s->d_gates) {
      if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "stream sync");
      cudaFree(s->d_gates);
      s->d_gates = nullptr;
    }
    const size_t cap = std::max<size_t>(total, 64 << 10);
    if ((e = cudaMalloc(&s->d_gates, cap)) != cudaSuccess) {
      s->d_gates_cap = 0;
      return set_error(SV_ERR_OOM, "device gate buffer allocation failed");
    }
    s->d_gates_cap = cap;
  }
  if (total > s->h_stage_cap) {
    if (s->h_stage) cudaFreeHost(s->h_stage);
    s->h_stage = nullptr;
    const size_t cap = std::max<size_t>(total, 64 << 10);
    if ((e = cudaMallocHost(&s->h_stage, cap)) != cudaSuccess) {
      s->h_stage_cap = 0;
      return set_error(SV_ERR_OOM, "pinned gate staging allocation failed");
    }
    s->h_stage_cap = cap;
  }
  plan_blob_fill(P, s->h_stage);
  if ((e = cudaMemcpyAsync(s->d_gates, s->h_stage, total, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
    return cuda_fail(e, "gate upload");
  if ((e = cudaEventRecord(s->stage_ev, s->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  s->stage_pending = true;
  *d_blob = s->d_gates;
  return SV_OK;
}

int f64_share_of(const sv_state *s) { return s->f64_share >= 0 ? s->f64_share : kDefaultF64Share; }

int ensure_scratch(sv_state *s) {
  cudaError_t e;
  if (!s->d_scalars && (e = cudaMalloc(&s->d_scalars, sizeof(double) * (norm_parts() + 1))) != cudaSuccess) {
    s->d_scalars = nullptr;
    return cuda_fail(e, "state scratch allocation");
  }
  if (!s->d_sched) {
    if ((e = cudaMalloc(&s->d_sched, sizeof(FusedSched))) != cudaSuccess) {
      s->d_sched = nullptr;
      return cuda_fail(e, "state scratch allocation");
    }
    if ((e = cudaMemsetAsync(s->d_sched, 0, sizeof(FusedSched), s->stream)) != cudaSuccess)
      return cuda_fail(e, "state scratch initialisation");
  }
  if (!s->stage_ev && (e = cudaEventCreateWithFlags(&s->stage_ev, cudaEventDisableTiming)) != cudaSuccess) {
    s->stage_ev = nullptr;
    return cuda_fail(e, "state scratch allocation");
  }
  return SV_OK;
}

int maybe_renormalize(sv_state *s, int applied) {
  if (s->renorm_period <= 0) return SV_OK;
  s->gates_since_renorm += applied;
  if (s->gates_since_renorm < s->renorm_period) return SV_OK;
  s->gates_since_renorm = 0;
  cudaError_t e = launch_norm(s->psi, s->n, mode_of(s), s->d_scalars, s->d_scalars + norm_parts(), s->stream);
  if (e == cudaSuccess) e = launch_scale(s->psi, s->n, mode_of(s), s->d_scalars + norm_parts(), s->stream);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "renormalise");
}

int ensure_event_pool(sv_state *s, size_t steps) {
  while (s->ev_pool.size() < 2 * steps) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(e, "profiling event");
    s->ev_pool.push_back(ev);
  }
  return SV_OK;
}

std::vector<int> step_kinds(const Plan &P) {
  std::vector<int> k;
  for (const Step &st : P.steps) k.push_back((int)st.kind);
  return k;
}

int run_plan(sv_state *s, const Plan &P, const void *d_blob, cudaStream_t st, const cudaEvent_t *evs,
             bool capturing) {
  const int mode = mode_of(s);
  const unsigned rec_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  for (size_t si = 0; si < P.steps.size(); ++si) {
    const Step &step = P.steps[si];
    cudaError_t e = cudaSuccess;
    if (evs && (e = cudaEventRecordWithFlags(evs[2 * si], st, rec_flags)) != cudaSuccess)
      return cuda_fail(e, "profiling event");
    if (step.kind == Step::FUSED) {
      PassDesc d = P.passes[step.index];
      d.psi = s->psi;
      plan_pass_pointers(P, step.index, d_blob, d);
      // A pass of pure exchanges (X / CNOT / Toffoli) moves doubles as they are: bit-exact in every mode.
      bool moves_only = mode == MODE_C128_DF32;
      for (int i = 0; moves_only && i < d.ngates; ++i)
        moves_only = P.fused_gates[P.pass_gate_offset[step.index] + i].cls == GC_X;
      e = launch_fused(d, moves_only ? (int)MODE_C128_F64 : mode, st, f64_share_of(s), s->d_sched);
      if (d.nblocks > 0) s->tc_used = true;
    } else {
      e = launch_sweep(s->psi, s->n, mode, P.sweep_gates[step.index], st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (evs && (e = cudaEventRecordWithFlags(evs[2 * si + 1], st, rec_flags)) != cudaSuccess)
      return cuda_fail(e, "profiling event");
    if (st == s->stream) {
      const int rc = maybe_renormalize(s, step.ngates);
      if (rc != SV_OK) return rc;
    }
  }
  return SV_OK;
}

int canonicalize_on(sv_state *s, std::vector<int> &perm, cudaStream_t st, int *npasses) {
  // Pure data movement: complex128 passes move doubles untouched (FP64 working form, no conversion).
  const int mode = mode_of(s) == MODE_C64_F32 ? (int)MODE_C64_F32 : (int)MODE_C128_F64;
  const std::vector<PassDesc> passes = canonicalize_passes(s->n, plan_config(s), perm);
  for (PassDesc d : passes) {
    d.psi = s->psi;
    cudaError_t e = launch_fused(d, mode, st);
    if (e != cudaSuccess) return cuda_fail(e, "bit-permutation pass");
  }
  if (npasses) *npasses = (int)passes.size();
  return SV_OK;
}

int canonicalize_now(sv_state *s) {
  int np = 0;
  const int rc = canonicalize_on(s, s->perm, s->stream, &np);
  s->st_remaps += np;
  return rc;
}

// ---- Product states (Sec. V: a state without entanglement is the Kronecker product of one-qubit states) ----

void set_basis_product(sv_state *s, uint64_t x) {
  s->pf.assign(4 * (size_t)s->n, 0.0);
  s->pm.assign(8 * (size_t)s->n, 0.0);
  for (int t = 0; t < s->n; ++t) {
    s->pf[4 * t + ((x >> t) & 1ull ? 2 : 0)] = 1.0;
    s->pm[8 * t + 0] = 1.0;  // M_t = identity
    s->pm[8 * t + 6] = 1.0;
  }
  s->product = true;
}

// Form psi = (x)_t M_t f_t on the GPU (every amplitude is written).
int expand_product(sv_state *s) {
  const size_t head = 12 * (size_t)s->n * sizeof(double);
  const size_t need = head + product_table_entries(s->n) * 2 * sizeof(double);
  cudaError_t e;
  if (s->d_prod_cap < need) {
    if (s->d_prod) {
      if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "stream sync");
      cudaFree(s->d_prod);
      s->d_prod = nullptr;
      s->d_prod_cap = 0;
    }
    if ((e = cudaMalloc(&s->d_prod, need)) != cudaSuccess) return set_error(SV_ERR_OOM, "product-state scratch allocation failed");
    s->d_prod_cap = need;
  }
  std::vector<double> fm(12 * (size_t)s->n);
  for (int t = 0; t < s->n; ++t) {
    std::memcpy(&fm[12 * t], &s->pf[4 * t], 4 * sizeof(double));
    std::memcpy(&fm[12 * t + 4], &s->pm[8 * t], 8 * sizeof(double));
  }
  // Pageable source: the call returns once the bytes are staged, so `fm` may go out of scope.
  if ((e = cudaMemcpyAsync(s->d_prod, fm.data(), head, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
    return cuda_fail(e, "product factors upload");
  for (int t = 0; t < s->n; ++t) s->perm[t] = t;
  e = launch_init_product(s->psi, s->n, mode_of(s), (const double *)s->d_prod, (char *)s->d_prod + head, s->stream);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "product state");
}

// While the state is a product state, move every single-qubit gate (and SWAP) that acts only on qubits no
// earlier remaining gate touches to the front and fold it into the qubits' factors: M_t <- U M_t (FP64), SWAP
// exchanges two qubits' factors.  Gates on disjoint qubits commute, so the order of the rest is kept and the
// result is unchanged.  `rest` receives the remaining records in order; returns the number folded.
int absorb_leading(int n, const sv_gate *gates, size_t ngates, std::vector<double> &pf, std::vector<double> &pm,
                   std::vector<sv_gate> &rest) {
  std::vector<char> touched(n, 0);
  int folded = 0;
  rest.clear();
  for (size_t i = 0; i < ngates; ++i) {
    const sv_gate &g = gates[i];
    if (g.kind == SV_GATE_U && g.ncontrols == 0 && !touched[g.target]) {
      double *m = &pm[8 * (size_t)g.target];
      double r[8];
      for (int row = 0; row < 2; ++row)
        for (int col = 0; col < 2; ++col) {
          double re = 0.0, im = 0.0;
          for (int j = 0; j < 2; ++j) {
            const double ur = g.U[4 * row + 2 * j], ui = g.U[4 * row + 2 * j + 1];
            const double mr = m[4 * j + 2 * col], mi = m[4 * j + 2 * col + 1];
            re += ur * mr - ui * mi;
            im += ur * mi + ui * mr;
          }
          r[4 * row + 2 * col] = re;
          r[4 * row + 2 * col + 1] = im;
        }
      std::memcpy(m, r, sizeof r);
      ++folded;
      continue;
    }
    if (g.kind == SV_GATE_SWAP && !touched[g.target] && !touched[g.target2]) {
      for (int j = 0; j < 4; ++j) std::swap(pf[4 * (size_t)g.target + j], pf[4 * (size_t)g.target2 + j]);
      for (int j = 0; j < 8; ++j) std::swap(pm[8 * (size_t)g.target + j], pm[8 * (size_t)g.target2 + j]);
      ++folded;
      continue;
    }
    touched[g.target] = 1;
    if (g.kind == SV_GATE_SWAP || g.kind == SV_GATE_U4) touched[g.target2] = 1;
    for (int c = 0; c < g.ncontrols; ++c) touched[g.controls[c]] = 1;
    rest.push_back(g);
    if (g.kind == SV_GATE_U4)  // its three row records go along (validated: they follow)
      for (int r = 1; r < 4; ++r) rest.push_back(gates[++i]);
  }
  return folded;
}

// Apply-call prologue for product states: fold what can be folded, re-form the amplitudes, and point
// (gates, ngates) at the remaining records (kept in `rest`).  Re-forming costs one write of the state, so
// the fold is taken when it leaves nothing else to run or folds at least max(2, n/4) gates (a gate inside a
// fused pass costs a fraction of a pass).  The state stays a product state only if nothing remains.
int product_prologue(sv_state *s, const sv_gate *&gates, size_t &ngates, std::vector<sv_gate> &rest) {
  s->st_absorbed = 0;
  if (!s->product || ngates == 0) return SV_OK;
  if (!s->product_start) {
    s->product = false;
    return SV_OK;
  }
  std::vector<double> pf = s->pf, pm = s->pm;
  const int folded = absorb_leading(s->n, gates, ngates, pf, pm, rest);
  if (folded > 0 && (rest.empty() || folded >= std::max(2, s->n / 4))) {
    s->pf.swap(pf);
    s->pm.swap(pm);
    const int rc = expand_product(s);
    if (rc != SV_OK) return rc;
    s->st_absorbed = folded;
    gates = rest.data();
    ngates = rest.size();
  }
  if (ngates > 0) s->product = false;
  return SV_OK;
}

int alloc_state(int n, sv_dtype dt, cudaStream_t st, sv_state **out, bool init_zero) {
  const size_t bytes = amp_bytes(dt) << n;
  // Host-side failure injection for tests: with SV_FAULT_ALLOC set, every state allocation fails as if
  // the device were out of memory (nothing is launched, the GPU is not touched).
  if (std::getenv("SV_FAULT_ALLOC")) return set_error(SV_ERR_OOM, "allocation failure injected (SV_FAULT_ALLOC)");
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
  if (bytes > free_b) return set_error(SV_ERR_OOM, "state of " + std::to_string(bytes) + " bytes exceeds free device memory");
  sv_state *s = new sv_state();
  s->n = n;
  s->dtype = dt;
  s->stream = st;
  s->perm.resize(n);
  for (int t = 0; t < n; ++t) s->perm[t] = t;
  if ((e = cudaMalloc(&s->psi, bytes)) != cudaSuccess) {
    delete s;
    cudaGetLastError();
    return set_error(SV_ERR_OOM, "cudaMalloc of the state failed");
  }
  int rc = ensure_scratch(s);
  if (rc != SV_OK) {
    sv_destroy(s);
    return rc;
  }
  if (init_zero) {
    if ((e = launch_init_basis(s->psi, n, mode_of(s), 0, st)) != cudaSuccess) {
      sv_destroy(s);
      return cuda_fail(e, "init");
    }
    set_basis_product(s, 0);
  }
  *out = s;
  return SV_OK;
}

} // namespace svi

// =========================================================================================================
extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }
const char *sv_version(void) { return "gb300-statevec 0.1 (sm_103a)"; }

static bool bad_dtype(sv_dtype dt) { return dt != SV_C64 && dt != SV_C128; }

sv_status sv_create(int n, sv_dtype dtype, void *stream, sv_state **out) {
  if (!out) return set_error(SV_ERR_ARG, "out is NULL");
  if (n < 1 || n > kMaxQubits) return set_error(SV_ERR_ARG, "n must be in [1, 36]");
  if (bad_dtype(dtype)) return set_error(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
  int rc = check_device();
  if (rc != SV_OK) return rc;
  return alloc_state(n, dtype, (cudaStream_t)stream, out, true);
}

sv_status sv_create_from_buffer(int n, sv_dtype dtype, void *dev_ptr, void *stream, sv_state **out) {
  if (!out || !dev_ptr) return set_error(SV_ERR_ARG, "out or dev_ptr is NULL");
  if (n < 1 || n > kMaxQubits) return set_error(SV_ERR_ARG, "n must be in [1, 36]");
  if (bad_dtype(dtype)) return set_error(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
  if (((uintptr_t)dev_ptr & 15u) != 0) return set_error(SV_ERR_ARG, "dev_ptr must be 16-byte aligned");
  int rc = check_device();
  if (rc != SV_OK) return rc;
  sv_state *s = new sv_state();
  s->n = n;
  s->dtype = dtype;
  s->stream = (cudaStream_t)stream;
  s->psi = dev_ptr;
  s->owned = false;
  s->canonical = 1;
  s->perm.resize(n);
  for (int t = 0; t < n; ++t) s->perm[t] = t;
  if ((rc = ensure_scratch(s)) != SV_OK) {
    sv_destroy(s);
    return rc;
  }
  *out = s;
  return SV_OK;
}

sv_status sv_destroy(sv_state *s) {
  if (!s) return SV_OK;
  cudaStreamSynchronize(s->stream);
  for (auto &kv : s->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.d_gates) cudaFree(kv.second.d_gates);
  }
  if (s->owned && s->psi) cudaFree(s->psi);
  if (s->d_gates) cudaFree(s->d_gates);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->d_scalars) cudaFree(s->d_scalars);
  if (s->d_sched) cudaFree(s->d_sched);
  if (s->d_read) cudaFree(s->d_read);
  if (s->d_prod) cudaFree(s->d_prod);
  if (s->stage_ev) cudaEventDestroy(s->stage_ev);
  for (cudaEvent_t ev : s->ev_pool) cudaEventDestroy(ev);
  for (auto &kv : s->graphs)
    for (cudaEvent_t ev : kv.second.evs) cudaEventDestroy(ev);
  delete s;
  return SV_OK;
}

sv_status sv_init_basis(sv_state *s, uint64_t x) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  if (x >= (1ull << s->n)) return set_error(SV_ERR_ARG, "basis index out of range");
  for (int t = 0; t < s->n; ++t) s->perm[t] = t;
  s->gates_since_renorm = 0;
  cudaError_t e = launch_init_basis(s->psi, s->n, mode_of(s), x, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init");
  set_basis_product(s, x);
  return SV_OK;
}

sv_status sv_init_product(sv_state *s, const double *factors) {
  if (!s || !factors) return set_error(SV_ERR_ARG, "NULL argument");
  for (int t = 0; t < s->n; ++t) {
    const double *f = factors + 4 * t;
    double nrm = 0.0;
    for (int j = 0; j < 4; ++j) {
      if (!std::isfinite(f[j])) return set_error(SV_ERR_ARG, "factor " + std::to_string(t) + " is not finite");
      nrm += f[j] * f[j];
    }
    if (std::fabs(nrm - 1.0) > 1e-10) return set_error(SV_ERR_ARG, "factor " + std::to_string(t) + " is not normalised");
  }
  set_basis_product(s, 0);
  std::memcpy(s->pf.data(), factors, 4 * (size_t)s->n * sizeof(double));
  s->gates_since_renorm = 0;
  const int rc = expand_product(s);
  if (rc != SV_OK) s->product = false;
  return rc;
}

sv_status sv_set_option(sv_state *s, int option, int64_t value) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  switch (option) {
    case SV_OPT_ARITH:
      if (value != SV_ARITH_AUTO && value != SV_ARITH_F64 && value != SV_ARITH_DF32)
        return set_error(SV_ERR_ARG, "bad arithmetic mode");
      s->arith = (int)value;
      return SV_OK;
    case SV_OPT_CHUNK_QUBITS:
      if (value != 0 && (value < 6 || value > kMaxChunkQubits)) return set_error(SV_ERR_ARG, "chunk qubits must be 0 or 6..13");
      s->chunk_k = (int)value;
      return SV_OK;
    case SV_OPT_FUSION: s->fusion = value ? 1 : 0; return SV_OK;
    case SV_OPT_CUBES: s->cubes = value ? 1 : 0; return SV_OK;
    case SV_OPT_TENSOR_BLOCKS:
      if (value < 0 || value > 64) return set_error(SV_ERR_ARG, "tensor blocks: 0 (off), 1 (on) or 2..64 (minimum size)");
      s->tensor_blocks = (int)value;
      return SV_OK;
    case SV_OPT_PRODUCT_START: s->product_start = value ? 1 : 0; return SV_OK;
    case SV_OPT_PROFILE: s->profile = value ? 1 : 0; return SV_OK;
    case SV_OPT_F64_SHARE:
      if (value < -1 || value > 99) return set_error(SV_ERR_ARG, "FP64 share must be -1 (default) or 0..99 percent");
      s->f64_share = (int)value;
      return SV_OK;
    case SV_OPT_RENORM_PERIOD:
      if (value < 0) return set_error(SV_ERR_ARG, "renormalisation period must be >= 0");
      s->renorm_period = value;
      return SV_OK;
    case SV_OPT_CANONICAL:
      if (!s->owned && !value) return set_error(SV_ERR_ARG, "buffer states stay in logical order");
      s->canonical = value ? 1 : 0;
      return SV_OK;
    default: return set_error(SV_ERR_ARG, "unknown option");
  }
}

sv_status sv_get_info(sv_state *s, int *n, sv_dtype *dtype, void **dev_ptr) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  if (n) *n = s->n;
  if (dtype) *dtype = s->dtype;
  if (dev_ptr) *dev_ptr = s->psi;
  return SV_OK;
}

sv_status sv_get_layout(sv_state *s, int *perm) {
  if (!s || !perm) return set_error(SV_ERR_ARG, "NULL argument");
  for (int t = 0; t < s->n; ++t) perm[t] = s->perm[t];
  return SV_OK;
}

sv_status sv_canonicalize(sv_state *s) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  return canonicalize_now(s);
}

static int apply_records(sv_state *s, const sv_gate *gates, size_t ngates, bool single) {
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
  PlanConfig cfg = plan_config(s);
  if (single) cfg.fusion = false;
  Plan P;
  make_plan(s->n, cfg, s->perm, gates, ngates, P);
  void *d_blob = nullptr;
  int rc = upload_plan(s, P, &d_blob);
  if (rc != SV_OK) return rc;
  const cudaEvent_t *evs = nullptr;
  s->last_evs = nullptr;
  s->last_kind.clear();
  if (s->profile) {
    if ((rc = ensure_event_pool(s, P.steps.size())) != SV_OK) return rc;
    evs = s->ev_pool.data();
    s->last_evs = evs;
    s->last_kind = step_kinds(P);
  }
  rc = run_plan(s, P, d_blob, s->stream, evs, false);
  if (rc != SV_OK) return rc;
  s->st_passes = (int)P.passes.size();
  s->st_fused = P.n_fused_gates;
  s->st_sweeps = P.n_sweep_gates;
  s->st_relabels = P.n_relabels;
  s->st_blocks = P.n_blocks;
  s->st_block_gates = P.n_block_gates;
  s->st_remaps = 0;
  if (s->canonical) return canonicalize_now(s);
  return SV_OK;
}

sv_status sv_apply_gate(sv_state *s, const double *U, int target, const int *controls, int ncontrols) {
  if (!s || !U) return set_error(SV_ERR_ARG, "NULL argument");
  if (ncontrols < 0 || ncontrols > SV_MAX_CONTROLS) return set_error(SV_ERR_ARG, "ncontrols out of range");
  if (ncontrols > 0 && !controls) return set_error(SV_ERR_ARG, "controls is NULL");
  sv_gate g;
  std::memset(&g, 0, sizeof g);
  std::memcpy(g.U, U, sizeof g.U);
  g.kind = SV_GATE_U;
  g.target = target;
  g.target2 = -1;
  g.ncontrols = ncontrols;
  for (int i = 0; i < SV_MAX_CONTROLS; ++i) g.controls[i] = i < ncontrols ? controls[i] : -1;
  return apply_records(s, &g, 1, true);
}

sv_status sv_apply_gate2q(sv_state *s, const double *V, int q0, int q1, const int *controls, int ncontrols) {
  if (!s || !V) return set_error(SV_ERR_ARG, "NULL argument");
  if (ncontrols < 0 || ncontrols > SV_MAX_CONTROLS) return set_error(SV_ERR_ARG, "ncontrols out of range");
  if (ncontrols > 0 && !controls) return set_error(SV_ERR_ARG, "controls is NULL");
  sv_gate g[4];
  std::memset(g, 0, sizeof g);
  for (int r = 0; r < 4; ++r) {
    std::memcpy(g[r].U, V + 8 * r, sizeof g[r].U);
    g[r].kind = r == 0 ? SV_GATE_U4 : SV_GATE_U4_ROW;
    g[r].target = q0;
    g[r].target2 = q1;
    for (int i = 0; i < SV_MAX_CONTROLS; ++i) g[r].controls[i] = -1;
  }
  g[0].ncontrols = ncontrols;
  for (int i = 0; i < ncontrols; ++i) g[0].controls[i] = controls[i];
  return apply_records(s, g, 4, true);
}

sv_status sv_apply_swap(sv_state *s, int a, int b) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  sv_gate g;
  std::memset(&g, 0, sizeof g);
  g.kind = SV_GATE_SWAP;
  g.target = a;
  g.target2 = b;
  return apply_records(s, &g, 1, true);
}

sv_status sv_apply_circuit(sv_state *s, const sv_gate *gates, size_t ngates) {
  if (!s || (!gates && ngates)) return set_error(SV_ERR_ARG, "NULL argument");
  return apply_records(s, gates, ngates, false);
}

sv_status sv_plan_dry_run(int n, sv_dtype dtype, int chunk_k, const sv_gate *gates, size_t ngates, int *nsteps,
                          int *step_of_gate, int *order_of_gate, uint64_t *step_qmask, int max_steps,
                          int *final_perm) {
  if (n < 1 || n > kMaxQubits) return set_error(SV_ERR_ARG, "n must be in [1, 36]");
  if (bad_dtype(dtype)) return set_error(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
  if (!gates && ngates) return set_error(SV_ERR_ARG, "gates is NULL");
  {
    std::string why;
    size_t bad = 0;
    const int rc = validate_records(gates, ngates, n, why, bad);
    if (rc != SV_OK) return set_error(rc, "gate " + std::to_string(bad) + ": " + why);
  }
  sv_state tmp;
  tmp.n = n;
  tmp.dtype = dtype;
  tmp.chunk_k = chunk_k;
  std::vector<int> perm(n);
  for (int t = 0; t < n; ++t) perm[t] = t;
  Plan P;
  make_plan(n, plan_config(&tmp), perm, gates, ngates, P);
  if (nsteps) *nsteps = (int)P.steps.size();
  for (size_t i = 0; i < ngates; ++i) {
    if (step_of_gate) step_of_gate[i] = P.gate_step[i];
    if (order_of_gate) order_of_gate[i] = P.gate_order[i];
  }
  if (step_qmask)
    for (int j = 0; j < max_steps && j < (int)P.step_qmask.size(); ++j) step_qmask[j] = P.step_qmask[j];
  if (final_perm)
    for (int t = 0; t < n; ++t) final_perm[t] = perm[t];
  return SV_OK;
}

sv_status sv_plan_dry_run_blocks(int n, sv_dtype dtype, int chunk_k, int tensor_blocks, const sv_gate *gates,
                                 size_t ngates, int *passes, int *passes_with_blocks, int *blocks, int *block_gates) {
  if (n < 1 || n > kMaxQubits) return set_error(SV_ERR_ARG, "n must be in [1, 36]");
  if (bad_dtype(dtype)) return set_error(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
  if (tensor_blocks < 0 || tensor_blocks > 64) return set_error(SV_ERR_ARG, "tensor_blocks must be in 0..64");
  if (chunk_k != 0 && (chunk_k < 6 || chunk_k > kMaxChunkQubits))
    return set_error(SV_ERR_ARG, "chunk_k must be 0 or 6..13");
  if (!gates && ngates) return set_error(SV_ERR_ARG, "gates is NULL");
  {
    std::string why;
    size_t bad = 0;
    const int rc = validate_records(gates, ngates, n, why, bad);
    if (rc != SV_OK) return set_error(rc, "gate " + std::to_string(bad) + ": " + why);
  }
  sv_state tmp;
  tmp.n = n;
  tmp.dtype = dtype;
  tmp.chunk_k = chunk_k;
  tmp.tensor_blocks = tensor_blocks;
  std::vector<int> perm(n);
  for (int t = 0; t < n; ++t) perm[t] = t;
  Plan P;
  make_plan(n, plan_config(&tmp), perm, gates, ngates, P);
  int with = 0;
  for (const PassDesc &d : P.passes) with += d.nblocks > 0;
  if (passes) *passes = (int)P.passes.size();
  if (passes_with_blocks) *passes_with_blocks = with;
  if (blocks) *blocks = P.n_blocks;
  if (block_gates) *block_gates = P.n_block_gates;
  return SV_OK;
}

sv_status sv_last_plan_blocks(sv_state *s, int *blocks, int *block_gates) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  if (blocks) *blocks = s->st_blocks;
  if (block_gates) *block_gates = s->st_block_gates;
  return SV_OK;
}

sv_status sv_profile_last(sv_state *s, int kind, int *launches, double *ms) {
  if (!s || !launches || !ms) return set_error(SV_ERR_ARG, "NULL argument");
  *launches = 0;
  *ms = 0.0;
  if (!s->last_evs) return SV_OK;
  for (size_t i = 0; i < s->last_kind.size(); ++i) {
    if (s->last_kind[i] != kind) continue;
    cudaError_t e = cudaEventSynchronize(s->last_evs[2 * i + 1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, s->last_evs[2 * i], s->last_evs[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "profiling event");
    ++*launches;
    *ms += t;
  }
  return SV_OK;
}

sv_status sv_sync(sv_state *s) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? check_tc_error(s) : cuda_fail(e, "stream sync");
}

sv_status sv_last_plan_stats(sv_state *s, int *passes, int *fused_gates, int *sweep_gates, int *relabels, int *remaps,
                             int *absorbed) {
  if (!s) return set_error(SV_ERR_ARG, "state is NULL");
  if (absorbed) *absorbed = s->st_absorbed;
  if (passes) *passes = s->st_passes;
  if (fused_gates) *fused_gates = s->st_fused;
  if (sweep_gates) *sweep_gates = s->st_sweeps;
  if (relabels) *relabels = s->st_relabels;
  if (remaps) *remaps = s->st_remaps;
  return SV_OK;
}

} // extern "C"
