// Host-side state handle and helpers shared by the API, the batch runner and the server.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>
#include <cuda_runtime.h>
#include "sv_internal.h"
#include "sv_plan.h"
#include "../../include/sv.h"

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  void *d_gates = nullptr;   // device blob: the plan's gates
  std::vector<cudaEvent_t> evs;   // profiling: two events per launch, recorded by the graph itself
  std::vector<int> ev_kind;
  std::vector<int> perm_before, perm_after;
  size_t nbytes = 0;
  // Everything the key hashes (gate records, layout, options, state address), kept so that a lookup compares
  // the bytes themselves and a hash collision can never replay another circuit's graph.
  std::vector<unsigned char> key_bytes;
};

struct sv_state {
  int n = 0;
  sv_dtype dtype = SV_C128;
  int arith = SV_ARITH_AUTO;
  void *psi = nullptr;
  bool owned = true;
  std::shared_ptr<void> arena;  // batch states: the shared allocation psi points into (freed with the last one)
  cudaStream_t stream = nullptr;
  std::vector<int> perm;      // logical qubit -> physical bit
  int chunk_k = 0;            // 0 = default
  int fusion = 1;
  int cubes = 1;              // complex64: register cubes in fused passes (SV_OPT_CUBES)
  int tensor_blocks = 0;      // dense tensor-core blocks in fused passes (SV_OPT_TENSOR_BLOCKS)
  bool tc_used = false;       // a tensor-core pass has run: read-backs check its error word
  int canonical = 0;
  int f64_share = -1;         // -1 = library default (SV_OPT_F64_SHARE)
  int64_t renorm_period = 0;
  int64_t gates_since_renorm = 0;
  // device gate buffer and its pinned staging copy
  void *d_gates = nullptr;   // device blob of the last plan's gates
  size_t d_gates_cap = 0;    // bytes
  void *h_stage = nullptr;   // pinned staging copy of that blob
  size_t h_stage_cap = 0;    // bytes
  cudaEvent_t stage_ev = nullptr;
  bool stage_pending = false;
  // norm scratch: norm_parts() partials + 1 result
  double *d_scalars = nullptr;
  svi::FusedSched *d_sched = nullptr;  // scratch of the mixed FP64 / double-float pass
  // read-out staging (device)
  void *d_read = nullptr;
  size_t d_read_cap = 0;
  // Product state (sv_init_product): while `product` holds, psi = (x)_t M_t f_t with f_t = pf[4t..4t+3]
  // (alpha_t, beta_t as re, im) and M_t = pm[8t..8t+7] (row-major re, im), the qubit's folded gates.
  bool product = false;
  int product_start = 1;      // SV_OPT_PRODUCT_START
  std::vector<double> pf, pm;
  void *d_prod = nullptr;     // device: 12 n doubles (f_t, M_t) then the two partial-product tables
  size_t d_prod_cap = 0;      // bytes
  // stats of the last apply
  int st_passes = 0, st_fused = 0, st_sweeps = 0, st_relabels = 0, st_remaps = 0, st_absorbed = 0;
  int st_blocks = 0, st_block_gates = 0;
  std::unordered_map<uint64_t, GraphEntry> graphs;
  // profiling (SV_OPT_PROFILE)
  int profile = 0;
  std::vector<cudaEvent_t> ev_pool;
  const cudaEvent_t *last_evs = nullptr;
  std::vector<int> last_kind;
};

namespace svi {

int set_error(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
int mode_of(const sv_state *s);
size_t amp_bytes(sv_dtype dt);
int check_device();
PlanConfig plan_config(const sv_state *s);
// Upload the plan's gates through the state's pinned staging buffer into its device blob.
int upload_plan(sv_state *s, const Plan &P, void **d_blob);
// Launch the steps of a plan (gates already on the device at d_fused / d_sweep) on stream st.
// evs: nullptr, or two timing events per step recorded around each launch (external records when capturing).
int run_plan(sv_state *s, const Plan &P, const void *d_blob, cudaStream_t st,
             const cudaEvent_t *evs = nullptr, bool capturing = false);
// Make sure the state's event pool holds at least 2 * steps events.
int ensure_event_pool(sv_state *s, size_t steps);
std::vector<int> step_kinds(const Plan &P);
int canonicalize_now(sv_state *s);
// Allocate the state's small scratch (norm partials, mixed-pass scheduler, staging event) if not done yet.
// Must not run inside a stream capture.
int ensure_scratch(sv_state *s);
// Product-state start: fold leading single-qubit gates into the factors and re-form psi; (gates, ngates)
// then name the remaining records, stored in `rest`.
int product_prologue(sv_state *s, const sv_gate *&gates, size_t &ngates, std::vector<sv_gate> &rest);
// Queue the bit-permutation passes that bring `perm` to the identity on stream st (perm is updated).
int canonicalize_on(sv_state *s, std::vector<int> &perm, cudaStream_t st, int *npasses);
// Percent of complex128 double-float chunks done in native FP64 alongside (see SV_OPT_F64_SHARE).
constexpr int kDefaultF64Share = SV_F64_SHARE_DEFAULT;
int f64_share_of(const sv_state *s);
int maybe_renormalize(sv_state *s, int applied);
// After a synchronisation: SV_ERR_TIMEOUT if a tensor-core pass of the state reported a wait that ran out
// (its error word is cleared); SV_OK otherwise.
int check_tc_error(sv_state *s);
int alloc_state(int n, sv_dtype dt, cudaStream_t st, sv_state **out, bool init_zero);

} // namespace svi
