/*
 * sv.h -- C ABI of the GB300 state-vector simulator.
 *
 * The library stores only the 2^n amplitudes of an n-qubit state and applies each single-qubit gate,
 * optionally controlled, to every amplitude pair whose indices differ in the target bit: the state-vector
 * method of LaRose, "Distributed Memory Techniques for Classical Simulation of Quantum Circuits"
 * (arXiv:1801.01037), Sec. V.A (the strided pair-update equation) and Sec. V.B (Algorithm 1 and its
 * controlled variant).
 *
 * Conventions shared by every entry point
 *   - Qubit t is bit t of the amplitude index (the paper's stride rule: qubit i pairs k with k + 2^i,
 *     Sec. V.A, Fig. "statevector").  Index k of a logical read is the integer sum_t b_t 2^t.
 *   - Amplitudes are interleaved complex numbers: SV_C128 = two IEEE doubles (16 B), SV_C64 = two floats (8 B).
 *   - Gate matrices are always given in double precision, row-major (q11, q12, q21, q22) as (re, im) pairs.
 *   - Every call returns an sv_status.  Arguments are validated on the host before any device work; on an
 *     error nothing is launched and sv_last_error() describes the problem.  No call aborts or throws.
 *   - A state handle is not thread-safe; its work is ordered on the CUDA stream given at creation
 *     (NULL = the legacy default stream).  Calls that return data to the host synchronise that stream.
 *   - Pointers named host_* are host memory; dev_ptr arguments are device memory of the current device.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sv_status;
#define SV_OK 0
#define SV_ERR_ARG (-1)          /* bad argument: NULL pointer, qubit out of range, duplicate qubits, ... */
#define SV_ERR_OOM (-2)          /* device (or pinned host) allocation failed, or over the server budget */
#define SV_ERR_CUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define SV_ERR_NOT_UNITARY (-4)  /* max |U^dagger U - I| > 1e-10 */
#define SV_ERR_TIMEOUT (-5)      /* a bounded device or host wait ran out */
#define SV_ERR_BUSY (-6)         /* the server cannot take the request now (queue full) */
#define SV_ERR_NOT_FOUND (-7)    /* unknown ticket */
#define SV_ERR_NO_DEVICE (-8)    /* no CUDA device, or not an sm_103 device */

typedef enum { SV_C64 = 1, SV_C128 = 2 } sv_dtype;

/* Arithmetic used for complex128 states.  The storage stays IEEE double in every mode.
 *   SV_ARITH_AUTO  : SV_ARITH_DF32 for complex128, FP32 for complex64 (the default).
 *   SV_ARITH_F64   : native FP64 multiply-adds (exact IEEE double, about 1/70 of the FP32 rate on GB300).
 *   SV_ARITH_DF32  : each double is split into a pair of floats (hi + lo, >= 47 significant bits) with
 *                    integer bit operations, each output of the 2x2 product is a compensated float dot
 *                    product (exact products by FMA, TwoSum accumulation) with the gate entries split exactly
 *                    into three floats, and the result is re-assembled into a double.  Error per gate: a few
 *                    2^-47 of the largest term (absolute), i.e. ~1e-14 for amplitudes of order 1.
 * complex64 states always use FP32 arithmetic. */
typedef enum { SV_ARITH_AUTO = 0, SV_ARITH_F64 = 1, SV_ARITH_DF32 = 2 } sv_arith;

#define SV_MAX_CONTROLS 4
#define SV_GATE_U 0     /* 2x2 unitary on `target`, acting where every control bit is 1 (Sec. V.B) */
#define SV_GATE_SWAP 1  /* exchange qubits `target` and `target2` (Sec. VI.B's relabelling) */
#define SV_GATE_U4 2    /* dense two-qubit unitary V (4x4) on qubits `target` and `target2`, acting where every
                           control bit is 1; V is indexed by b0 + 2 b1 with b0 the bit of `target` and b1 the
                           bit of `target2` (so V = A (x) B applies A to target2 and B to target, and the
                           paper's CNOT matrix of Sec. II.B is V with target2 = control).  Four consecutive
                           records: this one holds row 0 of V in U, the next three (SV_GATE_U4_ROW) rows 1..3. */
#define SV_GATE_U4_ROW 3 /* continuation record of SV_GATE_U4: U = row r of V (4 complex entries); target and
                            target2 repeat the first record's, ncontrols = 0 */

/* One gate record, 96 bytes. */
typedef struct sv_gate {
    double U[8];                       /* q11, q12, q21, q22 as (re, im); a row of V for SV_GATE_U4[_ROW];
                                          ignored for SV_GATE_SWAP */
    int32_t kind;                      /* SV_GATE_U, SV_GATE_SWAP, SV_GATE_U4 or SV_GATE_U4_ROW */
    int32_t target;                    /* target qubit, 0 <= target < n */
    int32_t target2;                   /* second qubit of SV_GATE_SWAP / SV_GATE_U4; -1 for SV_GATE_U */
    int32_t ncontrols;                 /* 0..SV_MAX_CONTROLS */
    int32_t controls[SV_MAX_CONTROLS]; /* distinct, != target (and target2), < n */
} sv_gate;

typedef struct sv_state sv_state;
typedef struct sv_server sv_server;

/* Options for sv_set_option. */
#define SV_OPT_ARITH 1          /* sv_arith value */
#define SV_OPT_CHUNK_QUBITS 2   /* k: 2^k amplitudes per fused chunk (0 = tuned default, else 6..13) */
#define SV_OPT_FUSION 3         /* 1 = fuse gates into chunk passes (default), 0 = one sweep kernel per gate */
#define SV_OPT_RENORM_PERIOD 4  /* renormalise every R applied gates (0 = never, the default) */
#define SV_OPT_CANONICAL 5      /* 1 = restore logical bit order after every apply call (default for
                                   sv_create_from_buffer states), 0 = keep the relabelled layout lazily */
#define SV_OPT_PROFILE 6        /* 1 = record a CUDA event before and after every launch of the apply calls
                                   (also inside captured graphs); read them with sv_profile_last */
#define SV_OPT_F64_SHARE 7      /* complex128 with SV_ARITH_DF32: percent (0..99) of each fused pass's chunks
                                   computed with native FP64 by one CTA per SM, in parallel with the
                                   double-float CTAs (the FP64 pipe is otherwise idle); -1 = default
                                   (SV_F64_SHARE_DEFAULT).
                                   Which chunks use FP64 depends only on their index: results are
                                   reproducible run to run. */
#define SV_F64_SHARE_DEFAULT 16
#define SV_OPT_PRODUCT_START 9  /* 1 = fold leading single-qubit gates into the factors while the state is a
                                   product state (sv_init_product), the default; 0 = never (every gate runs
                                   as a kernel, e.g. to time single-gate sweeps on a fresh state) */
#define SV_OPT_CUBES 8          /* complex64: 1 = apply runs of gates on at most 4 chunk bits from registers
                                   (one shared-memory round trip per run), the default; 0 = one
                                   shared-memory round trip per gate.  Results are identical either way. */
#define SV_OPT_TENSOR_BLOCKS 10 /* 1 = compose runs of gates on at most 4 chunk bits into one 16 x 16 unitary
                                   (FP64, host; Sec. II.B's multi-qubit gate as a matrix) and apply it with
                                   tcgen05 tensor-core MMAs; 0 = per-gate arithmetic (the default).
                                   complex64: three bfloat16 splits of each factor (24 bits), FP32 accumulation
                                   on the tensor cores, which drifts the state's norm by about 3e-7 per block
                                   (per-gate passes: far less), so the library's autotuner leaves it off.
                                   complex128 (double-float arithmetic, chunks of at most 2^12): six exact
                                   base-256 digits of each factor, integer products accumulated exactly per
                                   digit level in FP32 and combined in double-float (error a few 2^-47 of the
                                   chunk's 2-norm per block).  Used for fused passes with chunks of at least
                                   2^11 amplitudes, in passes where the blocks take at least 3/4 of the
                                   per-gate work.  A value v >= 2 turns blocks on and keeps only blocks that
                                   replace at least v dense one-qubit gate updates (1: at least 2). */

/* ---------------------------------------------------------------------------------------------------------
 * States
 * ------------------------------------------------------------------------------------------------------- */

/* Allocate a 2^n-amplitude state in device memory (library-owned) and set it to |0...0> (Sec. II.A).
 * n: 1 <= n <= 36 and the state must fit in free device memory.  stream: a cudaStream_t or NULL.
 * Errors: SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_NO_DEVICE.  *out is set only on success. */
sv_status sv_create(int n, sv_dtype dtype, void *stream, sv_state **out);

/* Wrap caller-owned device memory of 2^n amplitudes (e.g. a torch tensor's storage); the contents are
 * taken as the current state in logical order and are not modified here.  dev_ptr must be 16-byte
 * aligned and stay valid until sv_destroy.  The library never frees it.  The buffer is kept in logical
 * order after every call (SV_OPT_CANONICAL defaults to 1). */
sv_status sv_create_from_buffer(int n, sv_dtype dtype, void *dev_ptr, void *stream, sv_state **out);

/* Release the handle and, for sv_create states, the device memory.  NULL is accepted. */
sv_status sv_destroy(sv_state *s);

/* |x>: amplitude x = 1, all others 0.  x < 2^n.  Resets the layout to the identity.  Like sv_create's
 * |0...0>, the result is a product state (see sv_init_product). */
sv_status sv_init_basis(sv_state *s, uint64_t x);

/* Product state |psi_0 ... psi_{n-1}> (Sec. V, the per-qubit form of a state with no entanglement): qubit t
 * in alpha_t|0> + beta_t|1>, so amplitude k = prod_t (bit t of k ? beta_t : alpha_t).  factors: 4n doubles
 * in host memory, (re alpha_t, im alpha_t, re beta_t, im beta_t) for t = 0..n-1; each |alpha_t|^2 +
 * |beta_t|^2 must be 1 within 1e-10.  The amplitudes are formed on the GPU in FP64 (two tables of partial
 * products, one complex product per amplitude; complex64 states round the result).  Resets the layout.
 *
 * While a state is still a product state (since sv_create, sv_init_basis or sv_init_product, no gate has
 * entangled it), the apply calls fold every uncontrolled single-qubit gate (and SWAP) that acts on qubits no
 * earlier remaining gate of the call touches into those qubits' factors on the host (2x2 products in FP64),
 * as the paper suggests for the gates at the start of a circuit, re-form the amplitudes once, and plan only
 * the rest.  Re-forming writes the whole state, so the fold is taken only when nothing else remains or at
 * least max(2, n/4) gates fold (option SV_OPT_PRODUCT_START turns it off).  sv_last_plan_stats reports the
 * folded gates.
 * Errors: SV_ERR_ARG (NULL, non-finite or non-normalised factor), SV_ERR_CUDA. */
sv_status sv_init_product(sv_state *s, const double *factors);

/* Copy `count` amplitudes from host memory (state's dtype, logical order) into indices first..first+count-1
 * (checkpoint restore).  Errors: SV_ERR_ARG (NULL, range beyond 2^n, a non-finite component, or for complex128 a
 * component of magnitude >= 2^126: the double-float arithmetic holds components in float exponents), checked
 * on the host before anything is copied. */
sv_status sv_write_amplitudes(sv_state *s, uint64_t first, uint64_t count, const void *host_in);

sv_status sv_set_option(sv_state *s, int option, int64_t value);
sv_status sv_get_info(sv_state *s, int *n, sv_dtype *dtype, void **dev_ptr);

/* Logical-to-physical qubit map: perm[t] = index bit that currently holds qubit t (the paper's
 * non-sequential storage, Sec. VI.B).  perm must hold n ints. */
sv_status sv_get_layout(sv_state *s, int *perm);

/* Put the amplitudes back in logical order in device memory (perm = identity).  Done with gate-free chunk
 * passes whose store permutes bits: each pass moves a whole cycle (or a run of one) of the layout's bit
 * permutation at once, so a random layout of 30 qubits takes about 4 passes over the state. */
sv_status sv_canonicalize(sv_state *s);

/* ---------------------------------------------------------------------------------------------------------
 * Gates (Sec. V.A pair update; Sec. V.B controlled variant)
 * ------------------------------------------------------------------------------------------------------- */

/* Apply the 2x2 unitary U on qubit `target`, restricted to indices whose `ncontrols` control bits are all 1.
 * U: 8 doubles, row-major (re, im).  controls may be NULL when ncontrols == 0.
 * Errors: SV_ERR_ARG (qubit out of range, control == target, duplicate controls, > SV_MAX_CONTROLS),
 *         SV_ERR_NOT_UNITARY, SV_ERR_CUDA. */
sv_status sv_apply_gate(sv_state *s, const double *U, int target, const int *controls, int ncontrols);

/* Dense two-qubit unitary V (16 complex entries, row-major (re, im): 32 doubles) on qubits q0 (index bit b0)
 * and q1 (bit b1), entry order b0 + 2 b1, under `ncontrols` controls (see SV_GATE_U4).  Both qubits are brought
 * into the chunk of one fused pass and each quadruple of amplitudes is multiplied by V.
 * Errors: SV_ERR_ARG (qubits out of range or repeated), SV_ERR_NOT_UNITARY (max |V^dagger V - I| > 1e-10),
 *         SV_ERR_CUDA. */
sv_status sv_apply_gate2q(sv_state *s, const double *V, int q0, int q1, const int *controls, int ncontrols);

/* SWAP of qubits a and b.  Done as a relabelling of the layout map (no data movement); a canonical-only
 * (buffer) state is then put back in logical order by a bit-permutation pass at the end of the call. */
sv_status sv_apply_swap(sv_state *s, int a, int b);

/* Apply `ngates` gate records (host memory) in order.  All records are validated before any work; the
 * planner fuses runs of gates into passes over 2^k-amplitude chunks.  Error: index of the first bad gate in
 * sv_last_error(). */
sv_status sv_apply_circuit(sv_state *s, const sv_gate *gates, size_t ngates);

/* Same as sv_apply_circuit, but the gate list is captured once into a CUDA graph keyed by its contents
 * and the graph is replayed on later calls with identical gates and layout.  The key is a hash of the gate
 * records, the layout, the options and the state's address; a replay also compares all of those bytes, so a
 * hash collision only costs a new capture.  At most 64 graphs are kept per state. */
sv_status sv_apply_circuit_graph(sv_state *s, const sv_gate *gates, size_t ngates);

/* Host-only dry run of the planner for `ngates` records on n qubits of `dtype` (chunk_k = 0: the default
 * chunk size), starting from the identity layout.  No device work; works without a GPU.
 *   *nsteps            number of launches the plan makes (fused passes and single-gate sweeps)
 *   step_of_gate[i]    launch that applies gate i, or -1 for a SWAP folded into the layout / an identity
 *   order_of_gate[i]   position of gate i in execution order (the planner reorders only commuting gates:
 *                      gates that share a qubit keep their order)
 *   step_qmask[j]      physical index bits spanned by launch j's chunks (a sweep: its target bit), j < max_steps
 *   final_perm[t]      physical bit of logical qubit t after the circuit
 * Array outputs may be NULL.  Errors: SV_ERR_ARG, SV_ERR_NOT_UNITARY (as sv_apply_circuit). */
sv_status sv_plan_dry_run(int n, sv_dtype dtype, int chunk_k, const sv_gate *gates, size_t ngates, int *nsteps,
                          int *step_of_gate, int *order_of_gate, uint64_t *step_qmask, int max_steps,
                          int *final_perm);

/* ---------------------------------------------------------------------------------------------------------
 * Read-out and reductions
 * ------------------------------------------------------------------------------------------------------- */

/* Copy amplitudes first..first+count-1 (logical order) to host memory in the state's dtype.  Synchronises. */
sv_status sv_read_amplitudes(sv_state *s, uint64_t first, uint64_t count, void *host_out);

/* Same, but gather the logical indices listed in host array `idx` (count entries, each < 2^n). */
sv_status sv_read_amplitudes_at(sv_state *s, const uint64_t *idx, uint64_t count, void *host_out);

/* |alpha_k|^2 (Sec. II.A) for k = first..first+count-1, in double precision, to host memory. */
sv_status sv_read_probabilities(sv_state *s, uint64_t first, uint64_t count, double *host_out);

/* Measurement in the computational basis (the probabilities |alpha_k|^2 of Sec. II.A, normalised by their
 * sum).  The caller draws the random numbers: u[i] (host, count entries, each in [0, 1)) selects outcome
 * out[i] = the smallest logical index k with P_0 + ... + P_k > u[i], where P_j = |alpha_j|^2 / sum |alpha|^2
 * accumulated in FP64 in logical index order.  The state is not collapsed.  Synchronises.
 * Errors: SV_ERR_ARG (NULL, u outside [0, 1), zero state), SV_ERR_OOM, SV_ERR_CUDA. */
sv_status sv_sample(sv_state *s, const double *u, uint64_t count, uint64_t *out);

/* Expectation of the Pauli-Z product on the logical qubits set in `mask`:
 * sum_k |alpha_k|^2 (-1)^popcount(k & mask), accumulated like sv_norm (not divided by the norm).  Synchronises. */
sv_status sv_expect_z(sv_state *s, uint64_t mask, double *out);

/* sum_k |alpha_k|^2 accumulated in (at least) double precision.  Synchronises. */
sv_status sv_norm(sv_state *s, double *out);

/* Norm without any device allocation.  The paper has no counterpart: this entry point exists for callers
 * that must not allocate device memory themselves, e.g. a host framework that has already reserved the
 * GPU's memory for its own pool (so a cudaMalloc here would fail or fragment that pool), or a latency-critical
 * loop that cannot afford cudaMalloc's implicit device synchronisation.  They keep ownership of every buffer:
 *   psi    device pointer to 2^n amplitudes of `dtype` in physical order (16-byte aligned); the norm does not
 *          depend on the order
 *   d_out  device pointer to one double that receives sum_k |alpha_k|^2 (8-byte aligned)
 *   stream cudaStream_t or NULL; the work is queued on it and the call returns without waiting
 * The per-block partial sums go to a fixed scratch array of SV_NORM_NOALLOC_MAX_PARTIALS doubles (32 KiB)
 * compiled into the library: every GPU that loads the library keeps it until the process exits.  The first
 * call on a device does a one-time set-up (it looks up that array's device address, with the device
 * current); make that first call on each device before any stream capture.  With CUDA's lazy module loading
 * that look-up can be what makes the driver load the library's kernels onto the device, and the driver then
 * allocates their code and static data (this array included) itself: a caller that hands nearly all device
 * memory to its own pool should make one call (or any other call of this library) before reserving it.
 * The partial count is 4 per SM of the device current at the call.  Every call writes
 * each partial it later reads, so nothing needs clearing between calls, but all calls share the one array:
 * calls whose work overlaps on the GPU (e.g. on two streams) race and give wrong results.
 * Errors: SV_ERR_ARG (NULL or misaligned pointer, n outside [1, 36], bad dtype, or a GPU whose partial-sum
 * count exceeds SV_NORM_NOALLOC_MAX_PARTIALS), SV_ERR_NO_DEVICE, SV_ERR_CUDA.  The library itself calls no
 * allocating routine on any path (the one-time module load above is the driver's). */
#define SV_NORM_NOALLOC_MAX_PARTIALS 4096
sv_status sv_norm_noalloc(const void *psi, int n, sv_dtype dtype, void *stream, double *d_out);

/* Divide every amplitude by sqrt(sum |alpha_k|^2). */
sv_status sv_renormalize(sv_state *s);

/* Wait for all queued work of the state. */
sv_status sv_sync(sv_state *s);

/* Planner statistics of the last apply call: passes launched, gates applied inside fused passes, gates
 * applied by single-gate sweeps, SWAPs folded into the layout, bit-permutation passes run since the call
 * began (the canonicalisation that ends a call on a buffer state, and sv_canonicalize calls after it), and
 * gates folded into the factors of a product state (sv_init_product).  Any pointer may be NULL. */
sv_status sv_last_plan_stats(sv_state *s, int *passes, int *fused_gates, int *sweep_gates, int *relabels,
                             int *remaps, int *absorbed);

/* Host-only dry run of the dense-block planner (Sec. II.B: a run of gates on a few qubits as one matrix on
 * them) for `ngates` records on n qubits of `dtype`, from the identity layout, as a state with chunk size
 * chunk_k (0: the default) and SV_OPT_TENSOR_BLOCKS = tensor_blocks would plan them: fused passes, passes that
 * hold blocks, blocks, and the source gates they replace.  No device work; works without a GPU.  Output
 * pointers may be NULL.  Errors: SV_ERR_ARG (sizes, options), SV_ERR_NOT_UNITARY (as sv_apply_circuit). */
sv_status sv_plan_dry_run_blocks(int n, sv_dtype dtype, int chunk_k, int tensor_blocks, const sv_gate *gates,
                                 size_t ngates, int *passes, int *passes_with_blocks, int *blocks,
                                 int *block_gates);

/* Dense tensor-core blocks (SV_OPT_TENSOR_BLOCKS) of the last apply call: blocks applied and source gates they
 * replaced.  Any pointer may be NULL. */
sv_status sv_last_plan_blocks(sv_state *s, int *blocks, int *block_gates);

/* With SV_OPT_PROFILE on: device time of the launches of the most recent apply call (or graph replay) of one
 * kind (0 = fused chunk pass, 1 = single-gate sweep), summed over its launches.  Waits for those launches.
 * *launches = 0 when profiling is off or nothing of that kind ran. */
sv_status sv_profile_last(sv_state *s, int kind, int *launches, double *ms);

/* ---------------------------------------------------------------------------------------------------------
 * Batches and serving
 * ------------------------------------------------------------------------------------------------------- */

/* Run `count` independent circuits, circuit i on a fresh |0...0> state of n[i] qubits, all of one dtype,
 * with their passes interleaved in shared launches on `stream`.  out[i] receives a new library-owned
 * state (destroy each with sv_destroy).  Errors leave out[] untouched. */
sv_status sv_run_batch(int count, const int *n, sv_dtype dtype, const sv_gate *const *gates,
                       const size_t *ngates, void *stream, sv_state **out);

/* sv_run_batch with chunk sizes: chunk_k[i] (2^k amplitudes per fused chunk, 0 = the default, else 6..13)
 * for circuit i, e.g. from an autotuner; chunk_k may be NULL (all defaults).  Results do not depend on k
 * beyond rounding. */
sv_status sv_run_batch_k(int count, const int *n, sv_dtype dtype, const sv_gate *const *gates,
                         const size_t *ngates, const int *chunk_k, void *stream, sv_state **out);

/* Statistics of the last sv_run_batch / sv_run_batch_k call of this thread: rounds (steps of the batch: each
 * advances every circuit by one pass), rounds that ran in the FP64 / double-float split kernel (complex128
 * rounds with enough chunks to fill the GPU several times), the largest and the total chunk count of a round,
 * and rounds with a tensor-core launch (passes with dense blocks, see sv_batch_set_option). */
typedef struct sv_batch_stats {
    uint64_t rounds, mixed_rounds, max_round_chunks, total_chunks, tc_rounds;
} sv_batch_stats;
sv_status sv_last_batch_stats(sv_batch_stats *out);

/* Options for this host thread's later sv_run_batch / sv_run_batch_k calls (Sec. II.B's multi-qubit gates as
 * matrices, applied as dense blocks).  Only SV_OPT_TENSOR_BLOCKS is accepted, with the values of
 * sv_set_option (0, the default: off; 1: on; v >= 2: blocks must replace at least v dense one-qubit updates);
 * it applies to complex128 batches in double-float arithmetic, to the circuits whose passes use chunks of 2^12
 * amplitudes: their passes with blocks run in a tensor-core batched kernel beside the per-gate one in every
 * round.  A wait for the tensor cores that runs out fails the batch with SV_ERR_TIMEOUT.  Errors: SV_ERR_ARG
 * for another option or a value outside 0..64. */
sv_status sv_batch_set_option(int option, int value);

/* A serving loop on its own host thread and stream: admits requests while their states fit in
 * hbm_budget_bytes and fewer than max_active run, and advances every admitted request by one pass per
 * round (continuous batching: requests join and leave between rounds).  Each iteration of the loop launches
 * one round per dtype that has work (complex64 and complex128 requests advance side by side), up to four
 * rounds are queued on the server's stream ahead of the host, and admission (state allocation, planning and
 * the gate upload) runs outside the lock that sv_submit and sv_poll take.
 *
 * Budget: an admitted request's state counts against hbm_budget_bytes from admission until sv_poll hands
 * the finished state to the caller (who then owns it and frees it with sv_destroy).  A finished result that
 * is never polled keeps holding its share of the budget. */
sv_status sv_server_create(size_t hbm_budget_bytes, int max_active, sv_server **out);
sv_status sv_server_destroy(sv_server *srv);

/* Queue a circuit on |0...0> of n qubits; the gates are copied.  SV_ERR_BUSY when the pending queue is
 * full, SV_ERR_OOM when the state alone exceeds the budget.  The records are validated again when the
 * request is admitted; a request that fails then (or whose pass descriptors fail the host's checks before a
 * launch) reports its error through sv_poll and leaves the other requests running. */
sv_status sv_submit(sv_server *srv, int n, sv_dtype dtype, const sv_gate *gates, size_t ngates,
                    uint64_t *ticket);

/* Non-blocking: *done = 1 and *result = the final state (caller destroys it) once the request finished;
 * *done = 0 otherwise.  A finished ticket can be polled successfully once; a failed one returns its error
 * code once (with *done = 1, *result = NULL). */
sv_status sv_poll(sv_server *srv, uint64_t ticket, int *done, sv_state **result);

/* paused = 1: admit no new request (admitted ones keep running); 0: admit again.  Lets a caller queue a
 * burst of requests and have them admitted together. */
sv_status sv_server_pause(sv_server *srv, int paused);

typedef struct sv_server_stats {
    uint64_t submitted, admitted, completed, failed;
    uint64_t rounds;            /* launches of the batched pass */
    uint64_t mixed_rounds;      /* complex128 rounds run in the FP64 / double-float split kernel */
    uint64_t max_round_chunks;  /* largest number of chunks in one round */
    uint64_t active, pending;   /* requests admitted and not finished; requests waiting for admission */
    uint64_t budget_used;       /* bytes counted against the budget (see sv_server_create) */
} sv_server_stats;
sv_status sv_server_get_stats(sv_server *srv, sv_server_stats *out);

/* Thread-local description of the last error of this thread ("" if none). */
const char *sv_last_error(void);

/* Library version string. */
const char *sv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SV_H */
