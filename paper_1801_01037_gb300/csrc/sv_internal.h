// Internal structures shared by the host runtime (C++) and the CUDA kernels.  Not part of the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace svi {

constexpr int kMaxQubits = 36;
constexpr int kMaxChunkQubits = 13;

// Storage / arithmetic modes.  The storage of C128 is IEEE double in every mode.
enum Mode : int {
  MODE_C64_F32 = 0,   // complex64 storage, FP32 arithmetic
  MODE_C128_F64 = 1,  // complex128 storage, native FP64 arithmetic
  MODE_C128_DF32 = 2, // complex128 storage, double-float (hi+lo float pair) arithmetic
};

// Gate classes, decided on the host by exact comparisons of the FP64 matrix entries.
enum GateClass : uint32_t {
  GC_GENERAL = 0,   // dense 2x2
  GC_DIAG = 1,      // q12 = q21 = 0: each amplitude scaled by q11 or q22, no pairing
  GC_PHASE = 2,     // diagonal with q11 = 1: only amplitudes whose target bit is 1 change
  GC_ANTIDIAG = 3,  // q11 = q22 = 0: alpha_k <- q12 alpha_{k+2^t}, alpha_{k+2^t} <- q21 alpha_k
  GC_X = 4,         // q12 = q21 = 1, q11 = q22 = 0: the pair is exchanged (pure moves)
  GC_CUBE = 5,      // not a gate: header of a register cube (complex64 fused passes, see below)
  GC_DENSE4 = 6,    // dense two-qubit gate: this record holds row 0 of V, `target` the chunk bit of b0 and
                    //   `tmask` the chunk bit of b1 (both always inside the chunk); then three GC_ROW records
  GC_ROW = 7,       // rows 1..3 of the GC_DENSE4 record before it
  GC_BLOCK = 8,     // not a gate: a dense unitary on kBlockBits chunk-local bits applied with tcgen05 MMAs
                    //   (see below); `target` = number of source gates it replaces
};

// Dense block.  A header DevGate with cls = GC_BLOCK stands for the product of a run of gates whose qubits all
// lie in kBlockBits chunk-local bits (packed one per byte in `cmask`, ascending).  Every row of the chunk (the
// 2^kBlockBits amplitudes that differ only in those bits) is multiplied by the block's matrix in its real
// form W (kBlockK x kBlockK: outputs Re 0..15, Im 0..15 by inputs Re 0..15, Im 0..15): D = X W^T, one
// tcgen05.mma chain per 128 rows, A = the rows (shared memory, bfloat16 planes), B = W (bfloat16 planes).
// `gmask` = byte offset from the header to its operand planes in the device gate blob (kBlockPlaneBytes per
// plane, in the kernel's shared-memory layout).  complex64: three planes w = w0 + w1 + w2; the rows are split
// the same way and the six products with i + j <= 2 are accumulated in FP32 (24 bits of each factor).
// complex128: six planes of balanced base-256 digits of w * 2^47 against the rows' digits of x * 2^(47 - E)
// (E: a power of two above the chunk's 2-norm, which the pass's unitaries preserve); the products are exact
// integers, accumulated per digit level in FP32 (exactly: every partial sum stays below 2^22) and combined
// in double-float.
constexpr int kBlockBits = 4;
constexpr int kBlockDim = 1 << kBlockBits;   // complex amplitudes per row
constexpr int kBlockK = 2 * kBlockDim;       // reals per row (re | im)
constexpr int kBlockSplitsC64 = 3;
constexpr int kBlockDigitsC128 = 6;
constexpr size_t kBlockPlaneBytes = (size_t)kBlockK * kBlockK * 2;

// Register cube.  Inside a complex64 fused pass, a header DevGate with cls = GC_CUBE says that the next
// `target` gates act only on the `tmask` (= kCubeBits) chunk-local bits packed one per byte in `cmask`
// (ascending), apart from diagonal gates, which may sit on any bit.  Each thread then holds the 2^kCubeBits
// amplitudes that differ in those bits in registers and applies all of the cube's gates there: one
// shared-memory round trip for the run instead of one per gate.  The gates of a cube carry their in-cube
// control bits and target slot in the upper half of `cmask` (see group_cubes).  Five bits (32 registers
// of data per thread) measured the same speed and spilled at the 128-register cap.
constexpr int kCubeBits = 4;

// One gate as the kernels see it.  In a single-gate sweep, `target` and `cmask` are physical bits.  Inside
// a fused pass they are chunk-local bits; controls that lie outside the chunk go to `gmask` (physical bits
// that must all be 1 in the chunk's base index), and a diagonal gate whose target lies outside the chunk
// has target = -1 and its physical target bit in `tmask`.
struct DevGate {
  double q[8];       // q11, q12, q21, q22 (re, im), FP64
  float qh[8];       // q rounded to float (also the complex64 coefficients)
  float qm[8];       // three-float split q = qh + qm + ql, exact to 2^-72 relative: no systematic
  float ql[8];       //   coefficient error (a two-float split leaves ~1e-15, e.g. H off unitary by 6e-16)
  uint64_t cmask;
  uint64_t gmask;
  uint64_t tmask;
  int32_t target;
  uint32_t cls;
};
static_assert(sizeof(DevGate) == 192, "DevGate layout");

// One fused pass over all chunks of a state.  A chunk is the 2^k amplitudes whose indices agree outside
// the physical bits qpos[0..k-1]; qpos[j] = j for j < c, so each chunk is 2^(k-c) runs of 2^c contiguous
// amplitudes.  On store, chunk-local bit j goes to physical bit qpos_out[j] (a permutation of qpos over the
// same set of bits, so every chunk writes exactly the addresses it read: the pass stays in place).
struct PassDesc {
  void *psi;
  const DevGate *gates;   // device array, ngates entries
  uint64_t qmask;         // OR of 1 << qpos[j]
  uint64_t init_x;        // with init = 1: the pass starts from the basis state |init_x> (physical index)
  int32_t n, k, c, ngates;
  int8_t qpos[16];        // ascending; qpos[j] = j for j < c
  int8_t qpos_out[16];
  int32_t init;           // 0: read the chunk from HBM; 1: synthesise |init_x> restricted to the chunk
  int32_t permuted;       // 1 if qpos_out differs from qpos
  int8_t src_bit[16];     // permuted: bit j of the local amplitude stored at slot o is bit src_bit[j] of o
  int32_t nblocks;        // GC_BLOCK records among the gates (> 0: the pass needs the tensor-core kernel)
  int32_t tc_flags;      // tensor-core passes, test hook only: 1 = issue no MMA, so every wait runs out
};
static_assert(sizeof(PassDesc) == 112, "PassDesc layout");

// ---------------------------------------------------------------------------------------------------------
// Kernel launchers (sv_kernels.cu).  All return cudaGetLastError() of the launch.
// ---------------------------------------------------------------------------------------------------------
cudaError_t launch_init_basis(void *psi, int n, int mode, uint64_t x, cudaStream_t st);
// Product state from d_fm (12 doubles per qubit: f_t then M_t), using d_tab as scratch for
// product_table_entries(n) double2 values.
uint64_t product_table_entries(int n);
cudaError_t launch_init_product(void *psi, int n, int mode, const double *d_fm, void *d_tab, cudaStream_t st);

// Scratch of the mixed FP64 / double-float pass: one election slot per SM and one chunk counter per role.
constexpr int kSchedSlots = 256;
struct FusedSched {
  unsigned sm_slot[kSchedSlots];
  unsigned long long next[2];
  // Error word of the tensor-core pass: non-zero when a bounded wait for the tensor cores ran out (the kernel
  // then stops applying blocks).  Not cleared by the launches that reset the fields above; the host reads and
  // clears it (read_tc_error).
  unsigned tc_err;
  unsigned pad;
};
constexpr size_t kSchedResetBytes = offsetof(FusedSched, tc_err);

cudaError_t launch_sweep(void *psi, int n, int mode, const DevGate &g, cudaStream_t st);

// f64_share (complex128 double-float passes only): percent of the chunks done in native FP64 by one CTA per
// SM alongside the double-float CTAs (0 = all double-float); `sched` is device scratch for that split.
cudaError_t launch_fused(const PassDesc &p, int mode, cudaStream_t st, int f64_share = 0, FusedSched *sched = nullptr);
int fused_smem_bytes(int mode, int k);
// Logical-order gather: out[i] = psi[phys(idx_i)], idx_i = first + i (d_idx == nullptr) or d_idx[i].
// perm[t] = physical bit of logical qubit t.
cudaError_t launch_gather(const void *psi, int n, int mode, const int *perm, uint64_t first, uint64_t count,
                          const uint64_t *d_idx, void *d_out, cudaStream_t st);
cudaError_t launch_probs(const void *psi, int n, int mode, const int *perm, uint64_t first, uint64_t count,
                         double *d_out, cudaStream_t st);
// Sum of |psi_k|^2: stage 1 writes `nparts` partial sums (as double) to d_partials, stage 2 adds them in a
// fixed order into *d_out.  nparts must be norm_parts().
int norm_parts();
// pmask != 0: sum of (-1)^popcount(k & pmask) |psi_k|^2 over physical k instead (Pauli-Z expectation).
cudaError_t launch_norm(const void *psi, int n, int mode, double *d_partials, double *d_out, cudaStream_t st,
                        uint64_t pmask = 0);
// The same with an explicit partial count (`parts` blocks in stage 1, any value >= 1; the result's rounding
// depends on it), e.g. norm_parts_for_sms(SM count of the current device).
int norm_parts_for_sms(int sms);
cudaError_t launch_norm_parts(const void *psi, int n, int mode, double *d_partials, double *d_out, cudaStream_t st,
                              uint64_t pmask, int parts);
// Sampling: FP64 probability mass of each block of 2^b consecutive logical indices, then one lookup per shot
// inside its block (d_blk[i] = block, d_resid[i] = mass to skip inside it) -> logical index.
cudaError_t launch_block_probs(const void *psi, int n, int mode, const int *perm, int b, double *d_out,
                               cudaStream_t st);
cudaError_t launch_sample_block(const void *psi, int n, int mode, const int *perm, int b, const uint64_t *d_blk,
                                const double *d_resid, uint64_t count, uint64_t *d_out, cudaStream_t st);
cudaError_t launch_scale(void *psi, int n, int mode, const double *d_norm2, cudaStream_t st);

// Batched fused pass: `npass` pass descriptors in device memory; block b handles chunk b - chunk_start[p]
// of pass p, where chunk_start is an exclusive prefix sum over the passes' chunk counts (device array of
// npass + 1 entries).  All passes share `mode`; each has its own k <= kmax (shared memory is sized for kmax).
// f64_share / sched: as for launch_fused (complex128 double-float: that percent of the round's chunks, by
// their index in the round, run in native FP64 on one CTA per SM).  *used_mixed (if given) is set to 1 when
// the round ran in that split kernel (k_fused_batch_mixed), else 0.
// Raise the shared-memory grants of the batched kernels of `mode` for chunks of up to 2^kmax amplitudes (done
// by the launcher itself too; call it before a stream capture so that no attribute is set during one).
cudaError_t prepare_fused_batch(int mode, int kmax);
cudaError_t launch_fused_batch(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass,
                               uint64_t total_chunks, int mode, int kmax, cudaStream_t st, int f64_share = 0,
                               FusedSched *sched = nullptr, int *used_mixed = nullptr);

// Batched complex128 double-float passes with dense tensor-core blocks (every pass with k = kBatchTcK and blocks),
// indexed as for launch_fused_batch.  A wait for the tensor cores that runs out sets sched->tc_err (never
// cleared here).  prepare_fused_batch_tc raises the kernel's shared-memory grant outside a stream capture.
constexpr int kBatchTcK = 12;
cudaError_t prepare_fused_batch_tc();
cudaError_t launch_fused_batch_tc(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass,
                                  uint64_t total_chunks, cudaStream_t st, FusedSched *sched);

} // namespace svi
