// Fused chunk pass: one read and one write of the state applies a whole run of gates.
//
// The paper keeps the gates of "local" qubits (those whose amplitude pairs lie in one process's slice of
// the vector) free of communication (Sec. V.A, V.C) and proposes relabelling qubits so that the busy ones
// are local (Sec. VI.B).  On one GPU the analogue of a process's slice is a chunk of 2^k amplitudes held in
// shared memory: the amplitudes whose indices agree on every bit outside a chosen set Q of k physical bits.
// Q always holds the c lowest bits, so a chunk is 2^(k-c) runs of 2^c contiguous amplitudes (coalesced
// 256-byte rows); its other k - c bits can be any higher bits.  Every gate whose target lies in Q (and every
// diagonal gate, wherever its target) is applied to the chunk in shared memory with the pair update of
// Sec. V.A; control bits inside Q are inserted as fixed one-bits of the enumerated index (tested per
// amplitude inside complex64 register cubes), control bits outside Q are tested once per chunk.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "sv_internal.h"
#include "sv_arith.cuh"

namespace svi {
namespace {

constexpr int kFusedThreads = 256;
#ifndef SV_FUSED_MIN_BLOCKS
#define SV_FUSED_MIN_BLOCKS 3
#endif
#ifndef SV_FUSED_MIN_BLOCKS_C64
#define SV_FUSED_MIN_BLOCKS_C64 2
#endif
template <int MODE>
constexpr int min_blocks() { return MODE == MODE_C64_F32 ? SV_FUSED_MIN_BLOCKS_C64 : SV_FUSED_MIN_BLOCKS; }

__device__ __forceinline__ uint32_t ins0(uint32_t i, int t) {
  return ((i >> t) << (t + 1)) | (i & ((1u << t) - 1u));
}

// The i-th index, in ascending order, whose bits in `fix` equal those of `val`: the bits of i with the fixed
// bits inserted at their positions, lowest first.  Lets a controlled gate visit only the amplitudes it
// changes instead of testing every index.
__device__ __forceinline__ uint32_t expand_fixed(uint32_t i, uint32_t fix, uint32_t val) {
  for (uint32_t f = fix; f != 0u; f &= f - 1u) {
    const uint32_t b = (uint32_t)(__ffs((int)f) - 1), low = (1u << b) - 1u;
    i = ((i & ~low) << 1) | (val & (1u << b)) | (i & low);
  }
  return i;
}

// Unroll of the shared-memory pair loops: 2 for complex128 (the FP64 CTA and the controlled double-float
// gates run faster), 1 for complex64 (n = 30 random circuit: 462 -> 449 ms).
#ifndef SV_FUSED_PAIR_UNROLL
#define SV_FUSED_PAIR_UNROLL 2
#endif
#ifndef SV_FUSED_PAIR_UNROLL_C64
#define SV_FUSED_PAIR_UNROLL_C64 1
#endif
template <int MODE>
__host__ __device__ constexpr int pair_unroll() { return MODE == MODE_C64_F32 ? SV_FUSED_PAIR_UNROLL_C64 : SV_FUSED_PAIR_UNROLL; }

// Shared-memory slot of chunk-local amplitude o.  Complex64 chunks XOR bits 4..6 of the index into bits 1..3,
// so that the threads of a half-warp, whose register cubes differ in the lowest bits outside the cube, land
// on distinct banks.  Bit 0 is left alone, so amplitudes 2m and 2m+1 stay adjacent (one 16-byte copy); the
// map only permutes each aligned group of 128 slots, so it is a bijection for every k.
template <int MODE>
__device__ __forceinline__ uint32_t slot(uint32_t o) {
  if constexpr (MODE == MODE_C64_F32) return o ^ (((o >> 4) & 7u) << 1);
  else return o;
}

// 16-byte asynchronous copy global -> shared (no register staging), and the wait for this thread's copies.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// All pairs (j0, j0 | tb) of the chunk for one gate of class CLS, target bit t, local controls cm.
// PACK: dense double-float pairs in packed FP32x2 instructions (Arith::pair) or in scalar ones
// (Arith::pair_scalar, for the batched kernels, whose extra live state made the packed form spill).
template <int MODE, int CLS, bool PACK = true, int NT = kFusedThreads>
__device__ __forceinline__ void chunk_pairs(typename Arith<MODE>::S *sm, const typename Arith<MODE>::Coef &cf,
                                            uint32_t half, int t, uint32_t tb, uint32_t cm) {
  using S = typename Arith<MODE>::S;
  if constexpr (MODE == MODE_C128_DF32 && CLS == GC_GENERAL && PACK) {
    if (cm == 0 && (half % (2 * NT)) == 0) {
      // Double-float dense gates, no local control: two pairs per thread loaded before either is computed,
      // so their dependency chains interleave (the compiler cannot move a load above the previous pair's
      // stores to shared memory by itself).  Pairs i and i + NT are disjoint.
#pragma unroll 1
      for (uint32_t i = threadIdx.x; i < half; i += 2 * NT) {
        const uint32_t j0 = ins0(i, t), j1 = ins0(i + NT, t);
        const uint32_t s0 = slot<MODE>(j0), s1 = slot<MODE>(j0 | tb);
        const uint32_t s2 = slot<MODE>(j1), s3 = slot<MODE>(j1 | tb);
        S a = sm[s0], b = sm[s1], a1 = sm[s2], b1 = sm[s3];
        apply_pair<MODE, PACK>(CLS, cf, a, b);
        apply_pair<MODE, PACK>(CLS, cf, a1, b1);
        sm[s0] = a;
        sm[s1] = b;
        sm[s2] = a1;
        sm[s3] = b1;
      }
      return;
    }
  }
  if (cm != 0) {
    // Local controls: only the half >> popc(cm) pairs whose control bits are all 1, enumerated directly.
    const uint32_t cnt = half >> __popc(cm);
#pragma unroll pair_unroll<MODE>()
    for (uint32_t i = threadIdx.x; i < cnt; i += NT) {
      const uint32_t j0 = expand_fixed(i, tb | cm, cm);
      const uint32_t s0 = slot<MODE>(j0), s1 = slot<MODE>(j0 | tb);
      S a = sm[s0], b = sm[s1];
      apply_pair<MODE, PACK>(CLS, cf, a, b);
      sm[s0] = a;
      sm[s1] = b;
    }
    return;
  }
#pragma unroll pair_unroll<MODE>()
  for (uint32_t i = threadIdx.x; i < half; i += NT) {
    const uint32_t j0 = ins0(i, t);
    if ((j0 & cm) != cm) continue;
    const uint32_t s0 = slot<MODE>(j0), s1 = slot<MODE>(j0 | tb);
    S a = sm[s0], b = sm[s1];
    apply_pair<MODE, PACK>(CLS, cf, a, b);
    sm[s0] = a;
    sm[s1] = b;
  }
}

// All quadruples of the chunk for a dense two-qubit gate (GC_DENSE4 + three GC_ROW records): chunk bits t0
// (index bit b0 of the gate's matrix) and t1 (b1), local controls cm.  The four outputs are computed from
// the old values before any is stored.
template <int MODE, int NT = kFusedThreads>
__device__ __noinline__ void chunk_quads(typename Arith<MODE>::S *sm, const DevGate *rows, uint32_t nquads, int t0,
                                            int t1, uint32_t cm) {
  using M = Arith<MODE>;
  using S = typename M::S;
  const int lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
  const uint32_t b0 = 1u << t0, b1 = 1u << t1;
  for (uint32_t i = threadIdx.x; i < nquads; i += NT) {
    const uint32_t j = ins0(ins0(i, lo), hi);
    if ((j & cm) != cm) continue;
    const uint32_t s0 = slot<MODE>(j), s1 = slot<MODE>(j | b0), s2 = slot<MODE>(j | b1), s3 = slot<MODE>(j | b0 | b1);
    const S x0 = sm[s0], x1 = sm[s1], x2 = sm[s2], x3 = sm[s3];
    S r0, r1, r2, r3;
    if constexpr (MODE == MODE_C128_DF32) {
      r0 = M::row4g(rows[0], x0, x1, x2, x3);
      r1 = M::row4g(rows[1], x0, x1, x2, x3);
      r2 = M::row4g(rows[2], x0, x1, x2, x3);
      r3 = M::row4g(rows[3], x0, x1, x2, x3);
    } else {
      typename M::Coef cf;
      M::coef(cf, rows[0]);
      r0 = M::row4(cf, x0, x1, x2, x3);
      M::coef(cf, rows[1]);
      r1 = M::row4(cf, x0, x1, x2, x3);
      M::coef(cf, rows[2]);
      r2 = M::row4(cf, x0, x1, x2, x3);
      M::coef(cf, rows[3]);
      r3 = M::row4(cf, x0, x1, x2, x3);
    }
    sm[s0] = r0;
    sm[s1] = r1;
    sm[s2] = r2;
    sm[s3] = r3;
  }
}

// ---- Complex64 register cubes (GC_CUBE) ----------------------------------------------------------------
// v[s] holds the amplitude whose cube bits spell s (bit i of s = chunk bit pos[i]).  Each routine applies one
// gate to the 2^CB registers with the same arithmetic, in the same order, as the shared-memory pair loop, so
// the two paths give identical results.  cs: the gate's control bits inside the cube, as cube bits (the
// planner stores it, and the cube slot of the target, in the gate record; see GC_CUBE).
using C64 = Arith<MODE_C64_F32>;

template <int CB, int J, int CLS, bool CTL>
__device__ __forceinline__ void cube_pairs(float2 (&v)[1 << CB], const CoefF32 &cf, uint32_t cs) {
  if constexpr (J < CB) {
#pragma unroll
    for (int s = 0; s < (1 << CB); ++s) {
      if (s & (1 << J)) continue;
      if (CTL && ((uint32_t)s & cs) != cs) continue;
      apply_pair<MODE_C64_F32>(CLS, cf, v[s], v[s | (1 << J)]);
    }
  }
}

// CTL = false: the gate has no control bit inside the cube (cs = 0), so no per-pair test is compiled.
template <int CB, int CLS, bool CTL = true>
__device__ __forceinline__ void cube_pairs_at(int j, float2 (&v)[1 << CB], const CoefF32 &cf, uint32_t cs) {
  switch (j) {
    case 0: cube_pairs<CB, 0, CLS, CTL>(v, cf, cs); break;
    case 1: cube_pairs<CB, 1, CLS, CTL>(v, cf, cs); break;
    case 2: cube_pairs<CB, 2, CLS, CTL>(v, cf, cs); break;
    case 3: cube_pairs<CB, 3, CLS, CTL>(v, cf, cs); break;
    default: cube_pairs<CB, 4, CLS, CTL>(v, cf, cs); break;
  }
}

// Diagonal gate whose target bit is the same for all registers (one = that bit).
template <int CB>
__device__ __forceinline__ void cube_diag_uniform(float2 (&v)[1 << CB], const CoefF32 &cf, uint32_t cs, bool one,
                                                  bool phase) {
  if (!one && phase) return;
  const float qr = one ? cf.q[6] : cf.q[0], qi = one ? cf.q[7] : cf.q[1];
#pragma unroll
  for (int s = 0; s < (1 << CB); ++s) {
    if (((uint32_t)s & cs) != cs) continue;
    v[s] = make_float2(__fmaf_rn(qr, v[s].x, -qi * v[s].y), __fmaf_rn(qr, v[s].y, qi * v[s].x));
  }
}

// The slot map is linear over GF(2) (an XOR of shifted index bits), so the slot of base | (cube bits of s) is
// slot(base) XOR the slots of the cube bits set in s.
template <int CB>
__device__ __forceinline__ uint32_t cube_xoff(int s, const uint32_t (&soff)[CB]) {
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < CB; ++j)
    if (s & (1 << j)) x ^= soff[j];
  return x;
}

// The cube's `cnt` gates over the CB chunk bits packed in `posw` (one byte each, ascending), for every base
// index of the chunk.
template <int CB, int NT = kFusedThreads>
__device__ __forceinline__ void cube_run(const DevGate *gs, int cnt, uint64_t posw, uint64_t base, float2 *sm, int k) {
  int p[CB];
  uint32_t soff[CB], cube = 0;
#pragma unroll
  for (int j = 0; j < CB; ++j) {
    p[j] = (int)((posw >> (8 * j)) & 0xffu);
    cube |= 1u << p[j];
    soff[j] = slot<MODE_C64_F32>(1u << p[j]);
  }
  const uint32_t nbase = 1u << (k - CB);
  for (uint32_t bi = threadIdx.x; bi < nbase; bi += NT) {
    uint32_t bidx = bi;
#pragma unroll
    for (int j = 0; j < CB; ++j) bidx = ins0(bidx, p[j]);
    const uint32_t b0 = slot<MODE_C64_F32>(bidx);
    float2 v[1 << CB];
#pragma unroll
    for (int s = 0; s < (1 << CB); ++s) v[s] = sm[b0 ^ cube_xoff<CB>(s, soff)];
    for (int gi = 0; gi < cnt; ++gi) {
      const DevGate &g = gs[gi];
      if ((base & g.gmask) != g.gmask) continue;
      const uint64_t cmw = g.cmask;
      const uint32_t cb = (uint32_t)cmw & ~cube;
      if ((bidx & cb) != cb) continue;
      const uint32_t cs = (uint32_t)(cmw >> 32) & 31u;
      const int j = (int)((cmw >> 40) & 7u) - 1;
      const uint32_t cls = g.cls;
      CoefF32 cf;
      if (cls != GC_X) C64::coef(cf, g);
      switch (cls) {
        case GC_GENERAL:
          if (cs == 0) cube_pairs_at<CB, GC_GENERAL, false>(j, v, cf, cs);
          else cube_pairs_at<CB, GC_GENERAL>(j, v, cf, cs);
          break;
        case GC_ANTIDIAG: cube_pairs_at<CB, GC_ANTIDIAG>(j, v, cf, cs); break;
        case GC_X: cube_pairs_at<CB, GC_X>(j, v, cf, cs); break;
        default: {
          const int t = g.target;
          if (j >= 0 && cls == GC_DIAG) cube_pairs_at<CB, GC_DIAG>(j, v, cf, cs);
          else if (j >= 0) cube_pairs_at<CB, GC_PHASE>(j, v, cf, cs);
          else cube_diag_uniform<CB>(v, cf, cs, t >= 0 ? ((bidx >> t) & 1u) != 0 : (base & g.tmask) != 0, cls == GC_PHASE);
          break;
        }
      }
    }
    // Recompute the slots for the store (an opaque copy of b0 keeps the compiler from holding all 2^CB
    // load addresses live across the gates).
    uint32_t b1 = b0;
    asm volatile("" : "+r"(b1));
#pragma unroll
    for (int s = 0; s < (1 << CB); ++s) sm[b1 ^ cube_xoff<CB>(s, soff)] = v[s];
  }
}

// ---- Dense blocks on the tensor cores (GC_BLOCK) -----------------------------------------------------
// A block multiplies every row of the chunk (the 16 amplitudes that differ only in the block's 4 chunk bits)
// by the block's matrix: D = X W^T with X the rows in real form (Re 0..15 | Im 0..15) and W the real form of
// the 16 x 16 unitary.  X is written to shared memory as bfloat16 planes (A operand), W's planes come from the
// gate blob (B operand); one thread issues tcgen05.mma (M = 128 rows, N = 32, K = 16 per instruction) into a
// TMEM accumulator, commits to an mbarrier, and after the bounded wait every thread reads its row of D back
// with tcgen05.ld and stores the 16 new amplitudes into the chunk.

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor of an operand plane: no swizzle, K-major core matrices of 8 rows x 16 bytes,
// K-adjacent core matrices 128 bytes apart (leading byte offset), 8-row groups 512 bytes apart (stride byte
// offset), descriptor version 1 (bit 46).  The layout is the one sv_block.cpp writes for W.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor of kind::f16: f32 accumulator (bits 4-5 = 1), bfloat16 A and B (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128; N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
constexpr int kTcRowBytes = kBlockK * 2;          // one row of one plane
constexpr int kTcTileBytes = 128 * kTcRowBytes;   // 128 rows of one plane
constexpr uint64_t kTcWaitNs = 2000000000ull;     // bound of one wait for the tensor cores

// The planner keeps c >= min(3, k), so the row table never has more than max(1, 2^(k-3)) entries; 128 bytes
// of permuted-store table follow it.
template <int MODE>
__host__ __device__ constexpr int smem_bytes(int k) {
  return (int)(sizeof(typename Arith<MODE>::S) << k) + (int)(sizeof(uint64_t) << (k > 3 ? k - 3 : 0)) + 128;
}

// Tensor-core pass: the fused pass's shared memory, then (1024-byte aligned) the A planes of all rows, the B
// planes of one block, the mbarrier and the TMEM address slot.
template <int MODE>
__host__ __device__ constexpr int tc_planes() { return MODE == MODE_C64_F32 ? kBlockSplitsC64 : kBlockDigitsC128; }
template <int MODE>
__host__ __device__ constexpr int tc_smem_base(int k) { return (smem_bytes<MODE>(k) + 1023) & ~1023; }
// B planes per pair: complex128 keeps a zero plane in front of the block's six digit planes (see tc_issue).
template <int MODE>
__host__ __device__ constexpr int tc_bplanes() { return MODE == MODE_C64_F32 ? kBlockSplitsC64 : kBlockDigitsC128 + 1; }
template <int MODE>
__host__ __device__ constexpr int tc_smem_bytes(int k) {
  return tc_smem_base<MODE>(k) + tc_planes<MODE>() * ((1 << (k - kBlockBits)) * kTcRowBytes) +
         2 * tc_bplanes<MODE>() * (int)kBlockPlaneBytes + 256;
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
               : "memory");
}

// Bounded wait for the mbarrier phase with parity `ph`; false if it ran out.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t ph) {
  const uint32_t a = smem_addr(mbar);
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(a), "r"(ph)
                 : "memory");
    if (ok) return true;
    if (global_ns() - t0 > kTcWaitNs) return false;
  }
}

// Work split of the tensor-core pass (kTcThreads threads): warp groups 2p and 2p + 1 form pair p, which takes
// tiles p, p + kTcPairs, ..; in each tile, warp group 2p + h builds and reads back part h of every row
// (h = 0: the real parts, K columns 0..15 and outputs 0..15; h = 1: the imaginary parts, 16..31), so every
// warp group has work even for a chunk of two tiles.  TMEM lanes 32 (w % 4) .. + 31 belong to warp w, so each
// warp group reads all 128 lanes (rows) of a tile.
constexpr int kTcThreads = 512;
constexpr int kTcGroups = kTcThreads / 128;
constexpr int kTcPairs = kTcGroups / 2;
constexpr int kTcMaxTiles = 4;                    // 2^13-amplitude chunks: 512 rows
constexpr int kTcGateCopy = 64;                   // gate records staged in shared memory per pass

// Per-CTA state of the tensor-core pass (the same in every thread).
struct TcCtx {
  unsigned char *opA;   // A planes: plane-major, rows x kTcRowBytes each
  unsigned char *opB;   // B planes, one set per pair (kTcPairs x tc_bplanes x kBlockPlaneBytes)
  uint64_t *mbar;       // one mbarrier per tile
  uint32_t tmem;        // TMEM address of this CTA's accumulators (lane 0, first column)
  uint32_t phase;       // parity of the next phase of every tile's mbarrier
  int ok;               // 0 once a wait ran out: later blocks are skipped
  unsigned *err;        // global error word
  float *red;           // kTcThreads / 32 floats of shared scratch (complex128 chunk norm)
  float sc, isc;        // complex128: 2^(47 - E) and 2^(E - 62) for the current chunk's exponent E
  int fixed_in;         // complex128: the chunk holds the previous block's output in fixed point (see below)
  int no_mma;           // test hook: issue no MMA (every wait for the tensor cores then runs out)
};

// Row r's base slot (its index with zeros at the block bits, through the slot map).
template <int MODE>
__device__ __forceinline__ uint32_t tc_row_base(uint32_t r, const int (&pb)[kBlockBits]) {
  uint32_t bidx = r;
#pragma unroll
  for (int j = 0; j < kBlockBits; ++j) bidx = ins0(bidx, pb[j]);
  return slot<MODE>(bidx);
}

// Slot offset of element s of a row: the block bits set in s, through the slot map (linear over GF(2)).
template <int MODE>
__device__ __forceinline__ uint32_t tc_elem(int s, const int (&pb)[kBlockBits]) {
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < kBlockBits; ++j)
    if (s & (1 << j)) x ^= slot<MODE>(1u << pb[j]);
  return x;
}

// 16-byte store of eight bfloat16 values (four packed pairs).
__device__ __forceinline__ void st_planes(unsigned char *dst, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  *reinterpret_cast<uint4 *>(dst) = make_uint4(w0, w1, w2, w3);
}
__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }
__device__ __forceinline__ uint32_t bf2_pack(float a, float b) { return bf2_bits(__floats2bfloat162_rn(a, b)); }

__device__ __forceinline__ void pair_sync(uint32_t pair) {
  asm volatile("bar.sync %0, 256;" ::"r"(pair + 1u) : "memory");
}

// Issue tile t's MMAs and commit them to the tile's mbarrier.  Called by one thread.
// complex64: the six products x_i w_j with i + j <= 2 (i: A plane, j: B plane) into one 32-column accumulator.
// complex128: the products t_a u_b accumulate per digit level L = a + b = 4..10 in columns 32 (L - 4) .. + 31.
// The B planes sit in shared memory as [0, u_0, u_1, .., u_5] (a zero plane first, each plane 32 rows of N),
// and consecutive planes continue the 8-row-group stride, so for one A plane a the window of planes
// u_{4-a} .. u_{10-a} is a single B operand of N = 32 (levels) rows: one MMA computes t_a's products for
// every level at once.  a = 5 goes first over all seven levels (its window starts at the zero plane: level 4
// gets t_5 * 0) and initialises the accumulator; a = 4 .. 0 then add levels 4 .. a + 5 (N = 32 (a + 2)).  That
// is 6 MMAs per K step instead of one per digit pair (26), for the same products.
template <int MODE>
__device__ __forceinline__ void tc_issue(const TcCtx &tc, uint32_t t, uint32_t R, const unsigned char *myB) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t a0 = smem_addr(tc.opA) + t * kTcTileBytes, bb0 = smem_addr(myB);
  if constexpr (MODE == MODE_C64_F32) {
    const uint32_t d = tc.tmem + t * kBlockK;
    uint32_t acc = 0;
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
      const int i = pr == 2 || pr == 4 ? 1 : pr == 5 ? 2 : 0;
      const int j = pr == 1 || pr == 4 ? 1 : pr == 3 ? 2 : 0;
#pragma unroll
      for (int ks = 0; ks < kBlockK / 16; ++ks) {
        tc_mma(d, tc_desc(a0 + (uint32_t)i * R * kTcRowBytes + (uint32_t)ks * 256),
               tc_desc(bb0 + (uint32_t)j * (uint32_t)kBlockPlaneBytes + (uint32_t)ks * 256), tc_idesc(kBlockK), acc);
        acc = 1;
      }
    }
  } else {
    const uint32_t d = tc.tmem + t * (7 * kBlockK);
    uint32_t acc = 0;
#pragma unroll
    for (int a = kBlockDigitsC128 - 1; a >= 0; --a) {
      // window start: plane u_{4 - a} (index 5 - a in the array), the zero plane (index 0) for a = 5
      const uint32_t first = a == kBlockDigitsC128 - 1 ? 0u : (uint32_t)(5 - a);
      const uint32_t n = a == kBlockDigitsC128 - 1 ? 7u * kBlockK : (uint32_t)(a + 2) * kBlockK;
#pragma unroll
      for (int ks = 0; ks < kBlockK / 16; ++ks) {
        tc_mma(d, tc_desc(a0 + (uint32_t)a * R * kTcRowBytes + (uint32_t)ks * 256),
               tc_desc(bb0 + first * (uint32_t)kBlockPlaneBytes + (uint32_t)ks * 256), tc_idesc(n), acc);
        acc = 1;
      }
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(tc.mbar + t))
               : "memory");
}

// ---- complex64 parts ----
// A planes of part h of row r: the 16 components split into three bfloat16 planes x = x0 + x1 + x2.
__device__ __forceinline__ void tc_rows_c64(const float2 *sm, uint32_t b0, const int (&pb)[kBlockBits], uint32_t h,
                                            unsigned char *row, uint32_t R) {
  float x[kBlockDim];
#pragma unroll
  for (int s = 0; s < kBlockDim; ++s) {
    const float2 v = sm[b0 ^ tc_elem<MODE_C64_F32>(s, pb)];
    x[s] = h ? v.y : v.x;
  }
#pragma unroll
  for (int pl = 0; pl < kBlockSplitsC64; ++pl) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
      w[q] = bf2_bits(b);
      if (pl + 1 < kBlockSplitsC64) {
        const float2 f = __bfloat1622float2(b);
        x[2 * q] -= f.x;
        x[2 * q + 1] -= f.y;
      }
    }
    unsigned char *dst = row + (size_t)pl * R * kTcRowBytes + h * 256;
    st_planes(dst, w[0], w[1], w[2], w[3]);
    st_planes(dst + 128, w[4], w[5], w[6], w[7]);
  }
}

// Outputs 16 h .. 16 h + 15 of this lane's row (16 TMEM columns), load and wait in one asm statement.
__device__ __forceinline__ void tc_load16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- complex128 parts: exact digit products ----
// x (a double-float h + l with |x| < 2^E, E fixed per chunk: the chunk's 2-norm, which its unitary gates
// preserve, bounds every amplitude) is scaled to v = x 2^(47 - E), |v| <= 2^47, and written as six balanced
// base-256 digits t_a in [-128, 128] (v ~ sum_a t_a 256^a), each exact in bfloat16.  With the matrix's digits
// u_b of w 2^47 (host), every product t_a u_b is an exact integer below 2^14; the products of one digit level
// L = a + b, summed over K = 32 terms and at most 6 pairs, stay below 2^22, so the FP32 accumulation in TMEM
// is exact.  Levels 4..10 are kept (26 products): the dropped levels are below 2^-45 of |x|'s bound.
__device__ __forceinline__ float rint_small(float x) {  // round to nearest integer, |x| < 2^22
  return __fadd_rn(__fadd_rn(x, 12582912.0f), -12582912.0f);
}

// Six balanced base-256 digits of v = (h + l) * sc (see above); t[0] least significant.
__device__ __forceinline__ void df_digits(float h, float l, float sc, float (&t)[6]) {
  float H = __fmul_rn(h, sc), L = __fmul_rn(l, sc);
  t[5] = rint_small(__fmul_rn(H, 0x1p-40f));
  H = __fmaf_rn(-t[5], 0x1p40f, H);
  t[4] = rint_small(__fmul_rn(H, 0x1p-32f));
  H = __fmaf_rn(-t[4], 0x1p32f, H);
  float e;
  two_sum(H, L, H, e);
  L = e;
  t[3] = rint_small(__fmul_rn(H, 0x1p-24f));
  H = __fmaf_rn(-t[3], 0x1p24f, H);
  t[2] = rint_small(__fmul_rn(H, 0x1p-16f));
  H = __fmaf_rn(-t[2], 0x1p16f, H);
  two_sum(H, L, H, e);
  L = e;
  t[1] = rint_small(__fmul_rn(H, 0x1p-8f));
  H = __fmaf_rn(-t[1], 0x1p8f, H);
  t[0] = rint_small(__fadd_rn(H, L));
}

// A planes of part h of row r: six digit planes of the 16 components (groups of 8 columns).
__device__ __forceinline__ void tc_rows_c128(const float4 *sm, uint32_t b0, const int (&pb)[kBlockBits], uint32_t h,
                                             unsigned char *row, uint32_t R, float sc) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float dg[8][6];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float4 v = sm[b0 ^ tc_elem<MODE_C128_DF32>(q * 8 + e, pb)];
      if (h) df_digits(v.z, v.w, sc, dg[e]);
      else df_digits(v.x, v.y, sc, dg[e]);
    }
#pragma unroll
    for (int a = 0; a < kBlockDigitsC128; ++a)
      st_planes(row + (size_t)a * R * kTcRowBytes + h * 256 + q * 128, bf2_pack(dg[0][a], dg[1][a]),
                bf2_pack(dg[2][a], dg[3][a]), bf2_pack(dg[4][a], dg[5][a]), bf2_pack(dg[6][a], dg[7][a]));
  }
}

// Columns 4 g .. 4 g + 3 of part h of every digit level of one tile, for this lane (28 values), in one asm
// statement ending with the load wait.  a = TMEM address of level 0's first column of the part, + 4 g.
__device__ __forceinline__ void tc_load_levels(uint32_t a, float (&d)[7][4]) {
  uint32_t r[28];
  asm volatile(
      "{\n"
      ".reg .b32 ta;\n"
      "add.u32 ta, %28, 0;\n"   "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [ta];\n"
      "add.u32 ta, %28, 32;\n"  "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [ta];\n"
      "add.u32 ta, %28, 64;\n"  "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [ta];\n"
      "add.u32 ta, %28, 96;\n"  "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [ta];\n"
      "add.u32 ta, %28, 128;\n" "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16,%17,%18,%19}, [ta];\n"
      "add.u32 ta, %28, 160;\n" "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%20,%21,%22,%23}, [ta];\n"
      "add.u32 ta, %28, 192;\n" "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%24,%25,%26,%27}, [ta];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "}\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27])
      : "r"(a)
      : "memory");
#pragma unroll
  for (int L = 0; L < 7; ++L)
#pragma unroll
    for (int e = 0; e < 4; ++e) d[L][e] = __uint_as_float(r[4 * L + e]);
}

// S = sum_{i=0..6} D_i 256^i (D_i: digit level 4 + i, exact integers below 2^22) modulo 2^64, formed exactly
// in 64-bit integer arithmetic: each D_i enters as the bit pattern of D_i + 1.5 * 2^23, the patterns' constant
// part removed once at the end (all sums wrap modulo 2^64; S itself is below 2^62 in magnitude).  The block's
// output is y = 2^(E - 62) S.
__device__ __forceinline__ uint64_t levels_to_int(const float (&d)[7]) {
  uint32_t b[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) b[i] = __float_as_uint(__fadd_rn(d[i], 12582912.0f));
  constexpr uint64_t kMagic = 0x4B400000ull;
  constexpr uint64_t kBias = kMagic * (1ull + (1ull << 8) + (1ull << 16) + (1ull << 24) + (1ull << 32) + (1ull << 40) +
                                       (1ull << 48));
  const uint32_t top = b[4] + (b[5] << 8) + (b[6] << 16);
  return (uint64_t)b[0] + ((uint64_t)b[1] << 8) + ((uint64_t)b[2] << 16) + ((uint64_t)b[3] << 24) +
         ((uint64_t)top << 32) - kBias;
}

// y = 2^(E - 62) S as a normalised double-float: S split into 22-bit pieces that convert to float exactly.
__device__ __forceinline__ dfv int_to_df(uint64_t acc, float isc) {
  const uint32_t lo = (uint32_t)acc, hi = (uint32_t)(acc >> 32);
  const uint32_t c0 = lo & 0x3FFFFFu, c1 = __funnelshift_r(lo, hi, 22) & 0x3FFFFFu;
  const int32_t c2 = (int32_t)hi >> 12;
  const float f0 = __fadd_rn(__uint_as_float(0x4B000000u | c0), -8388608.0f);
  const float f1 = __fadd_rn(__uint_as_float(0x4B000000u | c1), -8388608.0f);
  const float f2 = __fadd_rn(__uint_as_float((uint32_t)(0x4B400000 + c2)), -12582912.0f);
  float h, e;
  two_sum(__fmul_rn(f2, 0x1p44f), __fmul_rn(f1, 0x1p22f), h, e);
  const dfv r = fast_two_sum(h, __fadd_rn(e, f0));
  return dfv{__fmul_rn(r.h, isc), __fmul_rn(r.l, isc)};
}

// Fixed-point hand-off between two blocks.  When the next gate record of the pass is also a block, a block
// writes each output component as w = v + kDigitBias in its 8-byte half of the slot, with v = round(S / 2^15)
// = round(y 2^(47 - E)): the very integer the next block's digit split would round y to (the chunk's E is the
// same for both).  With kDigitBias = 128 (1 + 256 + .. + 256^5), bytes 0..4 of w are t_0 + 128 .. t_4 + 128
// and w >> 40 = t_5 + 128 for balanced digits t_a of v (t_5 in [-128, 128]: |v| <= 2^47 keeps w in
// [0, 2^48 + 2^40)), so the next block reads its six digits with one byte select and one exact float
// subtraction each, and skips both the double-float conversion and the digit split.
constexpr uint64_t kDigitBias = 0x808080808080ull;

__device__ __forceinline__ uint2 int_to_fixed(uint64_t acc) {
  const uint64_t w = (uint64_t)(((int64_t)acc + (1ll << 14)) >> 15) + kDigitBias;
  return make_uint2((uint32_t)w, (uint32_t)(w >> 32));
}

// The float 2^23 + b for a byte b selected from x (0x4B0000bb), minus 2^23 + 128: b - 128 exactly.
__device__ __forceinline__ float byte_digit(uint32_t x, uint32_t sel) {
  return __fadd_rn(__uint_as_float(__byte_perm(x, 0x4B000000u, sel)), -8388736.0f);
}

__device__ __forceinline__ void fixed_digits(uint2 w, float (&t)[6]) {
  t[0] = byte_digit(w.x, 0x7650u);
  t[1] = byte_digit(w.x, 0x7651u);
  t[2] = byte_digit(w.x, 0x7652u);
  t[3] = byte_digit(w.x, 0x7653u);
  t[4] = byte_digit(w.y, 0x7650u);
  t[5] = __fadd_rn(__uint_as_float(0x4B000000u | (w.y >> 8)), -8388736.0f);
}

// A planes of part h of row r from the previous block's fixed-point output.
__device__ __forceinline__ void tc_rows_c128_fixed(const float4 *sm, uint32_t b0, const int (&pb)[kBlockBits],
                                                   uint32_t h, unsigned char *row, uint32_t R) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float dg[8][6];
#pragma unroll
    for (int e = 0; e < 8; ++e)
      fixed_digits(reinterpret_cast<const uint2 *>(&sm[b0 ^ tc_elem<MODE_C128_DF32>(q * 8 + e, pb)])[h], dg[e]);
#pragma unroll
    for (int a = 0; a < kBlockDigitsC128; ++a)
      st_planes(row + (size_t)a * R * kTcRowBytes + h * 256 + q * 128, bf2_pack(dg[0][a], dg[1][a]),
                bf2_pack(dg[2][a], dg[3][a]), bf2_pack(dg[4][a], dg[5][a]), bf2_pack(dg[6][a], dg[7][a]));
  }
}

// Sum of the squares of the chunk's high words (times `scale`), over the CTA; the same in every thread.
__device__ __forceinline__ float tc_sum_squares(const float4 *sm, uint32_t nloc, float scale, TcCtx &tc) {
  float part = 0.0f;
  for (uint32_t o = threadIdx.x; o < nloc; o += kTcThreads) {
    const float4 v = sm[o];
    const float a = __fmul_rn(v.x, scale), b = __fmul_rn(v.z, scale);
    part = __fmaf_rn(a, a, __fmaf_rn(b, b, part));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31u) == 0) tc.red[threadIdx.x >> 5] = part;
  __syncthreads();
  float tot = 0.0f;
#pragma unroll
  for (int w = 0; w < kTcThreads / 32; ++w) tot += tc.red[w];
  __syncthreads();  // tc.red is reused
  return tot;
}

// Chunk exponent of a complex128 chunk in working form: E with 2^E above the chunk's 2-norm (from the high
// words, with a margin of 2^-8 for the low words and rounding); sets tc.sc = 2^(47 - E), tc.isc = 2^(E - 62).
// The squares overflow FP32 once amplitudes reach 2^64: such chunks (the same decision in every thread) are
// summed again with the values scaled by 2^-100.  E is clamped to [-80, 150]: amplitudes below 2^-80 are then
// cut to a few 2^-127; every complex128 amplitude the library accepts (components below 2^126) leaves a chunk
// norm below 2^150.
__device__ __forceinline__ void tc_chunk_scale(const float4 *sm, uint32_t nloc, TcCtx &tc) {
  float tot = tc_sum_squares(sm, nloc, 1.0f, tc);
  int bias = 0;
  if (!(tot <= 3.0e38f)) {
    tot = tc_sum_squares(sm, nloc, 0x1p-100f, tc);
    bias = 100;
  }
  int E = 0;
  frexpf(sqrtf(__fmaf_rn(tot, 0x1p-8f, tot)) + 0x1p-126f, &E);
  E += bias;
  E = E < -80 ? -80 : (E > 150 ? 150 : E);
  tc.sc = __int_as_float((127 + 47 - E) << 23);
  const int ei = E - 62;
  tc.isc = ei >= -126 ? __int_as_float((127 + ei) << 23) : __int_as_float(1 << (ei + 149));
}

// One dense block (GC_BLOCK) on the chunk: every row of the chunk (the 16 amplitudes that differ only in the
// block's 4 chunk bits) times the block's matrix, D = X W^T.  Pair p writes the A planes of its tiles (each warp
// group one part), copies the matrix's planes, and one of its threads issues each tile's MMAs as soon as the
// tile is written (committed to the tile's mbarrier), so the tensor core works on tile t while the pair writes
// tile t + kTcPairs; then each warp group waits for its tiles and writes its part of the results back.  The
// CTA synchronises only at the end of the block (the next block's rows mix amplitudes of every tile).
template <int MODE>
__device__ __forceinline__ void tc_block(const DevGate &hdr, const DevGate *ghdr, typename Arith<MODE>::S *sm, int k,
                                         TcCtx &tc, bool next_block, uint32_t sx) {
  constexpr int planes = MODE == MODE_C64_F32 ? kBlockSplitsC64 : kBlockDigitsC128;
  const uint32_t tid = threadIdx.x, g = tid >> 7, pair = g >> 1, h = g & 1u, lane = tid & 127u;
  const uint32_t R = 1u << (k - kBlockBits), ntiles = R / 128;
  const unsigned char *src = reinterpret_cast<const unsigned char *>(ghdr) + hdr.gmask;  // offset from the blob record
  unsigned char *myB = tc.opB + (size_t)pair * tc_bplanes<MODE>() * kBlockPlaneBytes;
  unsigned char *myBd = myB + (MODE == MODE_C64_F32 ? 0 : kBlockPlaneBytes);  // the block's planes
  int pb[kBlockBits];
#pragma unroll
  for (int j = 0; j < kBlockBits; ++j) pb[j] = (int)((hdr.cmask >> (8 * j)) & 0xffu);
  int ok = tc.ok;
  if (pair < ntiles) {
    for (uint32_t u = tid & 255u; u < (uint32_t)(planes * kBlockPlaneBytes / 16); u += 256)
      cp_async16(myBd + 16u * u, src + 16u * u);
    for (uint32_t t = pair; t < ntiles; t += kTcPairs) {
      const uint32_t r = t * 128 + lane;
      const uint32_t b0 = tc_row_base<MODE>(r, pb) ^ sx;
      unsigned char *row = tc.opA + (r / 8) * 512 + (r % 8) * 16;
      if constexpr (MODE == MODE_C64_F32) tc_rows_c64(sm, b0, pb, h, row, R);
      else if (tc.fixed_in) tc_rows_c128_fixed(sm, b0, pb, h, row, R);
      else tc_rows_c128(sm, b0, pb, h, row, R, tc.sc);
      if (t == pair) cp_async_wait_all();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      pair_sync(pair);
      if ((tid & 255u) == 0 && ok && !tc.no_mma) tc_issue<MODE>(tc, t, R, myB);
    }
    for (uint32_t t = pair; t < ntiles; t += kTcPairs) {
      if (ok) ok = tc_wait(tc.mbar + t, tc.phase) ? 1 : 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t b0 = tc_row_base<MODE>(t * 128 + lane, pb) ^ sx;
      const uint32_t tl = tc.tmem + ((tid & 96u) << 16);
      if constexpr (MODE == MODE_C64_F32) {
        float dv[16];
        tc_load16(tl + t * kBlockK + h * kBlockDim, dv);
        if (ok) {
#pragma unroll
          for (int s = 0; s < kBlockDim; ++s)
            reinterpret_cast<float *>(&sm[b0 ^ tc_elem<MODE_C64_F32>(s, pb)])[h] = dv[s];
        }
      } else {
#pragma unroll 1
        for (uint32_t sg = 0; sg < kBlockDim / 4; ++sg) {
          float d[7][4];
          tc_load_levels(tl + t * (7 * kBlockK) + h * kBlockDim + 4u * sg, d);
          if (ok) {
            // elements 4 sg .. 4 sg + 3: block bits 0, 1 from e, bits 2, 3 from sg
            const uint32_t hiofs = tc_elem<MODE_C128_DF32>((int)(4 * sg), pb);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float lv[7];
#pragma unroll
              for (int L = 0; L < 7; ++L) lv[L] = d[L][e];
              const uint64_t acc = levels_to_int(lv);
              const uint32_t o = b0 ^ hiofs ^ tc_elem<MODE_C128_DF32>(e, pb);
              if (next_block) {
                reinterpret_cast<uint2 *>(&sm[o])[h] = int_to_fixed(acc);
              } else {
                const dfv y = int_to_df(acc, tc.isc);
                reinterpret_cast<float2 *>(&sm[o])[h] = make_float2(y.h, y.l);
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok);
  if (tc.ok) tc.phase ^= 1u;
  if (!ok && tc.ok && tid == 0) atomicOr(tc.err, 1u);
  tc.ok = ok;
  if constexpr (MODE == MODE_C128_DF32) tc.fixed_in = next_block ? 1 : 0;
}

// An exchange of a chunk bit with no control inside the chunk (its controls outside, if any, are tested per
// chunk before): a pure relabelling of the chunk's slots.
__device__ __forceinline__ bool lazy_x(const DevGate &g) {
  return g.cls == GC_X && g.target >= 0 && (uint32_t)g.cmask == 0u;
}

// Apply pending exchanges xm to the chunk's data: slots j and j ^ xm trade places.  Ends with a barrier.
template <int MODE, int NT>
__device__ __forceinline__ void apply_exchanges(typename Arith<MODE>::S *sm, uint32_t nloc, uint32_t xm) {
  for (uint32_t o = threadIdx.x; o < nloc; o += NT) {
    const uint32_t j = o ^ xm;
    if (o < j) {
      const typename Arith<MODE>::S a = sm[slot<MODE>(o)], b = sm[slot<MODE>(j)];
      sm[slot<MODE>(o)] = b;
      sm[slot<MODE>(j)] = a;
    }
  }
  __syncthreads();
}

// Shared-memory layout: 2^k working amplitudes, then 2^(k-c) row offsets (uint64), then 32 words for the
// permuted store's table.
template <int MODE, bool PACK = true, bool TC = false, int NT = kFusedThreads>
__device__ __forceinline__ void fused_chunk(const PassDesc &p, uint64_t chunk, typename Arith<MODE>::S *sm,
                                            uint64_t *rowoff, TcCtx *tc = nullptr, const DevGate *gcopy = nullptr) {
  // gate records: the pass's array in global memory, or a copy of it in shared memory (same order)
  const DevGate *const GR = gcopy ? gcopy : p.gates;
  using M = Arith<MODE>;
  using G = typename M::G;
  using S = typename M::S;
  const int k = p.k, c = p.c;
  const uint32_t nloc = 1u << k, half = nloc >> 1;
  const uint32_t nrows = 1u << (k - c), lowmask = (1u << c) - 1u;
  const uint32_t tid = threadIdx.x;

  // Base index of the chunk: the chunk number's bits spread over the positions outside Q.
  uint64_t base = chunk;
  for (int j = 0; j < k; ++j) {
    const int q = p.qpos[j];
    base = ((base >> q) << (q + 1)) | (base & ((1ull << q) - 1ull));
  }
  // Row offsets: row r's bits go to qpos[c..k-1].
  for (uint32_t r = tid; r < nrows; r += NT) {
    uint64_t off = 0;
    for (int j = c; j < k; ++j) off |= (uint64_t)((r >> (j - c)) & 1u) << p.qpos[j];
    rowoff[r] = off;
  }
  // Permuted store: the source slot of output slot o is the bit permutation P(o) = P(o mod 256) | P(o - o mod 256);
  // the table holds P(i * 256) for the 2^(k-8) values of i.
  uint32_t *ptab = (uint32_t *)(rowoff + nrows);
  if (p.permuted && tid < 32u && (tid << 8) < nloc) {
    uint32_t v = 0;
    for (int j = 0; j < k; ++j) v |= (((tid << 8) >> p.src_bit[j]) & 1u) << j;
    ptab[tid] = v;
  }
  __syncthreads();

  G *psi = (G *)p.psi;
  if (p.init) {
    // Basis state |init_x>: one amplitude of one chunk is 1.
    const bool mine = (p.init_x & ~p.qmask) == base;
    uint32_t lx = 0;
    for (int j = 0; j < k; ++j) lx |= (uint32_t)((p.init_x >> p.qpos[j]) & 1ull) << j;
    for (uint32_t o = tid; o < nloc; o += NT) sm[slot<MODE>(o)] = (mine && o == lx) ? M::one() : M::zero();
  } else {
    // The whole chunk in flight at once: one 16-byte asynchronous copy per amplitude (complex128) or per
    // adjacent pair (complex64), straight into its shared-memory slot.  Rows are 2^c >= 2 amplitudes long
    // and 16-byte aligned, so a pair never straddles two rows.
    constexpr uint32_t per = 16u / sizeof(G);
    for (uint32_t u = tid; u < nloc / per; u += NT) {
      const uint32_t o = u * per;
      cp_async16(&sm[slot<MODE>(o)], &psi[base + rowoff[o >> c] + (o & lowmask)]);
    }
    cp_async_wait_all();
    if constexpr (MODE == MODE_C128_DF32) {
      // Each thread converts the slots it copied, in place (double2 and the float4 working form are both
      // 16 bytes), so no barrier is needed before the conversion.
      for (uint32_t o = tid; o < nloc; o += NT) sm[o] = M::load(((const G *)sm)[o]);
    }
  }
  __syncthreads();
  if constexpr (TC && MODE == MODE_C128_DF32) {
    tc_chunk_scale(sm, nloc, *tc);
    tc->fixed_in = 0;
  }
  if constexpr (TC) tc->no_mma = p.tc_flags & 1;

  // Tensor-core passes apply an exchange (X) with no control inside the chunk lazily: the pending exchanges
  // form a mask xm, amplitude j of the chunk sits in slot slot(j ^ xm) (slot is linear over GF(2)), blocks read
  // and write through that map, and the mask is applied to the data only before a per-gate record or folded
  // into the final store.
  uint32_t xm = 0;
  for (int gi = 0; gi < p.ngates; ++gi) {
    const DevGate &g = GR[gi];
    if (g.cls == GC_BLOCK) {  // its gmask is the offset of its operand planes, not a control mask
      if constexpr (TC) {
        // a block followed by another block (lazy exchanges between them aside) hands its output over in
        // fixed point (complex128)
        int nx = gi + 1;
        while (nx < p.ngates && lazy_x(GR[nx])) ++nx;
        tc_block<MODE>(g, p.gates + gi, sm, k, *tc, nx < p.ngates && GR[nx].cls == GC_BLOCK, slot<MODE>(xm));
      }
      continue;
    }
    const uint64_t gmask = g.gmask;
    if ((base & gmask) != gmask) continue;  // a control bit outside the chunk is 0: the gate skips this chunk
    if constexpr (TC) {
      if (lazy_x(g)) {
        xm ^= 1u << g.target;
        continue;
      }
      if (xm != 0u) {
        apply_exchanges<MODE, NT>(sm, nloc, xm);
        xm = 0u;
      }
    }
    const uint32_t cls = g.cls;
    if (cls == GC_ROW) continue;  // consumed with its GC_DENSE4 record
    if (cls == GC_DENSE4) {
      chunk_quads<MODE, NT>(sm, GR + gi, nloc >> 2, g.target, (int)g.tmask, (uint32_t)g.cmask);
      gi += 3;
      __syncthreads();
      continue;
    }
    if (cls == GC_CUBE) {
      if constexpr (MODE == MODE_C64_F32) {
        cube_run<kCubeBits, NT>(GR + gi + 1, g.target, g.cmask, base, sm, k);
        gi += g.target;
        __syncthreads();
      }
      continue;  // other modes apply the cube's gates one by one
    }
    const int t = g.target;
    const uint32_t cm = (uint32_t)g.cmask;
    typename M::Coef cf;
    if (cls != GC_X) M::coef(cf, g);
    if (t >= 0) {
      const uint32_t tb = 1u << t;
      if (cls == GC_PHASE) {
        // Only the amplitudes with the target and every local control bit set.
        const uint32_t fix = tb | cm, cnt = nloc >> __popc(fix);
        for (uint32_t i = tid; i < cnt; i += NT) {
          const uint32_t j = expand_fixed(i, fix, fix);
          sm[slot<MODE>(j)] = M::cmul(cf, 3, sm[slot<MODE>(j)]);
        }
      } else {
        // One loop per class, so the class test is not inside the pair loop.
        switch (cls) {
          case GC_GENERAL: chunk_pairs<MODE, GC_GENERAL, PACK, NT>(sm, cf, half, t, tb, cm); break;
          case GC_DIAG: chunk_pairs<MODE, GC_DIAG, PACK, NT>(sm, cf, half, t, tb, cm); break;
          case GC_ANTIDIAG: chunk_pairs<MODE, GC_ANTIDIAG, PACK, NT>(sm, cf, half, t, tb, cm); break;
          default: chunk_pairs<MODE, GC_X, PACK, NT>(sm, cf, half, t, tb, cm); break;
        }
      }
    } else {
      // Diagonal gate on a qubit outside the chunk: every amplitude of the chunk has the same target bit.
      const bool one = (base & g.tmask) != 0;
      // Entry q22 (target bit 1) or q11 (0) on the amplitudes whose local control bits are all 1 (the entry
      // index stays a constant, so the coefficients stay in registers).
      const uint32_t cnt = nloc >> __popc(cm);
      if (one) {
        for (uint32_t i = tid; i < cnt; i += NT) {
          const uint32_t j = expand_fixed(i, cm, cm);
          sm[slot<MODE>(j)] = M::cmul(cf, 3, sm[slot<MODE>(j)]);
        }
      } else if (cls != GC_PHASE) {
        for (uint32_t i = tid; i < cnt; i += NT) {
          const uint32_t j = expand_fixed(i, cm, cm);
          sm[slot<MODE>(j)] = M::cmul(cf, 0, sm[slot<MODE>(j)]);
        }
      }
    }
    __syncthreads();
  }

  const uint32_t sx = slot<MODE>(xm);  // 0 unless lazy exchanges are pending (tensor-core passes)
  if (!p.permuted) {
    for (uint32_t o = tid; o < nloc; o += NT)
      psi[base + rowoff[o >> c] + (o & lowmask)] = M::store(sm[slot<MODE>(o) ^ sx]);
  } else {
    // Store with chunk-local bit j sent to physical bit qpos_out[j]: output slot o (bits in the ascending
    // order of Q) takes local amplitude P(o), bit j of P(o) = bit src_bit[j] of o.
    uint32_t plo = 0;
    for (int j = 0; j < k; ++j) plo |= (((tid & 255u) >> p.src_bit[j]) & 1u) << j;  // P(o mod 256), NT % 256 == 0
    const uint32_t *ptab = (const uint32_t *)(rowoff + nrows);
    for (uint32_t o = tid; o < nloc; o += NT)
      psi[base + rowoff[o >> c] + (o & lowmask)] = M::store(sm[slot<MODE>(plo | ptab[o >> 8]) ^ sx]);
  }
  __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(kFusedThreads, min_blocks<MODE>()) k_fused(const PassDesc p, uint64_t nchunks) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using S = typename Arith<MODE>::S;
  S *sm = (S *)smraw;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)sizeof(S) << p.k));
  for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) fused_chunk<MODE>(p, ch, sm, rowoff);
}

// Set-up of a tensor-core pass CTA for chunks of 2^k amplitudes: warp 0 allocates `ncols` TMEM columns for the
// CTA's accumulators (ncols * CTAs per SM <= 512, so the allocation never waits on a CTA of this launch), the
// first threads initialise the tiles' mbarriers the MMAs commit to, the zero plane in front of each pair's
// complex128 digit planes is cleared; both the columns and the barriers are released by tc_teardown.
template <int MODE>
__device__ __forceinline__ void tc_setup(unsigned char *smraw, int k, uint32_t ncols, unsigned *err, TcCtx &tc) {
  const uint32_t R = 1u << (k - kBlockBits);
  tc.opA = smraw + tc_smem_base<MODE>(k);
  tc.opB = tc.opA + (size_t)tc_planes<MODE>() * R * kTcRowBytes;
  tc.mbar = reinterpret_cast<uint64_t *>(tc.opB + (size_t)kTcPairs * tc_bplanes<MODE>() * kBlockPlaneBytes);
  if constexpr (MODE != MODE_C64_F32) {
    // the zero plane in front of each pair's digit planes (never written again)
    for (uint32_t u = threadIdx.x; u < (uint32_t)(kTcPairs * kBlockPlaneBytes / 16); u += kTcThreads) {
      const uint32_t pr = u / (kBlockPlaneBytes / 16), w = u % (kBlockPlaneBytes / 16);
      reinterpret_cast<uint4 *>(tc.opB + (size_t)pr * tc_bplanes<MODE>() * kBlockPlaneBytes)[w] = make_uint4(0, 0, 0, 0);
    }
  }
  uint32_t *tslot = reinterpret_cast<uint32_t *>(tc.mbar + kTcMaxTiles);
  tc.red = reinterpret_cast<float *>(tc.mbar + kTcMaxTiles + 1);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x < kTcMaxTiles) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(tc.mbar + threadIdx.x)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  tc.tmem = *tslot;
  tc.phase = 0;
  tc.ok = 1;
  tc.err = err;
  tc.fixed_in = 0;
  tc.no_mma = 0;
}

__device__ __forceinline__ void tc_teardown(const TcCtx &tc, uint32_t ncols) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(ncols) : "memory");
}

// Fused pass whose gates include dense blocks (GC_BLOCK) for the tensor cores.
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_fused_tc(const PassDesc p, uint64_t nchunks, uint32_t ncols,
                                                               unsigned *err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  using S = typename Arith<MODE>::S;
  S *sm = (S *)smraw;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)sizeof(S) << p.k));
  TcCtx tc;
  tc_setup<MODE>(smraw, p.k, ncols, err, tc);
  // The pass's gate records, copied once to shared memory (every chunk reads each of them); a pass with more
  // than kTcGateCopy records reads them from global memory.
  DevGate *gcopy = nullptr;
  if (p.ngates <= kTcGateCopy) {
    gcopy = reinterpret_cast<DevGate *>(smraw + tc_smem_bytes<MODE>(p.k));
    const uint4 *src = reinterpret_cast<const uint4 *>(p.gates);
    uint4 *dst = reinterpret_cast<uint4 *>(gcopy);
    for (uint32_t u = threadIdx.x; u < (uint32_t)p.ngates * (sizeof(DevGate) / 16); u += kTcThreads) dst[u] = src[u];
    __syncthreads();
  }
  for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x)
    fused_chunk<MODE, true, true, kTcThreads>(p, ch, sm, rowoff, &tc, gcopy);
  tc_teardown(tc, ncols);
}

// Complex128 pass split between the SM's two arithmetic units.  The double-float path keeps the FP32 pipes
// busy and leaves the FP64 pipe idle; GB300's FP64 pipe is slow (about 1.7 multiply-adds per clock per SM)
// but independent.  The first CTA to start on each SM (elected through `sched->sm_slot[%smid]`) processes
// chunks in native FP64, the others in double-float; each role takes its chunks from its own atomic counter.
// A chunk's arithmetic is fixed by its index (chunk c uses FP64 when c mod 100 < share), so results do not
// depend on scheduling.  `sched` must be zeroed before the launch.
__global__ void __launch_bounds__(kFusedThreads, SV_FUSED_MIN_BLOCKS)
    k_fused_mixed(const PassDesc p, uint64_t nchunks, int share, FusedSched *sched) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int role;
  __shared__ unsigned long long next;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)16 << p.k));
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    role = atomicAdd(&sched->sm_slot[smid % kSchedSlots], 1u) == 0u ? 1 : 0;
  }
  __syncthreads();
  if (role) {
    for (;;) {
      if (threadIdx.x == 0) next = atomicAdd(&sched->next[1], 1ull);
      __syncthreads();
      const uint64_t j = next;
      __syncthreads();
      const uint64_t c = (j / (uint64_t)share) * 100ull + (j % (uint64_t)share);
      if (c >= nchunks) break;
      fused_chunk<MODE_C128_F64>(p, c, (double2 *)smraw, rowoff);
    }
  } else {
    const uint64_t rest = (uint64_t)(100 - share);
    for (;;) {
      if (threadIdx.x == 0) next = atomicAdd(&sched->next[0], 1ull);
      __syncthreads();
      const uint64_t j = next;
      __syncthreads();
      const uint64_t c = (j / rest) * 100ull + (uint64_t)share + (j % rest);
      if (c >= nchunks) break;
      fused_chunk<MODE_C128_DF32>(p, c, (float4 *)smraw, rowoff);
    }
  }
}

// A batched round's pass descriptor, copied to shared memory for the chunk (a register copy of the 104-byte
// struct spilled).  Callers reach it after a barrier that ends the previous chunk, so no thread still reads
// the old one.
static_assert(sizeof(PassDesc) % 8 == 0, "PassDesc is copied in 8-byte words");
__device__ __forceinline__ void load_pass(PassDesc &dst, const PassDesc *src) {
  if (threadIdx.x < sizeof(PassDesc) / 8) ((uint64_t *)&dst)[threadIdx.x] = ((const uint64_t *)src)[threadIdx.x];
  __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(kFusedThreads, min_blocks<MODE>()) k_fused_batch(const PassDesc *__restrict__ passes,
                                                               const uint64_t *__restrict__ chunk_start, int npass,
                                                               uint64_t total, int kmax) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ PassDesc sp;
  using S = typename Arith<MODE>::S;
  S *sm = (S *)smraw;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)sizeof(S) << kmax));
  for (uint64_t b = blockIdx.x; b < total; b += gridDim.x) {
    int lo = 0, hi = npass - 1;  // last pass with chunk_start <= b
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    if constexpr (MODE == MODE_C64_F32) {
      // The complex64 kernel has registers to spare (no spill) and runs faster with its own copy.
      const PassDesc p = passes[lo];
      fused_chunk<MODE, false>(p, b - chunk_start[lo], sm, rowoff);
    } else {
      load_pass(sp, passes + lo);
      fused_chunk<MODE, false>(sp, b - chunk_start[lo], sm, rowoff);
    }
  }
}

// Batched pass with the FP64 / double-float split of k_fused_mixed: the round's chunks are numbered in order
// of their passes, chunk c runs in FP64 iff c mod 100 < share, and each role draws from its own counter.
__device__ __forceinline__ int batch_pass_of(const uint64_t *chunk_start, int npass, uint64_t b) {
  int lo = 0, hi = npass - 1;  // last pass with chunk_start <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunk_start[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Batched complex128 passes with dense blocks (double-float working form): every pass of the launch has chunks
// of 2^kBatchTcK amplitudes; the round's chunks are numbered in order of their passes and chunk b belongs to
// the last pass whose first chunk is <= b.  One CTA per SM, as k_fused_tc; the gate records are read from
// global memory (the passes change from chunk to chunk).
static_assert(kBatchTcK == kBlockBits + 8, "the batched tensor-core kernel is laid out for two 128-row tiles");

__global__ void __launch_bounds__(kTcThreads, 1)
    k_fused_batch_tc(const PassDesc *__restrict__ passes, const uint64_t *__restrict__ chunk_start, int npass,
                     uint64_t total, uint32_t ncols, unsigned *err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ PassDesc sp;
  float4 *sm = (float4 *)smraw;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)sizeof(float4) << kBatchTcK));
  TcCtx tc;
  tc_setup<MODE_C128_DF32>(smraw, kBatchTcK, ncols, err, tc);
  for (uint64_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int lo = batch_pass_of(chunk_start, npass, b);
    load_pass(sp, passes + lo);
    fused_chunk<MODE_C128_DF32, true, true, kTcThreads>(sp, b - chunk_start[lo], sm, rowoff, &tc);
  }
  tc_teardown(tc, ncols);
}

__global__ void __launch_bounds__(kFusedThreads, SV_FUSED_MIN_BLOCKS)
    k_fused_batch_mixed(const PassDesc *__restrict__ passes, const uint64_t *__restrict__ chunk_start, int npass,
                        uint64_t total, int kmax, int share, FusedSched *sched) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int role;
  __shared__ unsigned long long next;
  __shared__ PassDesc sp;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)16 << kmax));
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    role = atomicAdd(&sched->sm_slot[smid % kSchedSlots], 1u) == 0u ? 1 : 0;
  }
  __syncthreads();
  const uint64_t rest = (uint64_t)(100 - share);
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(&sched->next[role], 1ull);
    __syncthreads();
    const uint64_t j = next;
    __syncthreads();
    const uint64_t c = role ? (j / (uint64_t)share) * 100ull + (j % (uint64_t)share)
                            : (j / rest) * 100ull + (uint64_t)share + (j % rest);
    if (c >= total) break;
    const int pi = batch_pass_of(chunk_start, npass, c);
    load_pass(sp, passes + pi);
    if (role) fused_chunk<MODE_C128_F64>(sp, c - chunk_start[pi], (double2 *)smraw, rowoff);
    else fused_chunk<MODE_C128_DF32, false>(sp, c - chunk_start[pi], (float4 *)smraw, rowoff);
  }
}

// Largest dynamic shared-memory size already granted to kernel `fn` on the current device; raises it if
// `bytes` is larger.  One slot per (kernel, device); several host threads may call it (the serving thread and
// callers), so the slots are atomics and a raise keeps the larger value.
cudaError_t ensure_smem(const void *fn, int bytes, std::atomic<int> *granted_per_device) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (bytes <= granted_per_device[dev].load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) {
    int cur = granted_per_device[dev].load(std::memory_order_relaxed);
    while (cur < bytes && !granted_per_device[dev].compare_exchange_weak(cur, bytes, std::memory_order_release)) {
    }
  }
  return e;
}

// SM count of the device (one GPU per process), read once.
int sms() {
  static const int v = [] {
    int dev = 0, count = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    return count > 0 ? count : 1;
  }();
  return v;
}

template <int MODE>
cudaError_t fused_launch(const PassDesc &p, cudaStream_t st) {
  const int smem = smem_bytes<MODE>(p.k);
  static std::atomic<int> granted[64] = {};
  cudaError_t e = ensure_smem((const void *)k_fused<MODE>, smem, granted);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<MODE>, kFusedThreads, smem);
  if (occ < 1) occ = 1;
  const uint64_t nchunks = 1ull << (p.n - p.k);
  const uint64_t cap = (uint64_t)sms() * occ;
  const unsigned grid = (unsigned)(nchunks < cap ? nchunks : cap);
  k_fused<MODE><<<grid, kFusedThreads, smem, st>>>(p, nchunks);
  return cudaGetLastError();
}

template <int MODE>
std::atomic<int> *batch_granted() {
  static std::atomic<int> granted[64] = {};
  return granted;
}
std::atomic<int> *batch_mixed_granted() {
  static std::atomic<int> granted[64] = {};
  return granted;
}

template <int MODE>
cudaError_t fused_batch_launch(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass, uint64_t total,
                               int kmax, cudaStream_t st) {
  const int smem = smem_bytes<MODE>(kmax);
  cudaError_t e = ensure_smem((const void *)k_fused_batch<MODE>, smem, batch_granted<MODE>());
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_batch<MODE>, kFusedThreads, smem);
  if (occ < 1) occ = 1;
  const uint64_t cap = (uint64_t)sms() * occ;
  const unsigned grid = (unsigned)(total < cap ? (total > 0 ? total : 1) : cap);
  k_fused_batch<MODE><<<grid, kFusedThreads, smem, st>>>(d_passes, d_chunk_start, npass, total, kmax);
  return cudaGetLastError();
}

} // namespace

int fused_smem_bytes(int mode, int k) {
  return mode == MODE_C64_F32 ? smem_bytes<MODE_C64_F32>(k) : smem_bytes<MODE_C128_F64>(k);
}

template <int MODE>
cudaError_t tc_launch(const PassDesc &p, cudaStream_t st, FusedSched *sched) {
  const int smem = tc_smem_bytes<MODE>(p.k) + (p.ngates <= kTcGateCopy ? p.ngates * (int)sizeof(DevGate) : 0);
  static std::atomic<int> granted[64] = {};
  cudaError_t e = ensure_smem((const void *)k_fused_tc<MODE>, smem, granted);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_tc<MODE>, kTcThreads, smem);
  if (occ < 1) occ = 1;
  const uint32_t tiles = 1u << (p.k - kBlockBits - 7);
  const uint32_t levels = MODE == MODE_C64_F32 ? 1u : 7u;
  uint32_t ncols = 32;
  while (ncols < tiles * levels * (uint32_t)kBlockK) ncols <<= 1;
  if (ncols > 512) return cudaErrorInvalidValue;
  occ = std::min<int>(occ, (int)(512 / ncols));
  const uint64_t nchunks = 1ull << (p.n - p.k);
  const uint64_t cap = (uint64_t)sms() * occ;
  const unsigned grid = (unsigned)(nchunks < cap ? nchunks : cap);
  // Test hook: with SV_TEST_TC_NO_MMA set no MMA is issued, so the kernel's bounded waits run out and the
  // state reports SV_ERR_TIMEOUT (the failure path of a tensor core that never answers, without a fault).
  PassDesc q = p;
  q.tc_flags = std::getenv("SV_TEST_TC_NO_MMA") ? 1 : 0;
  k_fused_tc<MODE><<<grid, kTcThreads, smem, st>>>(q, nchunks, ncols, &sched->tc_err);
  return cudaGetLastError();
}

cudaError_t launch_fused(const PassDesc &p, int mode, cudaStream_t st, int f64_share, FusedSched *sched) {
  const uint64_t nchunks = 1ull << (p.n - p.k);
  if (p.nblocks > 0) {
    // dense blocks need the tensor-core kernel: chunks of at least 2^11 amplitudes (128-row tiles) and the
    // scratch that carries its error word
    if (sched == nullptr || p.k < kBlockBits + 7 || p.k > 13) return cudaErrorInvalidValue;
    if (mode == MODE_C64_F32) return tc_launch<MODE_C64_F32>(p, st, sched);
    if (mode == MODE_C128_DF32) return tc_launch<MODE_C128_DF32>(p, st, sched);
    return cudaErrorInvalidValue;
  }
  if (mode == MODE_C128_DF32 && f64_share > 0 && f64_share < 100 && sched != nullptr) {
    const int smem = smem_bytes<MODE_C128_DF32>(p.k);
    static std::atomic<int> granted[64] = {};
    cudaError_t e = ensure_smem((const void *)k_fused_mixed, smem, granted);
    if (e != cudaSuccess) return e;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_mixed, kFusedThreads, smem);
    if (occ < 1) occ = 1;
    const uint64_t grid = (uint64_t)sms() * occ;
    // Worth it only with several chunks per CTA and at least two CTAs per SM.
    if (occ >= 2 && nchunks >= 4 * grid) {
      cudaError_t e = cudaMemsetAsync(sched, 0, kSchedResetBytes, st);
      if (e != cudaSuccess) return e;
      k_fused_mixed<<<(unsigned)grid, kFusedThreads, smem, st>>>(p, nchunks, f64_share, sched);
      return cudaGetLastError();
    }
  }
  switch (mode) {
    case MODE_C64_F32: return fused_launch<MODE_C64_F32>(p, st);
    case MODE_C128_F64: return fused_launch<MODE_C128_F64>(p, st);
    default: return fused_launch<MODE_C128_DF32>(p, st);
  }
}

cudaError_t prepare_fused_batch(int mode, int kmax) {
  cudaError_t e;
  switch (mode) {
    case MODE_C64_F32:
      return ensure_smem((const void *)k_fused_batch<MODE_C64_F32>, smem_bytes<MODE_C64_F32>(kmax),
                         batch_granted<MODE_C64_F32>());
    case MODE_C128_F64:
      return ensure_smem((const void *)k_fused_batch<MODE_C128_F64>, smem_bytes<MODE_C128_F64>(kmax),
                         batch_granted<MODE_C128_F64>());
    default:
      e = ensure_smem((const void *)k_fused_batch<MODE_C128_DF32>, smem_bytes<MODE_C128_DF32>(kmax),
                      batch_granted<MODE_C128_DF32>());
      if (e != cudaSuccess) return e;
      return ensure_smem((const void *)k_fused_batch_mixed, smem_bytes<MODE_C128_DF32>(kmax), batch_mixed_granted());
  }
}

// The batched tensor-core kernel's shared memory: the pass of 2^kBatchTcK amplitudes and its block planes.
static std::atomic<int> *batch_tc_granted() {
  static std::atomic<int> g[64] = {};
  return g;
}

cudaError_t prepare_fused_batch_tc() {
  return ensure_smem((const void *)k_fused_batch_tc, tc_smem_bytes<MODE_C128_DF32>(kBatchTcK), batch_tc_granted());
}

cudaError_t launch_fused_batch_tc(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass, uint64_t total,
                                  cudaStream_t st, FusedSched *sched) {
  if (total == 0 || npass == 0) return cudaSuccess;
  if (sched == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = prepare_fused_batch_tc();
  if (e != cudaSuccess) return e;
  // two 128-row tiles of seven digit levels of 32 columns: 448 columns, allocated as 512
  const uint32_t ncols = 512;
  const uint64_t cap = (uint64_t)sms();
  const unsigned grid = (unsigned)(total < cap ? total : cap);
  k_fused_batch_tc<<<grid, kTcThreads, tc_smem_bytes<MODE_C128_DF32>(kBatchTcK), st>>>(d_passes, d_chunk_start, npass,
                                                                                         total, ncols, &sched->tc_err);
  return cudaGetLastError();
}

cudaError_t launch_fused_batch(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass, uint64_t total,
                               int mode, int kmax, cudaStream_t st, int f64_share, FusedSched *sched, int *used_mixed) {
  if (used_mixed) *used_mixed = 0;
  if (total == 0 || npass == 0) return cudaSuccess;
  if (mode == MODE_C128_DF32 && f64_share > 0 && f64_share < 100 && sched != nullptr) {
    const int smem = smem_bytes<MODE_C128_DF32>(kmax);
    cudaError_t e = ensure_smem((const void *)k_fused_batch_mixed, smem, batch_mixed_granted());
    if (e != cudaSuccess) return e;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_batch_mixed, kFusedThreads, smem);
    if (occ < 1) occ = 1;
    const uint64_t grid = (uint64_t)sms() * occ;
    if (occ >= 2 && total >= 4 * grid) {
      if ((e = cudaMemsetAsync(sched, 0, kSchedResetBytes, st)) != cudaSuccess) return e;
      k_fused_batch_mixed<<<(unsigned)grid, kFusedThreads, smem, st>>>(d_passes, d_chunk_start, npass, total, kmax,
                                                                        f64_share, sched);
      if (used_mixed) *used_mixed = 1;
      return cudaGetLastError();
    }
  }
  switch (mode) {
    case MODE_C64_F32: return fused_batch_launch<MODE_C64_F32>(d_passes, d_chunk_start, npass, total, kmax, st);
    case MODE_C128_F64: return fused_batch_launch<MODE_C128_F64>(d_passes, d_chunk_start, npass, total, kmax, st);
    default: return fused_batch_launch<MODE_C128_DF32>(d_passes, d_chunk_start, npass, total, kmax, st);
  }
}

} // namespace svi
