// Fused chunk pass: one read and one write of the state applies a whole run of gates.
//
// The paper keeps the gates of "local" qubits (those whose amplitude pairs lie in one process's slice of
// the vector) free of communication (Sec. V.A, V.C) and proposes relabelling qubits so that the busy ones
// are local (Sec. VI.B).  On one GPU the analogue of a process's slice is a chunk of 2^k amplitudes held in
// shared memory: the amplitudes whose indices agree on every bit outside a chosen set Q of k physical bits.
// Q always holds the c lowest bits, so a chunk is 2^(k-c) runs of 2^c contiguous amplitudes (coalesced
// 256-byte rows); its other k - c bits can be any higher bits.  Every gate whose target lies in Q (and every
// diagonal gate, wherever its target) is applied to the chunk in shared memory with the pair update of
// Sec. V.A; control bits inside Q are tested per amplitude, control bits outside Q once per chunk.
#include <cstdint>
#include <cuda_runtime.h>
#include "sv_internal.h"
#include "sv_arith.cuh"

namespace svi {
namespace {

constexpr int kFusedThreads = 256;
#ifndef SV_FUSED_MIN_BLOCKS
#define SV_FUSED_MIN_BLOCKS 3
#endif

__device__ __forceinline__ uint32_t ins0(uint32_t i, int t) {
  return ((i >> t) << (t + 1)) | (i & ((1u << t) - 1u));
}

#ifndef SV_FUSED_PAIR_UNROLL
#define SV_FUSED_PAIR_UNROLL 2
#endif
constexpr int kPairUnroll = SV_FUSED_PAIR_UNROLL;

// All pairs (j0, j0 | tb) of the chunk for one gate of class CLS, target bit t, local controls cm.
template <int MODE, int CLS>
__device__ __forceinline__ void chunk_pairs(typename Arith<MODE>::S *sm, const typename Arith<MODE>::Coef &cf,
                                            uint32_t half, int t, uint32_t tb, uint32_t cm) {
  using S = typename Arith<MODE>::S;
#pragma unroll kPairUnroll
  for (uint32_t i = threadIdx.x; i < half; i += kFusedThreads) {
    const uint32_t j0 = ins0(i, t);
    if ((j0 & cm) != cm) continue;
    S a = sm[j0], b = sm[j0 | tb];
    apply_pair<MODE>(CLS, cf, a, b);
    sm[j0] = a;
    sm[j0 | tb] = b;
  }
}

// Shared-memory layout: 2^k working amplitudes, then 2^(k-c) row offsets (uint64).
template <int MODE>
__device__ __forceinline__ void fused_chunk(const PassDesc &p, uint64_t chunk, typename Arith<MODE>::S *sm,
                                            uint64_t *rowoff) {
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
  for (uint32_t r = tid; r < nrows; r += kFusedThreads) {
    uint64_t off = 0;
    for (int j = c; j < k; ++j) off |= (uint64_t)((r >> (j - c)) & 1u) << p.qpos[j];
    rowoff[r] = off;
  }
  __syncthreads();

  G *psi = (G *)p.psi;
  if (p.init) {
    // Basis state |init_x>: one amplitude of one chunk is 1.
    const bool mine = (p.init_x & ~p.qmask) == base;
    uint32_t lx = 0;
    for (int j = 0; j < k; ++j) lx |= (uint32_t)((p.init_x >> p.qpos[j]) & 1ull) << j;
    for (uint32_t o = tid; o < nloc; o += kFusedThreads) sm[o] = (mine && o == lx) ? M::one() : M::zero();
  } else {
    // Issue four loads before converting, so each thread keeps several requests in flight.
    for (uint32_t o0 = tid; o0 < nloc; o0 += 4 * kFusedThreads) {
      G v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t o = o0 + u * kFusedThreads;
        if (o < nloc) v[u] = psi[base + rowoff[o >> c] + (o & lowmask)];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t o = o0 + u * kFusedThreads;
        if (o < nloc) sm[o] = M::load(v[u]);
      }
    }
  }
  __syncthreads();

  for (int gi = 0; gi < p.ngates; ++gi) {
    const DevGate &g = p.gates[gi];
    const uint64_t gmask = g.gmask;
    if ((base & gmask) != gmask) continue;  // a control bit outside the chunk is 0: the gate skips this chunk
    const uint32_t cls = g.cls;
    const int t = g.target;
    const uint32_t cm = (uint32_t)g.cmask;
    typename M::Coef cf;
    if (cls != GC_X) M::coef(cf, g);
    if (t >= 0) {
      const uint32_t tb = 1u << t;
      if (cls == GC_PHASE) {
        for (uint32_t i = tid; i < half; i += kFusedThreads) {
          const uint32_t j = ins0(i, t) | tb;
          if ((j & cm) == cm) sm[j] = M::cmul(cf, 3, sm[j]);
        }
      } else {
        // One loop per class, so the class test is not inside the pair loop.
        switch (cls) {
          case GC_GENERAL: chunk_pairs<MODE, GC_GENERAL>(sm, cf, half, t, tb, cm); break;
          case GC_DIAG: chunk_pairs<MODE, GC_DIAG>(sm, cf, half, t, tb, cm); break;
          case GC_ANTIDIAG: chunk_pairs<MODE, GC_ANTIDIAG>(sm, cf, half, t, tb, cm); break;
          default: chunk_pairs<MODE, GC_X>(sm, cf, half, t, tb, cm); break;
        }
      }
    } else {
      // Diagonal gate on a qubit outside the chunk: every amplitude of the chunk has the same target bit.
      const bool one = (base & g.tmask) != 0;
      if (one) {
        for (uint32_t j = tid; j < nloc; j += kFusedThreads)
          if ((j & cm) == cm) sm[j] = M::cmul(cf, 3, sm[j]);
      } else if (cls != GC_PHASE) {
        for (uint32_t j = tid; j < nloc; j += kFusedThreads)
          if ((j & cm) == cm) sm[j] = M::cmul(cf, 0, sm[j]);
      }
    }
    __syncthreads();
  }

  if (!p.permuted) {
    for (uint32_t o = tid; o < nloc; o += kFusedThreads) psi[base + rowoff[o >> c] + (o & lowmask)] = M::store(sm[o]);
  } else {
    // Store with chunk-local bit j sent to physical bit qpos_out[j]: output slot o (bits in the ascending
    // order of Q) takes local amplitude src(o), bit j of src(o) = bit pos(qpos_out[j]) of o.
    int8_t sp[16];
    for (int j = 0; j < k; ++j) {
      int s = 0;
      for (int i = 0; i < k; ++i)
        if (p.qpos[i] == p.qpos_out[j]) s = i;
      sp[j] = (int8_t)s;
    }
    for (uint32_t o = tid; o < nloc; o += kFusedThreads) {
      uint32_t src = 0;
      for (int j = 0; j < k; ++j) src |= ((o >> sp[j]) & 1u) << j;
      psi[base + rowoff[o >> c] + (o & lowmask)] = M::store(sm[src]);
    }
  }
  __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(kFusedThreads, SV_FUSED_MIN_BLOCKS) k_fused(const PassDesc p, uint64_t nchunks) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using S = typename Arith<MODE>::S;
  S *sm = (S *)smraw;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)sizeof(S) << p.k));
  for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) fused_chunk<MODE>(p, ch, sm, rowoff);
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

template <int MODE>
__global__ void __launch_bounds__(kFusedThreads, SV_FUSED_MIN_BLOCKS) k_fused_batch(const PassDesc *__restrict__ passes,
                                                               const uint64_t *__restrict__ chunk_start, int npass,
                                                               uint64_t total, int kmax) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using S = typename Arith<MODE>::S;
  S *sm = (S *)smraw;
  uint64_t *rowoff = (uint64_t *)(smraw + ((size_t)sizeof(S) << kmax));
  for (uint64_t b = blockIdx.x; b < total; b += gridDim.x) {
    int lo = 0, hi = npass - 1;  // last pass with chunk_start <= b
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const PassDesc p = passes[lo];
    fused_chunk<MODE>(p, b - chunk_start[lo], sm, rowoff);
  }
}

int g_sms = 0;
int sms() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms < 1) g_sms = 1;
  }
  return g_sms;
}

// The planner keeps c >= min(3, k), so the row table never has more than max(1, 2^(k-3)) entries.
template <int MODE>
int smem_bytes(int k) {
  return (int)(sizeof(typename Arith<MODE>::S) << k) + (int)(sizeof(uint64_t) << (k > 3 ? k - 3 : 0));
}

template <int MODE>
cudaError_t fused_launch(const PassDesc &p, cudaStream_t st) {
  const int smem = smem_bytes<MODE>(p.k);
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fused<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
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
cudaError_t fused_batch_launch(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass, uint64_t total,
                               int kmax, cudaStream_t st) {
  const int smem = smem_bytes<MODE>(kmax);
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_batch<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
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

cudaError_t launch_fused(const PassDesc &p, int mode, cudaStream_t st, int f64_share, FusedSched *sched) {
  const uint64_t nchunks = 1ull << (p.n - p.k);
  if (mode == MODE_C128_DF32 && f64_share > 0 && f64_share < 100 && sched != nullptr) {
    const int smem = smem_bytes<MODE_C128_DF32>(p.k);
    static int configured = 0;
    if (smem > configured) {
      cudaError_t e = cudaFuncSetAttribute(k_fused_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_mixed, kFusedThreads, smem);
    if (occ < 1) occ = 1;
    const uint64_t grid = (uint64_t)sms() * occ;
    // Worth it only with several chunks per CTA and at least two CTAs per SM.
    if (occ >= 2 && nchunks >= 4 * grid) {
      cudaError_t e = cudaMemsetAsync(sched, 0, sizeof(FusedSched), st);
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

cudaError_t launch_fused_batch(const PassDesc *d_passes, const uint64_t *d_chunk_start, int npass, uint64_t total,
                               int mode, int kmax, cudaStream_t st) {
  if (total == 0 || npass == 0) return cudaSuccess;
  switch (mode) {
    case MODE_C64_F32: return fused_batch_launch<MODE_C64_F32>(d_passes, d_chunk_start, npass, total, kmax, st);
    case MODE_C128_F64: return fused_batch_launch<MODE_C128_F64>(d_passes, d_chunk_start, npass, total, kmax, st);
    default: return fused_batch_launch<MODE_C128_DF32>(d_passes, d_chunk_start, npass, total, kmax, st);
  }
}

} // namespace svi
