// CUDA kernels for sm_103a: single-gate sweep, in-place bit swap, basis init, logical-order gather,
// probabilities, norm and scaling.  The fused chunk pass lives in sv_fused.cu.
#include <cstdint>
#include <cuda_runtime.h>
#include "sv_internal.h"
#include "sv_arith.cuh"

namespace svi {

namespace {

// SM count of the device (one GPU per process), read once; safe to call from several host threads.
int num_sms() {
  static const int v = [] {
    int dev = 0, count = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    return count > 0 ? count : 1;
  }();
  return v;
}

// Insert a zero bit at each of the `np` ascending positions pos[0..np).
__device__ __forceinline__ uint64_t insert_zeros(uint64_t i, const int8_t *pos, int np) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    if (j < np) {
      const int p = pos[j];
      i = ((i >> p) << (p + 1)) | (i & ((1ull << p) - 1));
    }
  }
  return i;
}

struct SweepArgs {
  DevGate g;
  uint64_t nitems;   // pairs (or single amplitudes for GC_PHASE)
  uint64_t setmask;  // OR'ed into the expanded index: control bits (and the target bit for GC_PHASE)
  int8_t pos[8];     // ascending bit positions where a zero is inserted (target and controls)
  int32_t npos;
};

constexpr int kSweepThreads = 256;
constexpr int kSweepUnroll = 4;

// One tile (kSweepThreads * kSweepUnroll items starting at `base`) of a single-gate sweep.  Each item is a pair
// (k, k + 2^t) with bit t of k zero and all control bits one (Algorithm 1, Sec. V.B); items are numbered by
// the remaining free bits, so consecutive threads touch consecutive addresses whenever the target and
// controls are not among the lowest index bits.  All loads of the tile are issued before any arithmetic.
template <int MODE, int CLS>
__device__ __forceinline__ void sweep_tile(typename Arith<MODE>::G *__restrict__ psi, const SweepArgs &a,
                                           const typename Arith<MODE>::Coef &c, uint64_t base) {
  using M = Arith<MODE>;
  using G = typename M::G;
  const uint64_t tstride = 1ull << a.g.target;
  uint64_t k0[kSweepUnroll];
  G va[kSweepUnroll], vb[kSweepUnroll];
#pragma unroll
  for (int u = 0; u < kSweepUnroll; ++u) {
    const uint64_t i = base + (uint64_t)u * kSweepThreads + threadIdx.x;
    k0[u] = insert_zeros(i, a.pos, a.npos) | a.setmask;
    if (i < a.nitems) {
      if (CLS == GC_PHASE) {
        vb[u] = psi[k0[u]];
      } else {
        va[u] = psi[k0[u]];
        vb[u] = psi[k0[u] + tstride];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kSweepUnroll; ++u) {
    const uint64_t i = base + (uint64_t)u * kSweepThreads + threadIdx.x;
    if (i >= a.nitems) continue;
    if (CLS == GC_X) {
      psi[k0[u]] = vb[u];
      psi[k0[u] + tstride] = va[u];
    } else if (CLS == GC_PHASE) {
      psi[k0[u]] = M::store(M::cmul(c, 3, M::load(vb[u])));
    } else {
      auto x = M::load(va[u]);
      auto y = M::load(vb[u]);
      apply_pair<MODE>(CLS, c, x, y);
      psi[k0[u]] = M::store(x);
      psi[k0[u] + tstride] = M::store(y);
    }
  }
}

// One gate over the whole state, tiles strided over the grid.
template <int MODE, int CLS>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(typename Arith<MODE>::G *__restrict__ psi, const SweepArgs a) {
  using M = Arith<MODE>;
  typename M::Coef c;
  if (CLS != GC_X) M::coef(c, a.g);
  const uint64_t tile = (uint64_t)kSweepThreads * kSweepUnroll;
  for (uint64_t base = (uint64_t)blockIdx.x * tile; base < a.nitems; base += (uint64_t)gridDim.x * tile)
    sweep_tile<MODE, CLS>(psi, a, c, base);
}

template <int MODE, int CLS>
cudaError_t sweep_launch(void *psi, const SweepArgs &a, cudaStream_t st) {
  static const int occ = [] {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_sweep<MODE, CLS>, kSweepThreads, 0);
    return o > 0 ? o : 1;
  }();
  const uint64_t tile = (uint64_t)kSweepThreads * kSweepUnroll;
  const uint64_t need = (a.nitems + tile - 1) / tile;
  const uint64_t cap = (uint64_t)num_sms() * occ;
  const unsigned grid = (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
  k_sweep<MODE, CLS><<<grid, kSweepThreads, 0, st>>>((typename Arith<MODE>::G *)psi, a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t sweep_mode(void *psi, const SweepArgs &a, cudaStream_t st) {
  switch (a.g.cls) {
    case GC_GENERAL: return sweep_launch<MODE, GC_GENERAL>(psi, a, st);
    case GC_DIAG: return sweep_launch<MODE, GC_DIAG>(psi, a, st);
    case GC_PHASE: return sweep_launch<MODE, GC_PHASE>(psi, a, st);
    case GC_ANTIDIAG: return sweep_launch<MODE, GC_ANTIDIAG>(psi, a, st);
    default: return sweep_launch<MODE, GC_X>(psi, a, st);
  }
}

// ------------------------------------------------------------------------------------------------------
template <typename G>
__global__ void k_set_one(G *psi, uint64_t x) {
  G v;
  v.x = 1; v.y = 0;
  psi[x] = v;
}

struct Perm { int8_t p[kMaxQubits]; };

__device__ __forceinline__ uint64_t logical_to_physical(uint64_t L, int n, const Perm &pm) {
  uint64_t P = 0;
  for (int t = 0; t < n; ++t) P |= ((L >> t) & 1ull) << pm.p[t];
  return P;
}

template <typename G>
__global__ void k_gather(const G *__restrict__ psi, int n, const Perm pm, uint64_t first, uint64_t count,
                         const uint64_t *__restrict__ idx, G *__restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t L = idx ? idx[i] : first + i;
    out[i] = psi[logical_to_physical(L, n, pm)];
  }
}

// |alpha|^2 = re*re + im*im in double, each product and the sum rounded once (no contraction).
template <typename G>
__global__ void k_probs(const G *__restrict__ psi, int n, const Perm pm, uint64_t first, uint64_t count,
                        double *__restrict__ out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const G v = psi[logical_to_physical(first + i, n, pm)];
    const double re = (double)v.x, im = (double)v.y;
    out[i] = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
  }
}

// ------------------------------------------------------------------------------------------------------
// Norm (the normalisation condition of Sec. II.A).  Each thread keeps an FP64 accumulator; the block adds the
// per-thread values in FP64 in a fixed tree order, and a second kernel adds the per-block partials with
// compensation in a fixed order, so the result does not depend on timing.  Every thread has kNormLoads 16-byte loads in flight per
// iteration (HBM latency needs that many bytes in flight per SM).
// * complex128: every component's square is added by one FP64 fused multiply-add on its exact value.
// * complex64: a float's square is exact as a pair p + e (one multiply, one FMA); the 16 squares of the
//   iteration's eight amplitudes are summed with error-free TwoSums into s, their errors and the e's summed
//   the same way into c, and only the errors of that second sum are rounded, into d (cascaded compensated
//   summation in the manner of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005: s + c + d is the
//   group's sum to about 2^-70 of it).  s, c and d, each converted exactly to double, enter the FP64
//   accumulator: three FP64 additions per eight amplitudes on GB300's slow FP64 pipe instead of two per
//   amplitude, and an error below that of one FP64 addition per group.  (Summing the small terms in a single
//   FP32 sum instead leaves a bias of about 2^-49 of each group's sum.)
// A sign (-1)^popcount(k & pmask) is applied by flipping one factor's sign bit (exact).
// ------------------------------------------------------------------------------------------------------
constexpr int kNormThreads = 256;
constexpr int kNormBlocksPerSm = 4;
constexpr int kNormLoads = 4;

// The exact double value of a float, with integer operations (the float -> double conversion instruction runs
// on GB300's slow FP64/conversion unit).  Normal floats: sign, exponent re-biased by 1023 - 127, mantissa
// shifted into place; subnormal floats (below 2^-126), zeros, infinities and NaNs take the conversion
// instruction (a branch that normalised states never take, apart from exact zeros).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = b & 0x7F800000u;
  if (e == 0u || e == 0x7F800000u) return (double)f;
  const uint32_t hi = (b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(b << 29));
}

__device__ __forceinline__ double flip_if(double x, bool neg) {
  return neg ? __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull) : x;
}
__device__ __forceinline__ float flipf_if(float x, bool neg) {
  return neg ? __uint_as_float(__float_as_uint(x) ^ 0x80000000u) : x;
}

// s + c + d += (+/-) x^2 (see above): x^2 = p + e exactly, s + r = s + p exactly, r + e = q + t exactly,
// c + q = c' + u exactly; only the small terms t + u (each below 2^-48 of the running sum) are rounded, into d.
__device__ __forceinline__ void sq_add(float x, bool neg, float &s, float &c, float &d) {
  const float xs = flipf_if(x, neg);
  const float p = __fmul_rn(xs, x);
  const float e = __fmaf_rn(xs, x, -p);
  float t1, r, q, t, u;
  two_sum(s, p, t1, r);
  s = t1;
  two_sum(r, e, q, t);
  two_sum(c, q, t1, u);
  c = t1;
  d = __fadd_rn(d, __fadd_rn(t, u));
}

// Stage 1 of sum_k (-1)^popcount(k & pmask) |psi_k|^2 over physical indices k (pmask = 0: the norm).
template <typename G, bool IS_DOUBLE>
__global__ void __launch_bounds__(kNormThreads) k_norm1(const G *__restrict__ psi, uint64_t N, uint64_t pmask,
                                                        double *__restrict__ partials) {
  constexpr uint64_t kPer = IS_DOUBLE ? 1 : 2;  // amplitudes per 16-byte load
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t NV = N / kPer;                  // 16-byte units
  double acc = 0.0;
  // main loop: kNormLoads units per thread per iteration, units tid + j * nthreads of the iteration's span
  const uint64_t span = nthreads * kNormLoads, full = NV / span * span;
  for (uint64_t base = 0; base < full; base += span) {
    if constexpr (IS_DOUBLE) {
      double2 v[kNormLoads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) v[j] = psi[base + tid + (uint64_t)j * nthreads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) {
        const bool neg = (__popcll((base + tid + (uint64_t)j * nthreads) & pmask) & 1) != 0;
        acc = __fma_rn(flip_if(v[j].x, neg), v[j].x, acc);
        acc = __fma_rn(flip_if(v[j].y, neg), v[j].y, acc);
      }
    } else {
      const float4 *p4 = reinterpret_cast<const float4 *>(psi);
      float4 v[kNormLoads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) v[j] = p4[base + tid + (uint64_t)j * nthreads];
      float s = 0.0f, c = 0.0f, d = 0.0f;
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) {
        const uint64_t k0 = 2 * (base + tid + (uint64_t)j * nthreads);
        const bool n0 = (__popcll(k0 & pmask) & 1) != 0, n1 = (__popcll((k0 + 1) & pmask) & 1) != 0;
        sq_add(v[j].x, n0, s, c, d);
        sq_add(v[j].y, n0, s, c, d);
        sq_add(v[j].z, n1, s, c, d);
        sq_add(v[j].w, n1, s, c, d);
      }
      // s + (c + d), with c + d formed first (both far below s)
      acc = __dadd_rn(acc, __dadd_rn(f2d_exact(s), __dadd_rn(f2d_exact(c), f2d_exact(d))));
    }
  }
  // the rest, one amplitude at a time (all of it when N < 2 span)
  for (uint64_t i = full * kPer + tid; i < N; i += nthreads) {
    const G v = psi[i];
    const bool neg = (__popcll(i & pmask) & 1) != 0;
    double x, y;
    if constexpr (IS_DOUBLE) {
      x = (double)v.x;
      y = (double)v.y;
    } else {
      x = f2d_exact((float)v.x);
      y = f2d_exact((float)v.y);
    }
    acc = __fma_rn(flip_if(x, neg), x, acc);
    acc = __fma_rn(flip_if(y, neg), y, acc);
  }
  __shared__ double red[kNormThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kNormThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// Error-free sum of two doubles (Knuth's TwoSum): s + e = a + b exactly.
__device__ __forceinline__ void two_sum_d(double a, double b, double &s, double &e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// Stage 2: the per-block partials added with compensation by one warp (lane l takes partials l, l + 32, ..
// in index order, keeping the rounding errors of its TwoSums in c; the 32 (s, c) pairs are then combined by a
// fixed butterfly of TwoSums), so the result is the correctly rounded sum of the partials up to a few units in
// the last place, in a fixed order.
__global__ void k_norm2(const double *__restrict__ partials, int nparts, double *__restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double s = 0.0, c = 0.0, e;
  for (int i = threadIdx.x; i < nparts; i += 32) {
    two_sum_d(s, partials[i], s, e);
    c = __dadd_rn(c, e);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double so = __shfl_xor_sync(0xffffffffu, s, off), co = __shfl_xor_sync(0xffffffffu, c, off);
    // the lower lane's pair first, so both lanes form the same sum
    const bool low = (threadIdx.x & off) == 0;
    two_sum_d(low ? s : so, low ? so : s, s, e);
    c = __dadd_rn(__dadd_rn(low ? c : co, low ? co : c), e);
  }
  if (threadIdx.x == 0) out[0] = __dadd_rn(s, c);
}

// psi *= 1 / sqrt(norm2), the factor f formed in FP64 once per thread.  complex128: one FP64 multiply per
// component.  complex64: f = fh + fl (two floats, fl = f - fh exactly rounded) and x f = fma(x, fh, x fl) in
// FP32, within an ulp of the correctly rounded product, without the FP64 pipe.  kNormLoads 16-byte units per
// thread per iteration, as in the norm.
template <typename G, bool IS_DOUBLE>
__global__ void k_scale(G *__restrict__ psi, uint64_t N, const double *__restrict__ norm2) {
  const double f = 1.0 / sqrt(norm2[0]);
  const float fh = (float)f, fl = (float)(f - (double)fh);
  constexpr uint64_t kPer = IS_DOUBLE ? 1 : 2;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t NV = N / kPer, span = nthreads * kNormLoads, full = NV / span * span;
  for (uint64_t base = 0; base < full; base += span) {
    if constexpr (IS_DOUBLE) {
      double2 v[kNormLoads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) v[j] = psi[base + tid + (uint64_t)j * nthreads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) {
        v[j].x *= f;
        v[j].y *= f;
        psi[base + tid + (uint64_t)j * nthreads] = v[j];
      }
    } else {
      float4 *p4 = reinterpret_cast<float4 *>(psi);
      float4 v[kNormLoads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) v[j] = p4[base + tid + (uint64_t)j * nthreads];
#pragma unroll
      for (int j = 0; j < kNormLoads; ++j) {
        v[j].x = __fmaf_rn(v[j].x, fh, __fmul_rn(v[j].x, fl));
        v[j].y = __fmaf_rn(v[j].y, fh, __fmul_rn(v[j].y, fl));
        v[j].z = __fmaf_rn(v[j].z, fh, __fmul_rn(v[j].z, fl));
        v[j].w = __fmaf_rn(v[j].w, fh, __fmul_rn(v[j].w, fl));
        p4[base + tid + (uint64_t)j * nthreads] = v[j];
      }
    }
  }
  for (uint64_t i = full * kPer + tid; i < N; i += nthreads) {
    G v = psi[i];
    if constexpr (IS_DOUBLE) {
      v.x *= f;
      v.y *= f;
    } else {
      v.x = __fmaf_rn(v.x, fh, __fmul_rn(v.x, fl));
      v.y = __fmaf_rn(v.y, fh, __fmul_rn(v.y, fl));
    }
    psi[i] = v;
  }
}

// Measurement sampling.  Logical indices are grouped in blocks of 2^b consecutive values; physical index of
// logical L = phys_hi(L >> b) | phys_lo(L & (2^b - 1)) because the layout map moves each bit independently.
// Stage 1: one warp per block adds |alpha|^2 (FP64) over the block in logical order.
template <typename G>
__global__ void k_block_probs(const G *__restrict__ psi, int n, const Perm pm, int b, uint64_t nblocks,
                              double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < nblocks; j += warps) {
    const uint64_t hi = logical_to_physical(j << b, n, pm);
    double acc = 0.0;
    for (uint32_t l = lane; l < (1u << b); l += 32) {
      const G v = psi[hi | logical_to_physical(l, b, pm)];
      const double re = (double)v.x, im = (double)v.y;
      acc += re * re + im * im;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[j] = acc;
  }
}

// Stage 2: one warp per shot walks its block in logical order (32 entries at a time, warp prefix sums) and
// returns the first index whose running sum exceeds the residual mass `resid` left after the earlier blocks.
template <typename G>
__global__ void k_sample_block(const G *__restrict__ psi, int n, const Perm pm, int b,
                               const uint64_t *__restrict__ blk, const double *__restrict__ resid, uint64_t count,
                               uint64_t *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += warps) {
    const uint64_t j = blk[i];
    const double r = resid[i];
    const uint64_t hi = logical_to_physical(j << b, n, pm);
    double run = 0.0;
    uint64_t found = ~0ull, last_nonzero = 0;
    for (uint32_t base = 0; base < (1u << b) && found == ~0ull; base += 32) {
      const uint32_t l = base + lane;
      double p = 0.0;
      if (l < (1u << b)) {
        const G v = psi[hi | logical_to_physical(l, b, pm)];
        const double re = (double)v.x, im = (double)v.y;
        p = re * re + im * im;
      }
      double incl = p;
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, p > 0.0 && run + incl > r);
      const unsigned nz = __ballot_sync(0xffffffffu, p > 0.0);
      if (nz) last_nonzero = base + 31 - __clz(nz);
      if (hit) found = base + __ffs(hit) - 1;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    // Rounding can leave r at or above the block's total: take its last non-zero entry.
    if (lane == 0) out[i] = (j << b) + (found != ~0ull ? found : last_nonzero);
  }
}

unsigned grid_for(uint64_t items, int threads) {
  const uint64_t need = (items + threads - 1) / threads;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  return (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
}

Perm make_perm(const int *perm, int n) {
  Perm p{};
  for (int t = 0; t < n; ++t) p.p[t] = (int8_t)perm[t];
  return p;
}

} // namespace

// ------------------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------------------
cudaError_t launch_sweep(void *psi, int n, int mode, const DevGate &g, cudaStream_t st) {
  SweepArgs a{};
  a.g = g;
  int pos[8], np = 0;
  pos[np++] = g.target;
  uint64_t cm = g.cmask;
  for (int b = 0; b < n; ++b)
    if (cm >> b & 1ull) pos[np++] = b;
  // ascending insertion sort (at most 5 entries)
  for (int i = 1; i < np; ++i)
    for (int j = i; j > 0 && pos[j - 1] > pos[j]; --j) { const int t = pos[j]; pos[j] = pos[j - 1]; pos[j - 1] = t; }
  for (int i = 0; i < np; ++i) a.pos[i] = (int8_t)pos[i];
  a.npos = np;
  a.nitems = 1ull << (n - np);
  a.setmask = cm | (g.cls == GC_PHASE ? (1ull << g.target) : 0ull);
  switch (mode) {
    case MODE_C64_F32: return sweep_mode<MODE_C64_F32>(psi, a, st);
    case MODE_C128_F64: return sweep_mode<MODE_C128_F64>(psi, a, st);
    default: return sweep_mode<MODE_C128_DF32>(psi, a, st);
  }
}

cudaError_t launch_init_basis(void *psi, int n, int mode, uint64_t x, cudaStream_t st) {
  const size_t bytes = (mode == MODE_C64_F32 ? 8ull : 16ull) << n;
  cudaError_t e = cudaMemsetAsync(psi, 0, bytes, st);
  if (e != cudaSuccess) return e;
  if (mode == MODE_C64_F32) k_set_one<float2><<<1, 1, 0, st>>>((float2 *)psi, x);
  else k_set_one<double2><<<1, 1, 0, st>>>((double2 *)psi, x);
  return cudaGetLastError();
}

// Product state (Sec. V): amplitude k = prod_t g_t[bit t of k] with g_t = M_t f_t.  Table entry i < 2^h
// holds the product over qubits 0..h-1 for low index bits i, entry 2^h + j the product over qubits h..n-1 for
// high index bits j (FP64, qubits in ascending order).
template <typename T>
__global__ void k_product_tables(const double *__restrict__ fm, int n, int h, T *__restrict__ tab) {
  const uint64_t nlo = 1ull << h, total = nlo + (1ull << (n - h));
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const bool lo = i < nlo;
    const uint64_t x = lo ? i : i - nlo;
    const int t0 = lo ? 0 : h, t1 = lo ? h : n;
    double re = 1.0, im = 0.0;
    for (int t = t0; t < t1; ++t) {
      const double *f = fm + 12 * t;
      const double *r = f + 4 + 4 * (int)((x >> (t - t0)) & 1ull);  // row b of M_t
      const double gr = r[0] * f[0] - r[1] * f[1] + r[2] * f[2] - r[3] * f[3];
      const double gi = r[0] * f[1] + r[1] * f[0] + r[2] * f[3] + r[3] * f[2];
      const double nr = re * gr - im * gi, ni = re * gi + im * gr;
      re = nr;
      im = ni;
    }
    tab[i] = T{(decltype(T::x))re, (decltype(T::x))im};  // complex64 tables are rounded once, here
  }
}

// One complex product per amplitude, in the state's precision (complex64: FP32 products of the rounded
// tables, relative error a few 2^-24).
template <typename G>
__global__ void k_init_product(G *__restrict__ psi, int n, int h, const G *__restrict__ tab) {
  const uint64_t N = 1ull << n, mlo = (1ull << h) - 1ull;
  const G *hi = tab + (1ull << h);
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < N; k += (uint64_t)gridDim.x * blockDim.x) {
    const G a = tab[k & mlo], b = hi[k >> h];
    psi[k] = G{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
  }
}

uint64_t product_table_entries(int n) { return (1ull << (n / 2)) + (1ull << (n - n / 2)); }

cudaError_t launch_init_product(void *psi, int n, int mode, const double *d_fm, void *d_tab, cudaStream_t st) {
  const int h = n / 2;
  const uint64_t entries = product_table_entries(n);
  const unsigned tgrid = grid_for(entries, 256), grid = grid_for(1ull << n, 256);
  if (mode == MODE_C64_F32) {
    k_product_tables<float2><<<tgrid, 256, 0, st>>>(d_fm, n, h, (float2 *)d_tab);
    k_init_product<float2><<<grid, 256, 0, st>>>((float2 *)psi, n, h, (const float2 *)d_tab);
  } else {
    k_product_tables<double2><<<tgrid, 256, 0, st>>>(d_fm, n, h, (double2 *)d_tab);
    k_init_product<double2><<<grid, 256, 0, st>>>((double2 *)psi, n, h, (const double2 *)d_tab);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(const void *psi, int n, int mode, const int *perm, uint64_t first, uint64_t count,
                          const uint64_t *d_idx, void *d_out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const Perm pm = make_perm(perm, n);
  const unsigned grid = grid_for(count, 256);
  if (mode == MODE_C64_F32)
    k_gather<float2><<<grid, 256, 0, st>>>((const float2 *)psi, n, pm, first, count, d_idx, (float2 *)d_out);
  else
    k_gather<double2><<<grid, 256, 0, st>>>((const double2 *)psi, n, pm, first, count, d_idx, (double2 *)d_out);
  return cudaGetLastError();
}

cudaError_t launch_probs(const void *psi, int n, int mode, const int *perm, uint64_t first, uint64_t count,
                         double *d_out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const Perm pm = make_perm(perm, n);
  const unsigned grid = grid_for(count, 256);
  if (mode == MODE_C64_F32)
    k_probs<float2><<<grid, 256, 0, st>>>((const float2 *)psi, n, pm, first, count, d_out);
  else
    k_probs<double2><<<grid, 256, 0, st>>>((const double2 *)psi, n, pm, first, count, d_out);
  return cudaGetLastError();
}

int norm_parts() { return num_sms() * kNormBlocksPerSm; }

int norm_parts_for_sms(int sms) { return (sms > 0 ? sms : 1) * kNormBlocksPerSm; }

cudaError_t launch_norm(const void *psi, int n, int mode, double *d_partials, double *d_out, cudaStream_t st,
                        uint64_t pmask) {
  return launch_norm_parts(psi, n, mode, d_partials, d_out, st, pmask, norm_parts());
}

cudaError_t launch_norm_parts(const void *psi, int n, int mode, double *d_partials, double *d_out, cudaStream_t st,
                              uint64_t pmask, int parts) {
  const uint64_t N = 1ull << n;
  if (mode == MODE_C64_F32)
    k_norm1<float2, false><<<parts, kNormThreads, 0, st>>>((const float2 *)psi, N, pmask, d_partials);
  else
    k_norm1<double2, true><<<parts, kNormThreads, 0, st>>>((const double2 *)psi, N, pmask, d_partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_norm2<<<1, 32, 0, st>>>(d_partials, parts, d_out);
  return cudaGetLastError();
}

cudaError_t launch_block_probs(const void *psi, int n, int mode, const int *perm, int b, double *d_out,
                               cudaStream_t st) {
  const Perm pm = make_perm(perm, n);
  const uint64_t nblocks = 1ull << (n - b);
  const unsigned grid = grid_for(nblocks * 32, 256);
  if (mode == MODE_C64_F32) k_block_probs<float2><<<grid, 256, 0, st>>>((const float2 *)psi, n, pm, b, nblocks, d_out);
  else k_block_probs<double2><<<grid, 256, 0, st>>>((const double2 *)psi, n, pm, b, nblocks, d_out);
  return cudaGetLastError();
}

cudaError_t launch_sample_block(const void *psi, int n, int mode, const int *perm, int b, const uint64_t *d_blk,
                                const double *d_resid, uint64_t count, uint64_t *d_out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const Perm pm = make_perm(perm, n);
  const unsigned grid = grid_for(count * 32, 256);
  if (mode == MODE_C64_F32)
    k_sample_block<float2><<<grid, 256, 0, st>>>((const float2 *)psi, n, pm, b, d_blk, d_resid, count, d_out);
  else
    k_sample_block<double2><<<grid, 256, 0, st>>>((const double2 *)psi, n, pm, b, d_blk, d_resid, count, d_out);
  return cudaGetLastError();
}

cudaError_t launch_scale(void *psi, int n, int mode, const double *d_norm2, cudaStream_t st) {
  const uint64_t N = 1ull << n;
  const unsigned grid = grid_for(N, 256);
  if (mode == MODE_C64_F32) k_scale<float2, false><<<grid, 256, 0, st>>>((float2 *)psi, N, d_norm2);
  else k_scale<double2, true><<<grid, 256, 0, st>>>((double2 *)psi, N, d_norm2);
  return cudaGetLastError();
}

} // namespace svi
