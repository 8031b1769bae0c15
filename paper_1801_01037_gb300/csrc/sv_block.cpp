// Dense gate blocks for the tensor cores (host side).
//
// A run of gates whose qubits all lie in the same kBlockBits chunk-local bits is one unitary on those bits
// (Sec. II.B: a multi-qubit gate is a matrix on its qubits' basis states; the product of the run's matrices,
// composed here in FP64 in gate order).  Applying it to a chunk is a matrix product: every row of the
// chunk (the 2^kBlockBits amplitudes that differ only in the block bits) is multiplied by the block's
// matrix, which the fused pass does with tcgen05 MMAs.  This file forms the blocks from a pass's gate run
// and encodes each block's matrix as the MMA's B operand in the exact shared-memory byte layout the kernel
// copies.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "sv_plan.h"

namespace svi {

namespace {

// Round a double to bfloat16 (round to nearest, ties to even, through float) and back.
uint16_t bf16_bits(double v) {
  const float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

// Byte offset of element (row i, column kk) of one 32 x 32 operand plane: 8-row x 16-byte core matrices,
// column-adjacent core matrices 128 bytes apart, 8-row groups 512 bytes apart (no swizzle, K-major).
size_t plane_offset(int i, int kk) {
  return (size_t)(i / 8) * 512 + (size_t)(kk / 8) * 128 + (size_t)(i % 8) * 16 + (size_t)(kk % 8) * 2;
}

// Qubit mask (chunk-local bits) of a gate record in a pass run, and whether it can join a block: its target
// and every control inside the chunk (no control outside it, not a diagonal on an outside qubit).
struct Item {
  size_t first;     // index in the run
  int nrec;         // records (4 for a two-qubit gate)
  uint32_t bits;    // chunk-local bits it touches
  bool blockable;
  double cost;      // per-gate work it saves, in dense one-qubit gate updates of the whole chunk
};

Item item_of(const std::vector<DevGate> &run, size_t i) {
  const DevGate &g = run[i];
  Item it{i, g.cls == GC_DENSE4 ? 4 : 1, 0u, true, 0.0};
  if (g.target >= 0) it.bits |= 1u << g.target;
  if (g.cls == GC_DENSE4) it.bits |= 1u << (int)g.tmask;
  it.bits |= (uint32_t)g.cmask;
  if (g.gmask != 0 || g.target < 0) it.blockable = false;
  // The per-gate pass touches only the amplitudes whose local control bits are all 1 (and, for a phase, whose
  // target bit is 1): the cost of the class, scaled by that fraction.
  switch (g.cls) {
    case GC_GENERAL: it.cost = 1.0; break;
    case GC_DENSE4: it.cost = 4.0; break;
    case GC_X: it.cost = 0.25; break;
    case GC_PHASE: it.cost = 0.25; break;
    default: it.cost = 0.5; break;  // diagonal, anti-diagonal
  }
  it.cost = std::ldexp(it.cost, -__builtin_popcount((uint32_t)g.cmask));
  return it;
}

// Apply record g (chunk-local bits; `slot` maps a chunk bit to its bit in the block index) to every column of
// the 2^B x 2^B complex matrix U (row-major, interleaved re/im): U <- G U, in FP64, with the pair update of
// Sec. V.A (old values on the right) and the controlled rule of Sec. V.B.
void apply_to_block(double *U, const std::vector<DevGate> &run, size_t i, const int *slot) {
  const int D = kBlockDim;
  const DevGate &g = run[i];
  uint32_t cm = 0;
  for (int b = 0; b < 32; ++b)
    if ((uint32_t)g.cmask >> b & 1u) cm |= 1u << slot[b];
  if (g.cls == GC_DENSE4) {
    const int b0 = slot[g.target], b1 = slot[(int)g.tmask];
    double V[32];
    for (int r = 0; r < 4; ++r) std::memcpy(V + 8 * r, run[i + r].q, 8 * sizeof(double));
    for (int col = 0; col < D; ++col)
      for (int x = 0; x < D; ++x) {
        if (x >> b0 & 1 || x >> b1 & 1 || (x & cm) != cm) continue;
        int idx[4];
        double ar[4], ai[4];
        for (int j = 0; j < 4; ++j) {
          idx[j] = x | ((j & 1) << b0) | ((j >> 1 & 1) << b1);
          ar[j] = U[2 * (idx[j] * D + col)];
          ai[j] = U[2 * (idx[j] * D + col) + 1];
        }
        for (int r = 0; r < 4; ++r) {
          double sr = 0.0, si = 0.0;
          for (int j = 0; j < 4; ++j) {
            const double vr = V[8 * r + 2 * j], vi = V[8 * r + 2 * j + 1];
            sr += vr * ar[j] - vi * ai[j];
            si += vr * ai[j] + vi * ar[j];
          }
          U[2 * (idx[r] * D + col)] = sr;
          U[2 * (idx[r] * D + col) + 1] = si;
        }
      }
    return;
  }
  const int t = slot[g.target];
  const double *q = g.q;
  for (int col = 0; col < D; ++col)
    for (int x = 0; x < D; ++x) {
      if (x >> t & 1 || (x & cm) != cm) continue;
      const int y = x | (1 << t);
      const double ar = U[2 * (x * D + col)], ai = U[2 * (x * D + col) + 1];
      const double br = U[2 * (y * D + col)], bi = U[2 * (y * D + col) + 1];
      U[2 * (x * D + col)] = (q[0] * ar - q[1] * ai) + (q[2] * br - q[3] * bi);
      U[2 * (x * D + col) + 1] = (q[0] * ai + q[1] * ar) + (q[2] * bi + q[3] * br);
      U[2 * (y * D + col)] = (q[4] * ar - q[5] * ai) + (q[6] * br - q[7] * bi);
      U[2 * (y * D + col) + 1] = (q[4] * ai + q[5] * ar) + (q[6] * bi + q[7] * br);
    }
}

// The real form of the block: output n (n < 16: Re y_n, else Im y_{n-16}) = sum_kk W[n][kk] x_kk with input kk
// (kk < 16: Re x_kk, else Im x_{kk-16}).
void real_form(const double *U, double (*W)[kBlockK]) {
  const int D = kBlockDim;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      const double ur = U[2 * (i * D + j)], ui = U[2 * (i * D + j) + 1];
      W[i][j] = ur;
      W[i][D + j] = -ui;
      W[D + i][j] = ui;
      W[D + i][D + j] = ur;
    }
}

// Operand planes of a block.  complex64: three bfloat16 planes w = w0 + w1 + w2 (each the rounding of what
// the planes before it leave, so the sum holds 24 bits of w).  complex128: six planes of balanced base-256
// digits of round(w * 2^47) (each in [-128, 128), the top one in [-128, 128] so that |w| = 1 is exact; all
// exact in bfloat16), digit 0 the least significant.
void encode_planes(int mode, const double (*W)[kBlockK], unsigned char *dst) {
  const int planes = mode == MODE_C64_F32 ? kBlockSplitsC64 : kBlockDigitsC128;
  std::memset(dst, 0, planes * kBlockPlaneBytes);
  for (int n = 0; n < kBlockK; ++n)
    for (int kk = 0; kk < kBlockK; ++kk) {
      uint16_t p[8];
      if (mode == MODE_C64_F32) {
        double r = W[n][kk];
        for (int s = 0; s < kBlockSplitsC64; ++s) {
          p[s] = bf16_bits(r);
          r -= bf16_value(p[s]);
        }
      } else {
        int64_t v = (int64_t)std::llround(std::ldexp(W[n][kk], 47));
        for (int s = 0; s < kBlockDigitsC128; ++s) {
          int64_t d = v;                          // the top digit keeps what is left: |v| <= 2^47 gives [-128, 128]
          if (s + 1 < kBlockDigitsC128) {
            d = ((v % 256) + 256) % 256;          // v mod 256 in [0, 256)
            if (d >= 128) d -= 256;               // balanced digit in [-128, 128)
          }
          p[s] = bf16_bits((double)d);
          v = (v - d) / 256;
        }
      }
      for (int s = 0; s < planes; ++s) std::memcpy(dst + s * kBlockPlaneBytes + plane_offset(n, kk), &p[s], 2);
    }
}

} // namespace

constexpr double kBlockPassShare = 0.75;

size_t block_data_bytes(int mode) {
  return (size_t)(mode == MODE_C64_F32 ? kBlockSplitsC64 : kBlockDigitsC128) * kBlockPlaneBytes;
}

// Greedy blocking of one pass's run (order of gates that share a qubit is kept; a gate joins a block only if
// its qubits are disjoint from every gate it would move ahead of).  A block is kept if the gates it absorbs
// save at least `min_cost` dense one-qubit gate updates; its header (GC_BLOCK) stands where its first gate
// stood.  Unused block bits are filled with the lowest free chunk bits.
int group_blocks(std::vector<DevGate> &run, int k, int mode, double min_cost, std::vector<unsigned char> &data) {
  std::vector<Item> items;
  for (size_t i = 0; i < run.size(); i += (run[i].cls == GC_DENSE4 ? 4 : 1)) items.push_back(item_of(run, i));
  std::vector<char> done(items.size(), 0);
  std::vector<DevGate> out;
  const size_t data0 = data.size();
  double total = 0.0, absorbed = 0.0;
  for (const Item &it : items) total += it.cost;
  int nblocks = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    if (done[i]) continue;
    const Item &a = items[i];
    std::vector<size_t> members;
    uint32_t bits = 0;
    if (a.blockable && __builtin_popcount(a.bits) <= kBlockBits) {
      members.push_back(i);
      bits = a.bits;
      uint32_t blocked = 0;
      for (size_t j = i + 1; j < items.size(); ++j) {
        if (done[j]) continue;
        const Item &b = items[j];
        if (b.blockable && !(b.bits & blocked) && __builtin_popcount(bits | b.bits) <= kBlockBits) {
          bits |= b.bits;
          members.push_back(j);
        } else {
          blocked |= b.bits;
        }
      }
    }
    double cost = 0.0;
    for (size_t m : members) cost += items[m].cost;
    if (members.size() < 2 || cost < min_cost) {
      for (int r = 0; r < a.nrec; ++r) out.push_back(run[a.first + r]);
      done[i] = 1;
      continue;
    }
    absorbed += cost;
    for (int b = 0; b < k && __builtin_popcount(bits) < kBlockBits; ++b) bits |= 1u << b;
    int pos[kBlockBits], np = 0, slot[32];
    for (int b = 0; b < 32; ++b) slot[b] = 0;
    for (int b = 0; b < k; ++b)
      if (bits >> b & 1u) { slot[b] = np; pos[np++] = b; }
    std::vector<double> U(2 * kBlockDim * kBlockDim, 0.0);
    for (int d = 0; d < kBlockDim; ++d) U[2 * (d * kBlockDim + d)] = 1.0;
    for (size_t m : members) {
      apply_to_block(U.data(), run, items[m].first, slot);
      done[m] = 1;
    }
    double W[kBlockK][kBlockK];
    real_form(U.data(), W);
    const size_t off = (data.size() + 127) & ~(size_t)127;
    data.resize(off + block_data_bytes(mode));
    encode_planes(mode, W, data.data() + off);
    DevGate h;
    std::memset(&h, 0, sizeof h);
    h.cls = GC_BLOCK;
    h.target = (int32_t)members.size();
    for (int s = 0; s < np; ++s) h.cmask |= (uint64_t)pos[s] << (8 * s);
    h.gmask = off;  // offset in the plan's block data; made relative to the header by plan_blob_fill
    out.push_back(h);
    ++nblocks;
  }
  // A pass with blocks runs in the tensor-core kernel, where the remaining gates go one by one more slowly
  // than in the per-gate pass: blocks are kept only if they take at least kBlockPassShare of the pass's work.
  if (nblocks > 0 && absorbed < kBlockPassShare * total) {
    data.resize(data0);
    return 0;
  }
  run.swap(out);
  return nblocks;
}

} // namespace svi
