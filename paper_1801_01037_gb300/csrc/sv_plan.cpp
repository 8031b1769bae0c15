// Host planner.  See sv_plan.h.
#include "sv_plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

namespace svi {

static bool eq(double a, double b) { return a == b; }

int classify(const double *U) {
  const bool q11_zero = eq(U[0], 0) && eq(U[1], 0), q12_zero = eq(U[2], 0) && eq(U[3], 0);
  const bool q21_zero = eq(U[4], 0) && eq(U[5], 0), q22_zero = eq(U[6], 0) && eq(U[7], 0);
  const bool q11_one = eq(U[0], 1) && eq(U[1], 0), q22_one = eq(U[6], 1) && eq(U[7], 0);
  if (q12_zero && q21_zero) {
    if (q11_one && q22_one) return -1;
    return q11_one ? GC_PHASE : GC_DIAG;
  }
  if (q11_zero && q22_zero) {
    const bool q12_one = eq(U[2], 1) && eq(U[3], 0), q21_one = eq(U[4], 1) && eq(U[5], 0);
    return (q12_one && q21_one) ? GC_X : GC_ANTIDIAG;
  }
  return GC_GENERAL;
}

void fill_coefficients(DevGate &g, const double *U) {
  for (int i = 0; i < 8; ++i) {
    g.q[i] = U[i];
    g.qh[i] = (float)U[i];
    const double r1 = U[i] - (double)g.qh[i];
    g.qm[i] = (float)r1;
    g.ql[i] = (float)(r1 - (double)g.qm[i]);
  }
}

int validate_gate(const sv_gate &g, int n, std::string &why) {
  char buf[160];
  if (g.kind == SV_GATE_SWAP) {
    if (g.target < 0 || g.target >= n || g.target2 < 0 || g.target2 >= n || g.target == g.target2) {
      snprintf(buf, sizeof buf, "SWAP qubits (%d, %d) must be distinct and in [0, %d)", g.target, g.target2, n);
      why = buf;
      return SV_ERR_ARG;
    }
    if (g.ncontrols != 0) {
      why = "controlled SWAP is not supported";
      return SV_ERR_ARG;
    }
    return SV_OK;
  }
  if (g.kind != SV_GATE_U) {
    snprintf(buf, sizeof buf, "unknown gate kind %d", g.kind);
    why = buf;
    return SV_ERR_ARG;
  }
  if (g.target < 0 || g.target >= n) {
    snprintf(buf, sizeof buf, "target %d out of range [0, %d)", g.target, n);
    why = buf;
    return SV_ERR_ARG;
  }
  if (g.ncontrols < 0 || g.ncontrols > SV_MAX_CONTROLS) {
    snprintf(buf, sizeof buf, "ncontrols %d out of range [0, %d]", g.ncontrols, SV_MAX_CONTROLS);
    why = buf;
    return SV_ERR_ARG;
  }
  uint64_t seen = 1ull << g.target;
  for (int i = 0; i < g.ncontrols; ++i) {
    const int c = g.controls[i];
    if (c < 0 || c >= n || (seen >> c & 1ull)) {
      snprintf(buf, sizeof buf, "control %d is out of range, equal to the target or repeated", c);
      why = buf;
      return SV_ERR_ARG;
    }
    seen |= 1ull << c;
  }
  // U^dagger U = I within 1e-10 (entries finite).
  const double *u = g.U;
  for (int i = 0; i < 8; ++i)
    if (!std::isfinite(u[i])) {
      why = "gate matrix has a non-finite entry";
      return SV_ERR_NOT_UNITARY;
    }
  double worst = 0;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      // (U^dagger U)_ij = sum_r conj(U_ri) U_rj
      double re = 0, im = 0;
      for (int r = 0; r < 2; ++r) {
        const double ar = u[4 * r + 2 * i], ai = -u[4 * r + 2 * i + 1];
        const double br = u[4 * r + 2 * j], bi = u[4 * r + 2 * j + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      worst = std::max(worst, std::fabs(re - (i == j ? 1.0 : 0.0)));
      worst = std::max(worst, std::fabs(im));
    }
  if (worst > 1e-10) {
    snprintf(buf, sizeof buf, "gate matrix is not unitary (max |U^dagger U - I| = %.3g)", worst);
    why = buf;
    return SV_ERR_NOT_UNITARY;
  }
  return SV_OK;
}

// A two-qubit gate: its four records, qubits, controls and the unitarity of V (16 complex entries).
static int validate_gate4(const sv_gate *g, size_t avail, int n, std::string &why) {
  char buf[160];
  if (avail < 4) {
    why = "two-qubit gate needs three SV_GATE_U4_ROW records after it";
    return SV_ERR_ARG;
  }
  const int q0 = g[0].target, q1 = g[0].target2;
  for (int r = 1; r < 4; ++r)
    if (g[r].kind != SV_GATE_U4_ROW || g[r].target != q0 || g[r].target2 != q1 || g[r].ncontrols != 0) {
      why = "two-qubit gate needs three SV_GATE_U4_ROW records with the same qubits after it";
      return SV_ERR_ARG;
    }
  if (q0 < 0 || q0 >= n || q1 < 0 || q1 >= n || q0 == q1) {
    snprintf(buf, sizeof buf, "two-qubit gate qubits (%d, %d) must be distinct and in [0, %d)", q0, q1, n);
    why = buf;
    return SV_ERR_ARG;
  }
  if (g[0].ncontrols < 0 || g[0].ncontrols > SV_MAX_CONTROLS) {
    snprintf(buf, sizeof buf, "ncontrols %d out of range [0, %d]", g[0].ncontrols, SV_MAX_CONTROLS);
    why = buf;
    return SV_ERR_ARG;
  }
  uint64_t seen = (1ull << q0) | (1ull << q1);
  for (int i = 0; i < g[0].ncontrols; ++i) {
    const int c = g[0].controls[i];
    if (c < 0 || c >= n || (seen >> c & 1ull)) {
      snprintf(buf, sizeof buf, "control %d is out of range, equal to a target or repeated", c);
      why = buf;
      return SV_ERR_ARG;
    }
    seen |= 1ull << c;
  }
  double v[32];
  for (int r = 0; r < 4; ++r) std::memcpy(v + 8 * r, g[r].U, sizeof g[r].U);
  for (int i = 0; i < 32; ++i)
    if (!std::isfinite(v[i])) {
      why = "gate matrix has a non-finite entry";
      return SV_ERR_NOT_UNITARY;
    }
  double worst = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double re = 0, im = 0;  // (V^dagger V)_ij = sum_r conj(V_ri) V_rj
      for (int r = 0; r < 4; ++r) {
        const double ar = v[8 * r + 2 * i], ai = -v[8 * r + 2 * i + 1];
        const double br = v[8 * r + 2 * j], bi = v[8 * r + 2 * j + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      worst = std::max(worst, std::fabs(re - (i == j ? 1.0 : 0.0)));
      worst = std::max(worst, std::fabs(im));
    }
  if (worst > 1e-10) {
    snprintf(buf, sizeof buf, "gate matrix is not unitary (max |V^dagger V - I| = %.3g)", worst);
    why = buf;
    return SV_ERR_NOT_UNITARY;
  }
  return SV_OK;
}

int validate_records(const sv_gate *g, size_t ngates, int n, std::string &why, size_t &bad) {
  for (size_t i = 0; i < ngates; ++i) {
    int rc;
    if (g[i].kind == SV_GATE_U4) {
      rc = validate_gate4(g + i, ngates - i, n, why);
      if (rc == SV_OK) {
        i += 3;
        continue;
      }
    } else if (g[i].kind == SV_GATE_U4_ROW) {
      why = "SV_GATE_U4_ROW record without its SV_GATE_U4 record";
      rc = SV_ERR_ARG;
    } else {
      rc = validate_gate(g[i], n, why);
    }
    if (rc != SV_OK) {
      bad = i;
      return rc;
    }
  }
  return SV_OK;
}

// Device blob: the DevGates of every pass, then (128-byte aligned) the operand planes of the dense blocks.
static size_t gates_bytes_aligned(const Plan &P) {
  const size_t b = P.fused_gates.size() * sizeof(DevGate);
  return P.block_data.empty() ? b : (b + 127) & ~(size_t)127;
}

size_t plan_blob_bytes(const Plan &P) { return gates_bytes_aligned(P) + P.block_data.size(); }

void plan_blob_fill(const Plan &P, void *dst) {
  if (!P.fused_gates.empty()) std::memcpy(dst, P.fused_gates.data(), P.fused_gates.size() * sizeof(DevGate));
  if (P.block_data.empty()) return;
  const size_t base = gates_bytes_aligned(P);
  std::memset((unsigned char *)dst + P.fused_gates.size() * sizeof(DevGate), 0,
              base - P.fused_gates.size() * sizeof(DevGate));
  std::memcpy((unsigned char *)dst + base, P.block_data.data(), P.block_data.size());
  // A block header's gmask becomes the byte distance from the header to its planes.
  DevGate *g = (DevGate *)dst;
  for (size_t i = 0; i < P.fused_gates.size(); ++i)
    if (g[i].cls == GC_BLOCK) g[i].gmask = base + P.fused_gates[i].gmask - i * sizeof(DevGate);
}

void plan_pass_pointers(const Plan &P, int idx, const void *d_blob, PassDesc &d) {
  d.gates = (const DevGate *)d_blob + P.pass_gate_offset[idx];
}

std::vector<std::pair<int, int>> canonicalize_steps(std::vector<int> &perm) {
  std::vector<std::pair<int, int>> out;
  const int n = (int)perm.size();
  for (int t = 0; t < n; ++t) {
    if (perm[t] == t) continue;
    int u = 0;
    while (perm[u] != t) ++u;
    out.emplace_back(perm[t], t);  // exchange physical bits perm[t] and t
    perm[u] = perm[t];
    perm[t] = t;
  }
  return out;
}

std::vector<PassDesc> canonicalize_passes(int n, const PlanConfig &cfg, std::vector<int> &perm) {
  int c = std::min(cfg.c, n);
  c = std::max(c, std::min(3, n));
  // At least two bits besides the low ones, so that every pass puts at least one bit in its place.
  const int k = std::min(n, std::max(cfg.k, c + 2));
  std::vector<PassDesc> out;
  for (int guard = 0; guard <= n; ++guard) {
    // dest[p]: physical bit that the data now at physical bit p belongs to (logical qubit t sits at perm[t]).
    int dest[64];
    bool done = true;
    for (int t = 0; t < n; ++t) {
      dest[perm[t]] = t;
      done = done && perm[t] == t;
    }
    if (done) break;
    // Q: the c low bits, then consecutive runs along the cycles of dest while bits are left.
    bool inq[64] = {false};
    int nbits = 0;
    for (int b = 0; b < c; ++b) { inq[b] = true; ++nbits; }
    bool seen[64] = {false};
    for (int b0 = 0; b0 < n && nbits < k; ++b0) {
      if (seen[b0] || dest[b0] == b0) continue;
      for (int b = b0; !seen[b]; b = dest[b]) {
        seen[b] = true;
        if (!inq[b]) {
          if (nbits == k) break;
          inq[b] = true;
          ++nbits;
        }
      }
    }
    for (int b = 0; b < n && nbits < k; ++b)
      if (!inq[b]) { inq[b] = true; ++nbits; }
    // sigma on Q: a bit whose destination is in Q sends its data there; the remaining ones fill, in order,
    // the bits of Q that nothing in Q is sent to.  The first kind is final; the pass is a bijection of Q.
    int sigma[64];
    bool hit[64] = {false};
    for (int b = 0; b < n; ++b)
      if (inq[b] && inq[dest[b]]) { sigma[b] = dest[b]; hit[dest[b]] = true; }
    int fill = 0;
    for (int b = 0; b < n; ++b) {
      if (!inq[b] || inq[dest[b]]) continue;
      while (!inq[fill] || hit[fill]) ++fill;
      sigma[b] = fill;
      hit[fill] = true;
    }
    PassDesc d;
    std::memset(&d, 0, sizeof d);
    d.n = n;
    d.k = k;
    d.c = c;
    int j = 0;
    for (int b = 0; b < n; ++b)
      if (inq[b]) {
        d.qpos[j] = (int8_t)b;
        d.qpos_out[j] = (int8_t)sigma[b];
        d.qmask |= 1ull << b;
        ++j;
      }
    d.permuted = 1;
    for (int jj = 0; jj < k; ++jj)
      for (int i = 0; i < k; ++i)
        if (d.qpos[i] == d.qpos_out[jj]) d.src_bit[jj] = (int8_t)i;
    out.push_back(d);
    for (int t = 0; t < n; ++t)
      if (inq[perm[t]]) perm[t] = sigma[perm[t]];
  }
  return out;
}

namespace {

struct Sched {
  int idx;        // source gate index (the first record of a two-qubit gate)
  int cls;        // gate class, or -2 (SWAP folded into the layout) / -1 (identity): no device work
  int pt;         // physical target (-1 for SWAP / identity entries)
  int pt2;        // two-qubit gate: physical bit of b1 (-1 otherwise)
  uint64_t pc;    // physical control mask
  uint64_t phys;  // physical bits the entry touches (target(s), controls; both bits of a SWAP)
  uint64_t logi;  // logical qubits the entry touches
};

bool needs_pairing(int cls) { return cls == GC_GENERAL || cls == GC_ANTIDIAG || cls == GC_X; }

DevGate to_sweep_gate(const sv_gate &g, const Sched &s) {
  DevGate d;
  std::memset(&d, 0, sizeof d);
  fill_coefficients(d, g.U);
  d.cls = (uint32_t)s.cls;
  d.target = s.pt;
  d.cmask = s.pc;
  return d;
}

} // namespace

// Split a pass's gate run (chunk-local targets) into register cubes, in order: a cube takes gates while the
// distinct targets of its pairing gates stay within kCubeBits bits; diagonal gates join any cube; a two-qubit
// gate ends the cube and is left outside any cube.  Unused cube bits are filled from the top of the chunk, which keeps the
// threads of a half-warp on distinct shared-memory banks for most bit sets.  Each gate in a cube gets its
// control bits inside the cube (as cube bits) in bits 32..36 of cmask and 1 + the cube slot of its target
// (0: not in the cube) in bits 40..42, so the kernel does no per-gate bit search.
void group_cubes(const std::vector<DevGate> &run, int k, std::vector<DevGate> &out) {
  const int cb = kCubeBits;
  size_t i = 0;
  while (i < run.size()) {
    if (run[i].cls == GC_DENSE4) {  // two-qubit gates run on their own, from shared memory (4 records)
      out.insert(out.end(), run.begin() + i, run.begin() + std::min(run.size(), i + 4));
      i += 4;
      continue;
    }
    if (run[i].cls == GC_BLOCK) {  // dense blocks run on the tensor cores, between cubes
      out.push_back(run[i]);
      ++i;
      continue;
    }
    uint32_t bits = 0;
    int nb = 0;
    size_t j = i;
    for (; j < run.size(); ++j) {
      const DevGate &g = run[j];
      if (g.cls == GC_DENSE4 || g.cls == GC_BLOCK) break;
      if (!needs_pairing((int)g.cls) || g.target < 0) continue;
      const uint32_t tb = 1u << g.target;
      if (bits & tb) continue;
      if (nb == cb) break;
      bits |= tb;
      ++nb;
    }
    for (int b = k - 1; b >= 0 && nb < cb; --b)
      if (!(bits >> b & 1u)) { bits |= 1u << b; ++nb; }
    int pos[8], np = 0;
    for (int b = 0; b < k; ++b)
      if (bits >> b & 1u) pos[np++] = b;
    DevGate h;
    std::memset(&h, 0, sizeof h);
    h.cls = GC_CUBE;
    h.target = (int32_t)(j - i);
    h.tmask = (uint64_t)cb;
    for (int s = 0; s < np; ++s) h.cmask |= (uint64_t)pos[s] << (8 * s);
    out.push_back(h);
    for (size_t x = i; x < j; ++x) {
      DevGate g = run[x];
      const uint32_t cm = (uint32_t)g.cmask;
      uint64_t cs = 0, slot1 = 0;
      for (int s = 0; s < np; ++s) {
        if (cm >> pos[s] & 1u) cs |= 1ull << s;
        if (g.target == pos[s]) slot1 = (uint64_t)(s + 1);
      }
      g.cmask = (uint64_t)cm | (cs << 32) | (slot1 << 40);
      out.push_back(g);
    }
    i = j;
  }
}

// Identity check of a two-qubit gate's four records.
static bool is_identity4(const sv_gate *g) {
  for (int r = 0; r < 4; ++r)
    for (int j = 0; j < 4; ++j) {
      const double re = g[r].U[2 * j], im = g[r].U[2 * j + 1];
      if (im != 0.0 || re != (r == j ? 1.0 : 0.0)) return false;
    }
  return true;
}

static void make_plan_records(int n, const PlanConfig &cfg, std::vector<int> &perm, const sv_gate *gates,
                              size_t ngates, Plan &P);

// Runs of uncontrolled one-qubit gates on one qubit, with no other record touching that qubit between them,
// become one gate whose matrix is their product, composed in FP64 on the host (later x earlier).  `groups[j]`
// lists the source records of reduced record j, in source order.  Returns the number of gates merged away.
static size_t merge_one_qubit_runs(int n, const sv_gate *gates, size_t ngates, std::vector<sv_gate> &red,
                                   std::vector<std::vector<int>> &groups) {
  std::vector<int> open(n, -1);  // reduced record holding the qubit's open run, or -1
  size_t merged = 0;
  for (size_t i = 0; i < ngates; ++i) {
    const sv_gate &g = gates[i];
    if (g.kind == SV_GATE_U && g.ncontrols == 0 && open[g.target] >= 0) {
      sv_gate &m = red[open[g.target]];
      double r[8];
      for (int row = 0; row < 2; ++row)
        for (int col = 0; col < 2; ++col) {
          double re = 0.0, im = 0.0;
          for (int j = 0; j < 2; ++j) {
            const double ur = g.U[4 * row + 2 * j], ui = g.U[4 * row + 2 * j + 1];
            const double mr = m.U[4 * j + 2 * col], mi = m.U[4 * j + 2 * col + 1];
            re += ur * mr - ui * mi;
            im += ur * mi + ui * mr;
          }
          r[4 * row + 2 * col] = re;
          r[4 * row + 2 * col + 1] = im;
        }
      std::memcpy(m.U, r, sizeof r);
      groups[open[g.target]].push_back((int)i);
      ++merged;
      continue;
    }
    const int recs = g.kind == SV_GATE_U4 ? 4 : 1;
    // every qubit this record touches closes its open run
    open[g.target] = -1;
    if (g.kind == SV_GATE_SWAP || g.kind == SV_GATE_U4) open[g.target2] = -1;
    if (g.kind != SV_GATE_SWAP)
      for (int c = 0; c < g.ncontrols; ++c) open[g.controls[c]] = -1;
    for (int r = 0; r < recs; ++r) {
      red.push_back(gates[i + r]);
      groups.push_back({(int)(i + r)});
    }
    if (g.kind == SV_GATE_U && g.ncontrols == 0) open[g.target] = (int)red.size() - 1;
    i += recs - 1;
  }
  return merged;
}

void make_plan(int n, const PlanConfig &cfg, std::vector<int> &perm, const sv_gate *gates, size_t ngates, Plan &P) {
  std::vector<sv_gate> red;
  std::vector<std::vector<int>> groups;
  red.reserve(ngates);
  groups.reserve(ngates);
  const size_t merged = cfg.merge ? merge_one_qubit_runs(n, gates, ngates, red, groups) : 0;
  if (merged == 0) {
    make_plan_records(n, cfg, perm, gates, ngates, P);
    return;
  }
  make_plan_records(n, cfg, perm, red.data(), red.size(), P);
  // Map the schedule record back to the source records: merged records share their step and take
  // consecutive positions in the execution order.
  std::vector<int> by_order(red.size());
  for (size_t j = 0; j < red.size(); ++j) by_order[P.gate_order[j]] = (int)j;
  std::vector<int> step(ngates, -1), ord(ngates, -1);
  int o = 0;
  for (int j : by_order)
    for (int src : groups[j]) {
      step[src] = P.gate_step[j];
      ord[src] = o++;
    }
  P.gate_step.swap(step);
  P.gate_order.swap(ord);
  P.n_merged = (int)merged;
}

static void make_plan_records(int n, const PlanConfig &cfg, std::vector<int> &perm, const sv_gate *gates,
                              size_t ngates, Plan &P) {
  P = Plan();
  P.gate_step.assign(ngates, -1);
  P.gate_order.assign(ngates, -1);
  int order = 0;
  const int k = std::min(cfg.k, n);
  int c = std::min(cfg.c, k);
  c = std::max(c, std::min(3, k));
  if (k < n) c = std::min(c, std::max(std::min(3, k), k - 2));  // room for both bits of a two-qubit gate

  auto records_of = [&](size_t i) { return gates[i].kind == SV_GATE_U4 ? 4 : 1; };
  auto sched_of = [&](size_t i, int cls) {
    Sched s;
    const sv_gate &g = gates[i];
    s.idx = (int)i;
    s.cls = cls;
    s.pc = 0;
    s.pt2 = -1;
    s.logi = 1ull << g.target;
    if (g.kind == SV_GATE_SWAP) {
      s.pt = -1;
      s.phys = (1ull << perm[g.target]) | (1ull << perm[g.target2]);
      s.logi |= 1ull << g.target2;
      return s;
    }
    for (int j = 0; j < g.ncontrols; ++j) {
      s.pc |= 1ull << perm[g.controls[j]];
      s.logi |= 1ull << g.controls[j];
    }
    s.pt = cls == -1 ? -1 : perm[g.target];
    s.phys = s.pc | (1ull << perm[g.target]);
    if (g.kind == SV_GATE_U4) {
      s.pt2 = cls == -1 ? -1 : perm[g.target2];
      s.phys |= 1ull << perm[g.target2];
      s.logi |= 1ull << g.target2;
    }
    return s;
  };
  auto cls_of_record = [&](size_t i) {
    if (gates[i].kind == SV_GATE_SWAP) return -2;
    if (gates[i].kind == SV_GATE_U4) return is_identity4(gates + i) ? -1 : (int)GC_DENSE4;
    return classify(gates[i].U);
  };
  // Execution-order bookkeeping: a two-qubit gate's four records keep consecutive positions.
  auto record_order = [&](int idx) {
    for (int r = 0; r < records_of(idx); ++r) P.gate_order[idx + r] = order++;
  };
  auto record_step = [&](int idx, int step) {
    for (int r = 0; r < records_of(idx); ++r) P.gate_step[idx + r] = step;
  };

  // One fused pass over the chunk bits inQ applying the entries pg (SWAP / identity entries included).
  auto emit_pass = [&](const bool *inQ_in, const std::vector<Sched> &pg, bool init_here) {
    bool inQ[64];
    int qcount = 0;
    for (int b = 0; b < n; ++b) {
      inQ[b] = inQ_in[b];
      qcount += inQ[b] ? 1 : 0;
    }
    // Fill Q up to k bits with the lowest unused bits, so every pass has chunks of exactly 2^k amplitudes.
    for (int b = 0; b < n && qcount < k; ++b)
      if (!inQ[b]) { inQ[b] = true; ++qcount; }
    PassDesc d;
    std::memset(&d, 0, sizeof d);
    d.n = n;
    d.k = k;
    d.c = c;
    int local[64];
    int j = 0;
    for (int b = 0; b < n; ++b)
      if (inQ[b]) {
        local[b] = j;
        d.qpos[j] = (int8_t)b;
        d.qpos_out[j] = (int8_t)b;
        d.qmask |= 1ull << b;
        ++j;
      }
    d.init = init_here ? 1 : 0;
    d.init_x = cfg.init_x;
    const int step_index = (int)P.steps.size();
    P.pass_gate_offset.push_back((int)P.fused_gates.size());
    int ng = 0;
    for (const Sched &s : pg) {
      record_order(s.idx);
      if (s.cls < 0) continue;
      record_step(s.idx, step_index);
      DevGate g;
      std::memset(&g, 0, sizeof g);
      fill_coefficients(g, gates[s.idx].U);
      g.cls = (uint32_t)s.cls;
      if (inQ[s.pt]) g.target = local[s.pt];
      else { g.target = -1; g.tmask = 1ull << s.pt; }
      if (s.cls == GC_DENSE4) g.tmask = (uint64_t)local[s.pt2];
      for (int b = 0; b < n; ++b)
        if (s.pc >> b & 1ull) {
          if (inQ[b]) g.cmask |= 1ull << local[b];
          else g.gmask |= 1ull << b;
        }
      P.fused_gates.push_back(g);
      if (s.cls == GC_DENSE4) {
        for (int r = 1; r < 4; ++r) {
          DevGate row;
          std::memset(&row, 0, sizeof row);
          fill_coefficients(row, gates[s.idx + r].U);
          row.cls = GC_ROW;
          row.target = g.target;
          row.tmask = g.tmask;
          P.fused_gates.push_back(row);
        }
      }
      ++ng;
    }
    d.nblocks = 0;
    if (cfg.block_mode >= 0 && k >= kBlockBits + 7 && k <= (cfg.block_mode == MODE_C64_F32 ? 13 : 12) && ng > 1) {
      const size_t first = P.pass_gate_offset.back();
      std::vector<DevGate> run(P.fused_gates.begin() + first, P.fused_gates.end());
      const int nb = group_blocks(run, k, cfg.block_mode, cfg.block_min_cost, P.block_data);
      if (nb > 0) {
        P.fused_gates.resize(first);
        P.fused_gates.insert(P.fused_gates.end(), run.begin(), run.end());
        d.nblocks = nb;
        P.n_blocks += nb;
        for (const DevGate &g : run)
          if (g.cls == GC_BLOCK) P.n_block_gates += g.target;
      }
    }
    if (cfg.cubes && k >= 8 && ng > 0) {
      const size_t first = P.pass_gate_offset.back();
      std::vector<DevGate> run(P.fused_gates.begin() + first, P.fused_gates.end());
      P.fused_gates.resize(first);
      group_cubes(run, k, P.fused_gates);
    }
    d.ngates = (int)(P.fused_gates.size() - P.pass_gate_offset.back());
    P.step_qmask.push_back(d.qmask);
    P.passes.push_back(d);
    P.steps.push_back({Step::FUSED, (int)P.passes.size() - 1, ng});
    P.n_fused_gates += ng;
  };
  auto low_bits = [&](bool *inQ) {
    for (int b = 0; b < n; ++b) inQ[b] = (k == n) || b < c;
  };

  if (!cfg.fusion) {
    for (size_t i = 0; i < ngates; ++i) {
      const sv_gate &g = gates[i];
      if (g.kind == SV_GATE_U4_ROW) continue;
      if (g.kind == SV_GATE_SWAP) {
        record_order((int)i);
        std::swap(perm[g.target], perm[g.target2]);
        ++P.n_relabels;
        continue;
      }
      const int cls = cls_of_record(i);
      if (cls < 0) {
        record_order((int)i);
        ++P.n_skipped;
        continue;
      }
      const Sched s = sched_of(i, cls);
      if (cls == GC_DENSE4) {  // no single-gate sweep for a two-qubit gate: a one-gate pass over both bits
        bool inQ[64];
        low_bits(inQ);
        inQ[s.pt] = inQ[s.pt2] = true;
        emit_pass(inQ, std::vector<Sched>{s}, false);
        continue;
      }
      record_order((int)i);
      P.sweep_gates.push_back(to_sweep_gate(g, s));
      record_step((int)i, (int)P.steps.size());
      P.step_qmask.push_back(1ull << s.pt);
      P.steps.push_back({Step::SWEEP, (int)P.sweep_gates.size() - 1, 1});
      ++P.n_sweep_gates;
    }
    return;
  }

  // Per-qubit queues of the gates touching each qubit; a gate is ready when it heads all of its queues.
  std::vector<std::vector<int>> q(n);
  std::vector<int> cls_of(ngates, -3);
  auto qubits_of = [&](size_t i, int *out) {
    int m = 0;
    const sv_gate &g = gates[i];
    out[m++] = g.target;
    if (g.kind == SV_GATE_SWAP || g.kind == SV_GATE_U4) out[m++] = g.target2;
    if (g.kind != SV_GATE_SWAP)
      for (int j = 0; j < g.ncontrols; ++j) out[m++] = g.controls[j];
    return m;
  };
  for (size_t i = 0; i < ngates; ++i) {
    if (gates[i].kind == SV_GATE_U4_ROW) continue;
    int qs[8];
    const int m = qubits_of(i, qs);
    for (int j = 0; j < m; ++j) q[qs[j]].push_back((int)i);
    cls_of[i] = cls_of_record(i);
  }
  std::vector<size_t> head(n, 0);
  auto is_ready = [&](int i) {
    int qs[8];
    const int m = qubits_of(i, qs);
    for (int j = 0; j < m; ++j)
      if (head[qs[j]] >= q[qs[j]].size() || q[qs[j]][head[qs[j]]] != i) return false;
    return true;
  };
  std::set<int> ready;
  for (int u = 0; u < n; ++u)
    if (!q[u].empty() && is_ready(q[u][0])) ready.insert(q[u][0]);
  auto pop = [&](int i) {
    ready.erase(i);
    int qs[8];
    const int m = qubits_of(i, qs);
    for (int j = 0; j < m; ++j) ++head[qs[j]];
    for (int j = 0; j < m; ++j) {
      const int u = qs[j];
      if (head[u] < q[u].size() && is_ready(q[u][head[u]])) ready.insert(q[u][head[u]]);
    }
  };
  // Can entry i run in a pass over chunk bits inQ?  Pairing gates need their target bit, two-qubit gates
  // both bits; diagonal gates, SWAPs and identities fit anywhere.
  auto fits = [&](int i, const bool *inQ) {
    const int cls = cls_of[i];
    if (cls < 0) return true;
    if (cls == GC_DENSE4) return inQ[perm[gates[i].target]] && inQ[perm[gates[i].target2]];
    return !needs_pairing(cls) || inQ[perm[gates[i].target]];
  };

  // Gates a pass over the chunk bits inQ plus `extra` would apply from the current frontier, counted on
  // copies of the scheduling state (SWAP relabels included).
  auto closure_with = [&](const bool *inQ, int extra) {
    bool q2[64];
    for (int x = 0; x < n; ++x) q2[x] = inQ[x];
    q2[extra] = true;
    std::vector<size_t> h = head;
    std::vector<int> pm = perm;
    std::set<int> rd = ready;
    auto ready_in = [&](int i) {
      int qs[8];
      const int m = qubits_of(i, qs);
      for (int j = 0; j < m; ++j)
        if (h[qs[j]] >= q[qs[j]].size() || q[qs[j]][h[qs[j]]] != i) return false;
      return true;
    };
    auto fits_in = [&](int i) {
      const int cls = cls_of[i];
      if (cls < 0) return true;
      if (cls == GC_DENSE4) return q2[pm[gates[i].target]] && q2[pm[gates[i].target2]];
      return !needs_pairing(cls) || q2[pm[gates[i].target]];
    };
    int run = 0;
    for (;;) {
      int ch = -1;
      for (int i : rd)
        if (fits_in(i)) { ch = i; break; }
      if (ch < 0) break;
      if (cls_of[ch] == -2) std::swap(pm[gates[ch].target], pm[gates[ch].target2]);
      else if (cls_of[ch] >= 0) ++run;
      rd.erase(ch);
      int qs[8];
      const int m = qubits_of(ch, qs);
      for (int j = 0; j < m; ++j) ++h[qs[j]];
      for (int j = 0; j < m; ++j) {
        const int u = qs[j];
        if (h[u] < q[u].size() && ready_in(q[u][h[u]])) rd.insert(q[u][h[u]]);
      }
    }
    return run;
  };

  bool first_pass = true;
  while (!ready.empty() || (first_pass && cfg.init_first)) {
    bool inQ[64] = {false};
    low_bits(inQ);
    int qcount = 0;
    for (int b = 0; b < n; ++b) qcount += inQ[b] ? 1 : 0;
    std::vector<Sched> pg;  // entries of this pass in scheduling order (SWAP / identity entries included)
    int nreal = 0, ndense4 = 0;
    for (;;) {
      int chosen = -1;
      for (int i : ready)
        if (fits(i, inQ)) { chosen = i; break; }
      if (chosen >= 0) {
        const int cls = cls_of[chosen];
        pg.push_back(sched_of(chosen, cls));
        if (cls == -2) {
          std::swap(perm[gates[chosen].target], perm[gates[chosen].target2]);
          ++P.n_relabels;
        } else if (cls == -1) {
          ++P.n_skipped;
        } else {
          ++nreal;
          ndense4 += cls == GC_DENSE4 ? 1 : 0;
        }
        pop(chosen);
        continue;
      }
      if (qcount >= k || ready.empty()) break;
      // Add the physical bit that the most ready gates are waiting for (ties: the earliest gate) ...
      int best_bit = -1, best_count = 0;
      int counts[64] = {0};
      for (int i : ready) {
        int bits[2] = {perm[gates[i].target], cls_of[i] == GC_DENSE4 ? perm[gates[i].target2] : -1};
        for (int b : bits)
          if (b >= 0 && !inQ[b] && ++counts[b] > best_count) { best_count = counts[b]; best_bit = b; }
      }
      if (best_bit < 0) break;
      // ... unless another bit lets more gates run in this pass: for every candidate bit, simulate the rest
      // of the pass (the gates that become ready as others run included) and take the largest count.
      if (cfg.lookahead) {
        int best_run = closure_with(inQ, best_bit);
        for (int b = 0; b < n; ++b) {
          if (inQ[b] || b == best_bit) continue;
          const int run = closure_with(inQ, b);
          if (run > best_run) { best_run = run; best_bit = b; }
        }
      }
      inQ[best_bit] = true;
      ++qcount;
    }
    const bool init_here = first_pass && cfg.init_first;
    first_pass = false;
    if (nreal == 0 && !init_here) {
      for (const Sched &e : pg) record_order(e.idx);
      continue;
    }
    if (nreal == 1 && ndense4 == 0 && cfg.single_as_sweep && !init_here) {
      for (const Sched &e : pg) {
        record_order(e.idx);
        if (e.cls < 0) continue;
        record_step(e.idx, (int)P.steps.size());
        P.step_qmask.push_back(1ull << e.pt);
        P.sweep_gates.push_back(to_sweep_gate(gates[e.idx], e));
        P.steps.push_back({Step::SWEEP, (int)P.sweep_gates.size() - 1, 1});
        ++P.n_sweep_gates;
      }
      continue;
    }
    emit_pass(inQ, pg, init_here);
  }
}

} // namespace svi
