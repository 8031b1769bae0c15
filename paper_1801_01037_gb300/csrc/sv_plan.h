// Host planner: gate classification, layout map (logical -> physical qubit) and fusion of gates into
// chunk passes.  Pure host code; it launches nothing.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include "sv_internal.h"
#include "../../include/sv.h"

namespace svi {

struct PlanConfig {
  int k = 12;               // chunk qubits (2^k amplitudes per chunk)
  int c = 4;                // contiguous low bits always in a chunk
  bool fusion = true;       // false: every gate becomes a single-gate sweep
  bool single_as_sweep = true;  // a pass holding one gate is emitted as a sweep instead
  bool init_first = false;  // the first pass starts from |init_x> (batched / served states)
  bool cubes = false;       // group each pass's gates into register cubes (complex64 passes, k >= 8)
  bool lookahead = true;    // grow a pass's chunk bits by simulated gate count (false: by immediate demand)
  bool merge = true;        // compose runs of one-qubit gates on one qubit into one matrix (FP64, host)
  uint64_t init_x = 0;
  int block_mode = -1;      // >= 0: form dense tensor-core blocks (GC_BLOCK) for this arithmetic mode
  double block_min_cost = 2.0;  // a block must replace at least this many dense one-qubit gate updates
};

struct Step {
  enum Kind { FUSED = 0, SWEEP = 1 } kind;
  int index;   // FUSED: pass index; SWEEP: sweep gate index
  int ngates;  // source gates this step applies
};

struct Plan {
  std::vector<Step> steps;
  std::vector<PassDesc> passes;      // psi / gates pointers are filled in at launch
  std::vector<int> pass_gate_offset; // first DevGate of each pass in fused_gates
  std::vector<DevGate> fused_gates;
  std::vector<DevGate> sweep_gates;
  int n_fused_gates = 0, n_sweep_gates = 0, n_relabels = 0, n_skipped = 0, n_merged = 0;
  int n_blocks = 0, n_block_gates = 0;
  std::vector<unsigned char> block_data;  // operand planes of the GC_BLOCK records (see sv_internal.h)
  // Schedule record per source gate: the step that applies it (-1: folded into the layout or skipped) and
  // its position in execution order; per step the physical bits its chunks span (a sweep: its target bit).
  std::vector<int> gate_step, gate_order;
  std::vector<uint64_t> step_qmask;
};

// The device copy of a plan's fused passes: its DevGates, in one byte blob.
size_t plan_blob_bytes(const Plan &P);
void plan_blob_fill(const Plan &P, void *dst);
// Point pass `idx` of P at its gates inside a device blob that holds plan_blob_fill's bytes.
void plan_pass_pointers(const Plan &P, int idx, const void *d_blob, PassDesc &d);

// Classify U (8 doubles) by exact comparisons; returns -1 for the identity.
int classify(const double *U);

// Fill q / qh / qm / ql of a DevGate from U.
void fill_coefficients(DevGate &g, const double *U);

// Validate one record against n qubits: qubits in range and distinct, U unitary within 1e-10.
// Returns SV_OK or an sv_status error with `why` set.
int validate_gate(const sv_gate &g, int n, std::string &why);

// Split one pass's gates (chunk-local targets, in order) into register cubes: appends to `out` a GC_CUBE
// header before each run.  Order is kept; every gate lands in exactly one cube.
void group_cubes(const std::vector<DevGate> &run, int k, std::vector<DevGate> &out);

// Replace runs of a pass's gates (chunk-local targets, in order) by dense blocks on kBlockBits bits where that
// saves at least `min_cost` dense one-qubit updates of the chunk; appends each block's operand planes to `data`
// (header gmask = their offset there).  The pass keeps its blocks only if they take at least 3/4 of its
// per-gate work (else `run` and `data` are left as they were).  Returns the number of blocks.
int group_blocks(std::vector<DevGate> &run, int k, int mode, double min_cost, std::vector<unsigned char> &data);
size_t block_data_bytes(int mode);

// Validate a record sequence (two-qubit gates take four records); on error `bad` is the first bad record.
int validate_records(const sv_gate *g, size_t ngates, int n, std::string &why, size_t &bad);

// Plan `ngates` validated records; perm (logical -> physical) is read and updated by SWAP relabelling.
void make_plan(int n, const PlanConfig &cfg, std::vector<int> &perm, const sv_gate *gates, size_t ngates, Plan &out);

// Transpositions (physical bit pairs) that bring `perm` back to the identity, in order; updates perm.
std::vector<std::pair<int, int>> canonicalize_steps(std::vector<int> &perm);

// The same transpositions as gate-free fused passes whose store permutes bits (the paper's relabelling,
// Sec. VI.B, done as data movement): consecutive transpositions on disjoint bits share a pass while their
// bits and the c low bits fit in the chunk.  Updates perm to the identity.
std::vector<PassDesc> canonicalize_passes(int n, const PlanConfig &cfg, std::vector<int> &perm);

} // namespace svi
