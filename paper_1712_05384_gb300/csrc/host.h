// Internal host-side structures shared by host.cpp (circuit, model, plan)
// and exec.cu (device execution).  Not part of the C ABI.
#pragma once

#include <algorithm>
#include <complex>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "qgm.h"

namespace qgm {

using cd = std::complex<double>;

void set_error(const char *fmt, ...);

// ---------------------------------------------------------------- circuit
struct Circuit {
  int n = 0, rows = 0, cols = 0, depth = 0;
  uint64_t seed = 0;
  int param = 0;
  std::vector<qgm_gate> gates;
  std::vector<int> param_gates;
};

// ------------------------------------------------------------------ model
// One factor per gate (Sec. III.B).  Table index = (bit(v[0]) << (nv-1)) | bit(v[1]).
struct MFactor {
  int nv = 0;
  int v[2] = {-1, -1};
  cd t[4];
  int gate = -1;
  int half_pow = 0;  // number of 2^{-1/2} factors pulled out of the table
};

struct Model {
  int n = 0, rows = 0, cols = 0;
  int n_vars = 0;
  std::vector<int> var_qubit, var_k, inputs, outputs;
  std::vector<MFactor> factors;
  int L = 0;                       // non-diagonal gates
  std::vector<int> param_factor;   // factor index of each RXY gate
  std::vector<qgm_gate> gates;     // copy of the circuit's gates
};

// ------------------------------------------------------------------- plan
constexpr int MAXIN = 8;    // tensors multiplied in one step
constexpr int MAXRUN = 16;  // contiguous bit runs of an index map
constexpr int MAXLEAFV = 4; // variables of a leaf factor (internal+slice+output)
constexpr int RES_WARPS = 8; // warps of a resident CTA

// Index map of one step input: the input's index is the union index with
// the bits of absent variables squeezed out (a "pext" by contiguous runs).
struct InDesc {
  int64_t off;       // byte offset of the tensor in the workspace
  int32_t meta;      // tensor metadata slot (intermediates), -1 for leaves
  int32_t batched;   // 1: rows of batch_padded complex values
  int32_t nruns;
  uint8_t src[MAXRUN], len[MAXRUN], dst[MAXRUN];
};

struct StepDesc {
  int32_t m;            // inputs
  int32_t k;            // variables summed (top k bits of the union index)
  int32_t w_out;        // output rank (binary variables)
  int32_t batched_out;
  int64_t out_off;
  int32_t out_meta;
  int32_t gemm;         // index of the step's GemmDesc, or -1
  // register tile: output bits (union positions < w_out) that the largest
  // input does not hold; a thread loads that input once per term and forms
  // the 2^tile_t outputs that share it
  int32_t tile_t;
  uint8_t tile_pos[4];
  InDesc in[MAXIN];
};

// A GEMM-shaped step: out[s, m, n] = sum_k A[s, m, k] B[s, n, k] with s the
// kept variables both operands hold, m (n) the kept variables only A (B)
// holds and k the summed variables (both hold all of them).  Each operand
// and the output are addressed through the bit positions of those
// variables in their own index (no transposition); the batch axis, when
// present, stays innermost.
constexpr int GMAXB = 24;
struct GemmDesc {
  int64_t a_off, b_off, o_off;
  int32_t a_meta, b_meta, o_meta;
  int32_t a_bat, b_bat, o_bat;
  int32_t nm, nn, nk, ns;
  // batch entry outermost (a tensor written by one tensor-core product per
  // entry and read only by another tensor-core step): entry beta's values
  // are a whole tensor of 2^rank complex64 at beta * 2^rank * 8 bytes
  int32_t a_bout, b_bout, o_bout;
  uint8_t mA[GMAXB], mO[GMAXB], nB[GMAXB], nO[GMAXB];
  uint8_t kA[GMAXB], kB[GMAXB], sA[GMAXB], sB[GMAXB], sO[GMAXB];
};

// Exchange the roles of the two operands: out[s, n, m] = sum_k B A is the
// same product.
inline void gemm_swap_roles(GemmDesc &g) {
  std::swap(g.a_off, g.b_off);
  std::swap(g.a_meta, g.b_meta);
  std::swap(g.a_bat, g.b_bat);
  std::swap(g.a_bout, g.b_bout);
  std::swap(g.nm, g.nn);
  for (int b = 0; b < GMAXB; ++b) {
    std::swap(g.mA[b], g.nB[b]);
    std::swap(g.mO[b], g.nO[b]);
    std::swap(g.kA[b], g.kB[b]);
    std::swap(g.sA[b], g.sB[b]);
  }
}

// Tensor-core form of a GEMM-shaped step.  One operand takes the MMA's M
// side (tiles of 128 rows), the other the N side (tiles of nt = min(256,
// 2^nN) rows); both are first split into planes of 16-bit terms stored as
// the MMA reads them.  When only one operand carries the batch axis it takes
// the M side and its batch entries become rows there (row = m * Bp + beta),
// so the other operand's tile serves every entry; when both carry it, each
// (shared index, batch entry) is a product of its own ("per entry").  A
// plane block holds, for one instance (shared index, and batch entry when
// per entry), one row tile and one chunk of 16 summed entries, P planes of
// TR x 16 terms in 8-row x 16-byte core matrices (row group stride 256 B,
// the two 8-entry halves of a row 128 B apart).
constexpr int TC_M = 128;
struct TcCfg {
  bool ok = false;
  bool swap = false;     // B takes the M side
  bool fold = false;     // batch entries are rows of the M side
  bool perbeta = false;  // one product per (shared index, batch entry)
  int nM = 0, nN = 0;    // private kept variables of the M and N sides
  int nt = 0;            // N tile
  int64_t mrows = 0, mtiles = 0, ntiles = 0, kc = 0, inst = 0;
  int64_t bytesM = 0, bytesN = 0;  // plane bytes of the M and N sides
};

// planes: 16-bit terms per complex value (4: FP16 high and low parts of the
// real and imaginary parts; 6: three BF16 terms of each)
inline TcCfg tc_config(const GemmDesc &g, int Bp, int planes, int nt_cap = 256) {
  TcCfg c;
  const bool one = g.o_bat && (g.a_bat != g.b_bat);
  c.swap = one ? (g.b_bat != 0) : (g.nn > g.nm);
  c.fold = one && Bp > 1;
  c.perbeta = g.o_bat && g.a_bat && g.b_bat && Bp > 1;
  c.nM = c.swap ? g.nn : g.nm;
  c.nN = c.swap ? g.nm : g.nn;
  if (g.nk < 1 || c.nN < 5 || g.ns > 15 || c.nM > 30) return c;
  c.mrows = ((int64_t)1 << c.nM) * (c.fold ? Bp : 1);
  if (c.mrows < TC_M) return c;
  c.mtiles = (c.mrows + TC_M - 1) / TC_M;
  c.nt = c.nN >= 8 ? 256 : (1 << c.nN);
  if (c.nt > nt_cap && nt_cap >= 32) c.nt = nt_cap;  // narrower N tiles: two CTAs per SM
  c.ntiles = ((int64_t)1 << c.nN) / c.nt;
  c.kc = (((int64_t)1 << g.nk) + 15) / 16;  // fewer than 16 summed entries: one chunk, zero-padded
  c.inst = ((int64_t)1 << g.ns) * (c.perbeta ? Bp : 1);
  if (c.inst * c.mtiles * c.ntiles >= ((int64_t)1 << 31)) return c;
  c.bytesM = c.inst * c.mtiles * c.kc * planes * TC_M * 32;
  c.bytesN = c.inst * c.ntiles * c.kc * planes * c.nt * 32;
  c.ok = true;
  return c;
}

// Launch parameters of one step chosen by the autotuner (qgm_plan_opts.autotune)
// by timing its candidates on the bound device; zeros are the fixed rules.
struct StepTune {
  int32_t nt_cap = 0;     // tensor-core GEMM: N tile at most 256, 128 or 64 (0: 256)
  int32_t T = 0;          // batched product-sum: term groups per row (0: rule)
  int32_t conv = 0;       // folded tensor-core step: 1 converts the M side in the product kernel
  int32_t U = 0;          // batched product-sum: terms in flight per thread (4 or 8, else 2)
  int32_t ps = 0;         // GEMM-shaped step: 1 runs it with the product-sum kernels
  float ms_rule = 0.f;    // measured time with the fixed rules (ms)
  float ms_best = 0.f;    // measured time of the chosen candidate (ms)
};

// A GEMM step runs on the tensor cores when its tensor-core form exists: the
// M side has at least 128 rows (batch entries counted when they become
// rows), the N side at least 32 (summed entries are zero-padded to whole
// chunks of 16, one MMA's K).
inline bool gemm_tc_eligible(const GemmDesc &g, int Bp) { return tc_config(g, Bp, 4).ok; }

// The FP32-core GEMM kernel's shapes: 64-row A tiles, 32- or 64-column B
// tiles, chunks of 16 summed entries.  Other GEMM steps (accepted for the
// tensor cores) run with the product-sum kernels where the tensor cores are
// not used.
inline bool gemm_fp32_ok(const GemmDesc &g) { return g.nk >= 4 && g.nm >= 6 && g.nn >= 5; }

// Leaf factor built on the device per slice: base table over
// (internal vars | slice vars | output vars), MSB first.
struct LeafDesc {
  int64_t base_off;  // complex64 base table (bytes into the workspace)
  int64_t out_off;   // built table
  int32_t n_int, n_slice, n_out, batched;
  int32_t slice_bit[MAXLEAFV];  // bit of the slice id for each slice var
  int32_t out_qubit[MAXLEAFV];  // qubit of each output var
};

// Resident executor: one CTA per chunk of Bc batch entries runs every step
// with its tensors in shared memory.  Offsets are bytes into dynamic smem.
// Input index = pext(row, runs) | (pext(e, emask) << rowbits): the summed
// variables are the top bits of the union index and, the input's variables
// being sorted the same way, the top bits of the input index too.
// One input of a resident step with its address tables precomputed by the
// planner (every input index is linear in the bits of the union index; all
// entries are byte offsets in shared memory):
//   lrow[b]  value of row bit b (b < r0), for a thread's first row;
//   lterm[b] value of summed bit b (b < lg), for a thread's first term;
//   rinc[t]  change when the thread's row counter carries into bit t;
//   tinc[t]  change when its term counter carries into bit t.
struct RIn {
  int32_t soff;      // smem byte offset of the tensor
  int32_t meta;      // smem metadata slot (intermediates), -1 for leaves
  int32_t batched;
  int32_t nlow;      // entries of lrow in use (min(r0, w_out))
  int32_t rinc[16];
  int32_t tinc[8];
  int32_t lrow[8];
  int32_t lterm[8];
};

struct RStep {
  int32_t m, k, w_out, batched_out;
  int32_t out_soff, out_meta;
  // warps [w0, w0 + nw) run the step with 2^lg lanes per output entry;
  // bit 16: the last step of its dependency level (a block barrier follows)
  int32_t sched;
  int32_t bytes;     // bytes of this descriptor in use (header + m inputs)
  RIn in[MAXIN];
};
constexpr int SCHED_LAST = 1 << 16;

struct RLeaf {        // leaf materialised in smem per chunk
  int32_t leaf;       // index into the LeafDesc table
  int32_t soff;
  int32_t batched;    // 1: rows x Bc entries from the bitstrings; 0: the table
  int32_t pad_;
};

// One row of a leaf staged into shared memory: entry (row, beta) is base
// entry src + (output bits of x_beta) stored at smem byte dst + 8 * beta
// (batched) or dst (unbatched).
struct RJob {
  int32_t src;      // float2 index into the workspace base tables
  int32_t dst;      // smem byte offset of (row, beta = 0)
  uint8_t n_out;    // output qubits of the leaf (0..2)
  uint8_t q0, q1;   // their qubits, most significant first
  uint8_t batched;
};

// Work list of the warps: entry = step | level << 12 | descriptor words << 22;
// warp w owns entries [wstart[w], wstart[w + 1]), ordered by level.
struct ResidentLayout {
  int chunk = 0;            // Bc
  int64_t smem_bytes = 0;   // dynamic shared memory per CTA
  std::vector<RStep> steps;
  std::vector<RLeaf> leaves;
  std::vector<RJob> jobs;
  std::vector<uint32_t> wlist;
  int32_t wstart[RES_WARPS + 1] = {0};
  int n_levels = 0;
  int wlist_soff = 0;       // smem byte offset of the work lists
  int final_soff = -1, final_meta = -1;
  std::vector<int> src_step, level;  // per entry of `steps`: plan step, dependency level
  // The bitstring-independent part: steps without a batch axis, run once per
  // call by a one-CTA kernel (compiled executor); `pre` lists their outputs
  // read by batched steps, staged through the workspace's pre region.
  struct PreT {
    int32_t soff;     // smem byte offset in this layout
    int32_t meta;     // metadata slot
    int32_t entries;  // complex64 entries
    int32_t goff;     // float2 index in the pre region's data
  };
  std::vector<PreT> pre;
  bool split_pre = false;  // the compiled executor runs the pre kernel
};

// Shared-memory bytes of the work lists, which sit between the metadata and
// the tensors (the compiled kernel has no work lists and drops them).
inline int64_t worklist_bytes(const ResidentLayout &L) { return ((int64_t)L.wlist.size() * 4 + 15) & ~int64_t(15); }
// Steps of the compiled resident kernel with a static bound on their output:
// every input is a leaf (gate tables: entries of modulus at most 1) or the
// output of such a step, scaled by the consumer to maxima at most 1/2, so
// |out| <= 2^k for k summed variables.  That bound, placed in the kernel's
// initial shared-memory image, serves as the recorded maximum (no run-time
// reduction); chains of such steps stop after three levels, so that the
// headroom a loose bound gives away stays far from FP32's range, and the
// final tensor is always measured (non-finite values reach it and set the
// status there).  Returns metadata slot -> (k, exponent), the exponent being
// the sum of the inputs' exponents and scale exponents, as at run time.
std::map<int, std::pair<int, int>> static_bounds(const ResidentLayout &L);
// Dynamic shared memory of the compiled resident kernel (16-byte multiple).
inline int64_t compiled_smem(const ResidentLayout &L) { return (L.smem_bytes - worklist_bytes(L) + 15) & ~int64_t(15); }

// Gradient of one parametrised gate (adjoint elimination): the adjoint of
// the leaf holding the gate, and the leaf's derivative tables with respect to
// theta and phi in the leaf's base-table layout.
struct GradParam {
  int64_t dbase_off[2];  // complex64 derivative base tables (bytes into the workspace)
  int64_t adj_off;       // adjoint of the leaf: rows x batch_padded complex64
  int32_t adj_meta;
  int32_t n_int, n_out, n_slice;  // derivative table over (internal | slice | output) variables
  int32_t out_qubit[MAXLEAFV];
  int32_t slice_bit[MAXLEAFV];    // bit of the slice id for each slice variable
};

struct SymTensor {
  std::vector<int> vars;  // sorted by elimination position
  bool batched = false;
  int leaf = -1;          // leaf index or -1
  int meta = -1;          // metadata slot for intermediates
  int64_t off = -1;       // byte offset in the workspace
  int64_t entries = 0;
};

struct StepRec {
  std::vector<int> inputs;  // SymTensor ids
  std::vector<int> uni;     // union vars (sorted)
  int k = 0;
  int out = -1;
  bool batched = false;
  double bytes = 0, flops = 0;
  bool gemm = false;        // two operands, run by the GEMM kernel
  // nested evaluation (compiled resident kernel): the last k_inner summed
  // variables occur only in the inputs flagged inner, so
  // out = sum_outer prod(outer inputs) * sum_inner prod(inner inputs)
  int k_inner = 0;
  std::vector<char> inner;
};

struct LeafFactor {          // merged factor after fixing the inputs
  std::vector<int> scope;    // var ids (table is C-order over scope)
  std::vector<cd> table;
  int half_pow = 0;
  std::vector<int> members; // model factor ids merged into it
};

struct SimResult {
  double bytes = 0, flops = 0, max_step_bytes = 0;
  int64_t max_entries = 0;
  int64_t arena_peak = 0;
  int max_clique = 0;
  std::vector<SymTensor> tensors;
  std::vector<StepRec> steps;
  std::vector<int> final_tensors;
  int final_tensor = -1;
  int tree_error = -1;  // a tensor consumed other than once (plan invariant broken)
};

}  // namespace qgm

struct qgm_circuit {
  qgm::Circuit c;
};
struct qgm_model {
  qgm::Model m;
};

struct qgm_exec_state;  // device-side state (exec.cu)

struct qgm_plan {
  const qgm::Model *model_copy_owner = nullptr;
  qgm::Model model;
  qgm_plan_opts opts{};
  int order_kind = 0;
  int output_mode = 0;
  int64_t batch = 1;
  int32_t Bp = 1;
  std::vector<int> order;        // eliminated vars
  std::vector<int> open_vars;    // never eliminated (open outputs)
  std::vector<int> slice_vars;
  std::vector<int> pos;          // elimination position per var (-1: not in graph)
  std::vector<int> var_role;     // 0 free, 1 input, 2 output(batched), 3 open, 4 slice
  std::vector<qgm::LeafFactor> leaves;
  qgm::cd constant = 1.0;        // product of scope-free factors and 2^{-L/2}
  int half_pow_total = 0;
  qgm::SimResult sim;
  // device layout
  std::vector<qgm::StepDesc> steps;
  std::vector<qgm::GemmDesc> gemms;
  std::vector<qgm::LeafDesc> leafdesc;
  std::vector<float> base_tables;  // interleaved complex64
  int n_meta = 0;
  int64_t off_header = 0, off_meta = 0, off_leafdesc = 0, off_base = 0, off_leaf = 0, off_bits = 0,
          off_outstage = 0, off_acc = 0, off_arena = 0, ws_bytes = 0;
  int64_t final_entries = 0;     // rows of the final tensor (2^n_open or 1)
  int open_in_batch = 0;         // open output qubits of a batch plan (k)
  int final_batched = 0;
  int64_t final_off = 0;
  int final_meta = -1;
  // adjoint elimination (qgm_plan_opts.gradients): forward steps that keep
  // every intermediate, the seed, backward steps, one record per parameter
  bool grad = false;
  std::vector<qgm::StepDesc> gfwd, gbwd;
  std::vector<qgm::GradParam> gparams;
  int64_t g_final_off = 0, g_seed_off = 0, off_gparams = 0;
  int g_final_meta = -1, g_seed_meta = -1, g_final_batched = 0;
  int n_meta_fwd = 0;
  // resident executor layouts for Bc = 1, 2, 4, 8 (empty when infeasible)
  std::vector<qgm::ResidentLayout> resident;
  int64_t off_rsteps = 0;   // workspace region for the chosen layout's steps
  int64_t off_pre = 0;      // pre region: per pre tensor (maxbits, exp), then the data (16-byte aligned)
  int64_t pre_data = 0;     // float2 index of the data inside the pre region
  int64_t off_image = 0;    // compiled resident kernel: initial shared-memory image (bitstring-independent leaves)
  int executor_pref = 0;    // qgm_plan_opts.executor
  bool gemm_ok = true;      // GEMM-shaped steps run by the GEMM kernel
  bool gemm_tc = false;     // eligible GEMM steps run on the tensor cores (split terms)
  int tc_planes = 4;        // 16-bit terms per complex value: 4 (FP16 x 2) or 6 (BF16 x 3)
  int64_t off_planes = 0;   // workspace region of the split operand planes
  int64_t planes_bytes = 0; // its size (the largest tensor-core step's two operands)
  int64_t ws_fwd_bytes = 0; // workspace the forward pass needs without that region
  std::vector<qgm::StepTune> tune;  // per step of `steps` (autotuner choices)
  // runs of consecutive small steps without a batch axis, run by one CTA in
  // one launch: plain_group[s] = steps in the run starting at s (0: none);
  // their descriptors are copied to the workspace at off_sdesc
  std::vector<int32_t> plain_group;
  int64_t off_sdesc = 0;
  // per leaf: table layout (internal | slice | output variables), offset of
  // its base table and of its derivative tables (floats), its RXY member
  std::vector<std::vector<int>> leaf_layout;
  std::vector<int64_t> base_at, dbase_at;
  std::vector<int> rxy_member;
  bool trees_ok = false;    // buckets of three or more inputs may run as contraction trees
  bool nest_ok = true;      // buckets may be marked for nested evaluation
  qgm_exec_state *exec = nullptr;
};

namespace qgm {
int build_plan(const Model &m, const qgm_plan_opts &o, qgm_plan *p);
int plan_set_params(qgm_plan *p, const double *params);
// CUDA source of the resident kernel specialised to one layout (jit.cpp):
// the whole pass, its batched part, or its bitstring-independent part
enum { RES_WHOLE = 0, RES_MAIN = 1, RES_PRE = 2 };
std::string resident_source(const qgm_plan *p, const ResidentLayout &L, const std::string &name, int minb,
                            int mode);
}
