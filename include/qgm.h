/*
 * qgm.h -- C ABI of the GB300 amplitude engine.
 *
 * Computes output amplitudes <x|C|0^n> of low-depth random grid circuits as
 * the partition function of a complex undirected graphical model, evaluated
 * by variable elimination (Boixo, Isakov, Smelyanskiy, Neven,
 * arXiv:1712.05384).  Host-side functions (circuit, model, plan) run on the
 * CPU; the elimination itself runs in hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: QGM_OK (0) or a negative
 *    QGM_ERR_* code.  No C++ exception crosses this boundary; the message of
 *    the last error on the calling thread is returned by qgm_last_error().
 *  - Handles (qgm_circuit, qgm_model, qgm_plan) are opaque, owned by the
 *    library, and released with the matching qgm_*_free (NULL is accepted).
 *  - Device buffers are owned by the caller: pointers are plain device
 *    addresses (cudaMalloc or a torch tensor's data_ptr) and `stream` is a
 *    cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Bit j of an output bitstring (uint64) is the value of qubit j; qubit
 *    q = r * cols + c on a rows x cols grid.
 *  - Complex results are complex128, stored as interleaved (re, im) doubles.
 */
#ifndef QGM_H
#define QGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  QGM_OK = 0,
  QGM_ERR_ARG = -1,       /* invalid argument, size or state */
  QGM_ERR_OOM = -2,       /* plan exceeds the memory budget / workspace too small */
  QGM_ERR_CUDA = -3,      /* a CUDA runtime call failed */
  QGM_ERR_TIMEOUT = -4,   /* a bounded device wait gave up */
  QGM_ERR_NONFINITE = -5, /* a tensor maximum became Inf/NaN */
  QGM_ERR_NOGPU = -6      /* no CUDA device is visible */
};

/* Gate kinds (paper Sec. "Numerical results": H, X^1/2, Y^1/2, T, CZ) plus
 * the parametrised one-qubit gate exp(-i theta (cos phi X + sin phi Y) / 2). */
enum {
  QGM_GATE_H = 0,
  QGM_GATE_X12 = 1,
  QGM_GATE_Y12 = 2,
  QGM_GATE_T = 3,
  QGM_GATE_CZ = 4,
  QGM_GATE_RXY = 5
};

typedef struct {
  int32_t kind;   /* QGM_GATE_* */
  int32_t cycle;  /* clock cycle t of Eq. fpath (0 = the H layer) */
  int32_t q0;     /* qubit */
  int32_t q1;     /* second qubit of a CZ, else -1 */
  double theta;   /* QGM_GATE_RXY only */
  double phi;     /* QGM_GATE_RXY only */
} qgm_gate;

typedef struct qgm_circuit qgm_circuit;
typedef struct qgm_model qgm_model;
typedef struct qgm_plan qgm_plan;

/* Message of the last failed call on this thread ("" if none). */
const char *qgm_last_error(void);

/* ---------------------------------------------------------------- circuit */

/* Random grid circuit, paper Sec. "Numerical results" (layout rules cited
 * there, read as: H layer in cycle 0; CZ layer (t-1) mod 8 of the rotation
 * [HZ0,HZ2,VT0,VT2,HZ1,HZ3,VT1,VT3] in cycle t; a qubit in a CZ at t-1 and
 * none at t gets T the first time, then X^1/2 or Y^1/2 from SplitMix64(seed)).
 * param_mode != 0 turns every X^1/2/Y^1/2 slot into RXY(theta, phi) with
 * theta = pi u1, phi = 2 pi u2 from two draws.  depth counts all cycles.
 * Errors: QGM_ERR_ARG for rows, cols, depth < 1 or rows*cols > 64. */
int qgm_circuit_grid(int rows, int cols, int depth, uint64_t seed, int param_mode,
                     qgm_circuit **out);

/* Circuit from an explicit host gate list (copied).  Gates act in list
 * order.  Errors: QGM_ERR_ARG for bad kinds or qubit indices. */
int qgm_circuit_from_gates(int n_qubits, const qgm_gate *gates, int64_t n_gates,
                           qgm_circuit **out);

/* Copies up to `cap` gates into `gates` (host) and stores the count in *n. */
int qgm_circuit_gates(const qgm_circuit *c, qgm_gate *gates, int64_t cap, int64_t *n);

/* Indices (into the gate list) of the RXY gates, in list order: the
 * parameter order of qgm_amplitude_grad (theta_p at 2p, phi_p at 2p+1). */
int qgm_circuit_param_gates(const qgm_circuit *c, int32_t *idx, int64_t cap, int64_t *n);

/* Expectation value of a Pauli string (Sec. III): for O = pauli[0] (x) ...
 * (character j, one of 'I', 'X', 'Y', 'Z', acts on qubit j), the gates of c
 * outside O's backward light cone cancel against their inverses and
 * <0|U^dagger O U|0> = phase * <0|W|0>, where W (written to *out, a new
 * circuit to free with qgm_circuit_free) applies the light-cone gates V,
 * then O, then V^dagger, on the qubits V touches, renumbered in increasing
 * order (qubit_of[j]: new index of qubit j or -1; may be NULL).  O and the
 * inverse gates are expressed exactly in the gate set (Z = T^4,
 * X = i RXY(pi, 0), Y = i RXY(pi, pi/2), T^-1 = T^7, (X^1/2)^-1 =
 * RXY(pi/2, pi), (Y^1/2)^-1 = RXY(pi/2, 3pi/2), RXY(t, f)^-1 = RXY(t, f + pi));
 * phase (double[2], re and im) collects the factors i.  The amplitude of the
 * all-zero bitstring of W then comes from any plan (qgm_plan_order, ...).
 * For O = I: *out = NULL and phase = 1.  Errors: QGM_ERR_ARG. */
int qgm_circuit_observable(const qgm_circuit *c, const char *pauli, qgm_circuit **out, double *phase,
                           int32_t *qubit_of);

/* Ordering study (Sec. IV.B, App. E, Fig. 6): the line graph of the
 * circuit's tensor network -- one vertex per wire segment between two gates
 * (segments to the fixed input and output vectors are fixed indices and drop
 * out), a clique per gate over its segments -- eliminated in min-fill order
 * (ties: fewest neighbours, then lowest segment number; segments numbered in
 * the order their consumer gates close them).  *max_clique: the largest
 * clique along that order (treewidth bound = *max_clique - 1);
 * *n_segments (may be NULL): vertices.  Errors: QGM_ERR_ARG. */
int qgm_circuit_line_graph_width(const qgm_circuit *c, int32_t *n_segments, int32_t *max_clique);

void qgm_circuit_free(qgm_circuit *c);

/* ------------------------------------------------------------------ model */

typedef struct {
  int32_t n_qubits;
  int32_t n_vars;      /* sum_j (d_j + 1): one variable b_j^k per qubit j and
                          per non-diagonal gate k, plus b_j^0 (Sec. III.A) */
  int32_t n_factors;   /* one factor per gate (Sec. III.B) */
  int32_t n_nondiag;   /* L of App. F: number of non-diagonal gates */
  int32_t n_params;    /* 2 * number of RXY gates */
} qgm_model_info;

/* Circuit -> graphical model (Sec. III.B, Eq. psi_x).  Diagonal gates (T, CZ)
 * add factors but no variable; H, X^1/2, Y^1/2, RXY add one variable each.
 * Variable ids: b_j^0 = j, then one id per non-diagonal gate in gate order. */
int qgm_build_model(const qgm_circuit *c, qgm_model **out);
int qgm_model_get_info(const qgm_model *m, qgm_model_info *info);

/* Per variable: qubit j and worldline index k (arrays of n_vars, host). */
int qgm_model_vars(const qgm_model *m, int32_t *qubit, int32_t *k);

/* Per factor f: scope size in nvar[f] (1 or 2) and the variable ids in
 * scope[2f], scope[2f+1] (-1 when unused). */
int qgm_model_factors(const qgm_model *m, int32_t *nvar, int32_t *scope);

void qgm_model_free(qgm_model *m);

/* ------------------------------------------------------------------- plan */

enum {
  QGM_ORDER_AUTO = 0,       /* cheapest of the orders below by the cost model */
  QGM_ORDER_MINFILL = 1,    /* min-fill; ties: fewest neighbours, smallest id */
  QGM_ORDER_VERTICAL = 2,   /* Sec. IV.A: worldlines in lexicographic (j, k),
                               j along the smaller lateral dimension first */
  QGM_ORDER_VERTICAL_T = 3, /* the same with the other lateral dimension */
  QGM_ORDER_GIVEN = 4       /* order passed in qgm_plan_opts.order */
};

enum {
  QGM_OUT_BATCH = 0,  /* outputs fixed per bitstring of a batch (batch axis) */
  QGM_OUT_OPEN = 1    /* all outputs left open: 2^n amplitudes (Eq. psi_x
                         without output deltas) */
};

typedef struct {
  int32_t order_kind;         /* QGM_ORDER_* */
  int32_t output_mode;        /* QGM_OUT_* */
  int64_t batch;              /* bitstrings per call (QGM_OUT_BATCH), >= 1 */
  int64_t mem_budget_bytes;   /* cap on live intermediates; 0 = 64 GiB */
  int32_t max_fuse;           /* max variables summed in one step (0 = 8) */
  int32_t n_order;            /* QGM_ORDER_GIVEN: length of `order` */
  const int32_t *order;       /* QGM_ORDER_GIVEN: elimination order (var ids) */
  int32_t executor;           /* QGM_EXEC_* */
  int32_t no_gemm;            /* 1: run GEMM-shaped steps with the product-sum
                                 kernel instead of the tiled GEMM kernel */
  int32_t gradients;          /* 1: also lay out the adjoint elimination of
                                 qgm_amplitude_grad (more workspace) */
  int32_t trees;              /* buckets of three or more inputs as contraction
                                 trees (pairs multiplied first, each variable
                                 summed once no other factor holds it) where that
                                 needs clearly fewer products: 1 on, -1 off,
                                 0 automatic (on for batch plans that no resident
                                 layout fits, when it saves 10% of the products) */
  uint64_t open_mask;         /* QGM_OUT_BATCH: qubits whose outputs stay open
                                 (Eq. psi_x without their deltas): each bitstring
                                 then yields 2^popcount(open_mask) amplitudes */
  int32_t resident_chunk;     /* bitstrings per CTA of the resident executor:
                                 1, 2, 4 or 8; 0 = chosen at bind (fewest
                                 waves x chunk on the bound device) */
  int32_t autotune;           /* 1: qgm_plan_bind times the candidate launch
                                 parameters of every step that has several (the
                                 tensor-core GEMM's N tile: 256, 128 or 64
                                 columns, and for a folded step whether its
                                 streamed operand is split in a pass of its own
                                 or inside the product kernel; the batched
                                 product-sum kernel's term
                                 groups: 1, 2 or 4, and terms in flight per
                                 thread: 2, 4 or 8; a GEMM-shaped step may run
                                 as a product-sum) on the bound device, on
                                 tensors from one pass over an all-zero batch,
                                 and keeps the fastest; 0: fixed rules */
  int32_t gemm_precision;     /* GEMM-shaped steps whose tensor-core form exists
                                 (one side >= 128 rows, batch entries counted
                                 when the other side has no batch axis; the
                                 other >= 32; 16 summed entries per chunk) run
                                 on the tensor cores with FP32 accumulation
                                 as split products of 16-bit terms:
                                 0 (default) or 2: split FP16 -- each scaled
                                 FP32 value x = h + l, h = fp16(x),
                                 l = fp16(x - h), the products h h' + h l' +
                                 l h' (22 significant bits, 12 MMAs per chunk
                                 of a complex product);
                                 1: split BF16 -- three 8-bit terms, the six
                                 term products above 2^-24 (24 MMAs);
                                 -1: every GEMM step on the FP32 cores (plain
                                 complex64) */
  int32_t n_keep;             /* QGM_OUT_BATCH: variables (model ids, not
                                 inputs) kept open like open outputs: the
                                 result then has 2^(k + n_keep) entries per
                                 bitstring, keep_vars[j] being bit j of the
                                 low n_keep bits of the entry index (e.g. an
                                 intermediate table of App. D, see
                                 qgm_eliminate_fixed) */
  const int32_t *keep_vars;   /* n_keep variable ids (copied at plan time) */
  int32_t tc_convert;         /* tensor-core steps whose batch entries are rows
                                 of M (one operand batch-free): 1 converts the
                                 batched operand to its 16-bit terms inside the
                                 product kernel, 0 (default) in a split pass of
                                 its own; with autotune on, the faster per step */
} qgm_plan_opts;

enum {
  QGM_EXEC_AUTO = 0,      /* compiled resident, else resident, when a chunk's live
                             set fits in shared memory; else stepwise */
  QGM_EXEC_STEPWISE = 1,  /* one kernel per step over the whole batch (CUDA graph) */
  QGM_EXEC_RESIDENT = 2,  /* one persistent launch: each CTA runs all steps for a
                             chunk of bitstrings out of shared memory, reading a
                             descriptor per step */
  QGM_EXEC_COMPILED = 3   /* the resident launch with a kernel generated for this
                             plan and compiled at bind time (NVRTC): offsets,
                             index maps and the warp schedule are constants */
};

typedef struct {
  int32_t order_kind;         /* the order actually used */
  int32_t n_free;             /* variables eliminated */
  int32_t max_clique;         /* induced width, size convention (Sec. IV.B) */
  int32_t n_steps;            /* kernel steps per slice */
  int32_t n_slice_vars;       /* variables sliced (conditioned on) */
  int32_t batch_padded;       /* batch axis length in memory */
  int64_t n_slices;           /* 2^n_slice_vars */
  int64_t max_tensor_entries; /* largest intermediate, complex64 entries */
  int64_t workspace_bytes;    /* device workspace qgm_plan_bind needs */
  int64_t arena_bytes;        /* of which live intermediates */
  double bytes_per_slice;     /* algorithmic bytes (inputs read + output written) */
  double flops_per_slice;     /* algorithmic real flops of the products and sums */
  double max_step_bytes;      /* algorithmic bytes of the largest step */
  int32_t n_gemm_steps;       /* steps run by the tiled GEMM kernel */
  int32_t n_tile_steps;       /* batched steps run with a register tile */
  int32_t n_nested_steps;     /* steps whose compiled form sums some variables
                                 in an inner loop over part of the inputs */
  int32_t n_gemm_tc_steps;    /* of the GEMM steps, those run on the tensor
                                 cores (qgm_plan_opts.gemm_precision) */
} qgm_plan_info;

/* Elimination order, slicing, step list and memory layout (Sec. IV, App. A).
 * Host only; deterministic.  Errors: QGM_ERR_ARG for bad options,
 * QGM_ERR_OOM when no slicing brings the live set under the budget. */
int qgm_plan_order(const qgm_model *m, const qgm_plan_opts *opts, qgm_plan **out);
int qgm_plan_get_info(const qgm_plan *p, qgm_plan_info *info);
/* The elimination order (n_free var ids) and the sliced variables. */
int qgm_plan_get_order(const qgm_plan *p, int32_t *order, int64_t cap, int64_t *n);
int qgm_plan_get_slice_vars(const qgm_plan *p, int32_t *vars, int64_t cap, int64_t *n);
/* Per-step record for tests and reports: for step s, out_rank[s] (binary
 * variables of the output), k[s] (variables summed), n_in[s], batched[s]. */
int qgm_plan_get_steps(const qgm_plan *p, int32_t *out_rank, int32_t *k, int32_t *n_in,
                       int32_t *batched, int64_t cap);
/* Kernel that runs step s in the stepwise executor: 0 product-sum without a
 * batch axis, 1 batched product-sum, 2 batched with a register tile, 3 tiled
 * GEMM, 4 a small step without a batch axis run with its neighbours of the
 * same kind in one single-CTA launch. */
int qgm_plan_get_step_kernels(const qgm_plan *p, int32_t *kind, int64_t cap);

/* Algorithmic cost of step s: bytes[s] (inputs read once + output written,
 * complex64) and flops[s] (real flops of the products and sums). */
int qgm_plan_get_step_cost(const qgm_plan *p, double *bytes, double *flops, int64_t cap);
/* Structure of step s for reports and tests: rec = [U, k, m, then per input
 * i: r_i, batched_i, and the positions in the step's union (summed variables
 * first, each group in elimination order) of its r_i variables].  *n = the
 * record's length; rec may be NULL to query it.  Host only. */
int qgm_plan_get_step_inputs(const qgm_plan *p, int32_t step, int32_t *rec, int64_t cap, int64_t *n);

/* Autotuner choices (qgm_plan_opts.autotune, after qgm_plan_bind): for the
 * c-th tuned step, rec[6c .. 6c+5] = step index, tensor-core N tile cap (0:
 * not a tensor-core step), product-sum term groups (0: not tuned), 1 when a
 * folded tensor-core step converts its streamed operand inside the product
 * kernel (instead of a separate split pass), product-sum terms in flight
 * per thread (4 or 8, or 0/2 for two), 1 when a GEMM-shaped step runs with the
 * product-sum kernels instead of a GEMM kernel, and
 * ms[2c], ms[2c+1] = milliseconds with the fixed rules and with the choice.
 * *n = the number of tuned steps; rec/ms may be NULL to query it. */
int qgm_plan_get_tuning(const qgm_plan *p, int32_t *rec, float *ms, int64_t cap, int64_t *n);

/* Sets launch parameters of steps by hand, in the records qgm_plan_get_tuning
 * returns (6 ints per step: step index, N tile cap 0/64/128/256, term groups
 * 0/1/2/4, in-kernel conversion 0/1, terms in flight 0/2/4/8, product-sum
 * form of a GEMM-shaped step 0/1 (only where no tensor of the step keeps its
 * batch entry outermost); a parameter that does not apply to the step is
 * ignored), e.g. to reuse a tuning saved
 * from an earlier bind without timing again.  After qgm_plan_bind (which
 * resets them); the next call re-captures its pass.  QGM_ERR_ARG on a bad
 * record (nothing changed). */
int qgm_plan_set_tuning(qgm_plan *p, const int32_t *rec, int64_t n);

/* Shapes of the GEMM-shaped steps (Sec. IV, Eq. par_sum with two large
 * operands sharing every summed variable): for the c-th such step, c < cap,
 * rec[12c .. 12c+11] = step index, nm, nn, nk, ns (variables private to A, to
 * B, summed, shared and kept), A batched, B batched, output batched, 1 when
 * the step runs on the tensor cores, 1 when its output is stored with the
 * batch entry outermost, 1 when an operand is (both for tensor-core steps
 * only: a product per batch entry read by another tensor-core step), and 1
 * when the tensor-core step folds its batch entries into M, so that the
 * product kernel can convert its batched operand itself
 * (qgm_plan_opts.tc_convert).  *n = the number of GEMM steps; rec may be
 * NULL to query it.  Host only. */
int qgm_plan_get_gemm(const qgm_plan *p, int32_t *rec, int64_t cap, int64_t *n);
void qgm_plan_free(qgm_plan *p);

/* ------------------------------------------------------------- execution */

/* Binds a caller-owned device workspace of at least info.workspace_bytes
 * (256-byte aligned) to the plan and uploads the plan's constant tables into
 * it on `stream`.  The caller keeps the workspace alive and untouched while
 * it is bound; binding again (or to another buffer) replaces the binding.
 * Errors: QGM_ERR_OOM if ws_bytes is too small, QGM_ERR_CUDA, QGM_ERR_NOGPU. */
int qgm_plan_bind(qgm_plan *p, void *d_workspace, size_t ws_bytes, void *stream);

/* Amplitudes of B <= opts.batch bitstrings (Sec. III-IV; App. A):
 * d_bitstrings: device uint64[B]; d_out: device double[2B] (re, im) written
 * with <x_b|C|0^n> for b < B.  With k = popcount(opts.open_mask) > 0, d_out
 * holds B * 2^k amplitudes: entry b * 2^k + c is x_b with its open qubits
 * set from c (bit i of c = the i-th lowest open qubit).  Runs every step of the plan, all slices, on
 * `stream` (asynchronous; the first call with a given pointer set also
 * builds a CUDA graph).  Requires QGM_OUT_BATCH and a bound workspace.
 * Errors: QGM_ERR_ARG (mode, B, unbound), QGM_ERR_CUDA. */
int qgm_amplitudes(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out,
                   void *stream);

/* The same with HOST bitstrings and a HOST result: copies in, runs, copies
 * out and synchronises `stream`.  Uses the bound workspace for staging; with
 * the resident executors and page-locked buffers the device can address
 * (cudaHostAlloc, cudaHostRegister), the kernel reads and writes them in
 * place instead. */
int qgm_amplitudes_host(qgm_plan *p, const uint64_t *h_bitstrings, int64_t B,
                        double *h_out, void *stream);

/* All 2^n amplitudes of a QGM_OUT_OPEN plan into device double[2 * 2^n]
 * (entry x has bit j = qubit j): Eq. psi_x with the output deltas omitted. */
int qgm_eliminate(qgm_plan *p, double *d_out, void *stream);

/* One contraction for a fixed output assignment (Eq. psi_x with the output
 * deltas fixed to fixed_assign[q], host uint8 of n_qubits values 0/1, qubit q
 * at index q): the final tensor as the elimination leaves it, before its
 * power-of-two exponent is applied.  d_out (device double[2 * 2^k], k =
 * popcount(open_mask) + n_keep) receives c * F[r], c the plan's constant
 * (scope-free factors, 2^{-1/2} per fixed gate pulled out), and *exp_out
 * (host) the exponent e: the value is d_out[r] * 2^e, which stays finite
 * where the product itself would leave FP64's range.  With kept variables
 * (qgm_plan_opts.keep_vars) it returns an intermediate table of App. A's
 * elimination, e.g. App. D's tau_2.  Runs the stepwise kernels whatever the
 * bound executor (the final tensor must be in the workspace); a sliced plan
 * returns the FP64 sum of its slices with *exp_out = 0.  Synchronises.
 * Errors: QGM_ERR_ARG (plan kind, values), QGM_ERR_CUDA. */
int qgm_eliminate_fixed(qgm_plan *p, const uint8_t *fixed_assign, double *d_out, int64_t *exp_out,
                        void *stream);

/* Report of one qgm_amplitudes call: the device status word (read and
 * cleared), the executor, milliseconds (CUDA events on the stream around
 * the call), the slices, the algorithmic bytes and flops of the plan's steps
 * over all slices (qgm_plan_info) and the kernel launches issued. */
typedef struct {
  int32_t status;
  int32_t executor;
  float ms;
  double bytes;
  double flops;
  int64_t slices;
  int64_t launches;
} qgm_report;

/* qgm_amplitudes with a report (synchronises `stream`); returns the device
 * status as an error when it is not QGM_OK. */
int qgm_amplitudes_report(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out, qgm_report *rep,
                          void *stream);

/* Timing pass for reports:/* Timing pass for reports: runs slice 0 of qgm_amplitudes kernel by kernel
 * (no graph) with CUDA events around each launch on `stream` and stores the
 * milliseconds in ms[0] (leaf build), ms[1 + s] (step s), ms[n_steps + 1]
 * (accumulation); ms must hold n_steps + 2 floats (host).  Synchronises. */
int qgm_plan_profile(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out,
                     float *ms, void *stream);

/* Per GEMM-shaped step (in step order, as qgm_plan_get_gemm lists them) of
 * slice 0 of a stepwise plan: milliseconds of the operand split into 16-bit
 * planes in ms_split[c] (0 for a step on the FP32 cores) and of the product
 * kernel in ms_product[c] (CUDA events on `stream` around each launch;
 * host float arrays of the number of GEMM steps).  Synchronises.  Errors:
 * QGM_ERR_ARG (not stepwise, bad sizes), QGM_ERR_CUDA. */
int qgm_plan_profile_gemm(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out,
                          float *ms_split, float *ms_product, void *stream);

/* Per step s of the last slice run on the bound workspace: the recorded
 * maximum of its output (float bits of max(|re|, |im|) of the scaled values,
 * maxbits[s]) and the output's power-of-two exponent (exps[s]); host arrays
 * of n_steps.  For tests and reports of the rescaling (A7).  Synchronises. */
int qgm_plan_step_stats(qgm_plan *p, uint32_t *maxbits, int32_t *exps, int64_t cap, void *stream);

/* Measurement utility (no counterpart in the paper): FP32 FMA throughput of
 * the current device in TFLOP/s (2 flops per FMA), from independent FMA
 * chains on every SM timed with CUDA events on `stream`; the peak against
 * which kernels bound by FP32 arithmetic are reported.  Synchronises. */
int qgm_measure_fp32_peak(double *tflops, void *stream);

/* Failure-detection self-test (no counterpart in the paper): runs the
 * bounded mbarrier wait every tensor-core kernel uses, on one barrier with an
 * arrival count of 1.  arrive = 0: nothing arrives, the wait gives up after
 * limit_ns (1 us .. 2 s, else QGM_ERR_ARG) and *status_out = QGM_ERR_TIMEOUT;
 * arrive = 1: the waiting thread arrives first and *status_out = QGM_OK.  The
 * context stays usable either way.  Host int32 out; synchronises. */
int qgm_selftest_wait_timeout(int64_t limit_ns, int32_t arrive, int32_t *status_out, void *stream);

/* Executor chosen at bind time:/* Executor chosen at bind time: *kind (QGM_EXEC_STEPWISE, _RESIDENT or
 * _COMPILED), the bitstrings per CTA *chunk and the dynamic shared memory per
 * CTA (resident and compiled). */
int qgm_plan_get_executor(const qgm_plan *p, int32_t *kind, int32_t *chunk, int64_t *smem_bytes);

/* CUDA source of the compiled resident kernel (QGM_EXEC_COMPILED) for this
 * plan, as qgm_plan_bind compiles it; needs no GPU.  chunk: bitstrings per
 * CTA of the layout (1, 2, 4 or 8); part: 0 the whole pass, 1 its batched
 * part, 2 its bitstring-independent part (the split used for batches of two
 * or more waves); min_blocks: CTAs per SM for the launch bounds (0: as many
 * as 228 KB of shared memory per SM hold, at most 8).  Copies up to cap - 1
 * bytes and a NUL into buf (may be NULL) and the full length into *len.
 * Errors: QGM_ERR_ARG (no such layout, bad part). */
int qgm_plan_kernel_source(const qgm_plan *p, int32_t chunk, int32_t part, int32_t min_blocks, char *buf,
                           int64_t cap, int64_t *len);

/* No counterpart in the paper: an allocation-free variant of qgm_amplitudes
 * for callers that cannot allocate device memory when they need amplitudes
 * (a framework whose pool allocator owns all device memory, or a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the
 * device).  Runs the plan with the stepwise kernels, their scratch being one
 * static device array of QGM_STATIC_SCRATCH_BYTES that every GPU loading this
 * library holds until exit; no qgm_plan_bind is needed and nothing is
 * allocated.  GEMM-shaped steps run on the FP32 cores here (the tensor-core
 * kernel's shared-memory limit is raised at bind).  d_bitstrings: device
 * uint64[B]; d_out: device double[2 * B * 2^k] with k = popcount(open_mask)
 * (entry b * 2^k + c as in qgm_amplitudes; k = 0 gives double[2B]).
 * The first call on a device (that device current) looks the array's device
 * address up with cudaGetSymbolAddress; make that first call before any
 * stream capture.  Calls share the array: each reloads the plan's tables and
 * clears what must start at zero, and calls that overlap on the GPU race.
 * Errors: QGM_ERR_OOM when the plan's workspace_bytes exceeds
 * QGM_STATIC_SCRATCH_BYTES (bind a workspace instead), QGM_ERR_ARG, QGM_ERR_CUDA. */
#define QGM_STATIC_SCRATCH_BYTES (64ull << 20)
int qgm_amplitudes_static(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out,
                          void *stream);

/* Cross-entropy benchmarking statistics (App. B) of B amplitudes a_b (device
 * double[2B], e.g. qgm_amplitudes' output): with p = |a|^2 and N = 2^n,
 * cross_entropy = -(1/B) sum log p (Eq. cee), alpha = (H0 - S)/(H0 - H) with
 * the Porter-Thomas H0 = log N + gamma, H = log N - 1 + gamma (Eq. ae),
 * mean_Np and second_moment = mean (N p)^2.  Sums are FP64 on the device
 * (d_scratch: caller-owned device double[4]); synchronises `stream`. */
typedef struct {
  double cross_entropy, alpha, mean_Np, second_moment;
} qgm_xeb_result;
int qgm_xeb_stats(const double *d_amps, int64_t B, int n_qubits, double *d_scratch,
                  qgm_xeb_result *out, void *stream);

/* Sampling from a computed set (App. C): m indices into the t amplitudes of
 * d_amps (device double[2t]) drawn with probability p_j / sum p, by inverse
 * transform of u_i = (SplitMix64(seed) draw i) >> 11 * 2^-53.  d_scratch:
 * caller-owned device double[t] (cumulative sums); d_idx: device int64[m]. */
int qgm_sample_from_set(const double *d_amps, int64_t t, int64_t m, uint64_t seed, double *d_scratch,
                        int64_t *d_idx, void *stream);

/* Reads and clears the device status word of the bound workspace
 * (synchronises `stream`): QGM_OK, QGM_ERR_NONFINITE or QGM_ERR_TIMEOUT. */
int qgm_status(qgm_plan *p, void *stream);

/* New angles for the parametrised gates of the plan's circuit (RXY, Sec.
 * "Numerical results" gate set extended by exp(-i theta (cos phi X + sin
 * phi Y) / 2)): params[2p] = theta_p, params[2p+1] = phi_p in the order of
 * qgm_circuit_param_gates, n = 2 * number of RXY gates.  The gate tables, the
 * merged leaf tables (and their derivative tables) and the constant are
 * recomputed on the host and, when a workspace is bound, copied into it on
 * `stream` (synchronised); the order, steps and layout are unchanged, so no
 * re-planning happens.  Later qgm_amplitudes / qgm_amplitude_grad calls use
 * the new angles.  Errors: QGM_ERR_ARG (count, structure), QGM_ERR_CUDA. */
int qgm_plan_set_params(qgm_plan *p, const double *params, int64_t n, void *stream);

/* Gradient (adjoint elimination) for a parametrised circuit.  The forward
 * elimination keeps every intermediate; the backward pass runs the steps in
 * reverse, each step of Eq. par_sum giving the adjoint of each input as the
 * product of the output's adjoint with the other inputs, summed over the
 * variables the input does not hold (bucket elimination is a tree, so every
 * tensor has exactly one consumer).  Needs a plan made with opts.gradients = 1.
 * A sliced plan (opts.mem_budget_bytes) recomputes, slice by slice, the
 * forward intermediates of that slice before its adjoint pass and adds each
 * slice's share of the gradient (a = sum_s a_s), so the live set stays that
 * of one slice.  Given
 * g_b = dL/d(conj a_b) for the B bitstrings (device double[2B]), writes
 * d_grad[i] = dL/dp_i = 2 Re sum_b conj(g_b) da_b/dp_i for the n_params
 * parameters (theta, phi of each RXY gate, see qgm_circuit_param_gates) into
 * device double[n_params], and the amplitudes into d_amp (device double[2B],
 * may be NULL).  Requires QGM_OUT_BATCH.  Asynchronous on `stream`; the
 * first call with a given set of pointers and B builds a CUDA graph of the
 * pass, later calls launch it.  Errors as qgm_amplitudes. */
int qgm_amplitude_grad(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B,
                       const double *d_dL_dconja, double *d_grad, double *d_amp,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QGM_H */
