/*
 * ajf.h -- C ABI of libajf: approximate equivalence checking of noisy quantum circuits by the
 * Jamiolkowski fidelity, computed on one GB300 (sm_103a) by contracting closed miter tensor
 * networks.
 *
 * The quantity (Sec. III, "Ease of calculation"): for an ideal circuit U on n qubits and a noisy
 * implementation E = {E_i} (a super-operator in Kraus form, Sec. II-B),
 *
 *     F_J(E, U) = (1/d^2) * sum_i |tr(U^dagger E_i)|^2,      d = 2^n.
 *
 * Problem 1 / Definition 1 (Sec. III): the two circuits are eps-equivalent iff F_J > 1 - eps.
 *
 * Two algorithms (Sec. IV):
 *   Alg. I  (Sec. IV-A): one single-layer miter U^dagger . E_i per Kraus combination; the
 *           library contracts all prod_k n_k combinations at once by giving every noise tensor
 *           an open Kraus index, so the result is the whole tensor t[j_1..j_m] of traces.
 *   Alg. II (Sec. IV-B): one doubled miter (U^dagger (x) U^T) . M_E with
 *           M_E built from V (x) V^* per gate and M_N = sum_k N_k (x) N_k^* per noisy gate;
 *           its value is sum_i |tr(U^dagger E_i)|^2 directly.
 *
 * Conventions shared by every call:
 *   - Matrices are complex128, interleaved (re, im), row-major, 2^a x 2^a for an a-qubit gate.
 *   - Qubit 0 is the most significant tensor factor of the circuit; within a gate matrix the
 *     first listed qubit is the most significant factor of the gate.
 *   - Gates apply in list order (the first gate acts first).
 *   - The caller owns every array it passes; the library copies what it needs before returning.
 *   - Every call returns an ajf_status; AJF_OK is 0. The library never aborts the process; the
 *     text of the last error is available from ajf_last_error.
 *   - A context is not thread-safe; different contexts may be used from different threads.
 *   - All device work is enqueued on the context's stream.
 */
#ifndef AJF_H
#define AJF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ajf_status;

enum {
  AJF_OK = 0,
  AJF_E_ARG = 1,         /* bad pointer, index, arity, size or option                         */
  AJF_E_NOT_UNITARY = 2, /* a gate is not unitary: ||G^dagger G - I||_F > 1e-10               */
  AJF_E_NOT_TP = 3,      /* a Kraus set is not trace preserving: ||sum K^dagger K - I||_F > 1e-10 */
  AJF_E_STATE = 4,       /* calls in the wrong order (e.g. a fidelity call before ajf_plan)    */
  AJF_E_BUDGET = 5,      /* the planned contraction does not fit the memory budget             */
  AJF_E_NOMEM = 6,       /* device or host allocation failed, or the workspace is too small    */
  AJF_E_CUDA = 7,        /* a CUDA runtime error; the message names the call                   */
  AJF_E_TIMEOUT = 8,     /* a bounded device-side wait expired                                 */
  AJF_E_UNSUPPORTED = 9  /* the request is valid but not supported on this device/build        */
};

enum { AJF_IDEAL = 0, AJF_IMPL = 1 };

enum {
  AJF_PLANNER_AUTO = 0,    /* best of greedy and min-fill by estimated time                     */
  AJF_PLANNER_GREEDY = 1,  /* randomised greedy pair selection (memory-removed cost)           */
  AJF_PLANNER_MINFILL = 2, /* min-fill elimination = tree decomposition of the line graph (Sec. IV-C) */
  AJF_PLANNER_LEARNED = 3  /* MLP merge scorer; the greedy planner is its fallback and judge     */
};

enum {
  AJF_PREC_F64 = 0,    /* FP64 arithmetic everywhere                                           */
  AJF_PREC_F32 = 1,    /* GEMM-class steps on FP32 CUDA cores (operands rounded to FP32)       */
  AJF_PREC_TF32 = 2,   /* GEMM-class steps: one-pass TF32 tensor-core GEMMs (tcgen05), FP32 accumulate */
  AJF_PREC_TF32X3 = 3, /* split TF32 hi/lo operands, three tcgen05 products, FP32 accumulate   */
  AJF_PREC_BF16X3 = 4, /* bf16 operands split in two terms, three tcgen05 products             */
  AJF_PREC_BF16X6 = 5, /* bf16 operands split in three terms, six tcgen05 products             */
  AJF_PREC_F16X3 = 6   /* fp16 operands in two terms scaled by a power of two per row and K block,
                          three tcgen05 products (the scale undone per K block in the epilogue) */
};
/* Tensors are planar complex in device memory: complex128 (FP64 planes), except the results of
 * the reduced modes' GEMM-class steps, which are complex64 (FP32 planes; each value is one FP32
 * register sum of the GEMM, so nothing is lost). A mode sets how the operands of the GEMM-class
 * steps are rounded or split. Leaves, small steps, the final contraction to a scalar,
 * sum_i |t_i|^2, F_J and 1 - F_J are FP64 in every mode. */

enum {
  AJF_LOWER_DEFAULT = 0,   /* GEMM-class steps on tensor cores / CUDA-core GEMMs, one launch per
                              level of small steps                                              */
  AJF_LOWER_PERSISTENT = 1 /* every step a CUDA-core gather or reduction step in FP64, so that one
                              thread block of the persistent kernel runs the whole network
                              (ajf_launch_persistent); meant for small networks                */
};

/* Simplifications of the closed composed sequence (implementation, then the ideal circuit's
 * adjoint, wires joined) before the network is built (Sec. IV-C; the paper's experiments run
 * without them). Flags for ajf_plan_opts.simplify; F_J is unchanged up to rounding.
 *   AJF_SIMPLIFY_SWAP: "SWAP elimination" -- every SWAP gate is dropped and the later elements are
 *     rewired, the closure joining each output wire to the input wire the SWAPs lead it to.
 *   AJF_SIMPLIFY_CANCEL: "local optimisations" -- adjacent unitary elements on the same ordered
 *     wires whose product is the identity are removed (also across the closed trace, "both ends"),
 *     as are elements equal to the identity; noises are never removed and block cancellation on
 *     their wires. Matrices count as the identity / SWAP within 1e-12 per entry.
 * The simplification depends on the gate matrices, not only the structure: a re-plan with new
 * values keeps its cached path only when the simplified sequence is the same. */
enum { AJF_SIMPLIFY_SWAP = 1, AJF_SIMPLIFY_CANCEL = 2 };

typedef struct ajf_ctx ajf_ctx;

typedef struct ajf_plan_opts {
  int32_t planner;         /* AJF_PLANNER_*                                                   */
  int32_t precision;       /* AJF_PREC_*                                                      */
  int32_t trials;          /* randomised restarts per planner; 0 = library default (32)       */
  int32_t use_graph;       /* 1: capture the device program in a CUDA graph on first run       */
  uint64_t seed;           /* planner random seed                                             */
  double mem_budget_bytes; /* 0 = 60% of the device's free memory at plan time                 */
  int32_t lowering;        /* AJF_LOWER_*; AJF_LOWER_PERSISTENT requires AJF_PREC_F64          */
  int32_t simplify;        /* AJF_SIMPLIFY_* flags; 0 = the sequence as given                  */
  int32_t alg1_slices;     /* Alg. I only: fix the Kraus index of this many noises per slice   */
                           /* (0 = none; see ajf_fidelity_alg1 for the early exit it enables)  */
  int32_t slice_bonds;     /* bond slicing: 0 = none; s > 0 = slice s closed labels; AJF_SLICE_AUTO */
                           /* = the fewest that bring the arena within mem_budget_bytes        */
  int32_t reserved[4];     /* must be zero                                                     */
} ajf_plan_opts;

/* opts.slice_bonds = AJF_SLICE_AUTO: slice only as far as the memory budget needs. */
enum { AJF_SLICE_AUTO = -1 };
/* At most this many sliced labels (2^24 contractions of the sliced network per evaluation). */
enum { AJF_MAX_SLICE_BONDS = 24 };

typedef struct ajf_plan_info {
  double cmacs;          /* sum over pairwise steps of M*N*K complex multiply-adds             */
  double flops;          /* 8 * cmacs (one complex multiply-add = 8 real flops)                */
  double bytes;          /* algorithmic bytes: sum over steps of (|A|+|B|+|C|) * element size   */
  double gemm_flops;     /* the part of `flops` done by the GEMM-class steps                    */
  double gemm_bytes;     /* the part of `bytes` moved by the GEMM-class steps                   */
  double arena_bytes;    /* device memory the plan needs (intermediates + scratch + inputs)     */
  double plan_seconds;   /* host time spent planning                                            */
  int32_t width;         /* log2 of the element count of the largest tensor                     */
  int32_t n_steps;       /* pairwise contraction steps                                          */
  int32_t n_gemm_steps;  /* steps lowered to permute + GEMM                                     */
  int32_t n_leaves;      /* tensors of the network before contraction                           */
  int32_t n_open_bits;   /* Alg. I: bits of the open Kraus-index result tensor; Alg. II: 0       */
  int32_t planner_used;  /* AJF_PLANNER_* that produced the chosen path                          */
  int32_t n_launches;    /* kernel launches one evaluation enqueues                              */
  int32_t n_tc_gemms;    /* GEMM launches that run on the tcgen05 tensor cores                   */
  int32_t plan_cached;   /* 1: the path was reused from the previous plan of the same structure  */
  int32_t n_removed;     /* gates removed by opts.simplify (SWAPs, cancelled pairs, identities)  */
  double upload_bytes;   /* host -> device bytes of one upload (descriptors + packed inputs)     */
  int32_t n_sliced_bonds; /* labels sliced (opts.slice_bonds): the evaluation runs 2^n_sliced_bonds */
                          /* contractions; cmacs, flops, bytes, gemm_* count all of them, width   */
                          /* and arena_bytes describe one                                          */
  int32_t reserved;
} ajf_plan_info;

/* Per-kernel-class timing collected while profiling is on (CUDA events around every launch on
 * the context's stream). Classes: 0 leaves, 1 small steps, 2 split-K, 3 operand gather,
 * 4 CUDA-core GEMM, 5 tensor-core GEMM, 6 final FP64 reduction. */
typedef struct ajf_kernel_stats {
  int64_t launches;    /* launches recorded                                                  */
  double ms;           /* summed device time (ms)                                            */
  double flops;        /* algorithmic flops of the complex steps these launches carried out  */
  double bytes;        /* algorithmic bytes of those steps                                   */
} ajf_kernel_stats;

typedef struct ajf_result {
  double F;            /* F_J(E, U)                                                          */
  double one_minus_F;  /* 1 - F_J, computed as (d^2 - S) / d^2 in FP64                         */
  double S;            /* sum_i |tr(U^dagger E_i)|^2                                            */
  int64_t traces_done; /* Alg. I: Kraus combinations evaluated; Alg. II: 0                      */
  int32_t equivalent;  /* eps < 0: -1; else 1 if F_J > 1 - eps (Definition 1), otherwise 0      */
  int32_t reserved;
} ajf_result;

/* Create a context on CUDA device `device` (device = -1: a host-only context that validates and
 * plans but cannot run; useful without a GPU). `cuda_stream` is a cudaStream_t that the library
 * borrows (never destroys); NULL makes the library create and own a non-blocking stream.
 * A device context also looks up the fixed 64 MiB arena of ajf_fidelity_noalloc, which makes the
 * device reserve it (once per process and device) if it has not already.
 * Errors: AJF_E_ARG (out == NULL), AJF_E_CUDA (bad device, or the fixed arena cannot be
 * reserved). */
ajf_status ajf_create(ajf_ctx **out, int device, void *cuda_stream);

/* Release everything the context owns (device memory it allocated, graphs, its own stream).
 * Borrowed workspace and streams are left alone. NULL is ignored. */
void ajf_destroy(ajf_ctx *ctx);

/* Text of the last error on this context ("" if none). Owned by the context. */
const char *ajf_last_error(const ajf_ctx *ctx);

/* Load a circuit (Sec. II-A: a sequence of gates on n qubits). role = AJF_IDEAL sets U;
 * role = AJF_IMPL sets the unitary skeleton of the noisy implementation (Fig. 2: the noisy
 * circuit's gates with the noisy gates taken out); without an AJF_IMPL load the skeleton is U.
 * arity[g] in {1, 2, 3}; qubits holds sum(arity) indices in [0, n); mats holds the gate matrices
 * one after another (complex128 interleaved, 2^a x 2^a each, row-major). Loading U clears the
 * noises and any previous skeleton; loading either invalidates the plan.
 * Errors: AJF_E_ARG (n_qubits not in [1, 62], bad arity/qubit/repeated qubit), AJF_E_NOT_UNITARY. */
ajf_status ajf_load_circuit(ajf_ctx *ctx, int role, int n_qubits, int n_gates,
                            const int32_t *arity, const int32_t *qubits, const double *mats);

/* Add a noisy gate N = {N_k} (Sec. II-B Kraus form; Example 2 lists the canonical ones) acting
 * right after skeleton gate `after_gate` (-1: before the first gate). Noises added after the same
 * gate act in the order added; Alg. I enumerates Kraus combinations with the last-added noise
 * varying fastest. kraus holds n_kraus matrices of 2^a x 2^a (complex128 interleaved, row-major).
 * Errors: AJF_E_STATE (no circuit loaded), AJF_E_ARG (bad index/arity/count, n_kraus > 256),
 * AJF_E_NOT_TP. */
ajf_status ajf_add_noise(ajf_ctx *ctx, int32_t after_gate, int32_t arity, const int32_t *qubits,
                         int32_t n_kraus, const double *kraus);

/* Remove every noise (keeps the circuits). Invalidates the plan. */
ajf_status ajf_clear_noise(ajf_ctx *ctx);

/* Build the network of algorithm `alg` (1: Alg. I with open Kraus indices, Sec. IV-A;
 * 2: Alg. II doubled network, Sec. IV-B; 0 = AJF_ALG_AUTO: plan both and keep the one whose
 * estimated run time is lower -- Sec. IV-B and V note that Alg. I wins when noises are few and
 * Alg. II when they are many; ajf_planned_alg tells which), choose a pairwise contraction
 * order, lower it to device kernels and size the device arena. opts may be NULL (defaults: AUTO
 * planner, AJF_PREC_F64, 32 trials, no graph). info may be NULL.
 * opts.alg1_slices = s > 0 (Alg. I, and Alg. I under AJF_ALG_AUTO): the s noises with the most
 * Kraus operators (earlier noise first on ties) get a fixed Kraus index; the network keeps the
 * open indices of the others, and ajf_fidelity_alg1 runs it once per combination of the fixed
 * indices. s must not exceed the number of noises; not with AJF_LOWER_PERSISTENT.
 * opts.slice_bonds (bond slicing; the paper contracts each network whole, Sec. IV-C, and has
 * no counterpart): a closed label b of the network is fixed to 0 in one contraction and to 1 in
 * another, in both tensors that carry it, and the two results are added. This is the same sum
 * over label values that the full contraction is, so the result is unchanged, while every tensor
 * carrying b is half the size. s labels give 2^s contractions of a network whose widest tensor
 * is up to 2^s times smaller: plans over the memory budget become runnable at the price of work.
 * The labels are chosen greedily on the planned path (those carried by the most of its widest
 * tensors first; Alg. I's open Kraus indices are never sliced, and no leaf loses its last
 * label), and the same path runs on the sliced network. s > 0 slices s labels (fewer when no
 * more can be sliced; info->n_sliced_bonds tells); AJF_SLICE_AUTO slices none when the plan fits the
 * budget, else the fewest that make it fit, and reports AJF_E_BUDGET beyond
 * AJF_MAX_SLICE_BONDS. Not with opts.alg1_slices or AJF_LOWER_PERSISTENT. Alg. II adds the
 * slices' scalars, Alg. I the slices' traces (complex, FP64, before |t|^2 is formed), both on the
 * host in FP64; eps decides only after every slice (no early exit).
 * Errors: AJF_E_STATE (no circuit), AJF_E_ARG (bad alg/option), AJF_E_BUDGET (the best plan's
 * arena exceeds the budget; info is still filled), AJF_E_UNSUPPORTED (tensor-core precision on
 * a device without tcgen05). */
ajf_status ajf_plan(ajf_ctx *ctx, int alg, const ajf_plan_opts *opts, ajf_plan_info *info);

enum { AJF_ALG_AUTO = 0 };

/* The algorithm (1 or 2) of the current plan. Errors: AJF_E_ARG, AJF_E_STATE (no plan). */
ajf_status ajf_planned_alg(const ajf_ctx *ctx, int *alg);

/* Run the planned algorithm: ajf_fidelity_alg1 or ajf_fidelity_alg2, whichever ajf_plan chose. */
ajf_status ajf_fidelity(ajf_ctx *ctx, double eps, ajf_result *out);

/* Lend the context `bytes` of device memory at `dev_ptr` (256-byte aligned) for its arena.
 * The caller keeps ownership and must keep it alive until ajf_destroy or the next
 * ajf_set_workspace. NULL returns to library-allocated memory.
 * Errors: AJF_E_ARG (misaligned pointer). AJF_E_NOMEM is reported at run time if it is too small. */
ajf_status ajf_set_workspace(ajf_ctx *ctx, void *dev_ptr, size_t bytes);

/* Device bytes the current plan needs (valid after ajf_plan). */
ajf_status ajf_workspace_size(const ajf_ctx *ctx, size_t *bytes);

/* Alg. I (Sec. IV-A): F_J from all prod_k n_k traces tr(U^dagger E_i), accumulated as
 * sum |t|^2 in FP64 on the device. eps < 0: no decision (equivalent = -1); eps in [0, 1]: also
 * decide Definition 1. Requires ajf_plan(ctx, 1, ...). Synchronises the context's stream.
 * Sliced plans (opts.alg1_slices > 0) run one contraction per combination of the fixed Kraus
 * indices, in decreasing order of weight prod ||K||_F^2 / 2^a, and add the slices' sums in FP64
 * on the host. With eps >= 0 they stop early once the partial F_J exceeds 1 - eps (the remark
 * after Alg. I: every term is non-negative, so the partial sum already decides equivalence):
 * then F, S and 1 - F describe the traces done (F is a lower bound of F_J), traces_done counts
 * them, equivalent = 1, and ajf_alg1_traces reports AJF_E_STATE.
 * Errors: AJF_E_STATE, AJF_E_ARG (eps > 1), AJF_E_NOMEM, AJF_E_CUDA. */
ajf_status ajf_fidelity_alg1(ajf_ctx *ctx, double eps, ajf_result *out);

/* Progress of a sliced Alg. I evaluation (checkpoint / resume; no paper counterpart). For Alg. I
 * over very many Kraus combinations the work can be split over calls, processes or machines:
 * the state is the next slice (in the plan's order, heaviest first) and the partial sum. */
typedef struct ajf_alg1_state {
  int64_t next_slice;  /* slices done                                                          */
  int64_t n_slices;    /* slices of the plan: prod of n_k over the fixed noises               */
  double S;            /* sum |t_i|^2 over the traces of the slices done (FP64)                */
  int64_t traces_done; /* traces of the slices done                                            */
  uint64_t plan_sig;   /* the plan's structure, slicing, precision and input values (hash)     */
} ajf_alg1_state;

/* Run up to max_slices more slices (max_slices <= 0: all that remain) of a sliced Alg. I plan,
 * from where the context stopped (the first call after ajf_plan starts at slice 0). eps >= 0
 * stops as soon as the partial F exceeds 1 - eps. out describes the slices done so far: F is a
 * lower bound of F_J until n_slices are done; equivalent = 1 once the partial F exceeds 1 - eps,
 * 0 once every slice is done and it does not, -1 while undecided (or eps < 0).
 * Errors: AJF_E_STATE (no sliced Alg. I plan, host-only context), AJF_E_ARG, AJF_E_CUDA. */
ajf_status ajf_alg1_continue(ajf_ctx *ctx, double eps, int64_t max_slices, ajf_result *out);

/* Copy the progress of the context's sliced Alg. I evaluation into *state (host only).
 * Errors: AJF_E_ARG, AJF_E_STATE (no sliced Alg. I plan). */
ajf_status ajf_alg1_checkpoint(const ajf_ctx *ctx, ajf_alg1_state *state);

/* Resume from a checkpoint: the context must hold the same sliced Alg. I plan of the same input
 * values (plan_sig). The next ajf_alg1_continue starts at state->next_slice with the partial
 * sum. The traces of the slices done before the checkpoint are not part of it, so
 * ajf_alg1_traces reports AJF_E_STATE after a resumed evaluation (F, S and 1 - F are complete).
 * Errors: AJF_E_ARG (NULL, another plan or other values, fields out of range), AJF_E_STATE. */
ajf_status ajf_alg1_restore(ajf_ctx *ctx, const ajf_alg1_state *state);

/* Host-side replay of the current plan's device program (no device needed; the paper has no
 * counterpart). It stands in for a device memory checker, which this library cannot rely on.
 * Every address a kernel of the program can form is a base plus distinct powers of two taken
 * from the step's index maps (which must address every bit of their operand, or elements would
 * be skipped): leaves, pairwise steps, operand gathers, GEMM operands, results,
 * K-split workspaces, partial sums, scalar slots and the final pass. The check makes sure that
 * each such address lies inside its buffer and the arena region that holds it. Replaying the
 * launches in stream order (each GEMM's shape must be that of the two gathers feeding it), it
 * also makes sure that:
 *   - every buffer read was written by an earlier launch;
 *   - no launch writes over a buffer that it, or a later launch, still reads;
 *   - no two writes of one launch overlap.
 * Errors: AJF_E_ARG (NULL), AJF_E_STATE (no plan, or a violation: the first is in
 * ajf_last_error). */
ajf_status ajf_check_plan(ajf_ctx *ctx);

/* Self-test of ajf_check_plan (tests only; no paper counterpart): plant one mistake in a copy of
 * the current plan's program and check it. mutation 1: a leaf past the end of the work region;
 * 2: an index-map position beyond its operand's bits; 3: a step writing over its own input;
 * 4: a step reading memory that no launch wrote; 5: two leaves in the same place; 6: a step of
 * the first launch writing over a leaf that a later launch still reads (3, 5 and 6 move their
 * buffer's readers along, so that only the overlap is wrong); 7: an operand bit that no index
 * map addresses (elements that would be skipped); 8: a GEMM whose K differs from its gathers'.
 * The context's
 * own program is not changed. Returns AJF_OK when the check reports the mistake (its message is
 * in ajf_last_error), AJF_E_STATE when it does not, AJF_E_ARG for an unknown mutation or a plan
 * without the needed step. */
ajf_status ajf_selftest_check_plan(ajf_ctx *ctx, int mutation);

/* Independent runs of one evaluation of the current plan (Sec. IV-A remarks that the traces are
 * independent; bond slices have no paper counterpart): the Kraus-index slices of a sliced
 * Alg. I plan (opts.alg1_slices), 2^n_sliced_bonds for a bond-sliced plan (opts.slice_bonds),
 * otherwise 1. These are the units for sharding one evaluation across devices or processes.
 * Errors: AJF_E_ARG (NULL), AJF_E_STATE (no plan). */
ajf_status ajf_slice_count(const ajf_ctx *ctx, int64_t *n);

/* Sharding one Alg. II evaluation (the paper has no counterpart; Sec. IV-B contracts the doubled
 * network whole). Runs the bond slices [first, first + count) of the context's Alg. II plan
 * (a plan without bond slicing has the one slice 0) and writes the sum of their scalars to
 * *S_part, in FP64. The slices partition the contraction's sum over label values, so S_part over
 * ranges that partition [0, ajf_slice_count) adds up to S, and F_J = S / 4^n: one FP64
 * all-reduce of S_part across devices or processes completes the evaluation. count = 0 gives
 * S_part = 0 without running anything. Synchronises the context's stream.
 * Errors: AJF_E_ARG (NULL, range outside [0, ajf_slice_count)), AJF_E_STATE (no Alg. II plan,
 * host-only context), AJF_E_NOMEM, AJF_E_CUDA, AJF_E_TIMEOUT. */
ajf_status ajf_alg2_slice_range(ajf_ctx *ctx, int64_t first, int64_t count, double *S_part);

/* The units that one evaluation of the current plan shards into, and how a rank runs a block of
 * them (the paper has no counterpart; Sec. IV-A notes the independence of Alg. I's traces):
 *   AJF_UNITS_KRAUS_SLICES: the Kraus-index slices of a sliced Alg. I plan (opts.alg1_slices); a
 *     block runs through ajf_alg1_restore (next_slice = first, S = 0) and ajf_alg1_continue, and
 *     its S is that block's sum of |t_i|^2;
 *   AJF_UNITS_BOND_SLICES: the 2^n_sliced_bonds bond slices of an Alg. II plan (1 when unsliced);
 *     a block runs through ajf_alg2_slice_range;
 *   AJF_UNITS_WHOLE: one unit, the whole evaluation (an Alg. I plan without Kraus slicing, bond
 *     sliced or not: its per-trace sums of slices are not additive in S, so it does not shard);
 *     the rank that holds it runs ajf_fidelity.
 * *kind and *n_units are written; every rank holding the same plan gets the same answer, so the
 * ranks agree on the split without communicating. Errors: AJF_E_ARG (NULL), AJF_E_STATE (no plan). */
enum { AJF_UNITS_WHOLE = 0, AJF_UNITS_KRAUS_SLICES = 1, AJF_UNITS_BOND_SLICES = 2 };
ajf_status ajf_shard_units(const ajf_ctx *ctx, int32_t *kind, int64_t *n_units);

/* Completes an evaluation from its sum S = sum_i |tr(U^dagger E_i)|^2 (Sec. III, "Ease of
 * calculation": F_J = S / d^2 with d = 2^n_qubits), e.g. after an all-reduce of the ranks' partial
 * sums: F = S / 4^n and 1 - F = (4^n - S) / 4^n in FP64 (exact scaling by a power of two; the
 * subtraction is the one rounding), equivalent per Definition 1 (F > 1 - eps; -1 when eps < 0),
 * traces_done copied. Needs no context and no device.
 * Errors: AJF_E_ARG (out NULL, n_qubits not in [1, 62], S negative or not finite, eps > 1). */
ajf_status ajf_fidelity_from_sum(int n_qubits, double S, double eps, int64_t traces_done, ajf_result *out);

/* Alg. II (Sec. IV-B): F_J from the one doubled network. Same contract as ajf_fidelity_alg1,
 * requiring ajf_plan(ctx, 2, ...). */
ajf_status ajf_fidelity_alg2(ajf_ctx *ctx, double eps, ajf_result *out);

/* Evaluate a planned context without allocating anything (the paper has no counterpart).
 * For callers that cannot allocate device memory: code whose device memory is reserved up front
 * and owned by another allocator, processes running under a hard device-memory cap, or paths
 * that must not enter the allocator (its latency and failure modes) once set up.
 * It runs the same device program as ajf_fidelity_alg1 (alg = 1) / ajf_fidelity_alg2 (alg = 2),
 * with the same results, but in a fixed device arena of 64 MiB that libajf declares as a static
 * __device__ array: every GPU that loads the library holds those 64 MiB until the process exits.
 * It calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating routine; inputs are copied
 * from the context's host memory and the result is read back synchronously. The context's own
 * arena, CUDA graph and Alg. I trace buffer are not touched (ajf_alg1_traces still returns the
 * last ajf_fidelity_alg1 result).
 * The arena's device address is looked up (cudaGetSymbolAddress, with the device current) by
 * ajf_create for every device context, which is also when the GPU reserves the array, so a
 * reservation failure surfaces there and this call itself performs no set-up. A context created
 * before a cudaDeviceReset keeps the old address: create a new context after a reset.
 * All calls on a device share the one arena and it keeps the last call's contents (the call
 * rewrites everything it reads, and zeroes its status words first). Calls whose device work
 * overlaps -- from different threads or different streams of one device -- race on the arena
 * and must be serialised by the caller.
 * Errors: AJF_E_ARG (alg, eps or out), AJF_E_STATE (no plan for `alg`, host-only context),
 * AJF_E_NOMEM (the plan's arena, ajf_workspace_size, exceeds 64 MiB), AJF_E_CUDA, AJF_E_TIMEOUT. */
ajf_status ajf_fidelity_noalloc(ajf_ctx *ctx, int alg, double eps, ajf_result *out);

/* After ajf_fidelity_alg1: copy the traces t_i = tr(U^dagger E_i) to `traces` (host, 2*count
 * doubles, interleaved), in enumeration order (lexicographic over noises in the order added,
 * last noise fastest; Sec. IV-A). count must equal prod_k n_k.
 * Errors: AJF_E_STATE (no Alg. I result), AJF_E_ARG (count mismatch). */
ajf_status ajf_alg1_traces(ajf_ctx *ctx, double *traces, int64_t count);

/* Enqueue one evaluation of the planned network on the context's stream without waiting:
 * uploads nothing (inputs must already be resident from an earlier fidelity call or
 * ajf_upload) and writes {S, F, 1-F} as three doubles to device memory `dev_result`.
 * With opts.use_graph the program is replayed from a CUDA graph.
 * Errors: AJF_E_STATE (no plan or inputs not uploaded), AJF_E_CUDA. */
ajf_status ajf_launch(ajf_ctx *ctx, double *dev_result);

/* Copy the circuit and noise inputs to the device (host -> device, on the context's stream)
 * and build the leaf tensors there. Called implicitly by the fidelity calls. */
ajf_status ajf_upload(ajf_ctx *ctx);

/* Alg. I over several contexts (independent circuits of uneven sizes; Sec. IV-A remarks that
 * the traces are independent): every context must have an Alg. I plan of the same precision
 * on the same device; every context's program is enqueued on that context's own stream (so the
 * circuits overlap on the GPU) and out[i] receives context i's result. eps as in ajf_fidelity_alg1.
 * Errors: AJF_E_ARG (n_ctx < 1, NULL entries, mixed device or precision), AJF_E_STATE. */
ajf_status ajf_fidelity_alg1_batch(ajf_ctx *const *ctxs, int n_ctx, double eps, ajf_result *out);

/* One kernel launch of a lowered plan, in the order an evaluation enqueues them. kind uses the
 * classes of ajf_kernel_stats (0 leaves ... 6 final); for GEMM launches M, N, K are the real GEMM
 * dimensions (2M', N', 2K' of the complex step) and terms the split terms (tensor cores). */
typedef struct ajf_launch_info {
  int32_t kind;
  int32_t terms;
  int64_t M, N, K;
  double flops;        /* algorithmic flops of the complex step(s) the launch carries out */
  double bytes;        /* algorithmic bytes of those steps                                 */
} ajf_launch_info;

/* List the launches of the current plan (valid after ajf_plan, also on host-only contexts):
 * up to `cap` records into `out`, the total count into *n. Errors: AJF_E_ARG, AJF_E_STATE. */
ajf_status ajf_plan_launches(const ajf_ctx *ctx, ajf_launch_info *out, int cap, int *n);

/* Turn per-launch timing on (1) or off (0) and clear the counters. While on, every run records
 * CUDA events around each launch (CUDA-graph replay is bypassed). */
ajf_status ajf_profile_enable(ajf_ctx *ctx, int on);

/* Read the counters: `stats` receives up to `cap` classes (8 are defined: 0 leaves, 1 small,
 * 2 split-K and tiled dot, 3 operand gather, 4 CUDA-core GEMM, 5 tensor-core GEMM, 6 final,
 * 7 persistent kernel -- counted on the context that leads the launch). Synchronises the
 * context's stream. Errors: AJF_E_ARG. */
ajf_status ajf_profile_read(ajf_ctx *ctx, ajf_kernel_stats *stats, int cap);

/* Self-test of the tensor-core GEMM kernel alone (no paper counterpart; used by the test suite):
 * C[M][N] = sum_{i + j < terms} A_i[M][K] . B_j[N][K]^T on device `device` for split operand
 * terms A_0..A_{terms-1}, B_0..B_{terms-1} (terms 1..3), FP32 accumulation promoted per K block.
 * kind 0: A and B hold terms * M * K (resp. N * K) FP32 values (read as TF32); kind 1: bf16 bit
 * patterns (uint16). All pointers are host memory; C receives M * N doubles (the kernel's FP32
 * results, widened exactly). The call allocates and frees its own device memory and synchronises
 * the device.
 * Errors: AJF_E_ARG, AJF_E_UNSUPPORTED (shape not tile-aligned: M % 128, N power of two >= 32,
 * K a multiple of 128 bytes), AJF_E_CUDA, AJF_E_TIMEOUT. */
ajf_status ajf_selftest_gemm(int device, int kind, int terms, int64_t M, int64_t N, int64_t K, const void *A,
                             const void *B, double *C);

/* Self-test of the step interpreter's failure path (no paper counterpart; used by the test suite):
 * one launch on device `device` whose second task waits for a first phase that can never
 * complete, with every wait bounded by wait_ms (0 < wait_ms <= 10000). The wait expires, the
 * kernel records code 21 in *code, every block stops taking tasks and returns, and the call
 * reports AJF_E_TIMEOUT; the device stays usable. Allocates and frees its own device memory and
 * synchronises the device. Errors: AJF_E_ARG, AJF_E_NOMEM, AJF_E_CUDA, AJF_E_TIMEOUT (expected). */
ajf_status ajf_selftest_queue_timeout(int device, double wait_ms, int32_t *code);

/* Self-test of one real product through the path's own operand preparation and tensor-core GEMM
 * (no paper counterpart; used by the test suite): C[M][N] = A[M][K] . B[N][K]^T for FP64 A and B
 * (row-major, host memory), on device `device`, in precision mode `precision` (AJF_PREC_TF32,
 * _TF32X3, _BF16X3, _BF16X6 or _F16X3). A and B enter as complex64 tensors with zero imaginary
 * part, as the reduced-precision modes store tensors (each value rounded to FP32, to nearest);
 * the gather splits them into the mode's operand terms (the leading term quantised per row and
 * K block) and the GEMM forms the product as it does in a contraction step (FP32 results, widened
 * exactly into C). M, N, K: powers of
 * two with M >= 16, N >= 16, K >= 8. C receives M * N doubles. The call allocates and frees its
 * own device memory and synchronises the device.
 * Errors: AJF_E_ARG, AJF_E_UNSUPPORTED (shape), AJF_E_NOMEM, AJF_E_CUDA, AJF_E_TIMEOUT. */
ajf_status ajf_selftest_split_gemm(int device, int precision, int64_t M, int64_t N, int64_t K, const double *A,
                                   const double *B, double *C);

/* Alg. I (alg = 1) or Alg. II (alg = 2) over several contexts at once: each context's device
 * program is enqueued on that context's own stream (give each context its own stream for the
 * circuits to overlap on the GPU), then all results are read back; out[i] receives context i's.
 * Contexts may differ in circuit size and precision. Sec. IV-A notes that the traces -- and so
 * the circuits -- are independent. A bond-sliced context (opts.slice_bonds) enqueues all its
 * runs on its stream at once when their staging fits 256 MiB of pinned memory (else it runs
 * chunk by chunk after the others are enqueued); Kraus-sliced Alg. I plans are refused.
 * Errors: AJF_E_ARG (n_ctx < 1, NULL entries, bad alg, contexts on different devices),
 * AJF_E_STATE (a context without a plan for `alg`, an alg1_slices plan), plus those of
 * ajf_fidelity_alg1/alg2. */
ajf_status ajf_fidelity_batch(ajf_ctx *const *ctxs, int n_ctx, int alg, double eps, ajf_result *out);

/* Persistent execution of many small networks in ONE kernel launch (no paper counterpart; the
 * independence of circuits and traces is Sec. IV-A's remark): one thread block per context runs
 * that context's whole program -- leaves, every pairwise step level by level, the FP64 trace,
 * sum |t_i|^2, F and 1 - F -- with its tensors in shared memory when the plan's work region
 * fits (96 KiB), otherwise in the context's device arena. Every context must be planned with
 * opts.lowering = AJF_LOWER_PERSISTENT, on one device; inputs not yet resident are uploaded on
 * each context's stream first. The launch goes on ctxs[0]'s stream, ordered after every
 * context's stream and before their later work (events). `dev_results` (device memory, 3 *
 * n_ctx doubles, may be NULL) receives {S, F, 1-F} per context; each context's own result and
 * Alg. I traces are written as by ajf_launch. Does not wait for the GPU.
 * Errors: AJF_E_ARG (n_ctx < 1, NULL entries, contexts on different devices or host-only),
 * AJF_E_STATE (a context without a persistent-lowered plan), AJF_E_NOMEM, AJF_E_CUDA. */
ajf_status ajf_launch_persistent(ajf_ctx *const *ctxs, int n_ctx, double *dev_results);

/* Persistent step interpreter (no paper counterpart for the kernel; Sec. IV-A remarks that the
 * evaluations of different circuits are independent): ONE launch of a persistent kernel, captured
 * in a CUDA graph, runs the default-lowered programs of all n_ctx contexts -- their leaves,
 * CUDA-core steps, operand gathers, tensor-core GEMM tiles (tcgen05) and final reductions -- as one
 * queue of tasks that the kernel's blocks (one per SM) take in order, each task after the previous
 * launch of its own program has completed. Contexts must be planned with the default lowering in a
 * tensor-core precision mode (or F64 plans without GEMM-class steps), unsliced, on one tcgen05
 * device; each context's inputs are uploaded if needed. The launch is enqueued on ctxs[0]'s stream
 * after the other contexts' streams (and they wait for it); results land in every context's own
 * result area (and in dev_results[3 i .. 3 i + 2] = S, F, 1 - F when dev_results is not NULL).
 * Errors: AJF_E_ARG, AJF_E_STATE (a context without a default-lowered unsliced plan),
 * AJF_E_UNSUPPORTED (CUDA-core GEMM steps or FP64 operands, no tcgen05 device), AJF_E_NOMEM,
 * AJF_E_CUDA. A device-side wait that expires is reported by ajf_fidelity_batch_queue. */
ajf_status ajf_launch_queue(ajf_ctx *const *ctxs, int n_ctx, double *dev_results);

/* Batch evaluation through one step-interpreter launch (ajf_launch_queue): out[i] receives
 * context i's result. Synchronises the contexts' streams.
 * Errors: those of ajf_launch_queue, AJF_E_ARG (alg, eps, out), AJF_E_STATE (a plan of the other
 * algorithm), AJF_E_TIMEOUT (a bounded device-side wait expired; the launch returned early). */
ajf_status ajf_fidelity_batch_queue(ajf_ctx *const *ctxs, int n_ctx, int alg, double eps, ajf_result *out);

/* Task-level timing of the step-interpreter launches led by ctx (no paper counterpart), taken by
 * launches made while ajf_profile_enable is on: for each kind of task k (0 leaves, 1 small steps,
 * 2 split-K, 3 split-K sums, 4 tiled traces, 5 operand gathers, 6 tensor-core GEMM work items,
 * 7 K-split sums, 8 open-tensor traces, 9 final), out[3k] = seconds the blocks spent running them,
 * out[3k + 1] = seconds they waited for the previous launch of the same program, out[3k + 2] =
 * tasks run; at most `cap` values. reset != 0 zeroes the counters. Synchronises ctx's stream.
 * Errors: AJF_E_ARG, AJF_E_STATE (no interpreter launch led by ctx), AJF_E_CUDA. */
ajf_status ajf_queue_profile(ajf_ctx *ctx, double *out, int cap, int reset);

/* Autotuner of the step interpreter's work decomposition (no paper counterpart): times `reps`
 * launches over the batch for each shape -- tensor-core GEMM work items (128 x BN tiles or K
 * splits) per task in {1, 2, 4}, and tasks per CUDA-core launch in {152, 304, 608} -- and keeps the
 * fastest for the process under the batch's signature (device and the programs' structures), used
 * by every later launch of a batch with that signature. The shape chosen is written to
 * *gemm_items and *body_tasks (either may be NULL). Synchronises the leading context's stream.
 * Errors: those of ajf_fidelity_batch_queue, AJF_E_ARG (reps < 1). */
ajf_status ajf_autotune_queue(ajf_ctx *const *ctxs, int n_ctx, int reps, int32_t *gemm_items, int32_t *body_tasks);

/* Autotune the persistent launch of this batch (no paper counterpart): its block size -- how many
 * output elements of a step one network's thread block computes at once -- is measured at 256,
 * 128 and 64 threads (CUDA events around `reps` launches each, after a warm-up launch), and the
 * fastest is kept (a smaller block must be at least 3% faster). The choice is remembered for
 * the process under the batch's signature (device and the networks' structures in order) and used
 * by every later persistent launch of a batch with that signature; *threads receives it. The
 * timed launches compute the batch's results as ajf_launch_persistent does. Synchronises the
 * leading context's stream. Errors: as ajf_launch_persistent, plus AJF_E_ARG (reps < 1,
 * threads NULL). */
ajf_status ajf_autotune_persistent(ajf_ctx *const *ctxs, int n_ctx, int reps, int32_t *threads);

/* Like ajf_fidelity_batch, with the contexts planned with AJF_LOWER_PERSISTENT run together in
 * one launch of the persistent kernel (ajf_launch_persistent) and the others on their own
 * streams, concurrently; waits and fills out[i] for every context. *n_persistent (may be NULL)
 * receives how many contexts ran in the persistent launch.
 * Errors: those of ajf_fidelity_batch and ajf_launch_persistent. */
ajf_status ajf_fidelity_batch_persistent(ajf_ctx *const *ctxs, int n_ctx, int alg, double eps, ajf_result *out,
                                         int32_t *n_persistent);

/* Self-test of the failure path of the device-side waits (no paper counterpart; used by the test
 * suite): runs the tensor-core GEMM kernel on a 128 x 32 x 32 problem with every wait bounded by
 * `wait_ms` and its producer told to issue no loads, so nothing ever completes the barriers the
 * other warps wait on. The kernel must give up after the bound, record which wait expired in
 * *code, release its TMEM and return; the device stays usable.
 * Returns AJF_E_TIMEOUT (the expected outcome, *code != 0) or AJF_OK (the waits did not report);
 * AJF_E_ARG (wait_ms not in (0, 10000], code NULL), AJF_E_NOMEM, AJF_E_CUDA. */
ajf_status ajf_selftest_wait_timeout(int device, double wait_ms, int32_t *code);

/* ---- Learned merge scorer (AJF_PLANNER_LEARNED). The paper orders contractions by a tree
 * decomposition (Sec. IV-C); this optional planner instead scores candidate pairwise merges with a
 * small MLP (16 features of the two operands, the result and the planner state; 16-224-192-1,
 * ReLU; 47,201 float32 parameters), trained to imitate the best paths that the greedy and min-fill
 * planners find with restarts. The greedy planner remains its fallback (no model loaded) and its
 * judge (the learned path is kept only if its estimated time is no worse). */

/* Number of float32 parameters of the scorer (47201). */
int32_t ajf_learned_param_count(void);

/* Give the context a scorer model (n must equal ajf_learned_param_count(); the library copies it;
 * NULL removes it). Invalidates the plan. Errors: AJF_E_ARG. */
ajf_status ajf_set_learned_model(ajf_ctx *ctx, const float *weights, int32_t n);

/* Training data from the loaded circuit: the network of `alg` is planned by the greedy and min-fill
 * planners (`trials` restarts, `seed`), and the best path is replayed; at every step the merge it
 * takes is paired with up to `negatives` other candidates. Each pair is 2 x 16 floats (the taken
 * merge's features, then the other's). Up to cap_pairs pairs go to `out` (host); *n_pairs gets the
 * total. Works on host-only contexts. Errors: AJF_E_ARG, AJF_E_STATE, AJF_E_BUDGET. */
ajf_status ajf_learned_dataset(ajf_ctx *ctx, int alg, int32_t trials, uint64_t seed, int32_t negatives, float *out,
                               int64_t cap_pairs, int64_t *n_pairs);

/* Train the scorer on device `device` with the hand-written CUDA training kernels: pairwise ranking
 * loss softplus(s(other) - s(taken)), minibatches of `batch` pairs, Adam (learning rate lr),
 * `epochs` passes, Glorot-initialised from `seed`. pairs: n_pairs x 2 x 16 floats (host).
 * Writes n_weights (= ajf_learned_param_count()) parameters and the last epoch's mean loss.
 * Errors: AJF_E_ARG, AJF_E_NOMEM, AJF_E_CUDA. */
ajf_status ajf_learned_train(int device, const float *pairs, int64_t n_pairs, int32_t epochs, int32_t batch, float lr,
                             uint64_t seed, float *weights, int32_t n_weights, double *final_loss);

/* Library version string, e.g. "ajf 0.1 sm_103a". */
const char *ajf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AJF_H */
