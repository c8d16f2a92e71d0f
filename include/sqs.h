/*
 * sqs.h -- C ABI of the GB300 sparse register-level quantum-state library.
 *
 * The library applies quantum operations to a state held only as its nonzero
 * branches, the representation of SparQSim (arXiv 2503.15118, Sec. II.C):
 *
 *     |psi> = sum_i a_i |v_i^0> |v_i^1> ... |v_i^{K-1}>          (Eq. 5)
 *
 * Each branch is a packed basis key -- register j occupies key bits
 * [off_j, off_j + w_j), off_0 = 0, off_j = sum_{i<j} w_i, so register 0 holds
 * the low bits and key bit q is qubit q of Eq. 4 -- plus one complex
 * amplitude.  Keys are one 64-bit word when sum(w_j) <= 64 and two words
 * (bits 64..127 in the second) up to 128 qubits.  A register is 1..64 bits
 * wide, the size of one StateStorage value (Table S2).
 *
 * Execution model.  All device memory belongs to the state; calls enqueue work
 * on the state's CUDA stream and return without waiting.  Runs of
 * non-interference operations (permutations, phases, QRAM, diagonal and
 * anti-diagonal single-qubit matrices) are queued and fused into the kernel
 * that next touches the state.  Only sqs_nnz, sqs_export, sqs_probabilities,
 * sqs_sync and sqs_state_destroy wait for the device.  Device-side failures
 * (capacity overflow, a bounded wait that ran out) are sticky: the next
 * waiting call returns them, and sqs_last_error() describes them.
 *
 * Threading: a state may be used by one host thread at a time.
 * Errors: every call checks its arguments on the host before enqueueing and
 * returns SQS_ERR_ARG without side effects when they are invalid.
 */
#ifndef SQS_H_
#define SQS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sqs_state sqs_state;
typedef struct sqs_table sqs_table;

typedef enum {
  SQS_OK = 0,
  SQS_ERR_ARG = -1,      /* invalid argument; nothing was enqueued          */
  SQS_ERR_OOM = -2,      /* device allocation failed                         */
  SQS_ERR_CAPACITY = -3, /* state would exceed the largest allowed capacity  */
  SQS_ERR_CUDA = -4,     /* a CUDA call failed (message in sqs_last_error)   */
  SQS_ERR_TIMEOUT = -5,  /* a bounded device-side wait ran out               */
  SQS_ERR_STATE = -6     /* the state is unusable after an earlier error     */
} sqs_status;

/* State-creation flags. */
#define SQS_AMP_FP64 0u           /* amplitudes stored as complex<double>       */
#define SQS_AMP_FP32 1u           /* stored as complex<float>.  Each child of
                                     an interference step is evaluated with
                                     compensated FP32 arithmetic (Dot2, float-
                                     float coefficients): the FP64 sum rounded
                                     once to FP32.  A component within rho
                                     (sqs_set_fp32_cancel) of its terms' size
                                     is set to zero (a cancellation the stored
                                     precision cannot resolve).  Norms and
                                     probabilities accumulate in FP64.          */
#define SQS_SIZING_EXACT 0u       /* output buffers sized from exact bounds     */
#define SQS_SIZING_LEARNED 2u     /* sized by the learned capacity predictor;
                                     an overflow is detected on the device and
                                     the operation re-run at the exact size     */
#define SQS_MERGE_AUTO 0u         /* default merge path (per-CTA buckets)       */
#define SQS_MERGE_HASH 4u         /* force the per-CTA bucket merge             */
#define SQS_MERGE_SORT 8u         /* force the radix-sort merge: LSD passes of
                                     8-bit digits over the pair-class key (the
                                     key without the target bit), windows
                                     skipping bits known constant, then one
                                     pass combining neighbours; states of 2^32
                                     or more branches use the bucket merge    */
#define SQS_MERGE_CLUSTER 16u     /* force the cluster (binned) merge           */
#define SQS_MERGE_TUNED 32u       /* measured choice per step: the first steps
                                     of each size class (log2 of the count
                                     bound, sort pass count) time the bucket
                                     and the sort merge with CUDA events; later
                                     steps of the class take the faster one.
                                     Both give bit-identical states.  A step
                                     whose target bit is known constant always
                                     takes the expansion path (no merge).     */
#define SQS_MERGE_PLAIN 64u       /* disable the host-proven shortcuts: the
                                     constant-bit expansion and the copy-pair
                                     fold (a target whose every partner is
                                     known to hold +-1 times the branch's
                                     amplitude).  Results are bit-identical
                                     either way; this flag exists to show it.
                                     Also runs every interference step alone
                                     (as SQS_FUSE_OFF).                       */
#define SQS_FUSE_OFF 128u         /* run every interference step alone.  By
                                     default (exact sizing, SQS_MERGE_AUTO or
                                     SQS_MERGE_TUNED) interference steps issued
                                     back to back on distinct target qubits,
                                     with no other operation queued between
                                     them and no step's controls or angle
                                     register on another step's target, are
                                     held and executed together when the run
                                     ends (Sec. II.D.2: each coherent group --
                                     the branches equal on every other qubit --
                                     is transformed as one vector of up to
                                     2^k entries, k <= 12).  The result is
                                     bit-identical to the steps run one by
                                     one, peak count included.  Runs end at
                                     the next operation of another kind that
                                     must execute, any read, sqs_flush, or
                                     when they reach 12 steps.  A held run
                                     executes fused when that is estimated to
                                     move less memory (sort passes plus the
                                     group pass against a scatter and a merge
                                     pass per step, one pass per constant-bit
                                     expansion) on at least 2^14 branches;
                                     otherwise its steps run one by one.     */
#define SQS_FUSE_ALWAYS 256u      /* execute every held run of two or more
                                     steps fused, whatever its size and
                                     estimated cost (exercises the fused path
                                     on small states)                        */
#define SQS_AUTOTUNE 512u         /* measure and pick, per (GPU, operation kind,
                                     key words, amplitude type, log2 of the
                                     branch count, bits to sort or run length):
                                     the radix digit width of every sort (6, 8,
                                     10 or 11 bits) and the tile size of fused
                                     runs.  Each candidate is timed twice with
                                     CUDA events on real steps (results do not
                                     depend on the choice), then the fastest
                                     median is kept.  Choices persist through
                                     sqs_tune_export / sqs_tune_import, or the
                                     file named by the environment variable
                                     SQS_TUNE_CACHE (read when the state is
                                     created, written when it is destroyed).
                                     Without this flag: 8-bit digits and the
                                     default tile rule.  The environment
                                     variable SQS_SORT_BITS (6, 8, 10 or 11),
                                     read when a state is created, forces one
                                     digit width for every sort of the state
                                     (tests, experiments).                    */

/*
 * One control (or predicate) qubit: bit `bit` of register `reg` must equal
 * `value` (1 for the textbook control of Sec. II.A, CU = |0><0| (x) I +
 * |1><1| (x) U; 0 is accepted as an extension).
 */
typedef struct {
  uint32_t reg, bit, value;
} sqs_ctrl;

#define SQS_MAX_CTRL 8    /* controls carried inline by one sqs_perm_op      */
#define SQS_MAX_PRED 128  /* controls / predicates passed as an array to the
                             sqs_apply_u1q, _h, _ry, _ry_reg and _phase calls:
                             one entry per qubit, so a predicate over whole
                             registers ("ancilla register = 0") fits       */

/*
 * Optional device allocator.  alloc(ctx, bytes, stream) returns device memory
 * usable on `stream` (or NULL on failure); free(ctx, ptr, stream) releases it.
 * When no allocator is given the library uses cudaMallocAsync/cudaFreeAsync.
 */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, void* stream);
} sqs_allocator;

/* Permutation operations (non-interference, Sec. II.D.1).  Each maps every
 * basis key to one key, bijectively, under its controls:
 *   SQS_PERM_X          flip bit `bit` of `reg` (X, CNOT, Toffoli: FlipBool of
 *                       Supp. B, controls attached as in ClassControllable)
 *   SQS_PERM_ADD_REG    reg := (reg + src_reg) mod 2^{w_reg}
 *   SQS_PERM_SUB_REG    reg := (reg - src_reg) mod 2^{w_reg}
 *   SQS_PERM_ADD_CONST  reg := (reg + constant) mod 2^{w_reg}
 *   SQS_PERM_SUB_CONST  reg := (reg - constant) mod 2^{w_reg}
 *   SQS_PERM_SWAP       exchange reg and src_reg (equal widths)
 * Sec. II.D.1 treats multiplication and division as arithmetic oracles built
 * the same way as addition: the multiply-add, multiply-by-odd-constant and
 * divide-XOR kinds are those oracles in their reversible forms (the sources, and the destination's previous value,
 * determine the result, so each map is a bijection on keys).  Sources must be
 * registers other than the destination; controls may not sit inside it. */
typedef enum {
  SQS_PERM_X = 0,
  SQS_PERM_ADD_REG = 1,
  SQS_PERM_SUB_REG = 2,
  SQS_PERM_ADD_CONST = 3,
  SQS_PERM_SUB_CONST = 4,
  SQS_PERM_SWAP = 5,
  SQS_PERM_MUL_ADD = 6,   /* reg := (reg + src_reg * src2_reg) mod 2^{w_reg}        */
  SQS_PERM_MUL_CONST = 7, /* reg := (reg * constant) mod 2^{w_reg}, constant odd      */
  SQS_PERM_DIV_XOR = 8    /* reg := reg XOR (src_reg / src2_reg) (integer quotient,
                             0 when src2_reg holds 0), truncated to w_reg          */
} sqs_perm_kind;

typedef struct {
  uint32_t kind;     /* sqs_perm_kind                                     */
  uint32_t reg;      /* target / destination register                     */
  uint32_t bit;      /* SQS_PERM_X: bit within reg                        */
  uint32_t src_reg;  /* *_REG and SWAP: source register (!= reg)          */
  uint64_t constant; /* *_CONST: added / subtracted value                 */
  uint32_t n_ctrl;   /* number of valid entries of ctrl (<= SQS_MAX_CTRL) */
  sqs_ctrl ctrl[SQS_MAX_CTRL];
  uint32_t src2_reg; /* MUL_ADD, DIV_XOR: second source register           */
} sqs_perm_op;

/* ---- state lifetime --------------------------------------------------- */

/* Creates a state over n_regs registers of the given widths (each 1..64, sum
 * 1..128) in |0...0> with amplitude 1 (one branch).  capacity_hint is the
 * branch count to pre-allocate for (0: small default; the state grows on
 * demand).  cuda_stream (a cudaStream_t, NULL = the legacy default stream)
 * orders every operation.  Errors: SQS_ERR_ARG (bad widths/flags),
 * SQS_ERR_OOM, SQS_ERR_CUDA.  *out is written only on SQS_OK. */
sqs_status sqs_state_create(const uint32_t* reg_widths, uint32_t n_regs, uint32_t flags,
                            uint64_t capacity_hint, const sqs_allocator* allocator,
                            void* cuda_stream, sqs_state** out);

/* Waits for the state's pending work, then releases its device memory. */
void sqs_state_destroy(sqs_state* st);

/* Resets to |0...0> (one branch, amplitude 1) keeping allocations and any
 * sticky error cleared.  Enqueued; does not wait. */
sqs_status sqs_state_reset(sqs_state* st);

/* FP32-storage states: the storage-precision cancellation threshold rho.
 * A component of a child of an interference step whose compensated value
 * is at most rho times the size of its terms (sum of |coefficient| x
 * |stored amplitude component|) is set to zero; the child is then pruned
 * when both components are zero.  Default 2^-19 (32 units of FP32 roundoff);
 * 0 disables the rule.  SQS_ERR_ARG outside [0, 2^-10].  Takes effect for
 * operations issued afterwards.  No effect on FP64 states. */
sqs_status sqs_set_fp32_cancel(sqs_state* st, double rho);

/* Threshold of the pruning step that ends every interference operation
 * (Sec. II.D.2: branches left at zero amplitude are removed).  A branch is
 * removed when |a| < eps (strict).  Default 1e-14; eps >= 0. */
sqs_status sqs_set_prune_eps(sqs_state* st, double eps);

/* ---- interference operations (Sec. II.D.2, rotation listing of Supp. B) --
 * Single-qubit matrix U on qubit `bit` of `reg`, on the branches whose
 * controls hold:   psi'(x) = sum_s U[x_t][s] psi(x with bit t := s),
 * U indexed [row = output bit][column = input bit].  Branches are split into
 * their two children, equal keys merged (amplitudes summed), and branches with
 * |a| < eps removed.  A control on the target qubit itself is SQS_ERR_ARG.
 * Diagonal and anti-diagonal U (the _operate_diagonal / _operate_off_diagonal
 * strategies of Supp. B) take the non-branching fused path; the result is the
 * same.  m is row-major {re00, im00, re01, im01, re10, im10, re11, im11}. */
sqs_status sqs_apply_u1q(sqs_state* st, uint32_t reg, uint32_t bit, const double m[8],
                         const sqs_ctrl* ctrl, uint32_t n_ctrl);
/* H = 2^{-1/2} [[1, 1], [1, -1]] (Sec. II.A). */
sqs_status sqs_apply_h(sqs_state* st, uint32_t reg, uint32_t bit, const sqs_ctrl* ctrl,
                       uint32_t n_ctrl);
/* RY(theta) = [[cos theta/2, -sin theta/2], [sin theta/2, cos theta/2]]. */
sqs_status sqs_apply_ry(sqs_state* st, uint32_t reg, uint32_t bit, double theta,
                        const sqs_ctrl* ctrl, uint32_t n_ctrl);
/* Register-valued rotation (angle_function_t of the rotation listing, Supp.
 * B): per branch, RY(scale * value(angle_reg) + offset) on (reg, bit).
 * angle_reg must not be reg. */
sqs_status sqs_apply_ry_reg(sqs_state* st, uint32_t reg, uint32_t bit, uint32_t angle_reg,
                            double scale, double offset, const sqs_ctrl* ctrl,
                            uint32_t n_ctrl);

/* ---- non-interference operations (Sec. II.D.1) --------------------------
 * Never change the number of branches and never prune. */
sqs_status sqs_apply_perm(sqs_state* st, const sqs_perm_op* ops, uint32_t n_ops);
/* a := a * e^{i phi} on every branch where all n_pred predicates hold (Z, S,
 * T and controlled phases; n_pred = 0 is a global phase). */
sqs_status sqs_apply_phase(sqs_state* st, const sqs_ctrl* pred, uint32_t n_pred, double phi);

/* ---- QRAM (Supp. C, Eq. S1) ----------------------------------------------
 * A table of n_entries little-endian unsigned entries of entry_bytes (1, 2, 4
 * or 8) copied from host memory to the device (the table is owned by the
 * state and freed with it).  Load maps |i>_A |j>_D -> |i>_A |j XOR d_i>_D with
 * d_i truncated to the data register's width (the word length); addresses at
 * or past n_entries read d = 0.  Unload applies the same map (it is its own
 * inverse). */
sqs_status sqs_table_create(sqs_state* st, const void* host_entries, uint64_t n_entries,
                            uint32_t entry_bytes, sqs_table** out);
sqs_status sqs_qram_load(sqs_state* st, uint32_t addr_reg, uint32_t data_reg,
                         const sqs_table* table);
sqs_status sqs_qram_unload(sqs_state* st, uint32_t addr_reg, uint32_t data_reg,
                           const sqs_table* table);
/* The same with the address formed by n_addr_regs consecutive registers
 * addr_reg, addr_reg + 1, ... (register addr_reg in the low bits), as the
 * controlled state preparation of a block-encoding queries a rotation-angle
 * tree at (column index, prepared prefix) (Supp. D, U_L).  The address is at
 * most 64 bits wide and the data register lies outside it (SQS_ERR_ARG). */
sqs_status sqs_qram_load_span(sqs_state* st, uint32_t addr_reg, uint32_t n_addr_regs,
                              uint32_t data_reg, const sqs_table* table);
sqs_status sqs_qram_unload_span(sqs_state* st, uint32_t addr_reg, uint32_t n_addr_regs,
                                uint32_t data_reg, const sqs_table* table);

/* ---- pruning, readout ---------------------------------------------------- */

/* Removes every branch with |a| < eps (ClearZero, Sec. II.D.2).  When nnz_out
 * is non-NULL the call waits and writes the remaining count. */
sqs_status sqs_prune(sqs_state* st, double eps, uint64_t* nnz_out);

/* Marginal probabilities of register `reg`: probs[v] = sum over branches with
 * reg = v of |a|^2, accumulated in FP64, for v in [0, 2^{w_reg}) (w_reg <= 26;
 * probs has 2^{w_reg} entries; NULL skips them).  norm2 (nullable) receives
 * sum |a|^2 over the whole state.  Waits. */
sqs_status sqs_probabilities(sqs_state* st, uint32_t reg, double* probs, double* norm2);

/* Same, written to device memory (probs_dev: 2^{w_reg} doubles, norm2_dev: 1
 * double, either nullable).  Enqueued; does not wait. */
sqs_status sqs_probabilities_device(sqs_state* st, uint32_t reg, double* probs_dev,
                                    double* norm2_dev);

/* Marginal probabilities of register `reg` in sparse form, for a register of
 * any width (up to 64 bits): the distinct values v the register holds over
 * the state's branches, ascending, in values[0..count), and probs[i] = sum
 * over the branches with reg = values[i] of |a|^2.  Sums are FP64, in a fixed
 * order (branches sorted by the register, each value's branches in key-sort
 * order), so repeated calls give identical results.  *count receives the
 * number of distinct values; when it exceeds cap nothing is copied and
 * SQS_ERR_ARG is returned (cap = 0 with NULL arrays asks for the count).
 * norm2 (nullable) receives sum |a|^2 over the whole state.  values and
 * probs are host memory.  The state must hold fewer than 2^32 branches
 * (SQS_ERR_CAPACITY otherwise).  Device scratch: a sorted copy of the state
 * and 16 bytes per branch.  Waits. */
sqs_status sqs_probabilities_sparse(sqs_state* st, uint32_t reg, uint64_t* values, double* probs,
                                    uint64_t cap, uint64_t* count, double* norm2);

/* Current branch count.  Waits. */
sqs_status sqs_nnz(sqs_state* st, uint64_t* out);

/* Largest branch count reached since creation or reset (max_system_size,
 * Table S1).  Waits. */
sqs_status sqs_peak_nnz(sqs_state* st, uint64_t* out);

/* Autotuner choices of the state (SQS_AUTOTUNE) as JSON text:
 * {"gpu": "<device name>", "entries": [{"site": "sort_bits" | "group_slots",
 * "kw": 1|2, "amp32": 0|1, "n_log2": L, "extra": E, "choice": V,
 * "cand": [...], "median_ms": [...]}, ...]} -- one entry per measured key, V
 * the value kept (-1 while still measuring).  Writes at most cap bytes
 * (including the terminating zero) to buf and the full length to *len;
 * SQS_ERR_ARG when it does not fit. */
sqs_status sqs_tune_export(const sqs_state* st, char* buf, uint64_t cap, uint64_t* len);
/* Loads choices from JSON text of the export's format; entries measured on a
 * GPU of another name are ignored.  Loaded choices are used without new
 * measurements when SQS_AUTOTUNE is set. */
sqs_status sqs_tune_import(sqs_state* st, const char* json);

/* Testing hook for the bounded device waits.  The cluster merge
 * (SQS_MERGE_CLUSTER) loads each CTA's slice of a bin with bulk copies that
 * complete on an mbarrier; every wait on it polls at most wait_limit times
 * (0 restores the default, about 6.7e7 polls), then records SQS_ERR_TIMEOUT
 * in the state, waits (bounded again) for copies in flight and lets the CTA
 * finish without its slice.  skip_copy_rank >= 0 makes the CTAs of that rank
 * in every cluster issue no copy, so that their wait runs out (a fault
 * injected on the host side of the copy, not on the GPU); -1 turns it off.
 * The next waiting call returns SQS_ERR_TIMEOUT; sqs_state_reset makes the
 * state usable again.  For tests only. */
sqs_status sqs_state_set_wait_test(sqs_state* st, uint32_t wait_limit, int32_t skip_copy_rank);

/* Copies the branches to host memory in ascending key order (the canonical
 * order of a state, which is a set; states of 2^32 or more branches are
 * copied in storage order).  keys receives kw words per branch (kw = 1 when
 * sum(w) <= 64, else 2: low word first); amps receives (re, im) FP64 pairs.
 * cap is the capacity of the arrays in branches; *n receives the branch count
 * (when it exceeds cap nothing is copied and SQS_ERR_ARG is returned).  The
 * sort runs on the device into scratch; the state keeps its own order.
 * Waits. */
sqs_status sqs_export(sqs_state* st, uint64_t* keys, double* amps, uint64_t cap, uint64_t* n);

/* Replaces the state with n branches from host memory (same layout as
 * sqs_export; keys must be distinct and fit the register widths).  Work
 * issued before and not yet executed (queued operations, a held run of
 * interference steps, queued learned-sizing steps) is dropped with the old
 * state; call sqs_flush first to execute it. */
sqs_status sqs_import(sqs_state* st, const uint64_t* keys, const double* amps, uint64_t n);

/* Executes everything queued and waits; returns any sticky device error. */
sqs_status sqs_sync(sqs_state* st);

/* Executes everything queued without waiting. */
sqs_status sqs_flush(sqs_state* st);

/* Number of key words per branch (1 or 2). */
uint32_t sqs_key_words(const sqs_state* st);

/* Kernel launches issued by this state since creation (host-side count). */
uint64_t sqs_launch_count(const sqs_state* st);

/* ---- tracing (profiling aid; replaces the per-operation wall-clock timer of
 * the paper's profiler helper, Supp. B, with CUDA events) ------------------
 * When enabled, every kernel launch is bracketed by two CUDA events on the
 * state's stream.  A record names the kernel, the index of the API call that
 * issued it (counted from the last sqs_trace_enable) and its device time. */
#define SQS_K_INIT 0u
#define SQS_K_APPLY 1u      /* fused non-interference run, in place        */
#define SQS_K_COMPACT 2u    /* fused run that may drop branches             */
#define SQS_K_PARTITION 3u  /* fused run + scatter into merge buckets       */
#define SQS_K_PAIR 4u       /* pair, 2x2, prune, compact (one CTA / bucket) */
#define SQS_K_PROB 5u       /* probabilities / norm                         */
#define SQS_K_CONVERT 6u    /* FP32 <-> FP64 staging for export / import    */
#define SQS_K_EXPAND 7u     /* constant target bit: children without merge  */
#define SQS_K_BIN 8u        /* cluster merge: coarse binning                */
#define SQS_K_PAIR_CLUSTER 9u /* cluster merge: pairing in a thread-block cluster */
#define SQS_K_SORT 10u      /* radix-sort merge: one LSD pass (histogram, scan, scatter) */
#define SQS_K_SORT_MERGE 11u /* radix-sort merge: neighbours combined, 2x2, prune */
#define SQS_K_FOLD 12u      /* copy-pair fold: both children from one member   */
#define SQS_K_GROUP_COUNT 13u /* fused run: coherent groups per bucket          */
#define SQS_K_GROUP 14u     /* fused run: every group transformed in shared memory */
typedef struct {
  uint32_t kernel; /* SQS_K_*                          */
  uint32_t call;   /* API call index (numbered from the last reset) that
                      issued the launch's work: a held interference step,
                      run when a later call closes its run, keeps its own
                      call's index                                          */
  float ms;        /* device time between the events    */
  uint32_t pad;
} sqs_trace_record;

/* Enables tracing for up to max_records launches (0 disables).  Allocates
 * events; call outside stream capture. */
sqs_status sqs_trace_enable(sqs_state* st, uint32_t max_records);
/* Waits, writes up to cap records, returns the count in *n, and starts a new
 * trace (records past max_records are dropped and counted in *n). */
sqs_status sqs_trace_read(sqs_state* st, sqs_trace_record* out, uint32_t cap, uint32_t* n);

/* Human-readable description of the last error on this state (never NULL). */
const char* sqs_last_error(const sqs_state* st);

/* Library version string. */
const char* sqs_version(void);

/* ---- learned capacity predictor ------------------------------------------
 * The paper sizes nothing in advance: its std::vector grows branch by branch
 * (Sec. II.C).  A device state must be sized before a merge runs.  In exact
 * mode the runtime uses the bound "an interference step at most doubles the
 * branches it acts on" and reads the exact count back when that bound would
 * outgrow the buffers.  In learned mode (SQS_SIZING_LEARNED plus an attached
 * predictor) interference steps are queued until the next flush; their
 * structural features go through one batched inference of this MLP, which
 * predicts log2(branches after / branches before) of each step; the merge
 * buckets are sized from the predicted counts; an undersized bucket is
 * detected on the device (no write goes out of bounds) and the step and
 * everything after it re-run at the exact size before the flush returns.
 *
 * Network: SQS_PRED_FEATURES inputs -> SQS_PRED_HIDDEN tanh -> SQS_PRED_HIDDEN
 * tanh -> 1, FP32.  Parameters (SQS_PRED_PARAMS floats) in the order W1[H][F],
 * b1[H], W2[H][H], b2[H], w3[H], b3.  Training minimises the mean squared
 * error with Adam, all on the device. */
#define SQS_PRED_FEATURES 16
#define SQS_PRED_HIDDEN 32
#define SQS_PRED_PARAMS 1633
typedef struct sqs_predictor sqs_predictor;
/* Deterministic initialisation from seed; work goes on cuda_stream. */
sqs_status sqs_predictor_create(uint64_t seed, void* cuda_stream, sqs_predictor** out);
void sqs_predictor_destroy(sqs_predictor* p);
sqs_status sqs_predictor_get_params(const sqs_predictor* p, float* out);
sqs_status sqs_predictor_set_params(sqs_predictor* p, const float* in);
/* Y[i] = net(X[i]) for n samples of SQS_PRED_FEATURES floats (host arrays). */
sqs_status sqs_predictor_predict(sqs_predictor* p, const float* X, uint32_t n, float* Y);
/* Gradient of the mean squared error over the n samples (host arrays). */
sqs_status sqs_predictor_gradient(sqs_predictor* p, const float* X, const float* T, uint32_t n,
                                  float* grad, float* loss);
/* Adam over `epochs` passes of mini-batches of `batch` samples. */
sqs_status sqs_predictor_train(sqs_predictor* p, const float* X, const float* T, uint32_t n,
                               uint32_t epochs, uint32_t batch, float lr, float* final_loss);
/* Attaches a predictor (owned by the caller) used when the state was created
 * with SQS_SIZING_LEARNED; NULL detaches. */
sqs_status sqs_state_set_predictor(sqs_state* st, sqs_predictor* p);
/* Records, for every interference step from now on, its feature vector and
 * the measured log2(branches after / branches before) (training traces). */
sqs_status sqs_state_record(sqs_state* st, uint32_t enable);
/* Waits, copies up to cap records (X: cap * SQS_PRED_FEATURES floats, y: cap
 * floats), writes the number available to *n and clears the records. */
sqs_status sqs_state_read_records(sqs_state* st, float* X, float* y, uint32_t cap, uint32_t* n);

/* ---- CUDA-graph capture -------------------------------------------------
 * Small states are bound by launch latency (tens of microseconds per gate);
 * a circuit that runs many times from |0...0> can be captured once and
 * replayed as one CUDA graph.
 *
 * sqs_capture_begin resets the state to |0...0> (now, and as the graph's
 * first node), sizes its buffers for static_bound branches and starts
 * capturing the state's stream (thread-local capture mode).  Until
 * sqs_capture_end, every call is recorded instead of run; the branch-count
 * bound is held at static_bound (an operation whose result would exceed it is
 * detected on the device and reported, sticky, at the next wait); calls that
 * wait for the device, copy to or from host memory or allocate return
 * SQS_ERR_STATE and make the capture fail (readouts, sqs_table_create,
 * sqs_import, sqs_sync; run the circuit once without capture first so that
 * QRAM tables and rotation tables exist).  Learned sizing and the sort,
 * cluster and measured merges cannot be captured, nor can a state created on
 * the legacy default stream (SQS_ERR_ARG).
 * sqs_capture_end closes the capture, instantiates the graph into *out and
 * leaves the state at |0...0> (nothing was run).  On failure nothing is
 * returned and the state is usable.
 * sqs_graph_launch replays the graph on the state's stream: the state becomes
 * what the captured calls make of |0...0>, asynchronously, exactly as if they
 * were issued again (pending operations are discarded as by a reset).  It
 * fails with SQS_ERR_STATE when the state's buffers were reallocated since
 * the capture (a larger state grew them): capture again.  Destroy graphs
 * before their state. */
typedef struct sqs_graph sqs_graph;
sqs_status sqs_capture_begin(sqs_state* st, uint64_t static_bound);
sqs_status sqs_capture_end(sqs_state* st, sqs_graph** out);
sqs_status sqs_graph_launch(sqs_state* st, sqs_graph* g);
void sqs_graph_destroy(sqs_graph* g);

typedef struct {
  uint64_t host_waits;       /* times the host read the device counts         */
  uint64_t overflow_reruns;  /* learned-mode steps re-run at the exact size    */
  uint64_t learned_steps;    /* steps sized from a prediction                  */
  uint64_t bytes_live;       /* device bytes currently held by the state       */
  uint64_t bytes_peak;       /* largest bytes_live since creation              */
  uint64_t steps_expand;     /* interference steps by path: constant target   */
  uint64_t steps_hash;       /*   per-CTA bucket merge                         */
  uint64_t steps_sort;       /*   radix-sort merge                             */
  uint64_t steps_cluster;    /*   binned cluster merge                         */
  uint64_t steps_fold;       /*   copy-pair fold                               */
  uint64_t runs_fused;       /* fused runs executed (SQS_FUSE_OFF unset)      */
  uint64_t steps_fused;      /*   interference steps inside them              */
  uint64_t ops_deferred;     /* queued operations kept queued past a step that
                                only merges (copy-pair target), applied later
                                to the smaller state                          */
} sqs_stats;
sqs_status sqs_state_stats(const sqs_state* st, sqs_stats* out);

/* ---- no-allocation variant --------------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: code embedded in a host framework that owns
 * every byte of device memory through its own pre-planned arena or budget,
 * and latency-bound callers that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may perform.  Such a caller
 * keeps its state in its own device buffers and passes them in and out.
 *
 * sqs_apply_u1q_noalloc applies the single-qubit matrix m (layout as in
 * sqs_apply_u1q) on bit `bit` of register `reg`, under the controls, to the
 * n_in branches in keys_lo_in / keys_hi_in / amps_in and writes the merged,
 * pruned (|a| < eps removed) result to keys_lo_out / keys_hi_out / amps_out:
 *   keys_lo_*: key bits 0..63, one uint64 per branch (device memory);
 *   keys_hi_*: key bits 64..127 (device memory; ignored, may be NULL, when
 *              sum(reg_widths) <= 64);
 *   amps_*:    (re, im) FP64 pairs, one per branch (device memory);
 *   n_out:     device pointer receiving the output count, or all ones when a
 *              device-side check failed.
 * Keys must be distinct.  The output order carries no meaning.  It never
 * allocates: its scratch space (buckets, output segments, offsets, a control
 * block) is one static device array of sqs_noalloc_scratch_bytes() bytes
 * (about 8.1 MiB), which every GPU that loads the library holds until the
 * process exits.  Inputs larger than SQS_NOALLOC_MAX_BRANCHES branches, or an
 * out_cap below 2 * n_in, are rejected with SQS_ERR_ARG before anything is
 * enqueued; sqs_noalloc_last_error() gives the reason.  The first call on a
 * device looks up the array's device address (set-up, once per device, with
 * that device current); make that first call before any stream capture.  All
 * calls share the one array and each clears what it needs at its start:
 * calls whose work overlaps on the GPU (other streams, or the same stream
 * from concurrent host threads) race and corrupt each other's results.
 * Enqueued on `stream`; returns without waiting. */
#define SQS_NOALLOC_MAX_BRANCHES 65536u
sqs_status sqs_apply_u1q_noalloc(const uint32_t* reg_widths, uint32_t n_regs, uint32_t reg,
                                 uint32_t bit, const double m[8], const sqs_ctrl* ctrl,
                                 uint32_t n_ctrl, double eps, const uint64_t* keys_lo_in,
                                 const uint64_t* keys_hi_in, const double* amps_in,
                                 uint64_t n_in, uint64_t* keys_lo_out, uint64_t* keys_hi_out,
                                 double* amps_out, uint64_t out_cap, uint64_t* n_out,
                                 void* stream);
/* Reason for the last SQS_ERR_* from sqs_apply_u1q_noalloc on this thread. */
const char* sqs_noalloc_last_error(void);
/* Size in bytes of the static scratch array of sqs_apply_u1q_noalloc. */
uint64_t sqs_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* SQS_H_ */
