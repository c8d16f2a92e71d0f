// Internal interfaces shared by the host runtime (sqs_api.cu) and the kernels
// (sqs_kernels.cu).  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace sqs {

// ---------------------------------------------------------------------------
// Fused non-interference operations.  A run of them is applied to each branch
// in registers by whichever kernel next streams the state (Sec. II.D.1: every
// branch is processed independently, so a run of such operations is one
// per-branch function and one pass over memory).
//
// Amplitude factors are folded: each OP_MUL / OP_MUL_XOR only records its
// outcome (not applied / factor c0 / factor c1) in a few bits of a per-branch
// index, and OP_TABLE multiplies the amplitude once by the product of the
// selected factors, precomputed on the host for every index.  FP64 arithmetic
// is the scarce resource on this GPU; integer work is not.
// ---------------------------------------------------------------------------
enum OpKind : uint32_t {
  OP_XOR = 0,        // key ^= xmask                                   (X, CNOT, Toffoli)
  OP_ADD_REG = 1,    // dst := dst + src  (mod 2^w)
  OP_SUB_REG = 2,    // dst := dst - src
  OP_ADD_CONST = 3,  // dst := dst + constant
  OP_SWAP = 4,       // exchange dst and src fields (equal width)
  OP_QRAM = 5,       // dst := dst XOR (T[src] & mask(w_dst)), src = address field
  OP_MUL = 6,        // record factor choice (bit sel of key: c1, else c0) (phases, diag U)
  OP_MUL_XOR = 7,    // the same, then key ^= xmask                     (anti-diagonal U)
  OP_TABLE = 8,      // amp *= tab[tab_off + idx] unless idx == 0; idx := 0
  OP_PRUNE = 9,      // drop the branch when |amp| < eps
  OP_MUL_ADD = 10,   // dst := dst + src * src2  (mod 2^w)
  OP_MUL_CONST = 11, // dst := dst * constant    (mod 2^w, constant odd)
  OP_DIV_XOR = 12    // dst := dst XOR (src / src2), 0 when src2 = 0
};

struct DevOp {
  uint32_t kind;
  uint32_t dst_off, dst_w;  // destination field (bit offset, width)
  uint32_t src_off, src_w;  // source field (register operand or QRAM address)
  uint32_t sel_bit;         // OP_MUL*: key bit choosing c0 / c1 (128 = no choice)
  uint32_t shift;           // OP_MUL*: position of this op's outcome in the index
  uint32_t tab_off;         // OP_TABLE: first entry of this group's table
  uint32_t src2_off, src2_w;   // OP_MUL_ADD / OP_DIV_XOR: second source field
  uint64_t pmask[2], pval[2];  // predicate: (key & pmask) == pval
  uint64_t xmask[2];           // OP_XOR / OP_MUL_XOR
  uint64_t constant;           // OP_ADD_CONST (already reduced mod 2^w); QRAM: entry bytes
  uint64_t n_entries;          // OP_QRAM table length
  const void* table;           // OP_QRAM device table
  double eps, eps2;            // OP_PRUNE
};

constexpr int kMaxOps = 64;      // fused operations per launch
constexpr int kTabEntries = 1024;  // folded factor entries per launch

struct OpList {
  uint32_t n;
  uint32_t touches_keys;  // some op changes keys
  uint32_t touches_amps;  // some op changes amplitudes
  uint32_t drops;         // some op may drop branches (OP_PRUNE)
  uint32_t n_tab;         // used entries of tab
  uint32_t pad[3];
  DevOp op[kMaxOps];
  double2 tab[kTabEntries];
};

// ---------------------------------------------------------------------------
// Device memory views.
// ---------------------------------------------------------------------------
// One SoA branch array.  Dense (seg_cnt == null): branches [0, n) with n in
// the control block.  Segmented: segment s holds seg_cnt[s] branches starting
// at s << seg_log2; the slots after them are unused.  Kernels that compact
// write one segment per CTA, which needs no global ordering.
struct Arr {
  uint64_t* k0;       // key bits 0..63
  uint64_t* k1;       // key bits 64..127 (null when keys are one word)
  void* amp;          // double2[cap] or float2[cap]
  uint64_t cap;       // capacity in branches
  unsigned int* seg_cnt;
  uint32_t seg_log2;
  uint32_t n_seg;
};

// Device control block.  The total branch count of the current array lives
// in a small ring: an operation that writes a new array adds into cnt[out]
// and clears cnt[(out + 1) & 3] for the operation after it.
struct Ctl {
  unsigned long long cnt[4];
  unsigned long long peak;
  unsigned long long need;     // branches an overflowing write needed
  unsigned int err;            // sticky error bits (kErr*)
  unsigned int err_where;      // launch sequence number of the first error
  double norm2;
  unsigned long long groups;     // fused run: coherent groups of its input
  unsigned long long items;      // fused run: branches of its input (after the queued run)
  unsigned long long stage[16];  // fused run: branches after each of its operations
  unsigned int buckets;          // bucket merge: buckets the partition filled
  unsigned int pair_next;        // bucket merge: next bucket a pair CTA takes (the partition zeroes it)
};

constexpr unsigned int kErrCapacity = 1u;  // output array too small
constexpr unsigned int kErrBucket = 2u;    // a hash bucket overflowed
constexpr unsigned int kErrProbe = 4u;     // a bounded hash probe ran out

struct Gate1 {            // the interference operation of one merge step
  uint32_t t;             // target key bit
  uint32_t mode;          // 0: complex U, 1: RY from a register value, 2: real U
  uint64_t cmask[2], cval[2];  // controls
  double u[8];            // U row-major (re, im)
  float uf[8];            // U rounded to FP32 (FP32-storage states)...
  float ufl[8];           // ...and the rest, u - uf rounded to FP32 (float-float)
  float rho32;            // FP32 storage: cancellation threshold (relative to the terms)
  // Product reuse: bit 0 set when U10 = +-U00 (bit 2: minus), bit 1 when
  // U11 = +-U01 (bit 3: minus); each column then costs one product per branch.
  uint32_t reuse;
  uint32_t ang_off, ang_w;     // mode 1: angle register field
  double scale, offset;        // mode 1: theta = scale * value + offset
  double eps, eps2;       // pruning threshold and its square (|a| < eps removes)
  float epsf;             // eps rounded to FP32
  uint32_t no_partners;   // the target bit is constant over the state: expand only
  // Host only: the operations queued before this step commute with it and
  // stay queued past it (the step can only merge: every partner exists).
  uint32_t defer_ops;
  uint32_t issue_call;  // host only: the API call that issued the step (trace attribution)
  uint64_t vary[2];       // key bits not known constant over the state (sort digits)
  // Copy-pair fold: +1 / -1 when every branch's partner across the target bit
  // is known to exist with amplitude exactly +1 / -1 times its own; 0 otherwise.
  int32_t fold_sign;
  // Fold with real U (mode 2) where child r's coefficient cancels exactly
  // (U[r][0] = -fold_sign * U[r][1]): that child is the rounding residue of
  // one product, below eps whenever both components of the branch's
  // amplitude are below fold_tmax (bit pattern, FP64 states; FP32 states
  // flush it always).  -1: no child cancels.
  int32_t fold_kill;
  // The surviving child's two coefficients are equal once the pair's sign is
  // applied (U[r][0] = fold_sign * U[r][1], H-like): the child
  // fma(U[r][0], a, round(U[r][0] a)) is exactly 2 round(U[r][0] a).
  uint32_t fold_twice;
  uint64_t fold_tmax;
  // Mode 1: (cos, sin) of the half angle per 16-bit digit of the angle
  // register's value, digit j at [j << 16, (j + 1) << 16), the offset folded
  // into digit 0 (device table owned by the state; null: direct sincos).
  const double2* ang_tab;
  uint32_t ang_digits;
};

// A fused run of interference operations on distinct target bits (Sec.
// II.D.2: the branches agreeing on every idle bit form a coherent group, and
// the operation acts on each group).  Operation j acts on key bit g[j].t,
// which is bit j of a branch's index inside its group; no operation's
// controls or angle register touch any target of the run, so each group
// either satisfies them as a whole or not at all.
constexpr int kMaxRun = 12;
struct GroupRun {
  uint32_t k;            // operations in the run (2 <= k <= kMaxRun)
  uint32_t pad;
  uint64_t tmask[2];     // union of the target bits
  Gate1 g[kMaxRun];
};

struct Launch {
  cudaStream_t stream;
  int sm_count;
  uint32_t seq;        // launch sequence number (error attribution)
  uint64_t n_hint;     // host-side upper bound of the branches streamed (grid size)
  // Bounded device waits (cluster merge): polls before giving up (0: the
  // default), and a testing hook -- a cluster rank whose CTAs issue no bulk
  // copy, so that their wait runs out (-1: none).
  uint32_t wait_limit = 0;
  int32_t skip_copy_rank = -1;
};

// Launchers (sqs_kernels.cu).  Each returns cudaGetLastError() after enqueueing.
// Fills tab[j << 16 | d] = (cos, sin)(scale / 2 * d * 2^(16 j) + (j == 0 ? offset / 2 : 0)).
cudaError_t launch_angle_table(cudaStream_t s, double2* tab, uint32_t digits, double scale,
                               double offset);
cudaError_t launch_init(const Launch& L, Ctl* ctl, Arr a, int slot, bool amp32);
cudaError_t launch_apply_inplace(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 const OpList& ops);
// Streams `in` through the run into a segmented `out` (one segment per
// 2^out.seg_log2 input slots), dropping pruned branches.
cudaError_t launch_apply_compact(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                                 int in_slot, Arr out, int out_slot, const OpList& ops);
// Streams `in` through the run and scatters every branch into the hash bucket
// of its pair class (key with the target bit cleared).  bk is segmented with
// bk.n_seg buckets of 2^bk.seg_log2 slots, counters zero on entry.
// Buckets follow the device count: ceil(count / fill_target) of them, at
// most bk.n_seg (the host's bound; fill_target 0 keeps bk.n_seg); the pair
// kernel leaves the others empty.
cudaError_t launch_partition(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                             const OpList& ops, const Gate1& g, Arr bk, uint32_t fill_target);

// Radix-sort merge (sqs_sort.cu).  One LSD pass: digit `shift` of the
// pair-class key (key with bit t deleted) of `in` -> `out` (dense), stable.
// With first_ops the fused run is applied on the way (in is the state as it
// lies, n_ptr its count); later passes read the dense count *n_ptr.  hist
// holds 2^8 * n_tiles counters, part sort_part_entries(); the pass stores the
// number of branches written in *n_dev.
int sort_tile();
int sort_radix_bits();                // default digit width (8)
int sort_radix_bits_max();            // widest digit supported (11)
bool sort_radix_bits_ok(int rb);      // a supported width: 6, 8, 10 or 11
uint32_t sort_merge_chunk_log2();
size_t sort_part_entries();
// With clear_mask (two words, non-zero) the sort key is the key with those
// bits cleared instead: a fused run's targets, so that every coherent group
// ends contiguous.
cudaError_t launch_rsort_pass(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                              const unsigned long long* n_ptr, uint32_t per_seg,
                              uint64_t n_tiles, const OpList* first_ops, uint32_t t,
                              uint32_t shift, unsigned int* hist, unsigned int* part,
                              unsigned long long* n_dev, Arr out,
                              const uint64_t* clear_mask = nullptr, int radix_bits = 8);
// Combines neighbours of the sorted array `in` (*n_ptr branches): chunk c of
// 2^sort_merge_chunk_log2() branches becomes segment c of `out` (twice the
// size).  Adds the count into cnt[out_slot], clears cnt[(out_slot + 1) & 3].
cudaError_t launch_rsort_merge(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                               const unsigned long long* n_ptr, const Gate1& g, Arr out,
                               int out_slot);
// Per bucket: pair, apply the 2x2, prune; bucket b's survivors become
// segment b of `out` (segment capacity 2 x bucket capacity).  One resident
// wave of CTAs draws the buckets the partition used (ctl->buckets) from a
// counter the partition zeroed (ctl->pair_next).  Resets the bucket counters.
cudaError_t launch_pair(const Launch& L, int kw, bool amp32, Ctl* ctl, const Gate1& g, Arr bk,
                        Arr out, int out_slot);
// Interference step whose target bit is constant over the state (no pair can
// exist): the fused run, then both children of every controlled branch,
// appended to the dense array `out` (count in cnt[out_slot]; input chunks of
// 2^12 slots, n_chunks of them).  With
// g.fold_sign set (every pair present with a1 = fold_sign * a0) the bit-0
// member of each controlled pair emits both children and the bit-1 member
// nothing: the copy-pair fold, with no partition and no pairing.
cudaError_t launch_expand(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                          uint64_t n_chunks, const OpList& ops, const Gate1& g, Arr out,
                          int out_slot);
// Copy-pair fold of a gate without controls (g.fold_sign != 0, no control
// bits): only the bit-0 members are read past their key and emit.
cudaError_t launch_fold(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                        uint64_t n_chunks, const OpList& ops, const Gate1& g, Arr out,
                        int out_slot);
cudaError_t launch_probabilities(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 uint32_t off, uint32_t w, double* probs, double* norm2);
// Copies a segmented array into a dense one given exclusive segment offsets.
cudaError_t launch_densify(const Launch& L, int kw, bool amp32, Arr in, const uint64_t* offsets,
                           Arr out);
cudaError_t launch_to_f64(const Launch& L, Ctl* ctl, Arr a, int slot, double* out);
// rec[0] = cnt[in_slot], rec[1] = cnt[out_slot] (one interference step's counts).
cudaError_t launch_record(const Launch& L, const Ctl* ctl, int in_slot, int out_slot,
                          unsigned long long* rec);
cudaError_t launch_from_f64(const Launch& L, Ctl* ctl, Arr a, const double* in, uint64_t n);

// Binned merge (thread-block clusters): bins of 2^cluster_bin_log2()
// branches, each paired by cluster_ctas() CTAs whose survivors go to output
// segments (bin * cluster_ctas() + rank) of 2^cluster_out_seg_log2() slots.
constexpr int kMaxBins = 2048;
int cluster_bin_log2();
int cluster_ctas();
int cluster_out_seg_log2();
cudaError_t launch_bin(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                       const OpList& ops, const Gate1& g, Arr bins);
cudaError_t launch_pair_cluster(const Launch& L, int kw, bool amp32, Ctl* ctl, const Gate1& g,
                                Arr bins, Arr out, int out_slot);

// Fused run (sqs_group.cu), over `in`: the dense array (count *n_ptr)
// sorted on the key with the run's targets cleared, so that each coherent
// group is contiguous.  launch_group_count adds the number of groups to
// ctl->groups and stores the count in ctl->items.  launch_group gives each
// CTA the groups that start in its tile of tile_len (<= 2048) branches and
// applies the run to them (in shared memory, each group a dense vector of
// 2^k amplitudes with presence flags, one operation after another with the
// pruning of each), appends the survivors to the dense `out` (count in
// cnt[out_slot]), adds the branch count after each operation into
// ctl->stage[j] and raises the peak to the largest of them.
constexpr uint32_t kGroupTile = 2048;
cudaError_t launch_group_count(const Launch& L, int kw, Ctl* ctl, Arr in,
                               const unsigned long long* n_ptr, const uint64_t tmask[2]);
cudaError_t launch_group(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                         const unsigned long long* n_ptr, uint32_t tile_len, uint64_t n_tiles,
                         Arr out, int out_slot, const GroupRun& run);
// Raises a kernel's dynamic shared-memory limit to `smem` bytes on the
// current device, once per device.  The attribute is per device; the
// bitmask of devices already configured is shared by host threads, so it is
// updated atomically (two threads that race both set the same attribute,
// which is harmless).
inline cudaError_t ensure_smem_optin(const void* func, size_t smem,
                                     std::atomic<unsigned long long>& configured) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
  const unsigned long long bit = 1ull << dev;
  if (configured.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) configured.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Sparse marginals (sqs_readout.cu) over `sorted`: the dense state (count
// *n_ptr) sorted by the field [off, off + w), ascending.  Writes the distinct
// field values in ascending order to values[] and the sum of |a|^2 over each
// value's branches to probs[], and their number to *total.  Scratch: runs[],
// lead_sum[], lead_full[] of run_tiles(n) entries each.
uint64_t run_tiles(uint64_t n);
cudaError_t launch_sparse_marginals(const Launch& L, int kw, bool amp32, const Ctl* ctl, Arr sorted,
                                    const unsigned long long* n_ptr, uint64_t n_tiles, uint32_t off,
                                    uint32_t w, unsigned int* runs, double* lead_sum,
                                    unsigned int* lead_full, unsigned long long* total,
                                    uint64_t* values, double* probs);

int pair_log2_capacity(int kw, bool amp32);  // log2 branches per bucket
size_t pair_smem_bytes(int kw, bool amp32);  // dynamic shared memory of one bucket CTA

}  // namespace sqs
