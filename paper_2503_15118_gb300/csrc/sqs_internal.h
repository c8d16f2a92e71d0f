// Internal interfaces shared by the host runtime (sqs_api.cu) and the kernels
// (sqs_kernels.cu).  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sqs {

// ---------------------------------------------------------------------------
// Fused non-interference operations.  A run of them is applied to each branch
// in registers by whichever kernel next streams the state (Sec. II.D.1: every
// branch is processed independently, so a run of such operations is one
// per-branch function and one pass over memory).
// ---------------------------------------------------------------------------
enum OpKind : uint32_t {
  OP_XOR = 0,        // key ^= xmask                                 (X, CNOT, Toffoli)
  OP_ADD_REG = 1,    // dst := dst + src  (mod 2^w)
  OP_SUB_REG = 2,    // dst := dst - src
  OP_ADD_CONST = 3,  // dst := dst + constant
  OP_SWAP = 4,       // exchange dst and src fields (equal width)
  OP_QRAM = 5,       // dst := dst XOR (T[src] & mask(w_dst)), src = address field
  OP_MUL = 6,        // amp *= (bit sel of key ? c1 : c0)             (phases, diag U)
  OP_MUL_XOR = 7,    // amp *= (bit sel ? c1 : c0); key ^= xmask        (anti-diagonal U)
  OP_PRUNE = 8       // drop the branch when |amp|^2 < eps2
};

struct DevOp {
  uint32_t kind;
  uint32_t dst_off, dst_w;  // destination field (bit offset, width)
  uint32_t src_off, src_w;  // source field (register operand or QRAM address)
  uint32_t sel_bit;         // OP_MUL*: key bit choosing c0 / c1 (128 = always c0)
  uint32_t entry_bytes;     // OP_QRAM: 1, 2, 4 or 8
  uint32_t pad0;
  uint64_t pmask[2], pval[2];  // predicate: (key & pmask) == pval
  uint64_t xmask[2];           // OP_XOR / OP_MUL_XOR
  uint64_t constant;           // OP_ADD_CONST (already reduced mod 2^w)
  uint64_t n_entries;          // OP_QRAM table length
  const void* table;           // OP_QRAM device table
  double c[4];                 // OP_MUL*: c0 = (c[0], c[1]), c1 = (c[2], c[3])
  double eps2;                 // OP_PRUNE
};

constexpr int kMaxOps = 48;  // fused operations per launch (kernel parameter space)

struct OpList {
  uint32_t n;
  uint32_t touches_keys;  // some op changes keys
  uint32_t touches_amps;  // some op changes amplitudes
  uint32_t drops;         // some op may drop branches (OP_PRUNE)
  DevOp op[kMaxOps];
};

// ---------------------------------------------------------------------------
// Device memory views.
// ---------------------------------------------------------------------------
struct Arr {          // one SoA branch array
  uint64_t* k0;       // key bits 0..63
  uint64_t* k1;       // key bits 64..127 (null when keys are one word)
  void* amp;          // double2[cap] or float2[cap]
  uint64_t cap;       // capacity in branches
};

// Device control block.  The branch count of the current array lives in a
// small ring: an operation that writes a new array appends into cnt[out] and
// clears cnt[(out + 1) & 3] for the operation after it.
struct Ctl {
  unsigned long long cnt[4];
  unsigned long long peak;
  unsigned long long need;     // branches an overflowing write needed
  unsigned int err;            // sticky error bits (kErr*)
  unsigned int err_where;      // launch sequence number of the first error
  double norm2;
  unsigned long long pad[2];
};

constexpr unsigned int kErrCapacity = 1u;  // output array too small
constexpr unsigned int kErrBucket = 2u;    // a hash bucket overflowed
constexpr unsigned int kErrProbe = 4u;     // a bounded hash probe ran out

struct Buckets {     // hash-partitioned staging for the merge
  uint64_t* k0;
  uint64_t* k1;
  void* amp;
  unsigned int* count;  // B counters, zero between uses
  uint32_t B, C;        // buckets, capacity per bucket (branches)
};

struct Gate1 {            // the interference operation of one merge step
  uint32_t t;             // target key bit
  uint32_t mode;          // 0: constant matrix U, 1: RY from a register value
  uint64_t cmask[2], cval[2];  // controls
  double u[8];            // U row-major (re, im)
  uint32_t ang_off, ang_w;     // mode 1: angle register field
  double scale, offset;        // mode 1: theta = scale * value + offset
  double eps2;            // prune threshold squared (strictly-less removes)
};

struct Launch {
  cudaStream_t stream;
  int sm_count;
  uint32_t seq;        // launch sequence number (error attribution)
  uint64_t n_hint;     // host-side upper bound of the branches streamed (grid size)
};

// Launchers (sqs_kernels.cu).  Each returns cudaGetLastError() after enqueueing.
cudaError_t launch_init(const Launch& L, Ctl* ctl, Arr a, int slot, bool amp32);
cudaError_t launch_apply_inplace(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 const OpList& ops);
cudaError_t launch_apply_compact(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                                 int in_slot, Arr out, int out_slot, const OpList& ops);
cudaError_t launch_partition(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                             const OpList& ops, const Gate1& g, Buckets bk, Arr out,
                             int out_slot);
cudaError_t launch_pair(const Launch& L, int kw, bool amp32, Ctl* ctl, const Gate1& g,
                        Buckets bk, Arr out, int out_slot);
cudaError_t launch_probabilities(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 uint32_t off, uint32_t w, double* probs, double* norm2);
cudaError_t launch_to_f64(const Launch& L, Ctl* ctl, Arr a, int slot, double* out);
cudaError_t launch_from_f64(const Launch& L, Ctl* ctl, Arr a, const double* in, uint64_t n);

int pair_capacity(int kw, bool amp32);       // branches per bucket
size_t pair_smem_bytes(int kw, bool amp32);  // dynamic shared memory of one bucket CTA

}  // namespace sqs
