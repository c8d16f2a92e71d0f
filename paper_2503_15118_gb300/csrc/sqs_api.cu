// Host runtime of the C ABI declared in include/sqs.h.
//
// It owns the device buffers of a state, translates every call into fused
// device operations, queues the non-interference ones, and launches the
// kernels of sqs_kernels.cu on the state's stream.  Sizing is exact: the host
// keeps an upper bound of the branch count (an interference step at most
// doubles the branches it acts on, Sec. II.D.2) and reads the exact count back
// only when that bound would outgrow the allocated capacity.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/sqs.h"
#include "sqs_internal.h"

using sqs::Arr;
using sqs::Ctl;
using sqs::DevOp;
using sqs::Gate1;
using sqs::GroupRun;
using sqs::OpList;

struct sqs_table {
  void* dev;
  uint64_t n;
  uint32_t bytes;
};

namespace {

constexpr uint32_t kBucketLog2 = 11;  // branches per merge bucket (shared-memory tile)
constexpr uint32_t kSegLog2 = 12;     // branches per output segment (2 x bucket)
// Mean bucket fill of the bucket merge.  Half of the 2048 slots up to 2^26
// branches: overflow is then about 32 sigma away, and the bucket counters
// the partition's atomics contend on see fewer branches each (measured 4%
// faster per step on the large random circuit, 2^24 branches at its peak,
// than a fill of three quarters).  Three quarters above 2^26 branches, and
// inside a graph capture, where every step sizes for the static bound: fewer,
// fuller buckets cost less memory and fewer merge CTAs (overflow about 18
// sigma away).
constexpr uint64_t kBucketFill = (1ull << kBucketLog2) / 2;
constexpr uint64_t kBucketFillLarge = (1ull << kBucketLog2) * 3 / 4;
uint64_t bucket_fill(uint64_t count_bound) {
  return count_bound <= (1ull << 26) ? kBucketFill : kBucketFillLarge;
}

// One branch buffer and its current layout.
struct Store {
  uint64_t* k0 = nullptr;
  uint64_t* k1 = nullptr;
  void* amp = nullptr;
  uint64_t cap = 0;
  unsigned int* segs = nullptr;  // per-segment counts (cap >> kBucketLog2 + 1 entries)
  bool segmented = false;
  uint32_t seg_log2 = 0;
  uint32_t n_seg = 0;

  Arr view() const {
    Arr a;
    a.k0 = k0;
    a.k1 = k1;
    a.amp = amp;
    a.cap = cap;
    a.seg_cnt = segmented ? segs : nullptr;
    a.seg_log2 = seg_log2;
    a.n_seg = n_seg;
    return a;
  }
  // Slots a kernel must visit: the segments, or the dense count bound.
  uint64_t slots(uint64_t count_ub) const {
    return segmented ? ((uint64_t)n_seg << seg_log2) : count_ub;
  }
  void set_dense() {
    segmented = false;
    seg_log2 = 0;
    n_seg = 0;
  }
  void set_segments(uint32_t log2, uint32_t n) {
    segmented = true;
    seg_log2 = log2;
    n_seg = n;
  }
};

// The host-side bookkeeping that describes the device state: buffer roles,
// the count slot and bound, and the per-qubit history.
struct HostSnap {
  Store cur, alt, bk;
  int cur_slot = 0;
  uint64_t ub = 1;
  uint32_t call = 0;
  std::vector<int64_t> last_branch;
  std::vector<uint32_t> writes_since, reads_since;
  std::vector<uint8_t> arith_since;
  std::vector<int8_t> const_val, pair_sign;
  int64_t n_branch = 0, last_target = -1;
};

// A queued non-interference operation; factors c0/c1 of amplitude operations
// stay on the host and are folded into the launch's factor table.
struct HostOp {
  DevOp d;
  std::complex<double> c0, c1;
};

}  // namespace

struct sqs_state {
  std::vector<uint32_t> width, offset;
  uint32_t total_bits = 0;
  int kw = 1;
  bool amp32 = false;
  uint32_t flags = 0;
  double eps = 1e-14;
  float rho32 = 0x1p-19f;  // FP32 storage: cancellation threshold (sqs_set_fp32_cancel)

  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 1;
  sqs_allocator alloc{};
  bool has_alloc = false;

  Store cur, alt, bk;
  int cur_slot = 0;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;    // pinned mirror
  double* scratch = nullptr;  // probabilities / format conversion / offsets
  size_t scratch_bytes = 0;

  std::vector<HostOp> pending;
  OpList ops_buf;   // staging for one launch's fused operations
  uint64_t ub = 1;  // upper bound of the current branch count
  uint32_t seq = 0;
  uint64_t launches = 0;
  std::vector<sqs_table*> tables;
  std::string err;
  sqs_status sticky = SQS_OK;

  // Tracing: event pairs around launches.
  std::vector<cudaEvent_t> ev;          // 2 per record
  std::vector<sqs_trace_record> trace;  // kernel / call of each used pair
  uint32_t trace_dropped = 0;
  uint32_t call = 0;                    // API call counter

  // Structural history per key bit: the features of the learned predictor.
  std::vector<int64_t> last_branch;  // index of the last interference step on the bit, -1: none
  std::vector<uint32_t> writes_since, reads_since;  // operations since that step
  std::vector<uint8_t> arith_since;  // the bit's register was an arithmetic destination since
  std::vector<int8_t> const_val;     // value when the bit is known constant, else -1
  // +1 / -1 when every branch's partner across the bit is known to exist with
  // exactly +1 / -1 times its amplitude (set by an uncontrolled expansion with
  // U[1][b] = +-U[0][b], kept while nothing reads or writes the bit), else 0.
  std::vector<int8_t> pair_sign;
  int64_t n_branch = 0;
  int64_t last_target = -1;

  // Training traces: features and (in, out) counts of every interference step.
  bool recording = false;
  std::vector<float> rec_x;
  unsigned long long* rec_dev = nullptr;
  uint32_t rec_cap = 0;

  // Learned sizing: queued interference steps (with the operations before
  // each), sized at the next flush from one batched inference.
  sqs_predictor* predictor = nullptr;
  struct Lazy {
    Gate1 g;
    std::vector<HostOp> ops;
    float x[SQS_PRED_FEATURES];
  };
  std::vector<Lazy> lazy;
  bool defer_frees = false;
  std::vector<void*> graveyard;
  uint64_t grow_hint_b = 0;  // learned mode: buckets at the predicted peak (growth target)

  // Radix-sort merge scratch: digit histograms, scan partials, count.
  unsigned char* sort_buf = nullptr;
  size_t sort_bytes = 0;
  // Bounded device waits: poll limit (0: default) and the testing hook of
  // sqs_state_set_wait_test.
  uint32_t wait_limit = 0;
  int32_t skip_copy_rank = -1;
  // Measured merge choice (SQS_MERGE_TUNED), per size class.
  struct Tune {
    float us_per_slot[2] = {-1.f, -1.f};  // bucket merge, sort merge
    int pending = -1;                     // path whose events are in flight
    uint64_t slots = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
  };
  std::map<uint32_t, Tune> tune;

  // Autotuner (SQS_AUTOTUNE): per key, the candidates, their timed samples
  // and the value kept; one measurement in flight per key.
  struct TuneKey {
    uint32_t site, kw, amp32, n_log2, extra;
    bool operator<(const TuneKey& o) const {
      return std::tie(site, kw, amp32, n_log2, extra) <
             std::tie(o.site, o.kw, o.amp32, o.n_log2, o.extra);
    }
  };
  struct TuneEntry {
    std::vector<int> cand;
    std::vector<std::vector<float>> ms;
    int choice = -1;   // value kept (-1: still measuring)
    int pending = -1;  // index of the candidate whose events are in flight
    cudaEvent_t ev[2] = {nullptr, nullptr};
  };
  std::map<TuneKey, TuneEntry> tuner;
  std::string gpu_name;
  int forced_sort_bits = 0;  // SQS_SORT_BITS: one digit width for every sort
  uint32_t trace_call = 0;   // when set, the call launches are attributed to

  // Half-angle tables of register-valued rotations, per (scale, offset,
  // digits); kept for the state's lifetime (queued steps may point to them).
  struct AngTab {
    double scale, offset;
    uint32_t digits;
    double2* dev;
  };
  std::vector<AngTab> ang_tabs;

  // Fused run (exact sizing): interference steps on distinct targets issued
  // back to back with nothing queued between them, held until the run ends.
  std::vector<Gate1> run_gates;
  std::vector<HostOp> run_pre;       // operations queued before the run's first step
  uint64_t run_tmask[2] = {0, 0};    // the run's target bits
  uint64_t run_reads[2] = {0, 0};    // control and angle bits its steps read

  // CUDA-graph capture (sqs_capture_begin / _end): while capturing, nothing
  // may wait for the device or allocate, and the branch-count bound is held
  // at static_ub (buffers are sized for it when the capture begins).
  bool capturing = false;
  uint64_t static_ub = 0;
  sqs_status capture_err = SQS_OK;
  HostSnap entry_snap;
  uint64_t launches_at_capture = 0;

  sqs_stats stats{};
  std::unordered_map<void*, size_t> sizes;
};

namespace {

const char* kVersion = "sqs 0.2 (sm_103a)";

sqs_status fail(sqs_state* st, sqs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (st) st->err = buf;
  return s;
}

sqs_status cuda_fail(sqs_state* st, cudaError_t e, const char* what) {
  st->sticky = SQS_ERR_CUDA;
  return fail(st, SQS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* dalloc(sqs_state* st, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (st->capturing) {
    st->capture_err = SQS_ERR_STATE;  // buffers are sized when the capture begins
    return nullptr;
  }
  if (st->has_alloc) {
    p = st->alloc.alloc(st->alloc.ctx, bytes, (void*)st->stream);
  } else if (cudaMallocAsync(&p, bytes, st->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    st->sizes[p] = bytes;
    st->stats.bytes_live += bytes;
    st->stats.bytes_peak = std::max(st->stats.bytes_peak, st->stats.bytes_live);
  }
  return p;
}

void dfree_now(sqs_state* st, void* p) {
  if (!p) return;
  auto it = st->sizes.find(p);
  if (it != st->sizes.end()) {
    st->stats.bytes_live -= it->second;
    st->sizes.erase(it);
  }
  if (st->has_alloc)
    st->alloc.free(st->alloc.ctx, p, (void*)st->stream);
  else
    cudaFreeAsync(p, st->stream);
}

// While a learned-sizing flush may still re-run a step, buffers that held
// its input are kept alive instead of being freed.
void dfree(sqs_state* st, void* p) {
  if (!p) return;
  if (st->defer_frees)
    st->graveyard.push_back(p);
  else
    dfree_now(st, p);
}

size_t amp_bytes(const sqs_state* st) { return st->amp32 ? 8 : 16; }

void free_store(sqs_state* st, Store& s) {
  dfree(st, s.k0);
  dfree(st, s.k1);
  dfree(st, s.amp);
  dfree(st, s.segs);
  s = Store{};
}

uint64_t round_cap(uint64_t need) {
  uint64_t c = 1ull << kSegLog2;
  while (c < need) c = c + c / 2;
  return (c + (1ull << kSegLog2) - 1) & ~((1ull << kSegLog2) - 1);
}

// Makes s hold at least `need` branches (contents are not kept).
bool ensure_store(sqs_state* st, Store& s, uint64_t need) {
  if (s.k0 && s.cap >= need) return true;
  if (st->capturing) {  // buffers are sized when a capture begins
    st->capture_err = SQS_ERR_STATE;
    return false;
  }
  free_store(st, s);
  const uint64_t cap = round_cap(need);
  const uint64_t nseg = (cap >> kBucketLog2) + 1;
  s.k0 = (uint64_t*)dalloc(st, cap * 8);
  s.k1 = st->kw == 2 ? (uint64_t*)dalloc(st, cap * 8) : nullptr;
  s.amp = dalloc(st, cap * amp_bytes(st));
  s.segs = (unsigned int*)dalloc(st, nseg * 4);
  s.cap = cap;
  if (!s.k0 || (st->kw == 2 && !s.k1) || !s.amp || !s.segs) {
    free_store(st, s);
    return false;
  }
  cudaMemsetAsync(s.segs, 0, nseg * 4, st->stream);
  return true;
}

uint64_t max_branches(const sqs_state* st) {
  return st->total_bits >= 62 ? (1ull << 62) : (1ull << st->total_bits);
}

// The count bound after an operation: v, held at the static bound while a
// graph is captured (the device checks every write against the buffers).
uint64_t bound_after(const sqs_state* st, uint64_t v) {
  return st->static_ub ? std::min(v, st->static_ub) : v;
}

// Brackets one launch with trace events when tracing is on.
struct Traced {
  sqs_state* st;
  int idx = -1;
  Traced(sqs_state* s, uint32_t kernel) : st(s) {
    if (st->ev.empty() || st->capturing) return;
    const size_t used = st->trace.size();
    if (2 * (used + 1) > st->ev.size()) {
      st->trace_dropped++;
      return;
    }
    idx = (int)used;
    st->trace.push_back(
        sqs_trace_record{kernel, st->trace_call ? st->trace_call : st->call, 0.f, 0u});
    cudaEventRecord(st->ev[2 * idx], st->stream);
  }
  ~Traced() {
    if (idx >= 0) cudaEventRecord(st->ev[2 * idx + 1], st->stream);
  }
};

sqs::Launch launch_of(sqs_state* st, uint64_t n_hint) {
  sqs::Launch L;
  L.stream = st->stream;
  L.sm_count = st->sm_count;
  L.seq = ++st->seq;
  L.n_hint = n_hint;
  L.wait_limit = st->wait_limit;
  L.skip_copy_rank = st->skip_copy_rank;
  st->launches++;
  return L;
}

// Predicate on the packed key from (reg, bit, value) triples.
bool encode_ctrls(sqs_state* st, const sqs_ctrl* c, uint32_t n, uint64_t mask[2],
                  uint64_t val[2]) {
  mask[0] = mask[1] = val[0] = val[1] = 0;
  if (n > SQS_MAX_PRED || (n && !c)) return false;
  for (uint32_t i = 0; i < n; ++i) {
    if (c[i].reg >= st->width.size() || c[i].bit >= st->width[c[i].reg] || c[i].value > 1)
      return false;
    const uint32_t q = st->offset[c[i].reg] + c[i].bit;
    mask[q >> 6] |= 1ull << (q & 63);
    if (c[i].value) val[q >> 6] |= 1ull << (q & 63);
  }
  return true;
}

bool ctrl_touches(const uint64_t mask[2], uint32_t q) { return (mask[q >> 6] >> (q & 63)) & 1; }

// Reads the control block (waits for the stream) and converts device errors.
// With report_only, a device error is returned without becoming sticky.
sqs_status sync_ctl(sqs_state* st, bool report_only = false) {
  if (st->capturing) {
    st->capture_err = SQS_ERR_STATE;
    return fail(st, SQS_ERR_STATE, "a host wait inside a graph capture (raise the static bound)");
  }
  cudaError_t e = cudaMemcpyAsync(st->ctl_host, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                  st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "synchronize");
  st->stats.host_waits++;
  const Ctl& c = *st->ctl_host;
  if (c.err && report_only) return SQS_ERR_CAPACITY;
  if (c.err) {
    st->sticky = (c.err & sqs::kErrProbe) ? SQS_ERR_TIMEOUT : SQS_ERR_CAPACITY;
    return fail(st, st->sticky,
                "device error 0x%x at launch %u (needed %llu branches); reset the state", c.err,
                c.err_where, (unsigned long long)c.need);
  }
  st->ub = c.cnt[st->cur_slot];
  return SQS_OK;
}

// Replaces the count bound by the exact count, mid-step.  Inside a learned-
// sizing flush a pending bucket overflow must reach the flush, which rolls
// back and replays; anywhere else a device error is sticky.
sqs_status sync_bound(sqs_state* st) {
  sqs_status s = sync_ctl(st, true);
  if (s == SQS_OK) return s;
  if (st->defer_frees && (st->ctl_host->err & ~sqs::kErrBucket) == 0) return s;
  return sync_ctl(st);
}

sqs_status check_usable(sqs_state* st) {
  if (!st) return SQS_ERR_ARG;
  return st->sticky;
}

// Calls that wait for the device or copy to or from host memory cannot be
// part of a graph capture.
sqs_status no_capture(sqs_state* st, const char* what) {
  if (!st) return SQS_ERR_ARG;
  if (!st->capturing) return SQS_OK;
  st->capture_err = SQS_ERR_STATE;
  return fail(st, SQS_ERR_STATE, "%s inside a graph capture", what);
}

// Folds the amplitude factors of one group of MUL ops into entries
// [n_tab, n_tab + 2^bits) of the factor table: entry idx is the product, in
// operation order, of the factors idx selects (2-bit or 1-bit fields).
struct Group {
  std::vector<const HostOp*> ops;
  std::vector<uint32_t> shift, nbits;
  uint32_t bits = 0;
};

void fold_group(Group& g, OpList& L) {
  if (g.ops.empty()) return;
  const uint32_t size = 1u << g.bits;
  for (uint32_t idx = 0; idx < size; ++idx) {
    std::complex<double> f(1.0, 0.0);
    for (size_t j = 0; j < g.ops.size(); ++j) {
      const uint32_t oc = (idx >> g.shift[j]) & ((1u << g.nbits[j]) - 1u);
      if (oc == 1) f *= g.ops[j]->c0;
      else if (oc == 2) f *= g.ops[j]->c1;
    }
    L.tab[L.n_tab + idx] = make_double2(f.real(), f.imag());
  }
  DevOp t;
  std::memset(&t, 0, sizeof(t));
  t.kind = sqs::OP_TABLE;
  t.sel_bit = 128;
  t.tab_off = L.n_tab;
  L.op[L.n++] = t;
  L.n_tab += size;
  g = Group{};
}

// Packs pending ops [from, ...) into one launch's list; returns how many
// were consumed (the list or its factor table filled up, or all done).
size_t pack_ops(const std::vector<HostOp>& ops, size_t from, OpList& L) {
  L.n = 0;
  L.n_tab = 0;
  L.touches_keys = L.touches_amps = L.drops = 0;
  Group g;
  size_t i = from;
  constexpr uint32_t kGroupBits = 10;
  for (; i < ops.size(); ++i) {
    const HostOp& h = ops[i];
    const uint32_t kind = h.d.kind;
    const bool mul = kind == sqs::OP_MUL || kind == sqs::OP_MUL_XOR;
    const uint32_t nb = mul ? (h.d.sel_bit < 128 ? 2u : 1u) : 0u;
    // Room for this op, the table ops still to come, and the factor table.
    const bool closes = (mul && g.bits + nb > kGroupBits) || kind == sqs::OP_PRUNE;
    const uint32_t pend_tab = g.ops.empty() ? 0 : (1u << g.bits);
    uint32_t need_tab = L.n_tab + pend_tab;
    if (mul) need_tab = closes ? need_tab + (1u << nb) : L.n_tab + (1u << (g.bits + nb));
    const uint32_t groups_after = (closes || g.ops.empty() ? 0u : 1u) + (mul ? 1u : 0u) +
                                  (closes && !g.ops.empty() ? 1u : 0u);
    if (L.n + 1 + groups_after > (uint32_t)sqs::kMaxOps || need_tab > (uint32_t)sqs::kTabEntries)
      break;
    if (closes) fold_group(g, L);
    DevOp d = h.d;
    if (mul) {
      d.shift = g.bits;
      g.ops.push_back(&h);
      g.shift.push_back(g.bits);
      g.nbits.push_back(nb);
      g.bits += nb;
      L.touches_amps = 1;
      if (kind == sqs::OP_MUL_XOR) L.touches_keys = 1;
    } else if (kind == sqs::OP_PRUNE) {
      L.drops = 1;
    } else {
      L.touches_keys = 1;
    }
    L.op[L.n++] = d;
  }
  fold_group(g, L);
  return i - from;
}

// Standalone pass over the current state with the packed list.
sqs_status run_list(sqs_state* st, const OpList& L) {
  cudaError_t e = cudaSuccess;
  const uint64_t in_slots = st->cur.slots(st->ub);
  if (L.drops) {
    // Output segment c holds what survives of input segment c (segmented
    // input, segments of any size) or of dense chunk c.
    const uint32_t seg_log2 =
        st->cur.segmented ? std::max<uint32_t>(kSegLog2, st->cur.seg_log2) : kSegLog2;
    const uint64_t chunks =
        st->cur.segmented ? std::max<uint64_t>(1, st->cur.n_seg)
                          : std::max<uint64_t>(1, (in_slots + (1ull << kSegLog2) - 1) >> kSegLog2);
    if (chunks > 0xffffffffull) return st->sticky = fail(st, SQS_ERR_CAPACITY, "state too large");
    if (!ensure_store(st, st->alt, chunks << seg_log2))
      return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                               (unsigned long long)(chunks << seg_log2));
    st->alt.set_segments(seg_log2, (uint32_t)chunks);
    const int out_slot = (st->cur_slot + 1) & 3;
    {
      Traced tr(st, SQS_K_COMPACT);
      e = sqs::launch_apply_compact(launch_of(st, in_slots), st->kw, st->amp32, st->ctl,
                                    st->cur.view(), st->cur_slot, st->alt.view(), out_slot, L);
    }
    std::swap(st->cur, st->alt);
    st->cur_slot = out_slot;
  } else if (L.touches_keys || L.touches_amps) {
    Traced tr(st, SQS_K_APPLY);
    e = sqs::launch_apply_inplace(launch_of(st, in_slots), st->kw, st->amp32, st->ctl,
                                  st->cur.view(), st->cur_slot, L);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "launch");
  return SQS_OK;
}

// Runs queued operations as standalone passes.  With keep_tail, the last
// launch-sized group is left packed in st->ops_buf for the kernel that
// follows to fuse; otherwise everything runs.
sqs_status flush_run(sqs_state* st);

sqs_status run_pending(sqs_state* st, bool keep_tail) {
  if (!st->run_gates.empty()) {
    sqs_status s = flush_run(st);  // the held run precedes everything queued
    if (s != SQS_OK) return s;
  }
  OpList& L = st->ops_buf;
  size_t from = 0;
  for (;;) {
    const size_t used = pack_ops(st->pending, from, L);
    const bool last = from + used >= st->pending.size();
    if (last && keep_tail) break;
    sqs_status s = run_list(st, L);
    if (s != SQS_OK) return s;
    from += used;
    if (last) {
      L.n = 0;
      L.n_tab = 0;
      L.touches_keys = L.touches_amps = L.drops = 0;
      break;
    }
  }
  st->pending.clear();
  return SQS_OK;
}

sqs_status densify(sqs_state* st);

// One interference step whose target bit is constant over the state: no
// pair exists, so k_expand writes both children of every controlled branch
// in one pass (the constant-bit path of the merge).
sqs_status run_expand(sqs_state* st, const Gate1& g, int64_t rec_idx) {
  const OpList& L = st->ops_buf;
  constexpr uint32_t kChunkLog2 = 12;  // input slots per chunk of the kernel
  // Output bound: an expansion at most doubles the branches, a fold keeps
  // their number (each pair's two members become its two children).
  auto out_bound = [&] {
    return g.fold_sign ? st->ub : std::min(max_branches(st), 2 * st->ub);
  };
  uint64_t need = std::max<uint64_t>(bound_after(st, out_bound()), 1);
  if (need > st->alt.cap && st->ub > 1) {
    sqs_status s = sync_bound(st);  // the bound outgrew the allocation: exact count
    if (s != SQS_OK) return s;
    need = std::max<uint64_t>(bound_after(st, out_bound()), 1);
  }
  const uint64_t in_slots = st->cur.slots(st->ub);
  const uint64_t chunks =
      st->cur.segmented
          ? std::max<uint64_t>(1, (uint64_t)st->cur.n_seg << (st->cur.seg_log2 - kChunkLog2))
          : std::max<uint64_t>(1, (st->ub + (1ull << kChunkLog2) - 1) >> kChunkLog2);
  if (st->alt.cap < need && !ensure_store(st, st->alt, need))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)need);
  st->alt.set_dense();
  const int out_slot = (st->cur_slot + 1) & 3;
  cudaError_t e;
  {
    Traced tr(st, g.fold_sign ? SQS_K_FOLD : SQS_K_EXPAND);
    const bool fold_only = g.fold_sign != 0 && g.cmask[0] == 0 && g.cmask[1] == 0;
    e = fold_only
            ? sqs::launch_fold(launch_of(st, in_slots), st->kw, st->amp32, st->ctl,
                               st->cur.view(), st->cur_slot, chunks, L, g, st->alt.view(),
                               out_slot)
            : sqs::launch_expand(launch_of(st, in_slots), st->kw, st->amp32, st->ctl,
                                 st->cur.view(), st->cur_slot, chunks, L, g, st->alt.view(),
                                 out_slot);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "expand launch");
  if (rec_idx >= 0) {
    e = sqs::launch_record(launch_of(st, 1), st->ctl, st->cur_slot, out_slot,
                           st->rec_dev + 2 * (size_t)rec_idx);
    if (e != cudaSuccess) return cuda_fail(st, e, "record launch");
  }
  std::swap(st->cur, st->alt);
  st->cur_slot = out_slot;
  st->ub = bound_after(st, out_bound());
  return SQS_OK;
}

// One interference step on the binned cluster path: k_bin then
// k_pair_cluster.  The fused run is already packed in st->ops_buf.
sqs_status run_binned(sqs_state* st, const Gate1& g, uint64_t B1, int64_t rec_idx) {
  const OpList& L = st->ops_buf;
  const uint32_t bin_log2 = (uint32_t)sqs::cluster_bin_log2();
  const uint32_t seg_log2 = (uint32_t)sqs::cluster_out_seg_log2();
  const uint64_t ctas = (uint64_t)sqs::cluster_ctas();
  const uint64_t Bcap = std::max<uint64_t>(B1, (st->grow_hint_b * kBucketFill) >> bin_log2);
  // One extra slice of padding: a bulk copy rounds its size up to 16 bytes.
  const uint64_t bin_need = (B1 << bin_log2) + 4096;
  const uint64_t out_need = (B1 * ctas) << seg_log2;
  if ((st->bk.cap < bin_need && !ensure_store(st, st->bk, ((Bcap << bin_log2) + 4096))) ||
      (st->alt.cap < out_need && !ensure_store(st, st->alt, (Bcap * ctas) << seg_log2)))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)out_need);
  st->bk.set_segments(bin_log2, (uint32_t)B1);
  st->alt.set_segments(seg_log2, (uint32_t)(B1 * ctas));
  const uint64_t in_slots = st->cur.slots(st->ub);
  const int out_slot = (st->cur_slot + 1) & 3;
  cudaError_t e;
  {
    Traced tr(st, SQS_K_BIN);
    e = sqs::launch_bin(launch_of(st, in_slots), st->kw, st->amp32, st->ctl, st->cur.view(),
                        st->cur_slot, L, g, st->bk.view());
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "bin launch");
  {
    Traced tr(st, SQS_K_PAIR_CLUSTER);
    e = sqs::launch_pair_cluster(launch_of(st, in_slots), st->kw, st->amp32, st->ctl, g,
                                 st->bk.view(), st->alt.view(), out_slot);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "cluster pair launch");
  if (rec_idx >= 0) {
    e = sqs::launch_record(launch_of(st, 1), st->ctl, st->cur_slot, out_slot,
                           st->rec_dev + 2 * (size_t)rec_idx);
    if (e != cudaSuccess) return cuda_fail(st, e, "record launch");
  }
  std::swap(st->cur, st->alt);
  st->cur_slot = out_slot;
  st->ub = bound_after(st, std::min(max_branches(st), 2 * st->ub));
  return SQS_OK;
}

// One interference step: fused pending run + partition + pair.  est_in < 0:
// buckets sized from the hard bound st->ub (exact mode); otherwise from the
// predicted input count est_in with a 20% margin (learned mode).
// One interference step on the per-CTA bucket merge (k_partition, k_pair),
// or on the binned cluster merge when requested.  The fused run is already
// packed in st->ops_buf.
sqs_status run_hashed(sqs_state* st, const Gate1& g, double est_in, int64_t rec_idx) {
  sqs_status s;
  const OpList& L = st->ops_buf;
  // A capture sized its buckets for the static bound at the eager fill, so a
  // replay partitions exactly as eager issue does.
  const uint64_t target = bucket_fill(st->ub);
  uint64_t want =
      est_in < 0 ? st->ub : std::min<uint64_t>(st->ub, (uint64_t)(est_in * 1.2) + 1);
  // The per-CTA bucket merge is the default (measured faster at every size
  // of the benchmark workload); the binned cluster merge runs when requested
  // and the state fits the bins one launch carries.
  const uint64_t bin_target = (3ull << sqs::cluster_bin_log2()) / 4;
  auto plan = [&](uint64_t w, uint64_t& B, uint64_t& B1) {
    B = std::max<uint64_t>(1, (w + target - 1) / target);
    B1 = std::max<uint64_t>(1, (w + bin_target - 1) / bin_target);
    const bool binned = (st->flags & SQS_MERGE_CLUSTER) && B1 <= (uint64_t)sqs::kMaxBins;
    return binned ? ((B1 * sqs::cluster_ctas()) << sqs::cluster_out_seg_log2())
                  : (B << kSegLog2);
  };
  uint64_t B, B1;
  uint64_t need = plan(want, B, B1);
  if (need > st->alt.cap && st->ub > 1) {
    // The bound (exact mode) or the estimate (learned mode) outgrew the
    // allocation: learn the exact count first.
    s = est_in < 0 ? sync_ctl(st) : sync_bound(st);
    if (s != SQS_OK) return s;
    want = st->ub;
    need = plan(want, B, B1);
  }
  if (B > 0x7fffffffull) return st->sticky = fail(st, SQS_ERR_CAPACITY, "too many buckets");
  if ((st->flags & SQS_MERGE_CLUSTER) && B1 <= (uint64_t)sqs::kMaxBins) {
    st->stats.steps_cluster++;
    return run_binned(st, g, B1, rec_idx);
  }
  st->stats.steps_hash++;
  // Learned mode grows buffers straight to the predicted peak (grow_hint_b),
  // or to this step's size when a predicted peak cannot be allocated.
  const uint64_t Bcap = std::max(B, st->grow_hint_b);
  auto grow = [&](uint64_t bc) {
    return (st->bk.cap >= (B << kBucketLog2) || ensure_store(st, st->bk, bc << kBucketLog2)) &&
           (st->alt.cap >= (B << kSegLog2) || ensure_store(st, st->alt, bc << kSegLog2));
  };
  if (!grow(Bcap) && (Bcap == B || !grow(B)))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)(B << kSegLog2));
  st->bk.set_segments(kBucketLog2, (uint32_t)B);
  st->alt.set_segments(kSegLog2, (uint32_t)B);

  const uint64_t in_slots = st->cur.slots(st->ub);
  const int out_slot = (st->cur_slot + 1) & 3;
  cudaError_t e;
  {
    Traced tr(st, SQS_K_PARTITION);
    e = sqs::launch_partition(launch_of(st, in_slots), st->kw, st->amp32, st->ctl,
                              st->cur.view(), st->cur_slot, L, g, st->bk.view(), (uint32_t)target);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "partition launch");
  {
    Traced tr(st, SQS_K_PAIR);
    e = sqs::launch_pair(launch_of(st, in_slots), st->kw, st->amp32, st->ctl, g, st->bk.view(),
                         st->alt.view(), out_slot);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "pair launch");
  if (rec_idx >= 0) {
    e = sqs::launch_record(launch_of(st, 1), st->ctl, st->cur_slot, out_slot,
                           st->rec_dev + 2 * (size_t)rec_idx);
    if (e != cudaSuccess) return cuda_fail(st, e, "record launch");
  }
  std::swap(st->cur, st->alt);
  st->cur_slot = out_slot;
  st->ub = bound_after(st, std::min(max_branches(st), 2 * st->ub));
  return SQS_OK;
}

// Digit windows of the radix-sort merge: start positions (in the pair-class
// key, the key with bit t deleted) of 8-bit digits covering every bit not
// known constant.  Known-constant bits order nothing and are skipped.
std::vector<uint32_t> sort_shifts(const sqs_state* st, const Gate1& g,
                                  uint32_t D = (uint32_t)sqs::sort_radix_bits()) {
  const uint32_t nb = st->total_bits;  // the class key has nb - 1 bits
  auto varying = [&](uint32_t q) {  // bit q of the class key
    const uint32_t kb = q < g.t ? q : q + 1;
    return ((g.vary[kb >> 6] >> (kb & 63)) & 1ull) != 0ull;
  };
  std::vector<uint32_t> shifts;
  for (uint32_t q = 0; q + 1 < nb;) {
    if (!varying(q)) {
      ++q;
      continue;
    }
    shifts.push_back(q);
    q += D;
  }
  if (shifts.empty()) shifts.push_back(0);  // one pass still applies the fused run
  return shifts;
}

// Scratch of the radix-sort passes: per-tile digit histograms, scan
// partials and the device count.
sqs_status sort_scratch(sqs_state* st, uint64_t tiles, unsigned int*& hist, unsigned int*& part,
                        unsigned long long*& n_dev, int radix_bits) {
  const uint64_t radix = 1ull << radix_bits;
  const size_t hist_bytes = (size_t)(radix * tiles * 4 + 255) & ~(size_t)255;
  const size_t part_bytes = (sqs::sort_part_entries() * 4 + 255) & ~(size_t)255;
  const size_t bytes = hist_bytes + part_bytes + 256;
  if (st->sort_bytes < bytes) {
    dfree(st, st->sort_buf);
    st->sort_buf = (unsigned char*)dalloc(st, bytes);
    st->sort_bytes = st->sort_buf ? bytes : 0;
    if (!st->sort_buf) return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate sort scratch");
  }
  hist = (unsigned int*)st->sort_buf;
  part = (unsigned int*)(st->sort_buf + hist_bytes);
  n_dev = (unsigned long long*)(st->sort_buf + hist_bytes + part_bytes);
  return SQS_OK;
}

// ---- autotuner (SQS_AUTOTUNE) ---------------------------------------------------
// Bits a sort orders: the positions in `keep` not known constant.
uint32_t bits_to_sort(const sqs_state* st, const uint64_t keep[2]) {
  uint32_t n = 0;
  for (uint32_t q = 0; q < st->total_bits; ++q)
    if (((keep[q >> 6] >> (q & 63)) & 1ull) && st->const_val[q] < 0) ++n;
  return n;
}

constexpr uint32_t kTuneSortBits = 1;    // radix digit width of a sort
constexpr uint32_t kTuneGroupSlots = 2;  // output slots per CTA tile of a fused run
constexpr int kTuneSamples = 2;          // timed runs per candidate

uint32_t log2_ceil(uint64_t v) {
  uint32_t lg = 0;
  while (lg < 63 && (1ull << lg) < v) ++lg;
  return lg;
}

// Picks the value for `key` among `cand` (cand[0] is the default, used when
// tuning is off).  While measuring, returns the candidate with the fewest
// samples and sets `timed`: the caller brackets its launches with
// tune_begin / tune_end.  A measurement still in flight is collected once its
// end event has completed (never waiting for it).
int tune_pick(sqs_state* st, const sqs_state::TuneKey& key, const std::vector<int>& cand,
              bool& timed) {
  timed = false;
  if (!(st->flags & SQS_AUTOTUNE) || st->capturing) {
    auto it = st->tuner.find(key);
    return (it != st->tuner.end() && it->second.choice >= 0) ? it->second.choice : cand[0];
  }
  sqs_state::TuneEntry& E = st->tuner[key];
  if (E.choice >= 0) return E.choice;
  if (E.cand.empty()) {
    E.cand = cand;
    E.ms.assign(cand.size(), {});
  }
  if (E.pending >= 0) {
    if (cudaEventQuery(E.ev[1]) != cudaSuccess) {
      cudaGetLastError();
      return E.cand[0];  // the last measurement is still running
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, E.ev[0], E.ev[1]) == cudaSuccess)
      E.ms[E.pending].push_back(ms);
    cudaGetLastError();
    E.pending = -1;
  }
  size_t pick = 0;
  for (size_t i = 1; i < E.cand.size(); ++i)
    if (E.ms[i].size() < E.ms[pick].size()) pick = i;
  if (E.ms[pick].size() >= (size_t)kTuneSamples) {
    double best = 1e300;
    for (size_t i = 0; i < E.cand.size(); ++i) {
      std::vector<float> v = E.ms[i];
      std::sort(v.begin(), v.end());
      const double med = v[v.size() / 2];
      if (med < best) {
        best = med;
        E.choice = E.cand[i];
      }
    }
    return E.choice;
  }
  if (!E.ev[0] && (cudaEventCreate(&E.ev[0]) != cudaSuccess ||
                   cudaEventCreate(&E.ev[1]) != cudaSuccess)) {
    cudaGetLastError();
    return E.cand[0];
  }
  E.pending = (int)pick;
  timed = true;
  return E.cand[pick];
}
void tune_begin(sqs_state* st, const sqs_state::TuneKey& key) {
  cudaEventRecord(st->tuner[key].ev[0], st->stream);
}
void tune_end(sqs_state* st, const sqs_state::TuneKey& key) {
  cudaEventRecord(st->tuner[key].ev[1], st->stream);
}

// Digit width of a sort over the kept, varying key bits (tuned per key
// words, amplitude type, size and number of bits to sort).
int pick_sort_bits(sqs_state* st, uint64_t n, uint32_t bits_to_sort, sqs_state::TuneKey& key,
                   bool& timed) {
  key = sqs_state::TuneKey{kTuneSortBits, (uint32_t)st->kw, st->amp32 ? 1u : 0u, log2_ceil(n),
                           bits_to_sort};
  if (st->forced_sort_bits) {
    timed = false;
    return st->forced_sort_bits;
  }
  return tune_pick(st, key, {sqs::sort_radix_bits(), 10, 11, 6}, timed);
}

std::string tune_json(const sqs_state* st) {
  std::ostringstream o;
  o << "{\"gpu\": \"" << st->gpu_name << "\", \"entries\": [";
  bool first = true;
  for (const auto& kv : st->tuner) {
    const auto& k = kv.first;
    const auto& E = kv.second;
    if (E.cand.empty()) continue;
    o << (first ? "" : ", ") << "{\"site\": \""
      << (k.site == kTuneSortBits ? "sort_bits" : "group_slots") << "\", \"kw\": " << k.kw
      << ", \"amp32\": " << k.amp32 << ", \"n_log2\": " << k.n_log2 << ", \"extra\": " << k.extra
      << ", \"choice\": " << E.choice << ", \"cand\": [";
    for (size_t i = 0; i < E.cand.size(); ++i) o << (i ? ", " : "") << E.cand[i];
    o << "], \"median_ms\": [";
    for (size_t i = 0; i < E.cand.size(); ++i) {
      std::vector<float> v = E.ms[i];
      std::sort(v.begin(), v.end());
      o << (i ? ", " : "") << (v.empty() ? -1.0 : (double)v[v.size() / 2]);
    }
    o << "]}";
    first = false;
  }
  o << "]}";
  return o.str();
}

// Integer value of "name": in [p, end) of one entry.
bool json_int(const char* p, const char* end, const char* name, long long& v) {
  const std::string pat = std::string("\"") + name + "\":";
  const char* q = std::search(p, end, pat.begin(), pat.end());
  if (q == end) return false;
  q += pat.size();
  while (q < end && *q == ' ') ++q;
  char* stop = nullptr;
  v = std::strtoll(q, &stop, 10);
  return stop != q;
}

// Loads entries measured on this GPU (the export's format).
void tune_load(sqs_state* st, const char* json) {
  const char* end = json + std::strlen(json);
  const std::string gpat = "\"gpu\": \"";
  const char* g = std::search(json, end, gpat.begin(), gpat.end());
  if (g == end) return;
  g += gpat.size();
  const char* ge = std::find(g, end, '"');
  if (std::string(g, ge) != st->gpu_name) return;
  const std::string epat = "{\"site\": \"";
  for (const char* p = std::search(ge, end, epat.begin(), epat.end()); p != end;) {
    const char* q = p + epat.size();
    const char* e = std::find(q, end, '}');
    const char* next = std::search(e, end, epat.begin(), epat.end());
    const std::string site(q, std::find(q, e, '"'));
    long long kw, amp32, nl, extra, choice;
    if (json_int(q, e, "kw", kw) && json_int(q, e, "amp32", amp32) &&
        json_int(q, e, "n_log2", nl) && json_int(q, e, "extra", extra) &&
        json_int(q, e, "choice", choice) && choice >= 0) {
      const uint32_t s = site == "sort_bits" ? kTuneSortBits
                         : site == "group_slots" ? kTuneGroupSlots : 0u;
      if (s && (s != kTuneSortBits || sqs::sort_radix_bits_ok((int)choice))) {
        sqs_state::TuneEntry& E = st->tuner[sqs_state::TuneKey{
            s, (uint32_t)kw, (uint32_t)amp32, (uint32_t)nl, (uint32_t)extra}];
        E.choice = (int)choice;
        // The candidate list, kept for the export ("cand": [a, b, ...]).
        E.cand.clear();
        const std::string cpat = "\"cand\": [";
        const char* c = std::search(q, e, cpat.begin(), cpat.end());
        if (c != e) {
          c += cpat.size();
          const char* ce = std::find(c, e, ']');
          while (c < ce) {
            char* stop = nullptr;
            const long v = std::strtol(c, &stop, 10);
            if (stop == c) break;
            E.cand.push_back((int)v);
            c = stop;
            while (c < ce && (*c == ',' || *c == ' ')) ++c;
          }
        }
        if (E.cand.empty()) E.cand.push_back((int)choice);
        E.ms.assign(E.cand.size(), {});
      }
    }
    p = next;
  }
}

// One interference step on the radix-sort merge: LSD passes ping-pong
// between the two scratch stores so that the sorted array always ends in
// st->bk, whose segment counters stay untouched (zero) for the bucket merge;
// the merge writes st->alt, which becomes the state.
sqs_status run_sorted(sqs_state* st, const Gate1& g, int64_t rec_idx) {
  const OpList& L = st->ops_buf;
  {
    // Tiles, histograms and buffers follow the count bound: a bound that
    // outgrew the allocation is replaced by the exact count first.
    const uint64_t c = 1ull << sqs::sort_merge_chunk_log2();
    const uint64_t out_need = std::max<uint64_t>(1, (st->ub + c - 1) / c) * 2 * c;
    if (st->ub > 1 && (st->bk.cap < st->ub || st->alt.cap < std::max(out_need, st->ub))) {
      sqs_status s = sync_bound(st);
      if (s != SQS_OK) return s;
    }
  }
  uint64_t all_bits[2] = {~0ull, ~0ull};
  all_bits[g.t >> 6] &= ~(1ull << (g.t & 63));
  sqs_state::TuneKey tkey;
  bool timed = false;
  const int rb = pick_sort_bits(st, st->ub, bits_to_sort(st, all_bits), tkey, timed);
  const std::vector<uint32_t> shifts = sort_shifts(st, g, (uint32_t)rb);
  const uint32_t npass = (uint32_t)shifts.size();
  const uint64_t tile = (uint64_t)sqs::sort_tile();
  const uint64_t in_slots = st->cur.slots(st->ub);
  uint32_t per_seg = 1;
  uint64_t tiles0;
  if (st->cur.segmented) {
    per_seg = (uint32_t)std::max<uint64_t>(1, ((1ull << st->cur.seg_log2) + tile - 1) / tile);
    tiles0 = std::max<uint64_t>(1, (uint64_t)st->cur.n_seg * per_seg);
  } else {
    tiles0 = std::max<uint64_t>(1, (st->ub + tile - 1) / tile);
  }
  const uint64_t tilesN = std::max<uint64_t>(1, (st->ub + tile - 1) / tile);
  unsigned int *hist, *part;
  unsigned long long* n_dev;
  {
    sqs_status s = sort_scratch(st, std::max(tiles0, tilesN), hist, part, n_dev, rb);
    if (s != SQS_OK) return s;
  }
  const uint32_t chunk_log2 = sqs::sort_merge_chunk_log2();
  const uint64_t nseg_out = std::max<uint64_t>(1, (st->ub + (1ull << chunk_log2) - 1) >> chunk_log2);
  if (nseg_out > 0xffffffffull) return st->sticky = fail(st, SQS_ERR_CAPACITY, "state too large");
  const uint64_t out_need = nseg_out << (chunk_log2 + 1);
  if ((st->bk.cap < st->ub && !ensure_store(st, st->bk, st->ub)) ||
      (st->alt.cap < std::max(out_need, st->ub) &&
       !ensure_store(st, st->alt, std::max(out_need, st->ub))))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)out_need);
  // Pass p writes buf[p & 1]; the last pass lands in bk.
  Store* buf[2];
  buf[0] = (npass & 1) ? &st->bk : &st->alt;
  buf[1] = (npass & 1) ? &st->alt : &st->bk;
  const unsigned long long* n_ptr = &st->ctl->cnt[st->cur_slot];
  Arr src = st->cur.view();
  cudaError_t e = cudaSuccess;
  if (timed) tune_begin(st, tkey);
  for (uint32_t p = 0; p < npass && e == cudaSuccess; ++p) {
    Store& dst = *buf[p & 1];
    dst.set_dense();
    Traced tr(st, SQS_K_SORT);
    e = sqs::launch_rsort_pass(launch_of(st, in_slots), st->kw, st->amp32, st->ctl, src, n_ptr,
                               p == 0 ? per_seg : 1u, p == 0 ? tiles0 : tilesN,
                               p == 0 ? &L : nullptr, g.t, shifts[p], hist, part, n_dev,
                               dst.view(), nullptr, rb);
    st->launches += 3;  // a pass is four kernels: histogram, two scan steps, scatter
    src = dst.view();
    n_ptr = n_dev;
  }
  if (timed) tune_end(st, tkey);
  if (e != cudaSuccess) return cuda_fail(st, e, "sort pass launch");
  const int out_slot = (st->cur_slot + 1) & 3;
  st->alt.set_segments(chunk_log2 + 1, (uint32_t)nseg_out);
  {
    Traced tr(st, SQS_K_SORT_MERGE);
    e = sqs::launch_rsort_merge(launch_of(st, in_slots), st->kw, st->amp32, st->ctl,
                                st->bk.view(), n_dev, g, st->alt.view(), out_slot);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "sort merge launch");
  st->bk.set_dense();
  if (rec_idx >= 0) {
    e = sqs::launch_record(launch_of(st, 1), st->ctl, st->cur_slot, out_slot,
                           st->rec_dev + 2 * (size_t)rec_idx);
    if (e != cudaSuccess) return cuda_fail(st, e, "record launch");
  }
  std::swap(st->cur, st->alt);
  st->cur_slot = out_slot;
  st->ub = bound_after(st, std::min(max_branches(st), 2 * st->ub));
  return SQS_OK;
}

// SQS_MERGE_TUNED: which merge this step takes, and whether it is timed.
// A size class is the log2 of the count bound with the sort pass count;
// its first steps time each path once (CUDA events, per slot visited),
// the rest take the faster.  A pending measurement is read only when its
// events have completed, so the choice never waits on the device.
int tuned_path(sqs_state* st, uint32_t key, bool& timed) {
  sqs_state::Tune& T = st->tune[key];
  timed = false;
  if (T.pending >= 0) {
    if (cudaEventQuery(T.ev[1]) != cudaSuccess) {
      cudaGetLastError();  // not ready: no new measurement this step
      return T.us_per_slot[1] >= 0.f && T.us_per_slot[1] < T.us_per_slot[0] ? 1 : 0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, T.ev[0], T.ev[1]);
    T.us_per_slot[T.pending] = 1e3f * ms / (float)std::max<uint64_t>(1, T.slots);
    T.pending = -1;
  }
  for (int p = 0; p < 2; ++p) {
    if (T.us_per_slot[p] < 0.f) {
      if (!T.ev[0] && (cudaEventCreate(&T.ev[0]) != cudaSuccess ||
                       cudaEventCreate(&T.ev[1]) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
      }
      timed = true;
      return p;
    }
  }
  return T.us_per_slot[1] < T.us_per_slot[0] ? 1 : 0;
}

// Attributes the launches of a step to the API call that issued it while in
// scope (a held step runs during a later call).
struct TraceCall {
  sqs_state* st;
  uint32_t saved;
  TraceCall(sqs_state* s, uint32_t call) : st(s), saved(s->trace_call) {
    if (call) st->trace_call = call;
  }
  ~TraceCall() { st->trace_call = saved; }
};

sqs_status run_branching(sqs_state* st, const Gate1& g, double est_in = -1.0,
                         int64_t rec_idx = -1) {
  TraceCall attribution(st, g.issue_call);
  sqs_status s = SQS_OK;
  if (g.defer_ops && st->run_gates.empty()) {
    // The queued operations stay queued past this step (defer_ops_ok).
    st->ops_buf.n = 0;
    st->ops_buf.n_tab = 0;
    st->ops_buf.touches_keys = st->ops_buf.touches_amps = st->ops_buf.drops = 0;
    st->stats.ops_deferred += st->pending.size();
  } else {
    s = run_pending(st, true);  // leaves the fused tail in ops_buf
    if (s != SQS_OK) return st->sticky = s;
  }
  if (g.no_partners || g.fold_sign) {
    if (g.fold_sign) st->stats.steps_fold++;
    else st->stats.steps_expand++;
    return run_expand(st, g, rec_idx);
  }
  const bool sort_ok = st->ub < (1ull << 31) && !(st->flags & SQS_MERGE_CLUSTER);
  int path = 0;
  bool timed = false;
  uint32_t key = 0;
  if (sort_ok && (st->flags & SQS_MERGE_SORT)) {
    path = 1;
  } else if (sort_ok && (st->flags & SQS_MERGE_TUNED)) {
    uint32_t lg = 0;
    while (lg < 63 && (1ull << lg) < st->ub) ++lg;
    key = lg | ((uint32_t)sort_shifts(st, g).size() << 8);
    path = tuned_path(st, key, timed);
  }
  if (timed) {
    sqs_state::Tune& T = st->tune[key];
    T.slots = st->cur.slots(st->ub);
    cudaEventRecord(T.ev[0], st->stream);
  }
  if (path == 1) {
    st->stats.steps_sort++;
    s = run_sorted(st, g, rec_idx);
  } else {
    s = run_hashed(st, g, est_in, rec_idx);
  }
  if (timed && s == SQS_OK) {
    sqs_state::Tune& T = st->tune[key];
    cudaEventRecord(T.ev[1], st->stream);
    T.pending = path;
  }
  return s;
}

// Digit windows of a fused run's sort: 8-bit windows over the key bits that
// are neither targets of the run nor known constant (the sort key is the key
// with the targets cleared; constant bits order nothing).
std::vector<uint32_t> group_shifts(const sqs_state* st, const GroupRun& run,
                                   uint32_t D = (uint32_t)sqs::sort_radix_bits()) {
  std::vector<uint32_t> shifts;
  for (uint32_t q = 0; q < st->total_bits;) {
    const bool target = (run.tmask[q >> 6] >> (q & 63)) & 1ull;
    const bool varying = (run.g[0].vary[q >> 6] >> (q & 63)) & 1ull;
    if (target || !varying) {
      ++q;
      continue;
    }
    shifts.push_back(q);
    q += D;
  }
  if (shifts.empty()) shifts.push_back(0);  // one pass still applies the queued run
  return shifts;
}

// A fused run of k >= 2 interference steps (Sec. II.D.2): the queued
// operations and a radix sort on the key with every target cleared (each
// coherent group becomes contiguous), the group count (the output holds at
// most 2^k branches per group), then every group transformed at once.
// Bit-identical to the k steps one by one.
sqs_status run_group(sqs_state* st, const std::vector<Gate1>& gates) {
  TraceCall attribution(st, gates.empty() ? 0u : gates[0].issue_call);
  sqs_status s = run_pending(st, true);  // leaves the fused operations in ops_buf
  if (s != SQS_OK) return st->sticky = s;
  const OpList& L = st->ops_buf;
  GroupRun run;
  std::memset(&run, 0, sizeof(run));
  run.k = (uint32_t)gates.size();
  for (uint32_t j = 0; j < run.k; ++j) {
    run.g[j] = gates[j];
    run.tmask[gates[j].t >> 6] |= 1ull << (gates[j].t & 63);
  }
  if (st->ub > 1 && (st->bk.cap < st->ub || st->alt.cap < st->ub)) {
    s = sync_bound(st);  // tiles and buffers follow the bound: exact count first
    if (s != SQS_OK) return s;
  }
  uint64_t keep_bits[2] = {~run.tmask[0], ~run.tmask[1]};
  sqs_state::TuneKey tkey;
  bool timed = false;
  const int rb = pick_sort_bits(st, st->ub, bits_to_sort(st, keep_bits), tkey, timed);
  const std::vector<uint32_t> shifts = group_shifts(st, run, (uint32_t)rb);
  const uint32_t npass = (uint32_t)shifts.size();
  const uint64_t tile = (uint64_t)sqs::sort_tile();
  const uint64_t in_slots = st->cur.slots(st->ub);
  uint32_t per_seg = 1;
  uint64_t tiles0;
  if (st->cur.segmented) {
    per_seg = (uint32_t)std::max<uint64_t>(1, ((1ull << st->cur.seg_log2) + tile - 1) / tile);
    tiles0 = std::max<uint64_t>(1, (uint64_t)st->cur.n_seg * per_seg);
  } else {
    tiles0 = std::max<uint64_t>(1, (st->ub + tile - 1) / tile);
  }
  const uint64_t tilesN = std::max<uint64_t>(1, (st->ub + tile - 1) / tile);
  unsigned int *hist, *part;
  unsigned long long* n_dev;
  {
    sqs_status s = sort_scratch(st, std::max(tiles0, tilesN), hist, part, n_dev, rb);
    if (s != SQS_OK) return s;
  }
  const uint64_t need_in = std::max<uint64_t>(st->ub, 1);
  if ((st->bk.cap < need_in && !ensure_store(st, st->bk, need_in)) ||
      (st->alt.cap < need_in && !ensure_store(st, st->alt, need_in)))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)need_in);
  // Pass p writes buf[p & 1]; the last pass lands in bk.
  Store* buf[2];
  buf[0] = (npass & 1) ? &st->bk : &st->alt;
  buf[1] = (npass & 1) ? &st->alt : &st->bk;
  const unsigned long long* n_ptr = &st->ctl->cnt[st->cur_slot];
  Arr src = st->cur.view();
  cudaError_t e = cudaSuccess;
  if (timed) tune_begin(st, tkey);
  for (uint32_t p = 0; p < npass && e == cudaSuccess; ++p) {
    Store& dst = *buf[p & 1];
    dst.set_dense();
    Traced tr(st, SQS_K_SORT);
    e = sqs::launch_rsort_pass(launch_of(st, in_slots), st->kw, st->amp32, st->ctl, src, n_ptr,
                               p == 0 ? per_seg : 1u, p == 0 ? tiles0 : tilesN,
                               p == 0 ? &L : nullptr, gates[0].t, shifts[p], hist, part, n_dev,
                               dst.view(), run.tmask, rb);
    st->launches += 3;  // a pass is four kernels: histogram, two scan steps, scatter
    src = dst.view();
    n_ptr = n_dev;
  }
  if (timed) tune_end(st, tkey);
  if (e != cudaSuccess) return cuda_fail(st, e, "sort pass launch");
  e = cudaMemsetAsync(&st->ctl->groups, 0,
                      sizeof(st->ctl->groups) + sizeof(st->ctl->items) + sizeof(st->ctl->stage),
                      st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "group counters");
  {
    Traced tr(st, SQS_K_GROUP_COUNT);
    e = sqs::launch_group_count(launch_of(st, st->ub), st->kw, st->ctl, st->bk.view(), n_dev,
                                run.tmask);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "group count launch");
  s = sync_ctl(st);  // the output holds at most 2^k branches per group
  if (s != SQS_OK) return s;
  const uint64_t G = st->ctl_host->groups, n = st->ctl_host->items;
  const uint64_t cap_all = max_branches(st);
  const uint64_t out_need = std::max<uint64_t>(1, G >= (cap_all >> run.k) ? cap_all : G << run.k);
  // Tiles short enough that groups which grow (up to 2^k branches each from
  // few) spread over many CTAs: about `slots` output slots per tile (2^15 by
  // default; tuned per run length and size under SQS_AUTOTUNE).
  const sqs_state::TuneKey gkey{kTuneGroupSlots, (uint32_t)st->kw, st->amp32 ? 1u : 0u,
                                log2_ceil(std::max<uint64_t>(n, 1)), run.k};
  bool gtimed = false;
  const int slots = tune_pick(st, gkey, {32768, 8192, 16384, 65536}, gtimed);
  uint32_t tile_len = sqs::kGroupTile;
  while (tile_len > 32 &&
         (double)tile_len * (double)out_need > (double)slots * (double)std::max<uint64_t>(n, 1))
    tile_len >>= 1;
  const uint64_t n_tiles = std::max<uint64_t>(1, (n + tile_len - 1) / tile_len);
  if (st->alt.cap < out_need && !ensure_store(st, st->alt, out_need))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)out_need);
  st->alt.set_dense();
  const int out_slot = (st->cur_slot + 1) & 3;
  {
    Traced tr(st, SQS_K_GROUP);
    if (gtimed) tune_begin(st, gkey);
    e = sqs::launch_group(launch_of(st, n), st->kw, st->amp32, st->ctl, st->bk.view(), n_dev,
                          tile_len, n_tiles, st->alt.view(), out_slot, run);
    if (gtimed) tune_end(st, gkey);
    st->launches++;  // the peak update after the run
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "group launch");
  st->bk.set_dense();
  std::swap(st->cur, st->alt);
  st->cur_slot = out_slot;
  st->ub = out_need;
  st->stats.runs_fused++;
  st->stats.steps_fused += run.k;
  return SQS_OK;
}

// Whether a held run is cheaper fused.  In passes over the state: the fused
// run costs its sort passes, the group count (keys only) and the group pass;
// the steps one by one cost a scatter and a merge pass each, or one pass for
// a constant-bit expansion.  Below 2^14 branches every launch is latency
// bound and the fused run's host wait does not pay.
bool fuse_pays(const sqs_state* st, const std::vector<Gate1>& gates) {
  if (st->flags & SQS_FUSE_ALWAYS) return true;
  if (st->ub < (1ull << 14)) return false;
  GroupRun run;
  std::memset(&run, 0, sizeof(run));
  run.k = (uint32_t)gates.size();
  run.g[0] = gates[0];
  for (const Gate1& g : gates) run.tmask[g.t >> 6] |= 1ull << (g.t & 63);
  double alone = 0.0;
  for (const Gate1& g : gates) alone += g.no_partners ? 1.0 : 2.0;
  const double fused = (double)group_shifts(st, run).size() + 1.5;
  return fused < alone;
}

// Executes the held run: alone (the per-step dispatch with its shortcuts) or
// fused.  Operations queued after the run stay queued after it.
sqs_status flush_run(sqs_state* st) {
  if (st->run_gates.empty()) return SQS_OK;
  std::vector<Gate1> gates;
  gates.swap(st->run_gates);
  std::vector<HostOp> after;
  after.swap(st->pending);
  st->pending.swap(st->run_pre);
  st->run_tmask[0] = st->run_tmask[1] = st->run_reads[0] = st->run_reads[1] = 0;
  sqs_status s = SQS_OK;
  if (gates.size() >= 2 && fuse_pays(st, gates)) {
    s = run_group(st, gates);
  } else {
    for (size_t j = 0; j < gates.size() && s == SQS_OK; ++j)
      s = run_branching(st, gates[j]);  // the queued operations go with the first
  }
  if (st->pending.empty()) st->pending.swap(after);
  else st->pending.insert(st->pending.end(), after.begin(), after.end());
  return s;
}

// Fused runs wait for the device (the group count sizes the output), so a
// graph capture runs every step alone.
bool fusing(const sqs_state* st) {
  return !(st->flags & (SQS_FUSE_OFF | SQS_MERGE_PLAIN | SQS_MERGE_HASH | SQS_MERGE_SORT |
                        SQS_MERGE_CLUSTER)) &&
         !st->recording && !st->capturing;
}

// Holds an interference step in the open run, or closes the run and opens a
// new one with it.  A step joins when nothing was queued since the run's
// last step, its target is new to the run and read by no step of it, and it
// reads (controls, angle register) none of the run's targets nor its own.
// A copy-pair fold always runs alone: one pass with no partition is cheaper
// than its share of a fused run.
sqs_status hold_step(sqs_state* st, const Gate1& g) {
  uint64_t reads[2] = {g.cmask[0], g.cmask[1]};
  if (g.mode == 1)
    for (uint32_t b = 0; b < g.ang_w; ++b) {
      const uint32_t q = g.ang_off + b;
      if (q < 128) reads[q >> 6] |= 1ull << (q & 63);
    }
  uint64_t tbit[2] = {0, 0};
  tbit[g.t >> 6] = 1ull << (g.t & 63);
  const bool alone = (reads[0] & tbit[0]) || (reads[1] & tbit[1]) || g.fold_sign != 0;
  const bool join = !st->run_gates.empty() && st->pending.empty() && !alone &&
                    st->run_gates.size() < (size_t)sqs::kMaxRun &&
                    !((st->run_tmask[0] | st->run_reads[0]) & tbit[0]) &&
                    !((st->run_tmask[1] | st->run_reads[1]) & tbit[1]) &&
                    !(reads[0] & st->run_tmask[0]) && !(reads[1] & st->run_tmask[1]);
  if (!join) {
    sqs_status s = flush_run(st);
    if (s != SQS_OK) return s;
    if (alone) return run_branching(st, g);
    st->run_pre.swap(st->pending);
  }
  st->run_gates.push_back(g);
  for (int w = 0; w < 2; ++w) {
    st->run_tmask[w] |= tbit[w];
    st->run_reads[w] |= reads[w];
  }
  return SQS_OK;
}

bool is_zero(double re, double im) { return re == 0.0 && im == 0.0; }

// ---- structural history (features of the learned predictor) ---------------
void history_reset(sqs_state* st, bool known_zero) {
  const uint32_t n = st->total_bits;
  st->last_branch.assign(n, -1);
  st->writes_since.assign(n, 0);
  st->reads_since.assign(n, 0);
  st->arith_since.assign(n, 0);
  st->const_val.assign(n, known_zero ? 0 : -1);
  st->pair_sign.assign(n, 0);
  st->n_branch = 0;
  st->last_target = -1;
}

template <class F>
void for_bits(const uint64_t m[2], uint32_t nbits, F f) {
  for (uint32_t q = 0; q < nbits; ++q)
    if ((m[q >> 6] >> (q & 63)) & 1ull) f(q);
}

// Every predicate bit known constant and equal to the required value?
// 1: always holds, 0: never holds, -1: unknown.
int predicate_known(const sqs_state* st, const uint64_t pm[2], const uint64_t pv[2]) {
  int res = 1;
  for (uint32_t q = 0; q < st->total_bits; ++q) {
    if (!((pm[q >> 6] >> (q & 63)) & 1ull)) continue;
    const int want = (int)((pv[q >> 6] >> (q & 63)) & 1ull);
    if (st->const_val[q] < 0) res = res == 0 ? 0 : -1;
    else if (st->const_val[q] != want) res = 0;
  }
  return res;
}

void note_field_write(sqs_state* st, uint32_t off, uint32_t w, bool arith) {
  for (uint32_t b = 0; b < w; ++b) {
    st->writes_since[off + b]++;
    st->const_val[off + b] = -1;
    if (arith) st->arith_since[off + b] = 1;
  }
}

void note_field_read(sqs_state* st, uint32_t off, uint32_t w) {
  for (uint32_t b = 0; b < w; ++b) st->reads_since[off + b]++;
}

// Updates the history for a queued non-interference operation.
void note_op(sqs_state* st, const HostOp& h) {
  const DevOp& d = h.d;
  for_bits(d.pmask, st->total_bits, [&](uint32_t q) { st->reads_since[q]++; });
  // Any bit the operation reads or writes loses its copy-pair property.
  {
    auto clear = [&](uint32_t q) {
      if (q < st->total_bits) st->pair_sign[q] = 0;
    };
    for_bits(d.pmask, st->total_bits, clear);
    switch (d.kind) {
      case sqs::OP_XOR:
        for_bits(d.xmask, st->total_bits, clear);
        break;
      case sqs::OP_MUL_XOR:
        for_bits(d.xmask, st->total_bits, clear);
        clear(d.sel_bit);
        break;
      case sqs::OP_MUL:
        clear(d.sel_bit);
        break;
      case sqs::OP_ADD_CONST:
      case sqs::OP_MUL_CONST:
        for (uint32_t b = 0; b < d.dst_w; ++b) clear(d.dst_off + b);
        break;
      case sqs::OP_MUL_ADD:
      case sqs::OP_DIV_XOR:
        for (uint32_t b = 0; b < d.dst_w; ++b) clear(d.dst_off + b);
        for (uint32_t b = 0; b < d.src_w; ++b) clear(d.src_off + b);
        for (uint32_t b = 0; b < d.src2_w; ++b) clear(d.src2_off + b);
        break;
      case sqs::OP_ADD_REG:
      case sqs::OP_SUB_REG:
      case sqs::OP_SWAP:
      case sqs::OP_QRAM:
        for (uint32_t b = 0; b < d.dst_w; ++b) clear(d.dst_off + b);
        for (uint32_t b = 0; b < d.src_w; ++b) clear(d.src_off + b);
        break;
      default:
        break;
    }
  }
  switch (d.kind) {
    case sqs::OP_XOR:
    case sqs::OP_MUL_XOR: {
      const int known = predicate_known(st, d.pmask, d.pval);
      for_bits(d.xmask, st->total_bits, [&](uint32_t q) {
        st->writes_since[q]++;
        if (st->const_val[q] >= 0) {
          if (known == 1) st->const_val[q] ^= 1;
          else if (known < 0) st->const_val[q] = -1;
        }
      });
      if (d.kind == sqs::OP_MUL_XOR && d.sel_bit < 128) st->reads_since[d.sel_bit]++;
      break;
    }
    case sqs::OP_ADD_REG:
    case sqs::OP_SUB_REG:
      note_field_read(st, d.src_off, d.src_w);
      note_field_write(st, d.dst_off, d.dst_w, true);
      break;
    case sqs::OP_ADD_CONST:
    case sqs::OP_MUL_CONST:
      note_field_write(st, d.dst_off, d.dst_w, true);
      break;
    case sqs::OP_MUL_ADD:
    case sqs::OP_DIV_XOR:
      note_field_read(st, d.src_off, d.src_w);
      note_field_read(st, d.src2_off, d.src2_w);
      note_field_write(st, d.dst_off, d.dst_w, true);
      break;
    case sqs::OP_SWAP:
      note_field_write(st, d.dst_off, d.dst_w, true);
      note_field_write(st, d.src_off, d.src_w, true);
      break;
    case sqs::OP_QRAM:
      note_field_read(st, d.src_off, d.src_w);
      note_field_write(st, d.dst_off, d.dst_w, true);
      break;
    case sqs::OP_MUL:
      if (d.sel_bit < 128) st->reads_since[d.sel_bit]++;
      break;
    default:
      break;
  }
}

void push_op(sqs_state* st, const HostOp& h) {
  note_op(st, h);
  st->pending.push_back(h);
}

// Feature vector of an interference step on key bit t (before it runs).
void features(const sqs_state* st, const Gate1& g, uint32_t n_ctrl, float* x) {
  const uint32_t t = g.t;
  const double lg = 1.0 / 4.0;
  int n_const = 0;
  for (uint32_t q = 0; q < st->total_bits; ++q) n_const += st->const_val[q] >= 0;
  bool ctrl_unknown = false;
  for_bits(g.cmask, st->total_bits, [&](uint32_t q) { ctrl_unknown |= st->const_val[q] < 0; });
  const bool branched = st->last_branch[t] >= 0;
  x[0] = (g.reuse & 0xfu) == (1u | 2u | 8u) ? 1.f : 0.f;  // H-like structure
  x[1] = g.mode == 2 ? 1.f : 0.f;
  x[2] = g.mode == 1 ? 1.f : 0.f;
  x[3] = g.mode == 0 ? 1.f : 0.f;
  x[4] = (float)n_ctrl / 4.f;
  x[5] = st->const_val[t] >= 0 ? 1.f : 0.f;
  x[6] = branched ? 1.f : 0.f;
  x[7] = branched && st->writes_since[t] == 0 && st->reads_since[t] == 0 ? 1.f : 0.f;
  x[8] = (float)(std::log2(1.0 + st->writes_since[t]) * lg);
  x[9] = (float)(std::log2(1.0 + st->reads_since[t]) * lg);
  x[10] = branched ? (float)(std::log2(1.0 + (double)(st->n_branch - st->last_branch[t])) * lg)
                   : 1.f;
  x[11] = st->total_bits ? (float)n_const / (float)st->total_bits : 0.f;
  x[12] = st->last_target == (int64_t)t ? 1.f : 0.f;
  x[13] = ctrl_unknown ? 1.f : 0.f;
  x[14] = st->arith_since[t] ? 1.f : 0.f;
  x[15] = 1.f;
}

void note_branch(sqs_state* st, const Gate1& g) {
  for_bits(g.cmask, st->total_bits, [&](uint32_t q) {
    st->reads_since[q]++;
    st->pair_sign[q] = 0;
  });
  if (g.mode == 1)
    for (uint32_t b = 0; b < g.ang_w; ++b)
      if (g.ang_off + b < st->total_bits) st->pair_sign[g.ang_off + b] = 0;
  const uint32_t t = g.t;
  st->last_branch[t] = st->n_branch++;
  st->writes_since[t] = st->reads_since[t] = 0;
  st->arith_since[t] = 0;
  st->const_val[t] = -1;
  st->last_target = t;
}

// Whether the operations queued before interference step g may stay queued
// past it.  The step must be one that can only merge: the copy-pair property
// of its target (every branch's partner present with +-1 times its
// amplitude, tracked the same way whatever merge path runs), which also
// guarantees that no queued operation reads or writes the target.  The
// queued operations must not write a control bit or an angle bit of the
// step, and none may prune.  The step is linear on the amplitudes of each
// pair and the operations permute keys and multiply amplitudes without
// touching the pair's bit, so the two orders give the same state; applied
// after the step, the operations stream half as many branches or fewer.
// Off in learned-sizing mode, whose queued steps carry their own operations.
bool defer_ops_ok(const sqs_state* st, const Gate1& g) {
  // The operations queued now are those between this step and anything held
  // before it (a held run keeps its own preceding operations), whatever the
  // merge path, so the decision is the same in every mode.
  if (st->pair_sign[g.t] == 0 || st->pending.empty()) return false;
  if (st->flags & SQS_SIZING_LEARNED) return false;
  uint64_t guard[2] = {g.cmask[0], g.cmask[1]};
  if (g.mode == 1)
    for (uint32_t b = 0; b < g.ang_w; ++b) {
      const uint32_t q = g.ang_off + b;
      if (q < 128) guard[q >> 6] |= 1ull << (q & 63);
    }
  auto field = [](uint64_t m[2], uint32_t off, uint32_t w) {
    for (uint32_t b = 0; b < w; ++b) {
      const uint32_t q = off + b;
      if (q < 128) m[q >> 6] |= 1ull << (q & 63);
    }
  };
  for (const HostOp& h : st->pending) {
    const sqs::DevOp& d = h.d;
    uint64_t w[2] = {0ull, 0ull};
    switch (d.kind) {
      case sqs::OP_PRUNE:
        return false;
      case sqs::OP_XOR:
      case sqs::OP_MUL_XOR:
        w[0] = d.xmask[0];
        w[1] = d.xmask[1];
        break;
      case sqs::OP_SWAP:
        field(w, d.dst_off, d.dst_w);
        field(w, d.src_off, d.src_w);
        break;
      case sqs::OP_MUL:
      case sqs::OP_TABLE:
        break;
      default:  // arithmetic and QRAM write their destination field
        field(w, d.dst_off, d.dst_w);
        break;
    }
    if ((w[0] & guard[0]) || (w[1] & guard[1])) return false;
  }
  return true;
}

constexpr size_t kLazyMax = 64;  // interference steps queued per learned-sizing flush
sqs_status run_lazy(sqs_state* st);

// Queues (learned mode) or runs (exact mode) one interference step.
sqs_status issue_branching(sqs_state* st, const Gate1& g_in, uint32_t n_ctrl) {
  float x[SQS_PRED_FEATURES];
  Gate1 g = g_in;
  features(st, g, n_ctrl, x);
  // Host-proven shortcuts (off under SQS_MERGE_PLAIN): a target bit known
  // constant over the whole state has no partner anywhere; a copy-paired bit
  // has every partner, holding +-1 times the branch's own amplitude.
  const bool plain = (st->flags & SQS_MERGE_PLAIN) != 0;
  const int8_t b0 = st->const_val[g.t];
  g.no_partners = (!plain && b0 >= 0) ? 1u : 0u;
  g.fold_sign = plain ? 0 : st->pair_sign[g.t];
  g.defer_ops = defer_ops_ok(st, g) ? 1u : 0u;
  g.issue_call = st->call;
  g.fold_kill = -1;
  g.fold_twice = 0;
  g.fold_tmax = 0;
  if (g.fold_sign && g.mode == 2 && g.eps > 0.0) {
    // Child r = (U[r][0] + s U[r][1]) a0 vanishes exactly when U[r][0] = -s U[r][1];
    // evaluated as fma(U[r][0], a0, round(U[r][1] * s a0)) it is the rounding
    // error of one product, at most 2^-53 |U[r][0] a0| per component, so it
    // falls below eps / 2 (and is pruned) while |a0| < eps 2^52 / |U[r][0]|.
    const double s = (double)g.fold_sign;
    for (int r = 0; r < 2; ++r) {
      const double ur0 = g.u[2 * (2 * r)], ur1 = g.u[2 * (2 * r + 1)];
      // FP32 states evaluate the child with compensated arithmetic, where the
      // two products cancel exactly: the child is zero and always pruned.
      if (ur0 == -s * ur1 && ur0 != 0.0) {
        const double t = std::ldexp(g.eps, 52) / std::fabs(ur0) * (1.0 - 1e-12);
        std::memcpy(&g.fold_tmax, &t, 8);
        g.fold_kill = r;
        const int k = 1 - r;  // the surviving child
        g.fold_twice = g.u[2 * (2 * k)] == s * g.u[2 * (2 * k + 1)] ? 1u : 0u;
        break;
      }
    }
  }
  // An expansion that always acts (no controls that can fail) with
  // U[1][b0] = +-U[0][b0] leaves every branch paired with +-1 times itself.
  int8_t new_sign = 0;
  if (b0 >= 0 && g.mode != 1 && predicate_known(st, g.cmask, g.cval) == 1) {
    // Compared as numbers (0.0 == -0.0): the children U[r][b0] * a then
    // agree, or agree after a sign flip, in every nonzero component, and a
    // signed zero sums like an unsigned one.
    const double* r0 = &g.u[2 * (0 * 2 + b0)];  // U[0][b0] (re, im)
    const double* r1 = &g.u[2 * (1 * 2 + b0)];  // U[1][b0]
    if (r0[0] == r1[0] && r0[1] == r1[1]) new_sign = 1;
    else if (r0[0] == -r1[0] && r0[1] == -r1[1]) new_sign = -1;
  }
  g.vary[0] = g.vary[1] = 0ull;
  for (uint32_t q = 0; q < st->total_bits; ++q)
    if (st->const_val[q] < 0) g.vary[q >> 6] |= 1ull << (q & 63);
  note_branch(st, g);
  st->pair_sign[g.t] = new_sign;
  if ((st->flags & SQS_SIZING_LEARNED) && st->predictor) {
    sqs_state::Lazy q;
    q.g = g;
    q.ops.swap(st->pending);
    std::memcpy(q.x, x, sizeof(x));
    st->lazy.push_back(std::move(q));
    // Long circuits flush every kLazyMax steps: a misprediction then re-runs
    // at most that many steps, and the chained estimate restarts from an
    // exact count.
    if (st->lazy.size() >= kLazyMax && !st->capturing) return run_lazy(st);
    return SQS_OK;
  }
  if (fusing(st)) return hold_step(st, g);
  sqs_status s = flush_run(st);
  if (s != SQS_OK) return s;
  int64_t rec = -1;
  if (st->recording && st->rec_x.size() / SQS_PRED_FEATURES < st->rec_cap) {
    rec = (int64_t)(st->rec_x.size() / SQS_PRED_FEATURES);
    st->rec_x.insert(st->rec_x.end(), x, x + SQS_PRED_FEATURES);
  }
  return run_branching(st, g, -1.0, rec);
}

// Growth factor used for sizing from a predicted log2 ratio: a quarter of a
// bit above the prediction, and never above the doubling bound, so that the
// estimates chained from step to step do not drift below the true counts.
double grow_factor(float y) {
  return std::exp2(std::min(1.0, std::max(-8.0, (double)y + 0.25)));
}

// Executes the queued interference steps of learned mode: one batched
// inference predicts every step's growth; buckets are sized from the
// predicted counts; a device-side bucket overflow rolls back to the failed
// step, whose input buffers were kept alive, and re-runs it and the steps
// after it at the exact size.
sqs_status run_lazy(sqs_state* st) {
  if (st->lazy.empty()) return SQS_OK;
  const size_t n = st->lazy.size();
  std::vector<float> X(n * SQS_PRED_FEATURES), Y(n);
  for (size_t i = 0; i < n; ++i)
    std::memcpy(&X[i * SQS_PRED_FEATURES], st->lazy[i].x, sizeof(st->lazy[i].x));
  sqs_status s = sqs_predictor_predict(st->predictor, X.data(), (uint32_t)n, Y.data());
  if (s != SQS_OK) return st->sticky = fail(st, s, "predictor inference failed");
  s = sync_ctl(st);  // exact count entering the first queued step
  if (s != SQS_OK) return s;
  std::vector<HostOp> tail;
  tail.swap(st->pending);  // operations queued after the last step

  struct Snap {
    Store cur, alt, bk;
    int cur_slot;
    uint32_t seq;
  };
  std::vector<Snap> snaps(n);
  st->defer_frees = true;
  // Estimated count entering each step.  Chained step by step with the
  // quarter-bit margin of grow_factor, and capped one bit plus a margin that
  // widens with the square root of the steps chained (the errors of
  // independent predictions add like a random walk) above the plain chained
  // prediction: over long flushes (hundreds of steps of a linear-system
  // walk) the per-step margins would otherwise compound into sizes far above
  // any real count.
  std::vector<double> est(n);
  {
    // No estimate above what the device could hold: the free memory plus the
    // state's own buffers, over the three buffers a merge keeps (input,
    // buckets, output) with the bucket and segment slack.
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    const double rb = (double)(8 * st->kw + amp_bytes(st));
    const double fit = ((double)free_b + (double)st->stats.bytes_live) / (rb * 3.0 * 2.7);
    const double lmax = std::min<double>((double)std::min<uint32_t>(st->total_bits, 62),
                                         std::log2(std::max(2.0, fit)));
    double e = (double)st->ub, chain = std::log2(std::max(1.0, (double)st->ub));
    for (size_t i = 0; i < n; ++i) {
      const double cap = std::exp2(std::min(lmax, chain + 1.0 + 0.25 * std::sqrt((double)i)));
      e = std::max(1.0, std::min(e, cap));
      est[i] = e;
      const double r = grow_factor(Y[i]);
      e = std::min(2.0 * e, std::max(1.0, e * r));
      chain += std::min(1.0, std::max(-8.0, (double)Y[i]));
    }
    // Buffers that must grow during the flush grow once, to the predicted
    // peak, so that few of them wait in the graveyard.
    const double peak = *std::max_element(est.begin(), est.end());
    const double fill = (double)bucket_fill((uint64_t)std::min(peak, 0x1p62));
    st->grow_hint_b = (uint64_t)std::min(peak * 1.2 / fill, 0x1p40) + 1;
  }
  for (size_t i = 0; i < n && s == SQS_OK; ++i) {
    snaps[i] = Snap{st->cur, st->alt, st->bk, st->cur_slot, st->seq};
    st->pending = st->lazy[i].ops;
    s = run_branching(st, st->lazy[i].g, est[i]);
  }
  st->stats.learned_steps += n;
  if (s == SQS_OK) s = sync_ctl(st, true);
  if (s == SQS_ERR_CAPACITY && (st->ctl_host->err & ~sqs::kErrBucket) == 0) {
    // Roll back to the first step whose launches include the failing one.
    const uint32_t where = st->ctl_host->err_where;
    size_t f = 0;
    while (f + 1 < n && snaps[f + 1].seq < where) ++f;
    for (Store* x : {&st->cur, &st->alt, &st->bk})
      for (void* ptr : {(void*)x->k0, (void*)x->k1, x->amp, (void*)x->segs})
        if (ptr) st->graveyard.push_back(ptr);
    st->cur = snaps[f].cur;
    st->alt = snaps[f].alt;
    st->bk = snaps[f].bk;
    st->cur_slot = snaps[f].cur_slot;
    Ctl* c = st->ctl;
    cudaMemsetAsync(&c->err, 0, sizeof(c->err) + sizeof(c->err_where), st->stream);
    cudaMemsetAsync(&c->need, 0, sizeof(c->need), st->stream);
    if (st->bk.segs)
      cudaMemsetAsync(st->bk.segs, 0, ((st->bk.cap >> kBucketLog2) + 1) * 4, st->stream);
    s = sync_ctl(st);  // exact input count of the failed step
    for (size_t i = f; i < n && s == SQS_OK; ++i) {
      st->pending = st->lazy[i].ops;
      s = run_branching(st, st->lazy[i].g);
      st->stats.overflow_reruns++;
    }
    if (s == SQS_OK) s = sync_ctl(st);
  } else if (s == SQS_ERR_CAPACITY) {
    s = sync_ctl(st);  // any other device error is sticky
  }
  st->defer_frees = false;
  st->grow_hint_b = 0;
  std::vector<void*> live;
  for (Store* x : {&st->cur, &st->alt, &st->bk})
    for (void* ptr : {(void*)x->k0, (void*)x->k1, x->amp, (void*)x->segs}) live.push_back(ptr);
  std::sort(st->graveyard.begin(), st->graveyard.end());
  st->graveyard.erase(std::unique(st->graveyard.begin(), st->graveyard.end()),
                      st->graveyard.end());
  for (void* p : st->graveyard)
    if (std::find(live.begin(), live.end(), p) == live.end()) dfree_now(st, p);
  st->graveyard.clear();
  st->lazy.clear();
  st->pending.swap(tail);
  return s;
}

HostOp blank_op(uint32_t kind) {
  HostOp o;
  std::memset(&o.d, 0, sizeof(o.d));
  o.d.kind = kind;
  o.d.sel_bit = 128;
  o.c0 = o.c1 = std::complex<double>(1.0, 0.0);
  return o;
}

void push_prune(sqs_state* st, double eps) {
  HostOp o = blank_op(sqs::OP_PRUNE);
  o.d.eps = eps;
  o.d.eps2 = eps * eps;
  st->pending.push_back(o);
}

sqs_status apply_1q(sqs_state* st, uint32_t reg, uint32_t bit, const double* m,
                    const sqs_ctrl* ctrl, uint32_t n_ctrl, int mode, uint32_t angle_reg,
                    double scale, double offset) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  if (reg >= st->width.size() || bit >= st->width[reg])
    return fail(st, SQS_ERR_ARG, "target (%u, %u) out of range", reg, bit);
  uint64_t cm[2], cv[2];
  if (!encode_ctrls(st, ctrl, n_ctrl, cm, cv)) return fail(st, SQS_ERR_ARG, "bad controls");
  const uint32_t t = st->offset[reg] + bit;
  if (ctrl_touches(cm, t)) return fail(st, SQS_ERR_ARG, "a control sits on the target qubit");
  if (mode == 1 && (angle_reg >= st->width.size() || angle_reg == reg))
    return fail(st, SQS_ERR_ARG, "bad angle register");

  if (mode == 0 && is_zero(m[2], m[3]) && is_zero(m[4], m[5])) {
    // Diagonal: phases only (the _operate_diagonal strategy, Supp. B).
    HostOp o = blank_op(sqs::OP_MUL);
    o.d.pmask[0] = cm[0], o.d.pmask[1] = cm[1], o.d.pval[0] = cv[0], o.d.pval[1] = cv[1];
    o.d.sel_bit = t;
    o.c0 = std::complex<double>(m[0], m[1]);
    o.c1 = std::complex<double>(m[6], m[7]);
    push_op(st, o);
    push_prune(st, st->eps);
    return SQS_OK;
  }
  if (mode == 0 && is_zero(m[0], m[1]) && is_zero(m[6], m[7])) {
    // Anti-diagonal: flip plus phase (the _operate_off_diagonal strategy).
    // A branch with bit 0 moves to bit 1 with factor U10; bit 1 moves to 0 with U01.
    HostOp o = blank_op(sqs::OP_MUL_XOR);
    o.d.pmask[0] = cm[0], o.d.pmask[1] = cm[1], o.d.pval[0] = cv[0], o.d.pval[1] = cv[1];
    o.d.sel_bit = t;
    o.c0 = std::complex<double>(m[4], m[5]);
    o.c1 = std::complex<double>(m[2], m[3]);
    o.d.xmask[t >> 6] = 1ull << (t & 63);
    push_op(st, o);
    push_prune(st, st->eps);
    return SQS_OK;
  }
  Gate1 g;
  std::memset(&g, 0, sizeof(g));
  g.t = t;
  g.mode = (uint32_t)mode;
  if (mode == 0 && m[1] == 0.0 && m[3] == 0.0 && m[5] == 0.0 && m[7] == 0.0) g.mode = 2;
  g.cmask[0] = cm[0], g.cmask[1] = cm[1], g.cval[0] = cv[0], g.cval[1] = cv[1];
  if (mode == 0)
    for (int i = 0; i < 8; ++i) g.u[i] = m[i];
  for (int i = 0; i < 8; ++i) {
    g.uf[i] = (float)g.u[i];
    g.ufl[i] = (float)(g.u[i] - (double)g.uf[i]);
  }
  if (mode == 0) {
    // Rows of a column equal up to sign share one product per branch.
    auto same = [&](int r0, int r1, double sgn) {
      return m[2 * r1] == sgn * m[2 * r0] && m[2 * r1 + 1] == sgn * m[2 * r0 + 1];
    };
    if (same(0, 2, 1.0)) g.reuse |= 1u;
    else if (same(0, 2, -1.0)) g.reuse |= 1u | 4u;
    if (same(1, 3, 1.0)) g.reuse |= 2u;
    else if (same(1, 3, -1.0)) g.reuse |= 2u | 8u;
  }
  g.ang_off = mode == 1 ? st->offset[angle_reg] : 0;
  g.ang_w = mode == 1 ? st->width[angle_reg] : 0;
  g.scale = scale;
  g.offset = offset;
  g.ang_tab = nullptr;
  g.ang_digits = 0;
  if (mode == 1) {
    const uint32_t digits = (g.ang_w + 15) / 16;
    for (const auto& t : st->ang_tabs)
      if (t.scale == scale && t.offset == offset && t.digits == digits) g.ang_tab = t.dev;
    if (!g.ang_tab && st->ang_tabs.size() < 32) {
      double2* dev = (double2*)dalloc(st, ((size_t)digits << 16) * sizeof(double2));
      if (dev && sqs::launch_angle_table(st->stream, dev, digits, scale, offset) == cudaSuccess) {
        st->ang_tabs.push_back(sqs_state::AngTab{scale, offset, digits, dev});
        g.ang_tab = dev;
      } else if (dev) {
        dfree_now(st, dev);
      }
      cudaGetLastError();
    }
    g.ang_digits = g.ang_tab ? digits : 0;
  }
  g.eps = st->eps;
  g.eps2 = st->eps * st->eps;
  g.epsf = (float)st->eps;
  g.rho32 = st->rho32;
  return issue_branching(st, g, n_ctrl);
}

sqs_status flush_all(sqs_state* st) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  s = run_lazy(st);
  if (s != SQS_OK) return s;
  return run_pending(st, false);
}

sqs_status ensure_scratch(sqs_state* st, size_t bytes) {
  if (st->scratch_bytes >= bytes && st->scratch) return SQS_OK;
  if (st->capturing) {
    st->capture_err = SQS_ERR_STATE;
    return fail(st, SQS_ERR_STATE, "scratch allocation inside a graph capture");
  }
  dfree(st, st->scratch);
  st->scratch = (double*)dalloc(st, bytes);
  st->scratch_bytes = st->scratch ? bytes : 0;
  return st->scratch ? SQS_OK : fail(st, SQS_ERR_OOM, "cannot allocate scratch");
}

// Copies a segmented current array into a dense one (waits).
sqs_status densify(sqs_state* st) {
  if (!st->cur.segmented) return SQS_OK;
  const uint32_t ns = st->cur.n_seg;
  std::vector<unsigned int> cnt(ns);
  cudaError_t e = cudaMemcpyAsync(cnt.data(), st->cur.segs, (size_t)ns * 4,
                                  cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "densify");
  std::vector<uint64_t> off(ns);
  uint64_t total = 0;
  for (uint32_t i = 0; i < ns; ++i) {
    off[i] = total;
    total += cnt[i];
  }
  sqs_status s = ensure_scratch(st, (size_t)ns * 8 + 16);
  if (s != SQS_OK) return s;
  if (!ensure_store(st, st->alt, std::max<uint64_t>(total, 1)))
    return st->sticky = fail(st, SQS_ERR_OOM, "densify");
  st->alt.set_dense();
  e = cudaMemcpyAsync(st->scratch, off.data(), (size_t)ns * 8, cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess)
    e = sqs::launch_densify(launch_of(st, total), st->kw, st->amp32, st->cur.view(),
                            (const uint64_t*)st->scratch, st->alt.view());
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "densify");
  std::swap(st->cur, st->alt);
  return SQS_OK;
}

HostSnap take_snap(const sqs_state* st) {
  HostSnap h;
  h.cur = st->cur;
  h.alt = st->alt;
  h.bk = st->bk;
  h.cur_slot = st->cur_slot;
  h.ub = st->ub;
  h.call = st->call;
  h.last_branch = st->last_branch;
  h.writes_since = st->writes_since;
  h.reads_since = st->reads_since;
  h.arith_since = st->arith_since;
  h.const_val = st->const_val;
  h.pair_sign = st->pair_sign;
  h.n_branch = st->n_branch;
  h.last_target = st->last_target;
  return h;
}

void put_snap(sqs_state* st, const HostSnap& h) {
  st->cur = h.cur;
  st->alt = h.alt;
  st->bk = h.bk;
  st->cur_slot = h.cur_slot;
  st->ub = h.ub;
  st->call = h.call;
  st->last_branch = h.last_branch;
  st->writes_since = h.writes_since;
  st->reads_since = h.reads_since;
  st->arith_since = h.arith_since;
  st->const_val = h.const_val;
  st->pair_sign = h.pair_sign;
  st->n_branch = h.n_branch;
  st->last_target = h.last_target;
}

}  // namespace

// A captured sequence of calls: the CUDA graph, and the host bookkeeping
// (buffer roles, count slot and bound, per-qubit history) before and after.
struct sqs_graph {
  sqs_state* st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  HostSnap entry, exit;
  uint64_t launches = 0;
};

// Sorts the current state (executed: nothing queued; n branches) into one
// of the two scratch stores, dense and ascending in (key & keep), with LSD
// passes of the radix sort over the kept bits not known constant.  The
// state itself is unchanged.  *sorted receives the store, *n_sorted the
// device count pointer of the sorted copy.  States of 2^32 or more branches
// are refused (32-bit counts).
sqs_status sort_copy(sqs_state* st, uint64_t n, const uint64_t keep[2], Store** sorted,
                     const unsigned long long** n_sorted) {
  if (n >= (1ull << 32)) return fail(st, SQS_ERR_CAPACITY, "sorting needs fewer than 2^32 branches");
  sqs_state::TuneKey tkey;
  bool timed = false;
  const int rb = pick_sort_bits(st, n, bits_to_sort(st, keep), tkey, timed);
  const uint32_t D = (uint32_t)rb;
  std::vector<uint32_t> shifts;
  for (uint32_t q = 0; q < st->total_bits;) {
    const bool kept = (keep[q >> 6] >> (q & 63)) & 1ull;
    if (!kept || st->const_val[q] >= 0) {
      ++q;
      continue;
    }
    shifts.push_back(q);
    q += D;
  }
  if (shifts.empty()) shifts.push_back(0);  // one pass still makes the dense copy
  const uint64_t tile = (uint64_t)sqs::sort_tile();
  uint32_t per_seg = 1;
  uint64_t tiles0;
  if (st->cur.segmented) {
    per_seg = (uint32_t)std::max<uint64_t>(1, ((1ull << st->cur.seg_log2) + tile - 1) / tile);
    tiles0 = std::max<uint64_t>(1, (uint64_t)st->cur.n_seg * per_seg);
  } else {
    tiles0 = std::max<uint64_t>(1, (n + tile - 1) / tile);
  }
  const uint64_t tilesN = std::max<uint64_t>(1, (n + tile - 1) / tile);
  unsigned int *hist, *part;
  unsigned long long* n_dev;
  sqs_status s = sort_scratch(st, std::max(tiles0, tilesN), hist, part, n_dev, rb);
  if (s != SQS_OK) return s;
  if ((st->bk.cap < n && !ensure_store(st, st->bk, n)) ||
      (st->alt.cap < n && !ensure_store(st, st->alt, n)))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot allocate %llu branches",
                             (unsigned long long)n);
  // Digits of key & keep: the clear mask drops every other bit.  With
  // nothing to drop, the pair-class key of a bit past the key is the key.
  uint64_t cm[2] = {~keep[0], ~keep[1]};
  if (st->kw == 1) cm[1] = 0;
  const bool whole = cm[0] == 0 && cm[1] == 0;
  const uint32_t t_none = 64u * (uint32_t)st->kw;
  Store* buf[2] = {&st->alt, &st->bk};
  const unsigned long long* n_ptr = &st->ctl->cnt[st->cur_slot];
  Arr src = st->cur.view();
  const uint32_t npass = (uint32_t)shifts.size();
  cudaError_t e = cudaSuccess;
  if (timed) tune_begin(st, tkey);
  for (uint32_t p = 0; p < npass && e == cudaSuccess; ++p) {
    Store& dst = *buf[p & 1];
    dst.set_dense();
    Traced tr(st, SQS_K_SORT);
    e = sqs::launch_rsort_pass(launch_of(st, n), st->kw, st->amp32, st->ctl, src, n_ptr,
                               p == 0 ? per_seg : 1u, p == 0 ? tiles0 : tilesN, nullptr, t_none,
                               shifts[p], hist, part, n_dev, dst.view(), whole ? nullptr : cm,
                               rb);
    st->launches += 3;
    src = dst.view();
    n_ptr = n_dev;
  }
  if (timed) tune_end(st, tkey);
  if (e != cudaSuccess) return cuda_fail(st, e, "sort pass launch");
  *sorted = buf[(npass - 1) & 1];
  *n_sorted = n_dev;
  return SQS_OK;
}

extern "C" {

const char* sqs_version(void) { return kVersion; }

sqs_status sqs_state_create(const uint32_t* reg_widths, uint32_t n_regs, uint32_t flags,
                            uint64_t capacity_hint, const sqs_allocator* allocator,
                            void* cuda_stream, sqs_state** out) {
  if (!out || !reg_widths || n_regs == 0 || n_regs > 128) return SQS_ERR_ARG;
  if (flags & ~(SQS_AMP_FP32 | SQS_SIZING_LEARNED | SQS_MERGE_HASH | SQS_MERGE_SORT |
                SQS_MERGE_CLUSTER | SQS_MERGE_TUNED | SQS_MERGE_PLAIN | SQS_FUSE_OFF |
                SQS_FUSE_ALWAYS | SQS_AUTOTUNE))
    return SQS_ERR_ARG;
  uint32_t total = 0;
  for (uint32_t j = 0; j < n_regs; ++j) {
    if (reg_widths[j] < 1 || reg_widths[j] > 64) return SQS_ERR_ARG;
    total += reg_widths[j];
  }
  if (total > 128) return SQS_ERR_ARG;
  if (allocator && (!allocator->alloc || !allocator->free)) return SQS_ERR_ARG;

  sqs_state* st = new sqs_state();
  uint32_t off = 0;
  for (uint32_t j = 0; j < n_regs; ++j) {
    st->width.push_back(reg_widths[j]);
    st->offset.push_back(off);
    off += reg_widths[j];
  }
  st->total_bits = total;
  st->kw = total > 64 ? 2 : 1;
  st->amp32 = (flags & SQS_AMP_FP32) != 0;
  st->flags = flags;
  st->stream = (cudaStream_t)cuda_stream;
  if (allocator) {
    st->alloc = *allocator;
    st->has_alloc = true;
  }
  cudaError_t e = cudaGetDevice(&st->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&st->sm_count, cudaDevAttrMultiProcessorCount, st->device);
  cudaDeviceProp prop;
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, st->device);
  if (e != cudaSuccess) {
    sqs_status s = SQS_ERR_CUDA;
    delete st;
    cudaGetLastError();
    return s;
  }
  st->gpu_name = prop.name;
  if (const char* rb = std::getenv("SQS_SORT_BITS")) {
    const int v = std::atoi(rb);
    if (sqs::sort_radix_bits_ok(v)) st->forced_sort_bits = v;
  }
  // Autotuner choices from an earlier run on this GPU (SQS_TUNE_CACHE).
  if (const char* path = std::getenv("SQS_TUNE_CACHE")) {
    std::ifstream f(path);
    if (f) {
      std::stringstream buf;
      buf << f.rdbuf();
      tune_load(st, buf.str().c_str());
    }
  }
  e = cudaMallocHost((void**)&st->ctl_host, sizeof(Ctl));
  if (e != cudaSuccess) {
    delete st;
    return SQS_ERR_OOM;
  }
  st->ctl = (Ctl*)dalloc(st, sizeof(Ctl));
  const uint64_t cap = round_cap(std::max<uint64_t>(capacity_hint, 1024));
  if (!st->ctl || !ensure_store(st, st->cur, cap) || !ensure_store(st, st->alt, cap)) {
    sqs_state_destroy(st);
    return SQS_ERR_OOM;
  }
  if (sqs_state_reset(st) != SQS_OK) {
    sqs_state_destroy(st);
    return SQS_ERR_CUDA;
  }
  *out = st;
  return SQS_OK;
}

void sqs_state_destroy(sqs_state* st) {
  if (!st) return;
  cudaStreamSynchronize(st->stream);
  // Autotuner choices to the cache file: merged with entries other states
  // wrote (this state's measured keys win), written through a temporary file.
  if (const char* path = std::getenv("SQS_TUNE_CACHE")) {
    bool any = false;
    for (auto& kv : st->tuner) {
      // Collect a last measurement that has completed by now.
      sqs_state::TuneEntry& E = kv.second;
      bool t = false;
      if (E.choice < 0 && !E.cand.empty()) tune_pick(st, kv.first, E.cand, t);
      any |= E.choice >= 0;
    }
    if (any) {
      sqs_state merged;
      merged.gpu_name = st->gpu_name;
      std::ifstream f(path);
      if (f) {
        std::stringstream buf;
        buf << f.rdbuf();
        tune_load(&merged, buf.str().c_str());
      }
      for (const auto& kv : st->tuner)
        if (kv.second.choice >= 0) {
          merged.tuner[kv.first] = kv.second;
          merged.tuner[kv.first].ev[0] = merged.tuner[kv.first].ev[1] = nullptr;
        }
      const std::string tmp = std::string(path) + ".tmp";
      {
        std::ofstream o(tmp);
        o << tune_json(&merged);
      }
      std::rename(tmp.c_str(), path);
    }
  }
  free_store(st, st->cur);
  free_store(st, st->alt);
  free_store(st, st->bk);
  dfree(st, st->rec_dev);
  dfree(st, st->ctl);
  dfree(st, st->scratch);
  dfree(st, st->sort_buf);
  for (auto& t : st->ang_tabs) dfree(st, t.dev);
  for (auto& kv : st->tune)
    for (cudaEvent_t e : kv.second.ev)
      if (e) cudaEventDestroy(e);
  for (auto& kv : st->tuner)
    for (cudaEvent_t e : kv.second.ev)
      if (e) cudaEventDestroy(e);
  for (sqs_table* t : st->tables) {
    dfree(st, t->dev);
    delete t;
  }
  cudaStreamSynchronize(st->stream);
  for (cudaEvent_t e : st->ev) cudaEventDestroy(e);
  if (st->ctl_host) cudaFreeHost(st->ctl_host);
  cudaGetLastError();
  delete st;
}

sqs_status sqs_state_reset(sqs_state* st) {
  if (!st) return SQS_ERR_ARG;
  st->pending.clear();
  st->lazy.clear();
  st->run_gates.clear();
  st->run_pre.clear();
  st->run_tmask[0] = st->run_tmask[1] = st->run_reads[0] = st->run_reads[1] = 0;
  st->sticky = SQS_OK;
  st->err.clear();
  st->cur_slot = 0;
  st->ub = 1;
  history_reset(st, true);
  if (st->bk.segs)
    cudaMemsetAsync(st->bk.segs, 0, ((st->bk.cap >> kBucketLog2) + 1) * 4, st->stream);
  st->cur.set_dense();
  st->call = 1;  // API calls are numbered from the reset
  Traced tr(st, SQS_K_INIT);
  cudaError_t e = sqs::launch_init(launch_of(st, 1), st->ctl, st->cur.view(), 0, st->amp32);
  if (e != cudaSuccess) return cuda_fail(st, e, "reset");
  return SQS_OK;
}

sqs_status sqs_tune_export(const sqs_state* st, char* buf, uint64_t cap, uint64_t* len) {
  if (!st || !len) return SQS_ERR_ARG;
  const std::string j = tune_json(st);
  *len = j.size();
  if (!buf || cap < j.size() + 1) return SQS_ERR_ARG;
  std::memcpy(buf, j.c_str(), j.size() + 1);
  return SQS_OK;
}

sqs_status sqs_tune_import(sqs_state* st, const char* json) {
  if (!st || !json) return SQS_ERR_ARG;
  tune_load(st, json);
  return SQS_OK;
}

sqs_status sqs_state_set_wait_test(sqs_state* st, uint32_t wait_limit, int32_t skip_copy_rank) {
  if (!st) return SQS_ERR_ARG;
  if (skip_copy_rank >= sqs::cluster_ctas()) return fail(st, SQS_ERR_ARG, "rank out of range");
  st->wait_limit = wait_limit;
  st->skip_copy_rank = skip_copy_rank < 0 ? -1 : skip_copy_rank;
  return SQS_OK;
}

sqs_status sqs_set_fp32_cancel(sqs_state* st, double rho) {
  if (!st || !(rho >= 0.0) || rho > 0x1p-10) return SQS_ERR_ARG;
  st->rho32 = (float)rho;
  return SQS_OK;
}

sqs_status sqs_set_prune_eps(sqs_state* st, double eps) {
  if (!st || !(eps >= 0.0) || std::isinf(eps)) return SQS_ERR_ARG;
  st->eps = eps;
  return SQS_OK;
}

sqs_status sqs_apply_u1q(sqs_state* st, uint32_t reg, uint32_t bit, const double m[8],
                         const sqs_ctrl* ctrl, uint32_t n_ctrl) {
  if (!m) return fail(st, SQS_ERR_ARG, "null matrix");
  for (int i = 0; i < 8; ++i)
    if (!std::isfinite(m[i])) return fail(st, SQS_ERR_ARG, "non-finite matrix entry");
  return apply_1q(st, reg, bit, m, ctrl, n_ctrl, 0, 0, 0.0, 0.0);
}

sqs_status sqs_apply_h(sqs_state* st, uint32_t reg, uint32_t bit, const sqs_ctrl* ctrl,
                       uint32_t n_ctrl) {
  const double r = 1.0 / std::sqrt(2.0);
  const double m[8] = {r, 0, r, 0, r, 0, -r, 0};
  return apply_1q(st, reg, bit, m, ctrl, n_ctrl, 0, 0, 0.0, 0.0);
}

sqs_status sqs_apply_ry(sqs_state* st, uint32_t reg, uint32_t bit, double theta,
                        const sqs_ctrl* ctrl, uint32_t n_ctrl) {
  if (!std::isfinite(theta)) return fail(st, SQS_ERR_ARG, "non-finite angle");
  const double c = std::cos(theta / 2), s = std::sin(theta / 2);
  const double m[8] = {c, 0, -s, 0, s, 0, c, 0};
  return apply_1q(st, reg, bit, m, ctrl, n_ctrl, 0, 0, 0.0, 0.0);
}

sqs_status sqs_apply_ry_reg(sqs_state* st, uint32_t reg, uint32_t bit, uint32_t angle_reg,
                            double scale, double offset, const sqs_ctrl* ctrl,
                            uint32_t n_ctrl) {
  if (!std::isfinite(scale) || !std::isfinite(offset))
    return fail(st, SQS_ERR_ARG, "non-finite angle map");
  const double m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  return apply_1q(st, reg, bit, m, ctrl, n_ctrl, 1, angle_reg, scale, offset);
}

sqs_status sqs_apply_perm(sqs_state* st, const sqs_perm_op* ops, uint32_t n_ops) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  if (n_ops && !ops) return fail(st, SQS_ERR_ARG, "null ops");
  std::vector<HostOp> add;
  add.reserve(n_ops);
  const uint32_t nr = (uint32_t)st->width.size();
  for (uint32_t i = 0; i < n_ops; ++i) {
    const sqs_perm_op& p = ops[i];
    if (p.reg >= nr) return fail(st, SQS_ERR_ARG, "op %u: bad register", i);
    uint64_t cm[2], cv[2];
    if (p.n_ctrl > SQS_MAX_CTRL || !encode_ctrls(st, p.ctrl, p.n_ctrl, cm, cv))
      return fail(st, SQS_ERR_ARG, "op %u: bad controls", i);
    HostOp h = blank_op(sqs::OP_XOR);
    DevOp& o = h.d;
    o.pmask[0] = cm[0], o.pmask[1] = cm[1], o.pval[0] = cv[0], o.pval[1] = cv[1];
    o.dst_off = st->offset[p.reg];
    o.dst_w = st->width[p.reg];
    const uint64_t wm = o.dst_w >= 64 ? ~0ull : ((1ull << o.dst_w) - 1);
    switch (p.kind) {
      case SQS_PERM_X: {
        if (p.bit >= st->width[p.reg]) return fail(st, SQS_ERR_ARG, "op %u: bad bit", i);
        const uint32_t q = o.dst_off + p.bit;
        if (ctrl_touches(cm, q)) return fail(st, SQS_ERR_ARG, "op %u: control on target", i);
        o.kind = sqs::OP_XOR;
        o.xmask[q >> 6] = 1ull << (q & 63);
        break;
      }
      case SQS_PERM_ADD_REG:
      case SQS_PERM_SUB_REG:
      case SQS_PERM_SWAP: {
        if (p.src_reg >= nr || p.src_reg == p.reg)
          return fail(st, SQS_ERR_ARG, "op %u: bad source register", i);
        if (p.kind == SQS_PERM_SWAP && st->width[p.src_reg] != st->width[p.reg])
          return fail(st, SQS_ERR_ARG, "op %u: swap needs equal widths", i);
        for (uint32_t b = 0; b < st->width[p.reg]; ++b)
          if (ctrl_touches(cm, o.dst_off + b))
            return fail(st, SQS_ERR_ARG, "op %u: control inside the target register", i);
        if (p.kind == SQS_PERM_SWAP)
          for (uint32_t b = 0; b < st->width[p.src_reg]; ++b)
            if (ctrl_touches(cm, st->offset[p.src_reg] + b))
              return fail(st, SQS_ERR_ARG, "op %u: control inside a swapped register", i);
        o.kind = p.kind == SQS_PERM_ADD_REG ? sqs::OP_ADD_REG
                 : p.kind == SQS_PERM_SUB_REG ? sqs::OP_SUB_REG
                                              : sqs::OP_SWAP;
        o.src_off = st->offset[p.src_reg];
        o.src_w = st->width[p.src_reg];
        break;
      }
      case SQS_PERM_MUL_ADD:
      case SQS_PERM_DIV_XOR: {
        if (p.src_reg >= nr || p.src_reg == p.reg || p.src2_reg >= nr || p.src2_reg == p.reg)
          return fail(st, SQS_ERR_ARG, "op %u: bad source registers", i);
        for (uint32_t b = 0; b < st->width[p.reg]; ++b)
          if (ctrl_touches(cm, o.dst_off + b))
            return fail(st, SQS_ERR_ARG, "op %u: control inside the target register", i);
        o.kind = p.kind == SQS_PERM_MUL_ADD ? sqs::OP_MUL_ADD : sqs::OP_DIV_XOR;
        o.src_off = st->offset[p.src_reg];
        o.src_w = st->width[p.src_reg];
        o.src2_off = st->offset[p.src2_reg];
        o.src2_w = st->width[p.src2_reg];
        break;
      }
      case SQS_PERM_MUL_CONST: {
        if (!(p.constant & 1ull))
          return fail(st, SQS_ERR_ARG, "op %u: the multiplier must be odd (a bijection)", i);
        for (uint32_t b = 0; b < st->width[p.reg]; ++b)
          if (ctrl_touches(cm, o.dst_off + b))
            return fail(st, SQS_ERR_ARG, "op %u: control inside the target register", i);
        o.kind = sqs::OP_MUL_CONST;
        o.constant = p.constant & wm;
        break;
      }
      case SQS_PERM_ADD_CONST:
      case SQS_PERM_SUB_CONST: {
        for (uint32_t b = 0; b < st->width[p.reg]; ++b)
          if (ctrl_touches(cm, o.dst_off + b))
            return fail(st, SQS_ERR_ARG, "op %u: control inside the target register", i);
        o.kind = sqs::OP_ADD_CONST;
        const uint64_t c = p.constant & wm;
        o.constant = p.kind == SQS_PERM_ADD_CONST ? c : ((0 - c) & wm);
        break;
      }
      default:
        return fail(st, SQS_ERR_ARG, "op %u: unknown kind %u", i, p.kind);
    }
    add.push_back(h);
  }
  for (const HostOp& h : add) push_op(st, h);
  return SQS_OK;
}

sqs_status sqs_apply_phase(sqs_state* st, const sqs_ctrl* pred, uint32_t n_pred, double phi) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  if (!std::isfinite(phi)) return fail(st, SQS_ERR_ARG, "non-finite phase");
  uint64_t cm[2], cv[2];
  if (!encode_ctrls(st, pred, n_pred, cm, cv)) return fail(st, SQS_ERR_ARG, "bad predicates");
  HostOp o = blank_op(sqs::OP_MUL);
  o.d.pmask[0] = cm[0], o.d.pmask[1] = cm[1], o.d.pval[0] = cv[0], o.d.pval[1] = cv[1];
  o.c0 = std::complex<double>(std::cos(phi), std::sin(phi));
  push_op(st, o);
  return SQS_OK;
}

sqs_status sqs_table_create(sqs_state* st, const void* host_entries, uint64_t n_entries,
                            uint32_t entry_bytes, sqs_table** out) {
  {
    sqs_status g = no_capture(st, "sqs_table_create");
    if (g != SQS_OK) return g;
  }
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (!out || (n_entries && !host_entries) ||
      !(entry_bytes == 1 || entry_bytes == 2 || entry_bytes == 4 || entry_bytes == 8))
    return fail(st, SQS_ERR_ARG, "bad table arguments");
  sqs_table* t = new sqs_table();
  t->n = n_entries;
  t->bytes = entry_bytes;
  t->dev = dalloc(st, n_entries * entry_bytes + 16);
  if (!t->dev) {
    delete t;
    return fail(st, SQS_ERR_OOM, "cannot allocate table");
  }
  if (n_entries) {
    cudaError_t e = cudaMemcpyAsync(t->dev, host_entries, n_entries * entry_bytes,
                                    cudaMemcpyHostToDevice, st->stream);
    // The host buffer belongs to the caller: finish the copy before returning.
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) {
      dfree(st, t->dev);
      delete t;
      return cuda_fail(st, e, "table upload");
    }
  }
  st->tables.push_back(t);
  *out = t;
  return SQS_OK;
}

static sqs_status qram(sqs_state* st, uint32_t addr_reg, uint32_t n_addr, uint32_t data_reg,
                       const sqs_table* t) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  const uint32_t nr = (uint32_t)st->width.size();
  if (!t || n_addr == 0 || addr_reg >= nr || n_addr > nr - addr_reg || data_reg >= nr ||
      (data_reg >= addr_reg && data_reg < addr_reg + n_addr))
    return fail(st, SQS_ERR_ARG, "bad QRAM arguments");
  uint32_t addr_w = 0;
  for (uint32_t r = addr_reg; r < addr_reg + n_addr; ++r) addr_w += st->width[r];
  if (addr_w > 64) return fail(st, SQS_ERR_ARG, "QRAM address wider than 64 bits");
  bool owned = false;
  for (sqs_table* x : st->tables) owned |= (x == t);
  if (!owned) return fail(st, SQS_ERR_ARG, "table belongs to another state");
  HostOp o = blank_op(sqs::OP_QRAM);
  o.d.dst_off = st->offset[data_reg];
  o.d.dst_w = st->width[data_reg];
  o.d.src_off = st->offset[addr_reg];  // registers are packed in order: one field
  o.d.src_w = addr_w;
  o.d.table = t->dev;
  o.d.n_entries = t->n;
  o.d.constant = t->bytes;
  push_op(st, o);
  return SQS_OK;
}

sqs_status sqs_qram_load(sqs_state* st, uint32_t addr_reg, uint32_t data_reg,
                         const sqs_table* table) {
  return qram(st, addr_reg, 1, data_reg, table);
}

sqs_status sqs_qram_unload(sqs_state* st, uint32_t addr_reg, uint32_t data_reg,
                           const sqs_table* table) {
  return qram(st, addr_reg, 1, data_reg, table);
}

sqs_status sqs_qram_load_span(sqs_state* st, uint32_t addr_reg, uint32_t n_addr_regs,
                              uint32_t data_reg, const sqs_table* table) {
  return qram(st, addr_reg, n_addr_regs, data_reg, table);
}

sqs_status sqs_qram_unload_span(sqs_state* st, uint32_t addr_reg, uint32_t n_addr_regs,
                                uint32_t data_reg, const sqs_table* table) {
  return qram(st, addr_reg, n_addr_regs, data_reg, table);
}

sqs_status sqs_prune(sqs_state* st, double eps, uint64_t* nnz_out) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (!(eps >= 0.0) || std::isinf(eps)) return fail(st, SQS_ERR_ARG, "bad eps");
  push_prune(st, eps);
  s = run_pending(st, false);
  if (s != SQS_OK) return s;
  if (nnz_out) {
    s = sync_ctl(st);
    if (s != SQS_OK) return s;
    *nnz_out = st->ctl_host->cnt[st->cur_slot];
  }
  return SQS_OK;
}


sqs_status sqs_probabilities_device(sqs_state* st, uint32_t reg, double* probs_dev,
                                    double* norm2_dev) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  s = flush_all(st);
  if (s != SQS_OK) return s;
  if (reg >= st->width.size() || (probs_dev && st->width[reg] > 26))
    return fail(st, SQS_ERR_ARG, "register too wide for dense marginals");
  const uint32_t w = st->width[reg];
  cudaError_t e = cudaSuccess;
  if (probs_dev) e = cudaMemsetAsync(probs_dev, 0, sizeof(double) << w, st->stream);
  if (e == cudaSuccess && norm2_dev) e = cudaMemsetAsync(norm2_dev, 0, sizeof(double), st->stream);
  if (e == cudaSuccess) {
    Traced tr(st, SQS_K_PROB);
    e = sqs::launch_probabilities(launch_of(st, st->cur.slots(st->ub)), st->kw, st->amp32,
                                  st->ctl, st->cur.view(), st->cur_slot, st->offset[reg], w,
                                  probs_dev, norm2_dev);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "probabilities");
  return SQS_OK;
}

sqs_status sqs_probabilities(sqs_state* st, uint32_t reg, double* probs, double* norm2) {
  {
    sqs_status g = no_capture(st, "sqs_probabilities");
    if (g != SQS_OK) return g;
  }
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (reg >= st->width.size() || (probs && st->width[reg] > 26))
    return fail(st, SQS_ERR_ARG, "register too wide for dense marginals");
  const uint32_t w = st->width[reg];
  const size_t nb = probs ? (sizeof(double) << w) : 0;
  s = ensure_scratch(st, nb + 16);
  if (s != SQS_OK) return s;
  double* pd = probs ? st->scratch : nullptr;
  double* nd = (double*)((char*)st->scratch + nb);
  s = sqs_probabilities_device(st, reg, pd, nd);
  if (s != SQS_OK) return s;
  cudaError_t e = cudaSuccess;
  if (probs) e = cudaMemcpyAsync(probs, pd, nb, cudaMemcpyDeviceToHost, st->stream);
  double n2 = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n2, nd, 8, cudaMemcpyDeviceToHost, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "probabilities readback");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  if (norm2) *norm2 = n2;
  return SQS_OK;
}

sqs_status sqs_nnz(sqs_state* st, uint64_t* out) {
  {
    sqs_status g = no_capture(st, "sqs_nnz");
    if (g != SQS_OK) return g;
  }
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (!out) return fail(st, SQS_ERR_ARG, "null output");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  *out = st->ctl_host->cnt[st->cur_slot];
  return SQS_OK;
}

sqs_status sqs_peak_nnz(sqs_state* st, uint64_t* out) {
  {
    sqs_status g = no_capture(st, "sqs_peak_nnz");
    if (g != SQS_OK) return g;
  }
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (!out) return fail(st, SQS_ERR_ARG, "null output");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  *out = std::max<uint64_t>(st->ctl_host->peak, st->ctl_host->cnt[st->cur_slot]);
  return SQS_OK;
}

sqs_status sqs_probabilities_sparse(sqs_state* st, uint32_t reg, uint64_t* values, double* probs,
                                    uint64_t cap, uint64_t* count, double* norm2) {
  {
    sqs_status g = no_capture(st, "sqs_probabilities_sparse");
    if (g != SQS_OK) return g;
  }
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (reg >= st->width.size()) return fail(st, SQS_ERR_ARG, "register out of range");
  if (!count) return fail(st, SQS_ERR_ARG, "null count");
  if (cap && (!values || !probs)) return fail(st, SQS_ERR_ARG, "null buffers");
  st->call++;
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  const uint64_t n = st->ctl_host->cnt[st->cur_slot];
  const uint32_t off = st->offset[reg], w = st->width[reg];
  const uint64_t tiles = sqs::run_tiles(n);
  // Scratch: values, probs (n each), runs, lead sums, lead flags (per tile),
  // the run total and the norm.
  const size_t a8 = 255;
  const size_t b_vals = (n * 8 + a8) & ~a8, b_probs = b_vals;
  const size_t b_runs = (tiles * 4 + a8) & ~a8, b_lead = (tiles * 8 + a8) & ~a8;
  const size_t bytes = b_vals + b_probs + 2 * b_runs + b_lead + 256;
  s = ensure_scratch(st, bytes);
  if (s != SQS_OK) return s;
  unsigned char* base = (unsigned char*)st->scratch;
  uint64_t* d_vals = (uint64_t*)base;
  double* d_probs = (double*)(base + b_vals);
  unsigned int* d_runs = (unsigned int*)(base + b_vals + b_probs);
  unsigned int* d_full = (unsigned int*)(base + b_vals + b_probs + b_runs);
  double* d_lead = (double*)(base + b_vals + b_probs + 2 * b_runs);
  unsigned long long* d_total = (unsigned long long*)(base + b_vals + b_probs + 2 * b_runs + b_lead);
  double* d_norm = (double*)(d_total + 1);
  cudaError_t e = cudaMemsetAsync(d_total, 0, 16, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "sparse marginals");
  if (n) {
    {
      Traced tr(st, SQS_K_PROB);
      e = sqs::launch_probabilities(launch_of(st, st->cur.slots(st->ub)), st->kw, st->amp32,
                                    st->ctl, st->cur.view(), st->cur_slot, off, w, nullptr, d_norm);
    }
    if (e != cudaSuccess) return cuda_fail(st, e, "sparse marginals");
    uint64_t km[2] = {0ull, 0ull};  // the register's key bits
    for (uint32_t b = 0; b < w; ++b) km[(off + b) >> 6] |= 1ull << ((off + b) & 63);
    Store* sorted = nullptr;
    const unsigned long long* n_sorted = nullptr;
    s = sort_copy(st, n, km, &sorted, &n_sorted);
    if (s != SQS_OK) return s;
    Traced tr(st, SQS_K_PROB);
    e = sqs::launch_sparse_marginals(launch_of(st, n), st->kw, st->amp32, st->ctl, sorted->view(),
                                     n_sorted, tiles, off, w, d_runs, d_lead, d_full, d_total,
                                     d_vals, d_probs);
    st->launches += 2;
    if (e != cudaSuccess) return cuda_fail(st, e, "sparse marginals");
  }
  unsigned long long head[2] = {0, 0};
  e = cudaMemcpyAsync(head, d_total, 16, cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "sparse marginals readback");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  const uint64_t total = head[0];
  double nv;
  std::memcpy(&nv, &head[1], 8);
  *count = total;
  if (norm2) *norm2 = nv;
  if (total > cap)
    return fail(st, SQS_ERR_ARG, "sparse marginals need %llu entries", (unsigned long long)total);
  if (total) {
    e = cudaMemcpyAsync(values, d_vals, total * 8, cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(probs, d_probs, total * 8, cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "sparse marginals readback");
  }
  return SQS_OK;
}

sqs_status sqs_export(sqs_state* st, uint64_t* keys, double* amps, uint64_t cap, uint64_t* n) {
  {
    sqs_status g = no_capture(st, "sqs_export");
    if (g != SQS_OK) return g;
  }
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (!n) return fail(st, SQS_ERR_ARG, "null count");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  const uint64_t cnt = st->ctl_host->cnt[st->cur_slot];
  *n = cnt;
  if (cnt > cap) return fail(st, SQS_ERR_ARG, "export needs %llu branches", (unsigned long long)cnt);
  if (cnt == 0) return SQS_OK;
  if (!keys || !amps) return fail(st, SQS_ERR_ARG, "null buffers");
  // Ascending keys: a sorted copy (the state keeps its own order).  States
  // of 2^32 or more branches are copied in storage order.
  Store* src = nullptr;
  if (cnt < (1ull << 32)) {
    const uint64_t all[2] = {~0ull, ~0ull};
    const unsigned long long* n_sorted = nullptr;
    s = sort_copy(st, cnt, all, &src, &n_sorted);
    if (s != SQS_OK) return s;
  } else {
    s = densify(st);
    if (s != SQS_OK) return s;
    src = &st->cur;
  }
  cudaError_t e;
  if (st->kw == 1) {
    e = cudaMemcpyAsync(keys, src->k0, cnt * 8, cudaMemcpyDeviceToHost, st->stream);
  } else {
    e = cudaMemcpy2DAsync(keys, 16, src->k0, 8, 8, cnt, cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(keys + 1, 16, src->k1, 8, 8, cnt, cudaMemcpyDeviceToHost,
                            st->stream);
  }
  if (e == cudaSuccess) {
    if (st->amp32) {
      s = ensure_scratch(st, cnt * 16);
      if (s != SQS_OK) return s;
      e = sqs::launch_to_f64(launch_of(st, cnt), st->ctl, src->view(), st->cur_slot,
                             st->scratch);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(amps, st->scratch, cnt * 16, cudaMemcpyDeviceToHost, st->stream);
    } else {
      e = cudaMemcpyAsync(amps, src->amp, cnt * 16, cudaMemcpyDeviceToHost, st->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "export");
  return SQS_OK;
}

sqs_status sqs_import(sqs_state* st, const uint64_t* keys, const double* amps, uint64_t n) {
  {
    sqs_status g = no_capture(st, "sqs_import");
    if (g != SQS_OK) return g;
  }
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (n && (!keys || !amps)) return fail(st, SQS_ERR_ARG, "null buffers");
  // Keys must fit the register widths.
  const uint32_t tb = st->total_bits;
  const uint64_t m0 = tb >= 64 ? ~0ull : ((1ull << tb) - 1);
  const uint64_t m1 = tb <= 64 ? 0ull : (tb >= 128 ? ~0ull : ((1ull << (tb - 64)) - 1));
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t lo = keys[i * st->kw];
    const uint64_t hi = st->kw == 2 ? keys[i * 2 + 1] : 0;
    if ((lo & ~m0) || (hi & ~m1)) return fail(st, SQS_ERR_ARG, "key %llu out of range",
                                              (unsigned long long)i);
  }
  // The imported state replaces the current one: queued operations and a
  // held run are dropped with it.
  st->pending.clear();
  st->run_gates.clear();
  st->run_pre.clear();
  st->run_tmask[0] = st->run_tmask[1] = st->run_reads[0] = st->run_reads[1] = 0;
  if (!ensure_store(st, st->cur, std::max<uint64_t>(n, 1)))
    return fail(st, SQS_ERR_OOM, "import");
  st->cur.set_dense();
  cudaError_t e = cudaSuccess;
  if (n) {
    if (st->kw == 1) {
      e = cudaMemcpyAsync(st->cur.k0, keys, n * 8, cudaMemcpyHostToDevice, st->stream);
    } else {
      e = cudaMemcpy2DAsync(st->cur.k0, 8, keys, 16, 8, n, cudaMemcpyHostToDevice, st->stream);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(st->cur.k1, 8, keys + 1, 16, 8, n, cudaMemcpyHostToDevice,
                              st->stream);
    }
    if (e == cudaSuccess) {
      if (st->amp32) {
        s = ensure_scratch(st, n * 16);
        if (s != SQS_OK) return s;
        e = cudaMemcpyAsync(st->scratch, amps, n * 16, cudaMemcpyHostToDevice, st->stream);
        if (e == cudaSuccess)
          e = sqs::launch_from_f64(launch_of(st, n), st->ctl, st->cur.view(), st->scratch, n);
      } else {
        e = cudaMemcpyAsync(st->cur.amp, amps, n * 16, cudaMemcpyHostToDevice, st->stream);
      }
    }
  }
  // Counts: the state now holds n branches in slot 0.
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.cnt[0] = n;
  c.peak = n;
  *st->ctl_host = c;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st->ctl, st->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "import");
  st->cur_slot = 0;
  st->ub = n;
  st->sticky = SQS_OK;
  st->lazy.clear();
  history_reset(st, false);
  return SQS_OK;
}

sqs_status sqs_sync(sqs_state* st) {
  {
    sqs_status g = no_capture(st, "sqs_sync");
    if (g != SQS_OK) return g;
  }
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  return sync_ctl(st);
}

sqs_status sqs_flush(sqs_state* st) { return flush_all(st); }

uint32_t sqs_key_words(const sqs_state* st) { return st ? (uint32_t)st->kw : 0; }

uint64_t sqs_launch_count(const sqs_state* st) { return st ? st->launches : 0; }

sqs_status sqs_trace_enable(sqs_state* st, uint32_t max_records) {
  if (!st) return SQS_ERR_ARG;
  for (cudaEvent_t e : st->ev) cudaEventDestroy(e);
  st->ev.clear();
  st->trace.clear();
  st->trace_dropped = 0;
  st->call = 0;
  for (uint32_t i = 0; i < 2 * max_records; ++i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(st, cudaGetLastError(), "event");
    st->ev.push_back(e);
  }
  return SQS_OK;
}

sqs_status sqs_trace_read(sqs_state* st, sqs_trace_record* out, uint32_t cap, uint32_t* n) {
  if (!st || !n || (cap && !out)) return SQS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "trace");
  const uint32_t used = (uint32_t)st->trace.size();
  for (uint32_t i = 0; i < used && i < cap; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, st->ev[2 * i], st->ev[2 * i + 1]);
    out[i] = st->trace[i];
    out[i].ms = ms;
  }
  *n = used + st->trace_dropped;
  st->trace.clear();
  st->trace_dropped = 0;
  st->call = 0;
  return SQS_OK;
}

sqs_status sqs_state_set_predictor(sqs_state* st, sqs_predictor* p) {
  if (!st) return SQS_ERR_ARG;
  sqs_status s = flush_all(st);  // steps queued under the old setting run first
  if (s != SQS_OK) return s;
  st->predictor = p;
  return SQS_OK;
}

sqs_status sqs_state_record(sqs_state* st, uint32_t enable) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (enable && !st->rec_dev) {
    st->rec_cap = 1u << 16;
    st->rec_dev = (unsigned long long*)dalloc(st, (size_t)st->rec_cap * 16);
    if (!st->rec_dev) return fail(st, SQS_ERR_OOM, "cannot allocate the record buffer");
  }
  st->recording = enable != 0;
  return SQS_OK;
}

sqs_status sqs_state_read_records(sqs_state* st, float* X, float* y, uint32_t cap, uint32_t* n) {
  {
    sqs_status g = no_capture(st, "sqs_state_read_records");
    if (g != SQS_OK) return g;
  }
  if (!st || !n || (cap && (!X || !y))) return SQS_ERR_ARG;
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  const size_t nrec = st->rec_x.size() / SQS_PRED_FEATURES;
  std::vector<unsigned long long> cnt(2 * std::max<size_t>(nrec, 1));
  if (nrec) {
    cudaError_t e = cudaMemcpyAsync(cnt.data(), st->rec_dev, nrec * 16, cudaMemcpyDeviceToHost,
                                    st->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "records");
  }
  // Steps whose input was empty carry no ratio and are skipped.
  uint32_t w = 0;
  for (size_t i = 0; i < nrec; ++i) {
    const unsigned long long a = cnt[2 * i], b = cnt[2 * i + 1];
    if (a == 0) continue;
    if (w < cap) {
      std::memcpy(X + (size_t)w * SQS_PRED_FEATURES, &st->rec_x[i * SQS_PRED_FEATURES],
                  SQS_PRED_FEATURES * sizeof(float));
      y[w] = (float)std::log2((double)std::max<unsigned long long>(b, 1) / (double)a);
    }
    ++w;
  }
  *n = w;
  st->rec_x.clear();
  return SQS_OK;
}

sqs_status sqs_capture_begin(sqs_state* st, uint64_t static_bound) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (st->capturing) return fail(st, SQS_ERR_ARG, "a capture is already open");
  if (st->flags & (SQS_SIZING_LEARNED | SQS_MERGE_SORT | SQS_MERGE_CLUSTER | SQS_MERGE_TUNED))
    return fail(st, SQS_ERR_ARG, "graph capture runs the bucket merge with exact sizing");
  if (static_bound == 0 || static_bound > max_branches(st))
    return fail(st, SQS_ERR_ARG, "static bound out of range");
  if (st->stream == nullptr)
    return fail(st, SQS_ERR_ARG, "graph capture needs a stream other than the legacy default");
  // Buffers for every operation on up to static_bound branches.
  // Enough buckets for eager issue on the same state as well (the smaller
  // fill), so that running the circuit eagerly between graph launches does
  // not move the buffers the graph holds.
  const uint64_t B = std::max<uint64_t>(1, (static_bound + kBucketFill - 1) / kBucketFill);
  const uint64_t cap = std::max<uint64_t>(B << kSegLog2, 2 * static_bound + 8192);
  if (!ensure_store(st, st->cur, cap) || !ensure_store(st, st->alt, cap) ||
      !ensure_store(st, st->bk, B << kBucketLog2))
    return st->sticky = fail(st, SQS_ERR_OOM, "cannot size buffers for the capture");
  s = sqs_state_reset(st);  // the state the graph starts from, now
  if (s != SQS_OK) return s;
  st->entry_snap = take_snap(st);
  st->launches_at_capture = st->launches;
  cudaError_t e = cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(st, e, "begin capture");
  st->capturing = true;
  st->static_ub = static_bound;
  st->capture_err = SQS_OK;
  return sqs_state_reset(st);  // ... and the graph's first node
}

sqs_status sqs_capture_end(sqs_state* st, sqs_graph** out) {
  if (!st || !out) return SQS_ERR_ARG;
  if (!st->capturing) return fail(st, SQS_ERR_ARG, "no capture is open");
  sqs_status s = st->sticky == SQS_OK ? run_pending(st, false) : st->sticky;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st->stream, &graph);
  const uint64_t launches = st->launches - st->launches_at_capture;
  HostSnap exit_snap = take_snap(st);
  st->capturing = false;
  st->static_ub = 0;
  put_snap(st, st->entry_snap);  // nothing ran: the device holds the entry state
  st->launches = st->launches_at_capture;
  st->pending.clear();
  if (s == SQS_OK && st->capture_err != SQS_OK) s = st->capture_err;
  if (s == SQS_OK && (e != cudaSuccess || !graph)) s = SQS_ERR_CUDA;
  cudaGraphExec_t exec = nullptr;
  if (s == SQS_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) s = SQS_ERR_CUDA;
  if (s != SQS_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    st->sticky = SQS_OK;
    return fail(st, s, "capture failed (%s)", st->err.c_str());
  }
  sqs_graph* g = new sqs_graph();
  g->st = st;
  g->graph = graph;
  g->exec = exec;
  g->entry = st->entry_snap;
  g->exit = std::move(exit_snap);
  g->launches = launches;
  *out = g;
  return SQS_OK;
}

sqs_status sqs_graph_launch(sqs_state* st, sqs_graph* g) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (!g || g->st != st) return fail(st, SQS_ERR_ARG, "graph of another state");
  if (st->capturing) return fail(st, SQS_ERR_STATE, "graph launch inside a capture");
  // The graph writes the buffers it was captured with, in their roles then.
  const void* now[3] = {st->cur.k0, st->alt.k0, st->bk.k0};
  const void* then[3] = {g->entry.cur.k0, g->entry.alt.k0, g->entry.bk.k0};
  for (const void* p : then)
    if (std::find(std::begin(now), std::end(now), p) == std::end(now))
      return fail(st, SQS_ERR_STATE, "the state's buffers changed since the capture");
  st->pending.clear();
  st->lazy.clear();
  put_snap(st, g->entry);
  cudaError_t e = cudaGraphLaunch(g->exec, st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "graph launch");
  put_snap(st, g->exit);
  st->launches += g->launches;
  return SQS_OK;
}

void sqs_graph_destroy(sqs_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

sqs_status sqs_state_stats(const sqs_state* st, sqs_stats* out) {
  if (!st || !out) return SQS_ERR_ARG;
  *out = st->stats;
  return SQS_OK;
}

const char* sqs_last_error(const sqs_state* st) {
  if (!st) return "null state";
  return st->err.c_str();
}

}  // extern "C"
