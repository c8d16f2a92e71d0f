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
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sqs.h"
#include "sqs_internal.h"

using sqs::Arr;
using sqs::Buckets;
using sqs::Ctl;
using sqs::DevOp;
using sqs::Gate1;
using sqs::OpList;

struct sqs_table {
  void* dev;
  uint64_t n;
  uint32_t bytes;
};

struct sqs_state {
  std::vector<uint32_t> width, offset;
  uint32_t total_bits = 0;
  int kw = 1;
  bool amp32 = false;
  uint32_t flags = 0;
  double eps = 1e-14;

  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 1;
  sqs_allocator alloc{};
  bool has_alloc = false;

  Arr cur{}, alt{};
  int cur_slot = 0;
  Buckets bk{};
  uint64_t bk_slots = 0;  // allocated branches in the bucket arrays
  uint32_t bk_counters = 0;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;  // pinned mirror
  double* scratch = nullptr;  // probabilities / format conversion
  size_t scratch_bytes = 0;

  std::vector<DevOp> pending;
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
};

namespace {

const char* kVersion = "sqs 0.1 (sm_103a)";

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
  if (st->has_alloc) {
    p = st->alloc.alloc(st->alloc.ctx, bytes, (void*)st->stream);
  } else if (cudaMallocAsync(&p, bytes, st->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dfree(sqs_state* st, void* p) {
  if (!p) return;
  if (st->has_alloc)
    st->alloc.free(st->alloc.ctx, p, (void*)st->stream);
  else
    cudaFreeAsync(p, st->stream);
}

size_t amp_bytes(const sqs_state* st) { return st->amp32 ? 8 : 16; }

void free_arr(sqs_state* st, Arr& a) {
  dfree(st, a.k0);
  dfree(st, a.k1);
  dfree(st, a.amp);
  a = Arr{};
}

bool alloc_arr(sqs_state* st, Arr& a, uint64_t cap) {
  a.k0 = (uint64_t*)dalloc(st, cap * 8);
  a.k1 = st->kw == 2 ? (uint64_t*)dalloc(st, cap * 8) : nullptr;
  a.amp = dalloc(st, cap * amp_bytes(st));
  a.cap = cap;
  if (!a.k0 || (st->kw == 2 && !a.k1) || !a.amp) {
    free_arr(st, a);
    return false;
  }
  return true;
}

uint64_t round_cap(uint64_t need) {
  uint64_t c = 1024;
  while (c < need) c = c + c / 2;
  return c;
}

uint64_t max_branches(const sqs_state* st) {
  return st->total_bits >= 63 ? (1ull << 63) : (1ull << st->total_bits);
}

// Brackets one launch with trace events when tracing is on.
struct Traced {
  sqs_state* st;
  int idx = -1;
  Traced(sqs_state* s, uint32_t kernel) : st(s) {
    if (st->ev.empty()) return;
    const size_t used = st->trace.size();
    if (2 * (used + 1) > st->ev.size()) {
      st->trace_dropped++;
      return;
    }
    idx = (int)used;
    st->trace.push_back(sqs_trace_record{kernel, st->call, 0.f, 0u});
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
  st->launches++;
  return L;
}

// Predicate on the packed key from (reg, bit, value) triples.
bool encode_ctrls(sqs_state* st, const sqs_ctrl* c, uint32_t n, uint64_t mask[2],
                  uint64_t val[2]) {
  mask[0] = mask[1] = val[0] = val[1] = 0;
  if (n > SQS_MAX_CTRL || (n && !c)) return false;
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
sqs_status sync_ctl(sqs_state* st) {
  cudaError_t e = cudaMemcpyAsync(st->ctl_host, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                  st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "synchronize");
  const Ctl& c = *st->ctl_host;
  if (c.err) {
    st->sticky = (c.err & sqs::kErrProbe) ? SQS_ERR_TIMEOUT : SQS_ERR_CAPACITY;
    return fail(st, st->sticky,
                "device error 0x%x at launch %u (needed %llu branches); reset the state", c.err,
                c.err_where, (unsigned long long)c.need);
  }
  st->ub = c.cnt[st->cur_slot];
  return SQS_OK;
}

sqs_status check_usable(sqs_state* st) {
  if (!st) return SQS_ERR_ARG;
  return st->sticky;
}

// Makes `alt` hold at least `need` branches.
sqs_status ensure_alt(sqs_state* st, uint64_t need) {
  if (st->alt.cap >= need && st->alt.k0) return SQS_OK;
  free_arr(st, st->alt);
  if (!alloc_arr(st, st->alt, round_cap(need)))
    return fail(st, SQS_ERR_OOM, "cannot allocate %llu branches", (unsigned long long)need);
  return SQS_OK;
}

sqs_status ensure_buckets(sqs_state* st, uint32_t B, uint32_t C) {
  const uint64_t slots = (uint64_t)B * C;
  if (st->bk_slots < slots || !st->bk.k0) {
    dfree(st, st->bk.k0);
    dfree(st, st->bk.k1);
    dfree(st, st->bk.amp);
    const uint64_t cap = round_cap(slots);
    st->bk.k0 = (uint64_t*)dalloc(st, cap * 8);
    st->bk.k1 = st->kw == 2 ? (uint64_t*)dalloc(st, cap * 8) : nullptr;
    st->bk.amp = dalloc(st, cap * amp_bytes(st));
    st->bk_slots = cap;
    if (!st->bk.k0 || (st->kw == 2 && !st->bk.k1) || !st->bk.amp)
      return fail(st, SQS_ERR_OOM, "cannot allocate merge buckets");
  }
  if (st->bk_counters < B || !st->bk.count) {
    dfree(st, st->bk.count);
    const uint32_t nc = std::max<uint32_t>(B, 1024);
    st->bk.count = (unsigned int*)dalloc(st, (size_t)nc * 4);
    if (!st->bk.count) return fail(st, SQS_ERR_OOM, "cannot allocate bucket counters");
    cudaMemsetAsync(st->bk.count, 0, (size_t)nc * 4, st->stream);
    st->bk_counters = nc;
  }
  st->bk.B = B;
  st->bk.C = C;
  return SQS_OK;
}

// Packs the queued operations into launch-sized lists.
void pack_ops(const std::vector<DevOp>& ops, size_t from, size_t to, OpList& L) {
  L.n = (uint32_t)(to - from);
  L.touches_keys = L.touches_amps = L.drops = 0;
  for (size_t i = from; i < to; ++i) {
    L.op[i - from] = ops[i];
    switch (ops[i].kind) {
      case sqs::OP_MUL:
        L.touches_amps = 1;
        break;
      case sqs::OP_MUL_XOR:
        L.touches_amps = 1;
        L.touches_keys = 1;
        break;
      case sqs::OP_PRUNE:
        L.drops = 1;
        break;
      default:
        L.touches_keys = 1;
        break;
    }
  }
}

// Runs queued operations as standalone passes, leaving at most kMaxOps for
// the kernel that follows (which fuses them).  keep_tail = false flushes all.
sqs_status run_pending(sqs_state* st, bool keep_tail) {
  size_t n = st->pending.size();
  size_t upto = keep_tail ? (n > (size_t)sqs::kMaxOps ? n - sqs::kMaxOps : 0) : n;
  size_t from = 0;
  OpList& L = st->ops_buf;
  while (from < upto) {
    const size_t to = std::min(upto, from + (size_t)sqs::kMaxOps);
    pack_ops(st->pending, from, to, L);
    cudaError_t e;
    if (L.drops) {
      const uint64_t need = st->ub;
      sqs_status s = ensure_alt(st, need);
      if (s != SQS_OK) return s;
      const int out_slot = (st->cur_slot + 1) & 3;
      Traced tr(st, SQS_K_COMPACT);
      e = sqs::launch_apply_compact(launch_of(st, st->ub), st->kw, st->amp32, st->ctl, st->cur,
                                    st->cur_slot, st->alt, out_slot, L);
      std::swap(st->cur, st->alt);
      st->cur_slot = out_slot;
    } else if (L.touches_keys || L.touches_amps) {
      Traced tr(st, SQS_K_APPLY);
      e = sqs::launch_apply_inplace(launch_of(st, st->ub), st->kw, st->amp32, st->ctl, st->cur,
                                    st->cur_slot, L);
    } else {
      e = cudaSuccess;
    }
    if (e != cudaSuccess) return cuda_fail(st, e, "launch");
    from = to;
  }
  st->pending.erase(st->pending.begin(), st->pending.begin() + upto);
  return SQS_OK;
}

// One interference step: fused pending run + partition + pair.
sqs_status run_branching(sqs_state* st, const Gate1& g) {
  sqs_status s = run_pending(st, true);
  if (s != SQS_OK) return s;
  OpList& L = st->ops_buf;
  pack_ops(st->pending, 0, st->pending.size(), L);
  st->pending.clear();
  // From here on a failure leaves the queue half-applied: errors are sticky.

  uint64_t out_ub = std::min(max_branches(st), 2 * st->ub);
  if (st->alt.cap < out_ub) {
    // The bound outgrew the allocation: learn the exact count first.
    s = sync_ctl(st);
    if (s != SQS_OK) return s;
    out_ub = std::min(max_branches(st), 2 * st->ub);
  }
  s = ensure_alt(st, out_ub);
  if (s != SQS_OK) return st->sticky = s;
  const uint32_t C = (uint32_t)sqs::pair_capacity(st->kw, st->amp32);
  const uint64_t target = (uint64_t)C * 3 / 4;
  const uint64_t B64 = std::max<uint64_t>(1, (st->ub + target - 1) / target);
  if (B64 > 0x7fffffffull) return st->sticky = fail(st, SQS_ERR_CAPACITY, "too many buckets");
  s = ensure_buckets(st, (uint32_t)B64, C);
  if (s != SQS_OK) return st->sticky = s;

  const int out_slot = (st->cur_slot + 1) & 3;
  cudaError_t e;
  {
    Traced tr(st, SQS_K_PARTITION);
    e = sqs::launch_partition(launch_of(st, st->ub), st->kw, st->amp32, st->ctl, st->cur,
                              st->cur_slot, L, g, st->bk, st->alt, out_slot);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "partition launch");
  {
    Traced tr(st, SQS_K_PAIR);
    e = sqs::launch_pair(launch_of(st, st->ub), st->kw, st->amp32, st->ctl, g, st->bk, st->alt,
                         out_slot);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "pair launch");
  std::swap(st->cur, st->alt);
  st->cur_slot = out_slot;
  st->ub = out_ub;
  return SQS_OK;
}

bool is_zero(double re, double im) { return re == 0.0 && im == 0.0; }

DevOp blank_op(uint32_t kind) {
  DevOp o;
  std::memset(&o, 0, sizeof(o));
  o.kind = kind;
  o.sel_bit = 128;
  return o;
}

void push_prune(sqs_state* st) {
  DevOp o = blank_op(sqs::OP_PRUNE);
  o.eps2 = st->eps * st->eps;
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
    DevOp o = blank_op(sqs::OP_MUL);
    o.pmask[0] = cm[0], o.pmask[1] = cm[1], o.pval[0] = cv[0], o.pval[1] = cv[1];
    o.sel_bit = t;
    o.c[0] = m[0], o.c[1] = m[1], o.c[2] = m[6], o.c[3] = m[7];
    st->pending.push_back(o);
    push_prune(st);
    return SQS_OK;
  }
  if (mode == 0 && is_zero(m[0], m[1]) && is_zero(m[6], m[7])) {
    // Anti-diagonal: flip plus phase (the _operate_off_diagonal strategy).
    // A branch with bit 0 moves to bit 1 with factor U10; bit 1 moves to 0 with U01.
    DevOp o = blank_op(sqs::OP_MUL_XOR);
    o.pmask[0] = cm[0], o.pmask[1] = cm[1], o.pval[0] = cv[0], o.pval[1] = cv[1];
    o.sel_bit = t;
    o.c[0] = m[4], o.c[1] = m[5], o.c[2] = m[2], o.c[3] = m[3];
    o.xmask[t >> 6] = 1ull << (t & 63);
    st->pending.push_back(o);
    push_prune(st);
    return SQS_OK;
  }
  Gate1 g;
  std::memset(&g, 0, sizeof(g));
  g.t = t;
  g.mode = (uint32_t)mode;
  g.cmask[0] = cm[0], g.cmask[1] = cm[1], g.cval[0] = cv[0], g.cval[1] = cv[1];
  if (mode == 0)
    for (int i = 0; i < 8; ++i) g.u[i] = m[i];
  g.ang_off = mode == 1 ? st->offset[angle_reg] : 0;
  g.ang_w = mode == 1 ? st->width[angle_reg] : 0;
  g.scale = scale;
  g.offset = offset;
  g.eps2 = st->eps * st->eps;
  return run_branching(st, g);
}

sqs_status flush_all(sqs_state* st) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  return run_pending(st, false);
}

}  // namespace

extern "C" {

const char* sqs_version(void) { return kVersion; }

sqs_status sqs_state_create(const uint32_t* reg_widths, uint32_t n_regs, uint32_t flags,
                            uint64_t capacity_hint, const sqs_allocator* allocator,
                            void* cuda_stream, sqs_state** out) {
  if (!out || !reg_widths || n_regs == 0 || n_regs > 128) return SQS_ERR_ARG;
  if (flags & ~(SQS_AMP_FP32 | SQS_SIZING_LEARNED | SQS_MERGE_HASH | SQS_MERGE_SORT))
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
  if (e != cudaSuccess) {
    sqs_status s = SQS_ERR_CUDA;
    delete st;
    cudaGetLastError();
    return s;
  }
  e = cudaMallocHost((void**)&st->ctl_host, sizeof(Ctl));
  if (e != cudaSuccess) {
    delete st;
    return SQS_ERR_OOM;
  }
  st->ctl = (Ctl*)dalloc(st, sizeof(Ctl));
  const uint64_t cap = round_cap(std::max<uint64_t>(capacity_hint, 1024));
  if (!st->ctl || !alloc_arr(st, st->cur, cap) || !alloc_arr(st, st->alt, cap)) {
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
  free_arr(st, st->cur);
  free_arr(st, st->alt);
  dfree(st, st->bk.k0);
  dfree(st, st->bk.k1);
  dfree(st, st->bk.amp);
  dfree(st, st->bk.count);
  dfree(st, st->ctl);
  dfree(st, st->scratch);
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
  st->sticky = SQS_OK;
  st->err.clear();
  st->cur_slot = 0;
  st->ub = 1;
  if (st->bk.count) cudaMemsetAsync(st->bk.count, 0, (size_t)st->bk_counters * 4, st->stream);
  st->call = 1;  // API calls are numbered from the reset
  Traced tr(st, SQS_K_INIT);
  cudaError_t e = sqs::launch_init(launch_of(st, 1), st->ctl, st->cur, 0, st->amp32);
  if (e != cudaSuccess) return cuda_fail(st, e, "reset");
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
  std::vector<DevOp> add;
  add.reserve(n_ops);
  const uint32_t nr = (uint32_t)st->width.size();
  for (uint32_t i = 0; i < n_ops; ++i) {
    const sqs_perm_op& p = ops[i];
    if (p.reg >= nr) return fail(st, SQS_ERR_ARG, "op %u: bad register", i);
    uint64_t cm[2], cv[2];
    if (!encode_ctrls(st, p.ctrl, p.n_ctrl, cm, cv))
      return fail(st, SQS_ERR_ARG, "op %u: bad controls", i);
    DevOp o = blank_op(sqs::OP_XOR);
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
    add.push_back(o);
  }
  st->pending.insert(st->pending.end(), add.begin(), add.end());
  return SQS_OK;
}

sqs_status sqs_apply_phase(sqs_state* st, const sqs_ctrl* pred, uint32_t n_pred, double phi) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  if (!std::isfinite(phi)) return fail(st, SQS_ERR_ARG, "non-finite phase");
  uint64_t cm[2], cv[2];
  if (!encode_ctrls(st, pred, n_pred, cm, cv)) return fail(st, SQS_ERR_ARG, "bad predicates");
  DevOp o = blank_op(sqs::OP_MUL);
  o.pmask[0] = cm[0], o.pmask[1] = cm[1], o.pval[0] = cv[0], o.pval[1] = cv[1];
  o.c[0] = std::cos(phi);
  o.c[1] = std::sin(phi);
  st->pending.push_back(o);
  return SQS_OK;
}

sqs_status sqs_table_create(sqs_state* st, const void* host_entries, uint64_t n_entries,
                            uint32_t entry_bytes, sqs_table** out) {
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

static sqs_status qram(sqs_state* st, uint32_t addr_reg, uint32_t data_reg, const sqs_table* t) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  st->call++;
  const uint32_t nr = (uint32_t)st->width.size();
  if (!t || addr_reg >= nr || data_reg >= nr || addr_reg == data_reg)
    return fail(st, SQS_ERR_ARG, "bad QRAM arguments");
  bool owned = false;
  for (sqs_table* x : st->tables) owned |= (x == t);
  if (!owned) return fail(st, SQS_ERR_ARG, "table belongs to another state");
  DevOp o = blank_op(sqs::OP_QRAM);
  o.dst_off = st->offset[data_reg];
  o.dst_w = st->width[data_reg];
  o.src_off = st->offset[addr_reg];
  o.src_w = st->width[addr_reg];
  o.table = t->dev;
  o.n_entries = t->n;
  o.entry_bytes = t->bytes;
  st->pending.push_back(o);
  return SQS_OK;
}

sqs_status sqs_qram_load(sqs_state* st, uint32_t addr_reg, uint32_t data_reg,
                         const sqs_table* table) {
  return qram(st, addr_reg, data_reg, table);
}

sqs_status sqs_qram_unload(sqs_state* st, uint32_t addr_reg, uint32_t data_reg,
                           const sqs_table* table) {
  return qram(st, addr_reg, data_reg, table);
}

sqs_status sqs_prune(sqs_state* st, double eps, uint64_t* nnz_out) {
  sqs_status s = check_usable(st);
  if (s != SQS_OK) return s;
  if (!(eps >= 0.0) || std::isinf(eps)) return fail(st, SQS_ERR_ARG, "bad eps");
  DevOp o = blank_op(sqs::OP_PRUNE);
  o.eps2 = eps * eps;
  st->pending.push_back(o);
  s = run_pending(st, false);
  if (s != SQS_OK) return s;
  if (nnz_out) {
    s = sync_ctl(st);
    if (s != SQS_OK) return s;
    *nnz_out = st->ctl_host->cnt[st->cur_slot];
  }
  return SQS_OK;
}

static sqs_status ensure_scratch(sqs_state* st, size_t bytes) {
  if (st->scratch_bytes >= bytes && st->scratch) return SQS_OK;
  dfree(st, st->scratch);
  st->scratch = (double*)dalloc(st, bytes);
  st->scratch_bytes = st->scratch ? bytes : 0;
  return st->scratch ? SQS_OK : fail(st, SQS_ERR_OOM, "cannot allocate scratch");
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
    e = sqs::launch_probabilities(launch_of(st, st->ub), st->kw, st->amp32, st->ctl, st->cur,
                                  st->cur_slot, st->offset[reg], w, probs_dev, norm2_dev);
  }
  if (e != cudaSuccess) return cuda_fail(st, e, "probabilities");
  return SQS_OK;
}

sqs_status sqs_probabilities(sqs_state* st, uint32_t reg, double* probs, double* norm2) {
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
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (!out) return fail(st, SQS_ERR_ARG, "null output");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  *out = st->ctl_host->cnt[st->cur_slot];
  return SQS_OK;
}

sqs_status sqs_peak_nnz(sqs_state* st, uint64_t* out) {
  sqs_status s = flush_all(st);
  if (s != SQS_OK) return s;
  if (!out) return fail(st, SQS_ERR_ARG, "null output");
  s = sync_ctl(st);
  if (s != SQS_OK) return s;
  *out = std::max<uint64_t>(st->ctl_host->peak, st->ctl_host->cnt[st->cur_slot]);
  return SQS_OK;
}

sqs_status sqs_export(sqs_state* st, uint64_t* keys, double* amps, uint64_t cap, uint64_t* n) {
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
  cudaError_t e;
  if (st->kw == 1) {
    e = cudaMemcpyAsync(keys, st->cur.k0, cnt * 8, cudaMemcpyDeviceToHost, st->stream);
  } else {
    e = cudaMemcpy2DAsync(keys, 16, st->cur.k0, 8, 8, cnt, cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(keys + 1, 16, st->cur.k1, 8, 8, cnt, cudaMemcpyDeviceToHost,
                            st->stream);
  }
  if (e == cudaSuccess) {
    if (st->amp32) {
      s = ensure_scratch(st, cnt * 16);
      if (s != SQS_OK) return s;
      e = sqs::launch_to_f64(launch_of(st, cnt), st->ctl, st->cur, st->cur_slot, st->scratch);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(amps, st->scratch, cnt * 16, cudaMemcpyDeviceToHost, st->stream);
    } else {
      e = cudaMemcpyAsync(amps, st->cur.amp, cnt * 16, cudaMemcpyDeviceToHost, st->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(st, e, "export");
  return SQS_OK;
}

sqs_status sqs_import(sqs_state* st, const uint64_t* keys, const double* amps, uint64_t n) {
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
  st->pending.clear();
  if (st->cur.cap < n) {
    free_arr(st, st->cur);
    if (!alloc_arr(st, st->cur, round_cap(n))) return fail(st, SQS_ERR_OOM, "import");
  }
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
          e = sqs::launch_from_f64(launch_of(st, n), st->ctl, st->cur, st->scratch, n);
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
  return SQS_OK;
}

sqs_status sqs_sync(sqs_state* st) {
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

const char* sqs_last_error(const sqs_state* st) {
  if (!st) return "null state";
  return st->err.c_str();
}

}  // extern "C"
