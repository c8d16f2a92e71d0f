// sqs_apply_u1q_noalloc: one interference step on a state that the caller
// keeps in its own device memory, for callers that cannot allocate device
// memory at all (see include/sqs.h for who they are and the contract).
//
// The merge needs scratch space -- hash buckets, per-bucket output segments,
// segment offsets and a control block -- which the state-based entry points
// allocate.  Here it lives in one file-scope device array of fixed size,
// resident on every device that loads the library until the process exits.
// Host code must not use the array's name as a device address: it gets the
// address from cudaGetSymbolAddress once per device and passes it on.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/sqs.h"
#include "sqs_internal.h"

namespace {

using sqs::Arr;
using sqs::Ctl;
using sqs::Gate1;

constexpr uint32_t kBucketLog2 = 11;   // same tile as the state-based merge
constexpr uint32_t kSegLog2 = 12;      // output segment = 2 x bucket
constexpr uint64_t kTarget = 1536;     // mean fill per bucket
constexpr uint64_t kMaxB = (SQS_NOALLOC_MAX_BRANCHES + kTarget - 1) / kTarget;

// Scratch layout (bytes, each region 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kCtlOff = 0;
constexpr size_t kBkK0Off = align256(kCtlOff + sizeof(Ctl));
constexpr size_t kBkSlots = kMaxB << kBucketLog2;
constexpr size_t kBkK1Off = align256(kBkK0Off + kBkSlots * 8);
constexpr size_t kBkAmpOff = align256(kBkK1Off + kBkSlots * 8);
constexpr size_t kBkCntOff = align256(kBkAmpOff + kBkSlots * 16);
constexpr size_t kOutSlots = kMaxB << kSegLog2;
constexpr size_t kOutK0Off = align256(kBkCntOff + kMaxB * 4);
constexpr size_t kOutK1Off = align256(kOutK0Off + kOutSlots * 8);
constexpr size_t kOutAmpOff = align256(kOutK1Off + kOutSlots * 8);
constexpr size_t kOutCntOff = align256(kOutAmpOff + kOutSlots * 16);
constexpr size_t kOffsetsOff = align256(kOutCntOff + kMaxB * 4);
constexpr size_t kScratchBytes = align256(kOffsetsOff + kMaxB * 8);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-device address of the array (set-up once per device).
constexpr int kMaxDevices = 64;
unsigned char* g_base[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;
thread_local char g_msg[256] = "";

sqs_status say(sqs_status s, const char* msg) {
  std::strncpy(g_msg, msg, sizeof(g_msg) - 1);
  g_msg[sizeof(g_msg) - 1] = 0;
  return s;
}

// Clears the control block, the bucket counters and the output-segment
// counters, then records the input count: every call starts from zero state
// whatever the previous call left.  A merge that stops on a device-side error
// leaves some output segments unwritten; their counters must read zero then,
// not the previous call's counts, or the final copy would run past out_cap.
__global__ void k_noalloc_begin(Ctl* ctl, unsigned int* bucket_cnt, unsigned int* seg_cnt,
                                uint32_t B, uint64_t n_in) {
  for (uint32_t i = threadIdx.x; i < B; i += blockDim.x) {
    bucket_cnt[i] = 0u;
    seg_cnt[i] = 0u;
  }
  if (threadIdx.x == 0) {
    unsigned long long* w = (unsigned long long*)ctl;
    for (size_t i = 0; i < sizeof(Ctl) / sizeof(unsigned long long); ++i) w[i] = 0ull;
    ctl->cnt[0] = n_in;
  }
}

// Exclusive offsets of the output segments and the total count, written to
// the caller's counter (all-ones when the merge flagged an error).  After an
// error every segment count is zeroed, so the final copy writes nothing into
// the caller's output arrays.
__global__ void k_noalloc_offsets(const Ctl* ctl, unsigned int* seg_cnt, uint32_t B,
                                  uint64_t out_cap, unsigned long long* offsets,
                                  unsigned long long* n_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long run = 0;
  for (uint32_t s = 0; s < B; ++s) {
    offsets[s] = run;
    run += seg_cnt[s];
  }
  const bool bad = ctl->err != 0u || run > out_cap;
  if (bad)
    for (uint32_t s = 0; s < B; ++s) seg_cnt[s] = 0u;
  *n_out = bad ? ~0ull : run;
}

}  // namespace

extern "C" sqs_status sqs_apply_u1q_noalloc(const uint32_t* reg_widths, uint32_t n_regs,
                                            uint32_t reg, uint32_t bit, const double m[8],
                                            const sqs_ctrl* ctrl, uint32_t n_ctrl, double eps,
                                            const uint64_t* keys_lo_in,
                                            const uint64_t* keys_hi_in, const double* amps_in,
                                            uint64_t n_in, uint64_t* keys_lo_out,
                                            uint64_t* keys_hi_out, double* amps_out,
                                            uint64_t out_cap, uint64_t* n_out, void* stream) {
  // ---- arguments (host-side checks; nothing is enqueued on failure) ----
  if (!reg_widths || n_regs == 0 || n_regs > 128 || !m || !n_out)
    return say(SQS_ERR_ARG, "null argument or bad register count");
  uint32_t total = 0, off = 0, t = 0;
  for (uint32_t j = 0; j < n_regs; ++j) {
    if (reg_widths[j] < 1 || reg_widths[j] > 64) return say(SQS_ERR_ARG, "register width");
    if (j == reg) t = off + bit;
    off += reg_widths[j];
  }
  total = off;
  if (total > 128) return say(SQS_ERR_ARG, "more than 128 qubits");
  if (reg >= n_regs || bit >= reg_widths[reg]) return say(SQS_ERR_ARG, "target out of range");
  if (n_in > SQS_NOALLOC_MAX_BRANCHES)
    return say(SQS_ERR_ARG, "input has more branches than SQS_NOALLOC_MAX_BRANCHES");
  if (out_cap < 2 * n_in) return say(SQS_ERR_ARG, "out_cap must be at least 2 * n_in");
  const int kw = total > 64 ? 2 : 1;
  if (n_in && (!keys_lo_in || !amps_in || (kw == 2 && !keys_hi_in)))
    return say(SQS_ERR_ARG, "null input arrays");
  if (!keys_lo_out || !amps_out || (kw == 2 && !keys_hi_out))
    return say(SQS_ERR_ARG, "null output arrays");
  if (!(eps >= 0.0) || eps == __builtin_inf()) return say(SQS_ERR_ARG, "bad eps");
  if (n_ctrl > SQS_MAX_CTRL || (n_ctrl && !ctrl)) return say(SQS_ERR_ARG, "bad controls");
  Gate1 g;
  std::memset(&g, 0, sizeof(g));
  for (uint32_t i = 0; i < n_ctrl; ++i) {
    if (ctrl[i].reg >= n_regs || ctrl[i].bit >= reg_widths[ctrl[i].reg] || ctrl[i].value > 1)
      return say(SQS_ERR_ARG, "bad controls");
    uint32_t q = ctrl[i].bit;
    for (uint32_t j = 0; j < ctrl[i].reg; ++j) q += reg_widths[j];
    if (q == t) return say(SQS_ERR_ARG, "a control sits on the target qubit");
    g.cmask[q >> 6] |= 1ull << (q & 63);
    if (ctrl[i].value) g.cval[q >> 6] |= 1ull << (q & 63);
  }
  for (int i = 0; i < 8; ++i) {
    if (!(m[i] == m[i]) || m[i] == __builtin_inf() || m[i] == -__builtin_inf())
      return say(SQS_ERR_ARG, "non-finite matrix entry");
    g.u[i] = m[i];
    g.uf[i] = (float)m[i];
    g.ufl[i] = (float)(m[i] - (double)g.uf[i]);
  }
  g.t = t;
  g.mode = (m[1] == 0.0 && m[3] == 0.0 && m[5] == 0.0 && m[7] == 0.0) ? 2u : 0u;
  g.reuse = 0;  // every product computed: same results, no flags needed
  g.eps = eps;
  g.eps2 = eps * eps;
  g.epsf = (float)eps;
  g.rho32 = 0x1p-19f;  // unused: FP64 amplitudes

  // ---- set-up: the array's device address, once per device ----
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return say(SQS_ERR_CUDA, "no device");
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_base[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return say(SQS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_base[dev] = (unsigned char*)p;
    }
  }
  unsigned char* base = g_base[dev];
  cudaStream_t s = (cudaStream_t)stream;

  // ---- views into the scratch array ----
  const uint32_t B = (uint32_t)(n_in ? (n_in + kTarget - 1) / kTarget : 1);
  Ctl* ctl = (Ctl*)(base + kCtlOff);
  Arr in{};
  in.k0 = (uint64_t*)keys_lo_in;
  in.k1 = kw == 2 ? (uint64_t*)keys_hi_in : nullptr;
  in.amp = (void*)amps_in;
  in.cap = n_in;
  Arr bk{};
  bk.k0 = (uint64_t*)(base + kBkK0Off);
  bk.k1 = kw == 2 ? (uint64_t*)(base + kBkK1Off) : nullptr;
  bk.amp = base + kBkAmpOff;
  bk.cap = kBkSlots;
  bk.seg_cnt = (unsigned int*)(base + kBkCntOff);
  bk.seg_log2 = kBucketLog2;
  bk.n_seg = B;
  Arr seg{};
  seg.k0 = (uint64_t*)(base + kOutK0Off);
  seg.k1 = kw == 2 ? (uint64_t*)(base + kOutK1Off) : nullptr;
  seg.amp = base + kOutAmpOff;
  seg.cap = kOutSlots;
  seg.seg_cnt = (unsigned int*)(base + kOutCntOff);
  seg.seg_log2 = kSegLog2;
  seg.n_seg = B;
  Arr out{};
  out.k0 = keys_lo_out;
  out.k1 = kw == 2 ? keys_hi_out : nullptr;
  out.amp = amps_out;
  out.cap = out_cap;
  unsigned long long* offsets = (unsigned long long*)(base + kOffsetsOff);

  static const sqs::OpList kNoOps = [] {
    sqs::OpList L;
    std::memset(&L, 0, sizeof(L));
    return L;
  }();
  sqs::Launch L;
  L.stream = s;
  L.sm_count = 152;
  cudaDeviceGetAttribute(&L.sm_count, cudaDevAttrMultiProcessorCount, dev);
  L.seq = 1;
  L.n_hint = n_in;

  // ---- the merge: clear, partition, pair, offsets, dense copy ----
  k_noalloc_begin<<<1, 256, 0, s>>>(ctl, bk.seg_cnt, seg.seg_cnt, B, n_in);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = sqs::launch_partition(L, kw, false, ctl, in, 0, kNoOps, g, bk, 0u);
  if (e == cudaSuccess) e = sqs::launch_pair(L, kw, false, ctl, g, bk, seg, 1);
  if (e == cudaSuccess) {
    k_noalloc_offsets<<<1, 32, 0, s>>>(ctl, seg.seg_cnt, B, out_cap, offsets,
                                       (unsigned long long*)n_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = sqs::launch_densify(L, kw, false, seg, (const uint64_t*)offsets, out);
  if (e != cudaSuccess) return say(SQS_ERR_CUDA, cudaGetErrorString(e));
  return say(SQS_OK, "");
}

extern "C" const char* sqs_noalloc_last_error(void) { return g_msg; }

extern "C" uint64_t sqs_noalloc_scratch_bytes(void) { return (uint64_t)kScratchBytes; }
