// CUDA kernels of the sparse register-level state library (sm_103a).
//
// The state is a structure of arrays: k0[] (key bits 0..63), k1[] (bits
// 64..127, two-word keys only) and amp[] (complex<double> or complex<float>),
// with its branch count in device memory (Ctl::cnt).  Every kernel here is a
// bandwidth-bound stream over those arrays; nothing is a dense contraction, so
// no tensor cores are used.
//
//  k_apply_inplace   runs of non-interference operations, fused (Sec. II.D.1)
//  k_apply_compact   the same when the run may drop branches (pruning)
//  k_partition       fused run + the first half of an interference operation:
//                    scatters each controlled branch into a hash bucket keyed
//                    by its pair class (key with the target bit cleared), so
//                    the two members of a coherent pair (Sec. II.D.2: branches
//                    equal on every idle qubit) meet in one bucket
//  k_pair            one CTA per bucket: pairs the members in a shared-memory
//                    open-addressing table, applies the 2x2 (FP64), drops
//                    |a| < eps, appends the survivors with warp-ballot
//                    compaction
//  k_probabilities   FP64 marginal probabilities and norm
#include <cuda_runtime.h>
#include <stdint.h>

#include "sqs_internal.h"

namespace sqs {

typedef unsigned __int128 u128;

template <int KW>
struct KT;
template <>
struct KT<1> {
  typedef uint64_t T;
};
template <>
struct KT<2> {
  typedef u128 T;
};

template <int KW>
__device__ __forceinline__ typename KT<KW>::T mk(uint64_t lo, uint64_t hi);
template <>
__device__ __forceinline__ uint64_t mk<1>(uint64_t lo, uint64_t) {
  return lo;
}
template <>
__device__ __forceinline__ u128 mk<2>(uint64_t lo, uint64_t hi) {
  return (((u128)hi) << 64) | (u128)lo;
}

__device__ __forceinline__ uint64_t lo64(uint64_t k) { return k; }
__device__ __forceinline__ uint64_t lo64(u128 k) { return (uint64_t)k; }
__device__ __forceinline__ uint64_t hi64(uint64_t) { return 0; }
__device__ __forceinline__ uint64_t hi64(u128 k) { return (uint64_t)(k >> 64); }

__device__ __forceinline__ uint64_t wmask(uint32_t w) {
  return w >= 64 ? ~0ull : ((1ull << w) - 1ull);
}

template <class K>
__device__ __forceinline__ uint64_t get_field(K k, uint32_t off, uint32_t w) {
  return (uint64_t)(k >> off) & wmask(w);
}

template <class K>
__device__ __forceinline__ K set_field(K k, uint32_t off, uint32_t w, uint64_t v) {
  const K m = ((K)wmask(w)) << off;
  return (k & ~m) | (((K)(v & wmask(w))) << off);
}

// splitmix64 finalizer (Steele, Lea, Flood 2014): a bijective 64-bit mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t khash(uint64_t k) { return mix64(k); }
__device__ __forceinline__ uint64_t khash(u128 k) {
  return mix64((uint64_t)k ^ mix64((uint64_t)(k >> 64) + 0x9e3779b97f4a7c15ull));
}

// ---- amplitudes ------------------------------------------------------------
__device__ __forceinline__ double2 ld_amp(const double2* p, uint64_t i) { return p[i]; }
__device__ __forceinline__ double2 ld_amp(const float2* p, uint64_t i) {
  const float2 f = p[i];
  return make_double2((double)f.x, (double)f.y);
}
__device__ __forceinline__ void st_amp(double2* p, uint64_t i, double2 v) { p[i] = v; }
__device__ __forceinline__ void st_amp(float2* p, uint64_t i, double2 v) {
  p[i] = make_float2((float)v.x, (float)v.y);
}

// (a.x + i a.y)(b.x + i b.y), each product rounded, then one rounded sum.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                      __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double norm2(double2 a) {
  return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}

// ---- keys --------------------------------------------------------------------
template <int KW>
__device__ __forceinline__ typename KT<KW>::T ld_key(const Arr& a, uint64_t i);
template <>
__device__ __forceinline__ uint64_t ld_key<1>(const Arr& a, uint64_t i) {
  return a.k0[i];
}
template <>
__device__ __forceinline__ u128 ld_key<2>(const Arr& a, uint64_t i) {
  return mk<2>(a.k0[i], a.k1[i]);
}
template <int KW>
__device__ __forceinline__ void st_key(const Arr& a, uint64_t i, typename KT<KW>::T k) {
  a.k0[i] = lo64(k);
  if (KW == 2) a.k1[i] = hi64(k);
}

// ---- errors --------------------------------------------------------------------
__device__ __forceinline__ void raise_err(Ctl* ctl, unsigned int bit, uint32_t seq,
                                          unsigned long long need) {
  if (atomicOr(&ctl->err, bit) == 0u) ctl->err_where = seq;
  atomicMax(&ctl->need, need);
}

// ---- fused operation run ---------------------------------------------------------
template <int KW>
__device__ __forceinline__ bool apply_ops(const OpList& L, typename KT<KW>::T& k, double2& a) {
  typedef typename KT<KW>::T K;
#pragma unroll 1
  for (uint32_t o = 0; o < L.n; ++o) {
    const DevOp& op = L.op[o];
    const bool on = (k & mk<KW>(op.pmask[0], op.pmask[1])) == mk<KW>(op.pval[0], op.pval[1]);
    switch (op.kind) {
      case OP_XOR:
        if (on) k ^= mk<KW>(op.xmask[0], op.xmask[1]);
        break;
      case OP_ADD_REG:
        if (on)
          k = set_field<K>(k, op.dst_off, op.dst_w,
                           get_field(k, op.dst_off, op.dst_w) + get_field(k, op.src_off, op.src_w));
        break;
      case OP_SUB_REG:
        if (on)
          k = set_field<K>(k, op.dst_off, op.dst_w,
                           get_field(k, op.dst_off, op.dst_w) - get_field(k, op.src_off, op.src_w));
        break;
      case OP_ADD_CONST:
        if (on)
          k = set_field<K>(k, op.dst_off, op.dst_w, get_field(k, op.dst_off, op.dst_w) + op.constant);
        break;
      case OP_SWAP:
        if (on) {
          const uint64_t v1 = get_field(k, op.dst_off, op.dst_w);
          const uint64_t v2 = get_field(k, op.src_off, op.src_w);
          k = set_field<K>(set_field<K>(k, op.dst_off, op.dst_w, v2), op.src_off, op.src_w, v1);
        }
        break;
      case OP_QRAM:
        if (on) {
          const uint64_t addr = get_field(k, op.src_off, op.src_w);
          uint64_t d = 0;
          if (addr < op.n_entries) {
            switch (op.entry_bytes) {
              case 1: d = __ldg((const uint8_t*)op.table + addr); break;
              case 2: d = __ldg((const uint16_t*)op.table + addr); break;
              case 4: d = __ldg((const uint32_t*)op.table + addr); break;
              default: d = __ldg((const unsigned long long*)op.table + addr); break;
            }
          }
          k = set_field<K>(k, op.dst_off, op.dst_w, get_field(k, op.dst_off, op.dst_w) ^ d);
        }
        break;
      case OP_MUL:
      case OP_MUL_XOR:
        if (on) {
          const bool one = op.sel_bit < 128 && ((k >> op.sel_bit) & (K)1) != (K)0;
          const double2 c = one ? make_double2(op.c[2], op.c[3]) : make_double2(op.c[0], op.c[1]);
          a = cmul(a, c);
          if (op.kind == OP_MUL_XOR) k ^= mk<KW>(op.xmask[0], op.xmask[1]);
        }
        break;
      case OP_PRUNE:
        if (norm2(a) < op.eps2) return false;
        break;
      default:
        break;
    }
  }
  return true;
}

// Warp-aggregated append of up to one branch per lane into `out`; returns the
// base reserved for the warp's survivors.  Lanes with keep == false write
// nothing.  Every lane of the warp must call it.
template <int KW, class AT>
__device__ __forceinline__ void warp_append(Ctl* ctl, uint32_t seq, Arr out, int out_slot,
                                            bool keep, typename KT<KW>::T k, double2 a) {
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int ball = __ballot_sync(0xffffffffu, keep);
  if (ball == 0u) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&ctl->cnt[out_slot], (unsigned long long)__popc(ball));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (keep) {
    const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
    if (pos < out.cap) {
      st_key<KW>(out, pos, k);
      st_amp((AT*)out.amp, pos, a);
    } else {
      raise_err(ctl, kErrCapacity, seq, pos + 1);
    }
  }
}

template <class AT>
__global__ void k_init(Ctl* ctl, Arr a, int slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    a.k0[0] = 0;
    if (a.k1) a.k1[0] = 0;
    st_amp((AT*)a.amp, 0, make_double2(1.0, 0.0));
    for (int s = 0; s < 4; ++s) ctl->cnt[s] = 0;
    ctl->cnt[slot] = 1;
    ctl->peak = 1;
    ctl->need = 0;
    ctl->err = 0;
    ctl->err_where = 0;
    ctl->norm2 = 0;
  }
}

// ---------------------------------------------------------------------------
template <int KW, class AT, bool TK, bool TA>
__global__ void __launch_bounds__(256) k_apply_inplace(Ctl* ctl, Arr a, int slot,
                                                       const __grid_constant__ OpList ops,
                                                       uint32_t seq) {
  if (ctl->err) return;
  const unsigned long long n = ctl->cnt[slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, n);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    typename KT<KW>::T k = ld_key<KW>(a, i);
    double2 v = TA ? ld_amp((const AT*)a.amp, i) : make_double2(0.0, 0.0);
    apply_ops<KW>(ops, k, v);
    if (TK) st_key<KW>(a, i, k);
    if (TA) st_amp((AT*)a.amp, i, v);
  }
}

template <int KW, class AT>
__global__ void __launch_bounds__(256) k_apply_compact(Ctl* ctl, Arr in, int in_slot, Arr out,
                                                       int out_slot,
                                                       const __grid_constant__ OpList ops,
                                                       uint32_t seq) {
  if (ctl->err) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[(out_slot + 1) & 3] = 0;
  const unsigned long long n = ctl->cnt[in_slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, n);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // The loop bound is rounded up to whole warps so every lane joins the ballot.
  const uint64_t n_pad = (n + 31ull) & ~31ull;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
    bool keep = false;
    typename KT<KW>::T k = 0;
    double2 v = make_double2(0.0, 0.0);
    if (i < n) {
      k = ld_key<KW>(in, i);
      v = ld_amp((const AT*)in.amp, i);
      keep = apply_ops<KW>(ops, k, v);
    }
    warp_append<KW, AT>(ctl, seq, out, out_slot, keep, k, v);
  }
}

// ---------------------------------------------------------------------------
template <int KW, class AT>
__global__ void __launch_bounds__(256) k_partition(Ctl* ctl, Arr in, int in_slot,
                                                   const __grid_constant__ OpList ops, Gate1 g,
                                                   Buckets bk, Arr out, int out_slot,
                                                   uint32_t seq) {
  typedef typename KT<KW>::T K;
  if (ctl->err) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[(out_slot + 1) & 3] = 0;
  const unsigned long long n = ctl->cnt[in_slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, n);
  const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
  const K cval = mk<KW>(g.cval[0], g.cval[1]);
  const K bmask = ((K)1) << g.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n_pad = (n + 31ull) & ~31ull;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
    bool alive = false;
    K k = 0;
    double2 v = make_double2(0.0, 0.0);
    if (i < n) {
      k = ld_key<KW>(in, i);
      v = ld_amp((const AT*)in.amp, i);
      alive = apply_ops<KW>(ops, k, v);
    }
    const bool ctrl = alive && ((k & cmask) == cval);
    if (ctrl) {
      const uint64_t h = khash(k & ~bmask);
      const uint32_t b = (uint32_t)(((h >> 32) * (uint64_t)bk.B) >> 32);
      const unsigned int pos = atomicAdd(&bk.count[b], 1u);
      if (pos < bk.C) {
        const uint64_t j = (uint64_t)b * bk.C + pos;
        bk.k0[j] = lo64(k);
        if (KW == 2) bk.k1[j] = hi64(k);
        st_amp((AT*)bk.amp, j, v);
      } else {
        raise_err(ctl, kErrBucket, seq, (unsigned long long)pos + 1);
      }
    }
    // Branches the controls leave alone go straight to the output.
    warp_append<KW, AT>(ctl, seq, out, out_slot, alive && !ctrl, k, v);
  }
}

// ---------------------------------------------------------------------------
// One CTA per bucket.  Shared memory: keys[C], amps[C] (storage type),
// slots[S] (S = 2C, 0 = empty, else index + 1), partner[C].
constexpr int kPairThreads = 256;

template <int KW, class AT>
__global__ void __launch_bounds__(kPairThreads) k_pair(Ctl* ctl, Gate1 g, Buckets bk, Arr out,
                                                       int out_slot, uint32_t seq) {
  typedef typename KT<KW>::T K;
  extern __shared__ __align__(16) unsigned char smem[];
  if (ctl->err) return;
  const uint32_t C = bk.C;
  const uint32_t S = 2u * C;
  K* skey = (K*)smem;
  AT* samp = (AT*)(smem + (size_t)C * sizeof(K));
  unsigned int* slot = (unsigned int*)(smem + (size_t)C * (sizeof(K) + sizeof(AT)));
  int* partner = (int*)(slot + S);

  const uint32_t b = blockIdx.x;
  const uint32_t n = bk.count[b];
  if (n > C) return;  // overflow already flagged by the partition
  const uint64_t base = (uint64_t)b * C;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    skey[i] = mk<KW>(bk.k0[base + i], KW == 2 ? bk.k1[base + i] : 0ull);
    samp[i] = ((const AT*)bk.amp)[base + i];
    partner[i] = -1;
  }
  for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) slot[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) bk.count[b] = 0u;  // bucket is clean for the next use

  const K bmask = ((K)1) << g.t;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const K p = skey[i] & ~bmask;
    uint32_t h = (uint32_t)khash(p) & (S - 1u);
    // At most C entries live in 2C slots, so a free slot or the partner is
    // always found within S probes; the bound only guards against misuse.
    uint32_t probe = 0;
    for (; probe < S; ++probe) {
      const unsigned int old = atomicCAS(&slot[h], 0u, i + 1u);
      if (old == 0u) break;
      const uint32_t j = old - 1u;
      if ((skey[j] & ~bmask) == p) {
        partner[i] = (int)j;
        partner[j] = (int)i;
        break;
      }
      h = (h + 1u) & (S - 1u);
    }
    if (probe == S) raise_err(ctl, kErrProbe, seq, 0);
  }
  __syncthreads();

  // Emission in two sweeps over the same rounds: the first counts the
  // surviving children of every (round, warp), a scan turns the counts into
  // offsets and one atomic per CTA reserves the output run; the second sweep
  // recomputes the children and writes them, each warp to a contiguous range.
  const uint32_t rounds = (n + blockDim.x - 1u) / blockDim.x;
  const uint32_t nwarps = blockDim.x >> 5;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const unsigned int lt = (1u << lane) - 1u;
  unsigned long long* woff = (unsigned long long*)(partner + C);  // rounds * nwarps + 1
  for (int sweep = 0; sweep < 2; ++sweep) {
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t i = r * blockDim.x + threadIdx.x;
      bool keep0 = false, keep1 = false;
      K p = 0;
      double2 o0 = make_double2(0.0, 0.0), o1 = make_double2(0.0, 0.0);
      if (i < n) {
        const K k = skey[i];
        const bool kt = (k & bmask) != (K)0;
        const int j = partner[i];
        if (!(kt && j >= 0)) {  // the bit-1 member of a pair is emitted by its partner
          p = k & ~bmask;
          double2 U00, U01, U10, U11;
          if (g.mode == 1) {
            const double theta = g.scale * (double)get_field(p, g.ang_off, g.ang_w) + g.offset;
            double sn, cs;
            sincos(theta * 0.5, &sn, &cs);
            U00 = make_double2(cs, 0.0);
            U01 = make_double2(-sn, 0.0);
            U10 = make_double2(sn, 0.0);
            U11 = make_double2(cs, 0.0);
          } else {
            U00 = make_double2(g.u[0], g.u[1]);
            U01 = make_double2(g.u[2], g.u[3]);
            U10 = make_double2(g.u[4], g.u[5]);
            U11 = make_double2(g.u[6], g.u[7]);
          }
          const double2 ai = ld_amp(samp, i);
          if (!kt) {
            o0 = cmul(U00, ai);
            o1 = cmul(U10, ai);
            if (j >= 0) {
              const double2 aj = ld_amp(samp, (uint64_t)j);
              o0 = cadd(o0, cmul(U01, aj));
              o1 = cadd(o1, cmul(U11, aj));
            }
          } else {
            o0 = cmul(U01, ai);
            o1 = cmul(U11, ai);
          }
          keep0 = !(norm2(o0) < g.eps2);
          keep1 = !(norm2(o1) < g.eps2);
        }
      }
      const unsigned int b0 = __ballot_sync(0xffffffffu, keep0);
      const unsigned int b1 = __ballot_sync(0xffffffffu, keep1);
      if (sweep == 0) {
        if (lane == 0) woff[r * nwarps + warp] = (unsigned long long)(__popc(b0) + __popc(b1));
        continue;
      }
      const unsigned long long wbase = woff[r * nwarps + warp];
      if (keep0) {
        const unsigned long long pos = wbase + __popc(b0 & lt);
        if (pos < out.cap) {
          st_key<KW>(out, pos, p);
          st_amp((AT*)out.amp, pos, o0);
        } else {
          raise_err(ctl, kErrCapacity, seq, pos + 1);
        }
      }
      if (keep1) {
        const unsigned long long pos = wbase + __popc(b0) + __popc(b1 & lt);
        if (pos < out.cap) {
          st_key<KW>(out, pos, p | bmask);
          st_amp((AT*)out.amp, pos, o1);
        } else {
          raise_err(ctl, kErrCapacity, seq, pos + 1);
        }
      }
    }
    if (sweep == 0) {
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (uint32_t q = 0; q < rounds * nwarps; ++q) {
          const unsigned long long c = woff[q];
          woff[q] = run;
          run += c;
        }
        const unsigned long long base = run ? atomicAdd(&ctl->cnt[out_slot], run) : 0ull;
        for (uint32_t q = 0; q < rounds * nwarps; ++q) woff[q] += base;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
constexpr int kProbThreads = 256;
constexpr uint32_t kSmemBinsLog2 = 11;

template <int KW, class AT>
__global__ void __launch_bounds__(kProbThreads) k_probabilities(Ctl* ctl, Arr a, int slot,
                                                                uint32_t off, uint32_t w,
                                                                double* probs, double* nrm) {
  __shared__ double bins[1u << kSmemBinsLog2];
  __shared__ double red[kProbThreads / 32];
  if (ctl->err) return;
  const bool smem_bins = probs != nullptr && w <= kSmemBinsLog2;
  if (smem_bins)
    for (uint32_t v = threadIdx.x; v < (1u << w); v += blockDim.x) bins[v] = 0.0;
  __syncthreads();
  const unsigned long long n = ctl->cnt[slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, n);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double2 v = ld_amp((const AT*)a.amp, i);
    const double p = norm2(v);
    acc += p;
    if (probs) {
      const uint64_t val = get_field(ld_key<KW>(a, i), off, w);
      if (smem_bins)
        atomicAdd(&bins[val], p);
      else
        atomicAdd(&probs[val], p);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31u) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kProbThreads / 32; ++q) t += red[q];
    if (nrm) atomicAdd(nrm, t);
  }
  if (smem_bins)
    for (uint32_t v = threadIdx.x; v < (1u << w); v += blockDim.x)
      if (bins[v] != 0.0) atomicAdd(&probs[v], bins[v]);
}

__global__ void k_to_f64(Ctl* ctl, const float2* amp, int slot, double2* out) {
  const unsigned long long n = ctl->cnt[slot];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)amp[i].x, (double)amp[i].y);
}

__global__ void k_from_f64(const double2* in, uint64_t n, float2* amp) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    amp[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int stream_grid(const Launch& L, int threads) {
  // Enough resident CTAs to cover every SM several times; the kernels are
  // grid-stride loops over the device-resident count.
  uint64_t want = (L.n_hint + threads - 1) / threads;
  uint64_t cap = (uint64_t)L.sm_count * 8;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

cudaError_t launch_init(const Launch& L, Ctl* ctl, Arr a, int slot, bool amp32) {
  if (amp32)
    k_init<float2><<<1, 32, 0, L.stream>>>(ctl, a, slot);
  else
    k_init<double2><<<1, 32, 0, L.stream>>>(ctl, a, slot);
  return cudaGetLastError();
}

template <int KW, class AT>
static void apply_inplace_t(const Launch& L, Ctl* ctl, Arr a, int slot, const OpList& ops) {
  const int g = stream_grid(L, 256);
  if (ops.touches_keys && ops.touches_amps)
    k_apply_inplace<KW, AT, true, true><<<g, 256, 0, L.stream>>>(ctl, a, slot, ops, L.seq);
  else if (ops.touches_keys)
    k_apply_inplace<KW, AT, true, false><<<g, 256, 0, L.stream>>>(ctl, a, slot, ops, L.seq);
  else
    k_apply_inplace<KW, AT, false, true><<<g, 256, 0, L.stream>>>(ctl, a, slot, ops, L.seq);
}

cudaError_t launch_apply_inplace(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 const OpList& ops) {
  if (kw == 1) {
    if (amp32) apply_inplace_t<1, float2>(L, ctl, a, slot, ops);
    else apply_inplace_t<1, double2>(L, ctl, a, slot, ops);
  } else {
    if (amp32) apply_inplace_t<2, float2>(L, ctl, a, slot, ops);
    else apply_inplace_t<2, double2>(L, ctl, a, slot, ops);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_compact(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                                 int in_slot, Arr out, int out_slot, const OpList& ops) {
  const int g = stream_grid(L, 256);
#define SQS_AC(KW_, AT_) \
  k_apply_compact<KW_, AT_><<<g, 256, 0, L.stream>>>(ctl, in, in_slot, out, out_slot, ops, L.seq)
  if (kw == 1) {
    if (amp32) SQS_AC(1, float2);
    else SQS_AC(1, double2);
  } else {
    if (amp32) SQS_AC(2, float2);
    else SQS_AC(2, double2);
  }
#undef SQS_AC
  return cudaGetLastError();
}

cudaError_t launch_partition(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                             const OpList& ops, const Gate1& g, Buckets bk, Arr out,
                             int out_slot) {
  const int grid = stream_grid(L, 256);
#define SQS_PT(KW_, AT_)                                                                    \
  k_partition<KW_, AT_><<<grid, 256, 0, L.stream>>>(ctl, in, in_slot, ops, g, bk, out, out_slot, \
                                                    L.seq)
  if (kw == 1) {
    if (amp32) SQS_PT(1, float2);
    else SQS_PT(1, double2);
  } else {
    if (amp32) SQS_PT(2, float2);
    else SQS_PT(2, double2);
  }
#undef SQS_PT
  return cudaGetLastError();
}

int pair_capacity(int kw, bool amp32) {
  (void)kw;
  (void)amp32;
  return 2048;
}

size_t pair_smem_bytes(int kw, bool amp32) {
  const size_t C = (size_t)pair_capacity(kw, amp32);
  const size_t woff = ((C + kPairThreads - 1) / kPairThreads) * (kPairThreads / 32) + 1;
  return C * (kw == 1 ? 8 : 16) + C * (amp32 ? 8 : 16) + 2 * C * 4 + C * 4 + woff * 8;
}

template <int KW, class AT>
static cudaError_t pair_t(const Launch& L, Ctl* ctl, const Gate1& g, Buckets bk, Arr out,
                          int out_slot) {
  const size_t smem = pair_smem_bytes(KW, sizeof(AT) == 8);
  // The opt-in to more than 48 KB of dynamic shared memory is per device.
  static unsigned long long configured = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !(configured & (1ull << dev))) {
    cudaError_t e = cudaFuncSetAttribute(k_pair<KW, AT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured |= 1ull << dev;
  }
  k_pair<KW, AT><<<bk.B, kPairThreads, smem, L.stream>>>(ctl, g, bk, out, out_slot, L.seq);
  return cudaGetLastError();
}

cudaError_t launch_pair(const Launch& L, int kw, bool amp32, Ctl* ctl, const Gate1& g,
                        Buckets bk, Arr out, int out_slot) {
  if (kw == 1) return amp32 ? pair_t<1, float2>(L, ctl, g, bk, out, out_slot)
                            : pair_t<1, double2>(L, ctl, g, bk, out, out_slot);
  return amp32 ? pair_t<2, float2>(L, ctl, g, bk, out, out_slot)
               : pair_t<2, double2>(L, ctl, g, bk, out, out_slot);
}

cudaError_t launch_probabilities(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 uint32_t off, uint32_t w, double* probs, double* nrm) {
  const int g = stream_grid(L, kProbThreads);
#define SQS_PR(KW_, AT_) \
  k_probabilities<KW_, AT_><<<g, kProbThreads, 0, L.stream>>>(ctl, a, slot, off, w, probs, nrm)
  if (kw == 1) {
    if (amp32) SQS_PR(1, float2);
    else SQS_PR(1, double2);
  } else {
    if (amp32) SQS_PR(2, float2);
    else SQS_PR(2, double2);
  }
#undef SQS_PR
  return cudaGetLastError();
}

cudaError_t launch_to_f64(const Launch& L, Ctl* ctl, Arr a, int slot, double* out) {
  k_to_f64<<<stream_grid(L, 256), 256, 0, L.stream>>>(ctl, (const float2*)a.amp, slot,
                                                       (double2*)out);
  return cudaGetLastError();
}

cudaError_t launch_from_f64(const Launch& L, Ctl* ctl, Arr a, const double* in, uint64_t n) {
  (void)ctl;
  k_from_f64<<<stream_grid(L, 256), 256, 0, L.stream>>>((const double2*)in, n, (float2*)a.amp);
  return cudaGetLastError();
}

}  // namespace sqs
