// Device helpers shared by the kernels of the sparse-state library: key
// packing, complex arithmetic in the storage type, the pruning test, the
// fused operation interpreter and the 2x2 of one interference step.
#pragma once
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

// Key with only bit t set, built from its two 64-bit words (no variable
// 128-bit shift, whose results for t >= 64 one compiled instantiation got
// wrong), and the mask of bits below t likewise.
template <int KW>
__device__ __forceinline__ typename KT<KW>::T bit_mask(uint32_t t) {
  const uint64_t lo = t < 64 ? (1ull << t) : 0ull;
  const uint64_t hi = (t >= 64 && t < 128) ? (1ull << (t - 64)) : 0ull;
  return mk<KW>(lo, hi);
}
template <int KW>
__device__ __forceinline__ typename KT<KW>::T low_mask_bits(uint32_t t) {
  const uint64_t lo = t >= 64 ? ~0ull : ((1ull << t) - 1ull);
  const uint64_t hi = t <= 64 ? 0ull : (t >= 128 ? ~0ull : ((1ull << (t - 64)) - 1ull));
  return mk<KW>(lo, hi);
}

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

// Visiting order of the parts of a segment.  Kernels hand out the parts of
// segmented arrays round-robin (part u of the array is part u & (2^l - 1) of
// segment u >> l); with that order and a grid that is a multiple of 2^l every
// CTA would always take the same part of each segment, and segments that are
// not full keep their live branches in their first parts, so the CTAs of the
// last parts would idle.  spread(sg, l) is an l-bit multiplicative hash of
// the segment index (Knuth's golden-ratio constant); XOR-ing it into the part
// index permutes the parts of each segment, so each CTA meets every part
// equally often.
__device__ __forceinline__ uint64_t spread(uint64_t sg, uint32_t l) {
  return l ? (sg * 0x9E3779B97F4A7C15ull) >> (64u - l) : 0ull;
}

// Part visited at round-robin position u (2^l parts per segment): a
// permutation of the parts of each segment.
__device__ __forceinline__ uint64_t spread_visit(uint64_t u, uint32_t l) {
  if (!l) return u;
  const uint64_t sg = u >> l;
  return (sg << l) | ((u ^ spread(sg, l)) & ((1ull << l) - 1ull));
}

// log2 of the parts per segment when that is a power of two, else 0 (the
// identity order: spread_visit permutes within aligned groups of 2^l parts,
// which must tile the part range exactly).
__device__ __forceinline__ uint32_t log2_pow2(uint32_t x) {
  return (x == 0u || (x & (x - 1u))) ? 0u : 31u - (uint32_t)__clz(x);
}
__device__ __forceinline__ uint64_t khash(u128 k) {
  return mix64((uint64_t)k ^ mix64((uint64_t)(k >> 64) + 0x9e3779b97f4a7c15ull));
}

// ---- amplitudes ------------------------------------------------------------
// FP64 states compute in FP64.  FP32-storage states keep the non-interference
// factors (phase tables) in FP32, and evaluate every child of an interference
// step with compensated FP32 arithmetic (error-free products and sums, below)
// that matches an FP64 accumulation rounded once to FP32: the FP32 pipe is 64x
// wider than the FP64 pipe on this GPU.
// Complex product with one product fused into the sum (two instructions per
// component): one rounding fewer than the host's complex<double> product.
// The sign sits on an input of the FMA (a negated multiplicand), never on a
// product, so no separate negation is issued.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(__fma_rn(-a.y, b.y, __dmul_rn(a.x, b.x)),
                      __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(-a.y, b.y, __fmul_rn(a.x, b.x)),
                     __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
// u * a + p (real u), fused per component.
__device__ __forceinline__ double2 rfma(double u, double2 a, double2 p) {
  return make_double2(__fma_rn(u, a.x, p.x), __fma_rn(u, a.y, p.y));
}
__device__ __forceinline__ float2 rfma(float u, float2 a, float2 p) {
  return make_float2(__fmaf_rn(u, a.x, p.x), __fmaf_rn(u, a.y, p.y));
}
// u * a - p (real u), fused per component: the same bits as u * a + (-p),
// with the sign flip carried by the FMA's addend instead of an instruction.
__device__ __forceinline__ double2 rfms(double u, double2 a, double2 p) {
  return make_double2(__fma_rn(u, a.x, -p.x), __fma_rn(u, a.y, -p.y));
}
__device__ __forceinline__ float2 rfms(float u, float2 a, float2 p) {
  return make_float2(__fmaf_rn(u, a.x, -p.x), __fmaf_rn(u, a.y, -p.y));
}
// c * a + p (complex c), fused.
__device__ __forceinline__ double2 cfma(double2 c, double2 a, double2 p) {
  return make_double2(__fma_rn(c.x, a.x, __fma_rn(-c.y, a.y, p.x)),
                      __fma_rn(c.x, a.y, __fma_rn(c.y, a.x, p.y)));
}
__device__ __forceinline__ float2 cfma(float2 c, float2 a, float2 p) {
  return make_float2(__fmaf_rn(c.x, a.x, __fmaf_rn(-c.y, a.y, p.x)),
                     __fmaf_rn(c.x, a.y, __fmaf_rn(c.y, a.x, p.y)));
}
// Real coefficient: (u + 0i)(a.x + i a.y) evaluated as above is exactly these
// two products.
__device__ __forceinline__ double2 rmul(double u, double2 a) {
  return make_double2(__dmul_rn(u, a.x), __dmul_rn(u, a.y));
}
__device__ __forceinline__ float2 rmul(float u, float2 a) {
  return make_float2(__fmul_rn(u, a.x), __fmul_rn(u, a.y));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}
// Exact negation by the sign bits, written as an integer XOR in PTX so that
// it stays an integer instruction and never occupies the FP64 pipe.
__device__ __forceinline__ double neg_bits(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  asm("xor.b64 %0, %0, 0x8000000000000000;" : "+l"(u));
  return __longlong_as_double((long long)u);
}
// Magnitude and sign bits of an FP64 value, as integer ANDs in PTX.  Written
// as C++ masks of the value's bits, the compiler recognises the magnitude as
// an absolute value and evaluates it on the FP64 pipe (a counted DADD per
// component), this GPU's scarcest unit.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  asm("and.b64 %0, %0, 0x7fffffffffffffff;" : "+l"(u));
  return u;
}
__device__ __forceinline__ unsigned long long sign_bits(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  asm("and.b64 %0, %0, 0x8000000000000000;" : "+l"(u));
  return u;
}
__device__ __forceinline__ double2 cneg(double2 a) {
  return make_double2(neg_bits(a.x), neg_bits(a.y));
}
__device__ __forceinline__ float2 cneg(float2 a) {
  return make_float2(__int_as_float(__float_as_int(a.x) ^ (int)0x80000000u),
                     __int_as_float(__float_as_int(a.y) ^ (int)0x80000000u));
}
__device__ __forceinline__ double norm2(double2 a) {
  return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}
__device__ __forceinline__ double norm2(float2 a) {
  const double x = (double)a.x, y = (double)a.y;
  return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
}
// |a| >= eps?  Certain, without floating-point arithmetic, when one component
// already reaches eps in magnitude (IEEE order of non-negative values is
// integer order); otherwise |a|^2 is compared with eps^2 in FP64.
__device__ __forceinline__ bool keep_amp(double2 a, double eps, float, double eps2) {
  const unsigned long long e = (unsigned long long)__double_as_longlong(eps);
  const unsigned long long ax = abs_bits(a.x);
  const unsigned long long ay = abs_bits(a.y);
  if (ax >= e || ay >= e) return true;
  if ((ax | ay) == 0ull) return e == 0ull;  // exact zero: kept only when eps = 0
  // Both components below eps/2 (the exponent of a normal eps minus one):
  // |a|^2 < eps^2 / 2, a removal the FP64 test below would decide the same
  // way.  Cancellation residues take this exit without FP64 arithmetic.
  const unsigned long long eh = e > (1ull << 52) ? e - (1ull << 52) : 0ull;
  if (ax < eh && ay < eh) return false;
  return !(norm2(a) < eps2);
}
__device__ __forceinline__ bool keep_amp(float2 a, double, float epsf, double eps2) {
  const unsigned int e = (unsigned int)__float_as_int(epsf);
  const unsigned int ax = (unsigned int)__float_as_int(a.x) & 0x7fffffffu;
  const unsigned int ay = (unsigned int)__float_as_int(a.y) & 0x7fffffffu;
  if (ax >= e || ay >= e) return true;
  if ((ax | ay) == 0u) return eps2 == 0.0;
  const unsigned int eh = e > (1u << 23) ? e - (1u << 23) : 0u;  // epsf / 2, as above
  if (ax < eh && ay < eh) return false;
  return !(norm2(a) < eps2);
}
__device__ __forceinline__ void to_amp(double2& out, double2 v) { out = v; }
__device__ __forceinline__ void to_amp(float2& out, double2 v) {
  out = make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 to_f64(double2 v) { return v; }
__device__ __forceinline__ double2 to_f64(float2 v) { return make_double2(v.x, v.y); }

// ---- keys --------------------------------------------------------------------
template <int KW>
__device__ __forceinline__ typename KT<KW>::T ld_key(const Arr& a, uint64_t i) {
  return mk<KW>(a.k0[i], KW == 2 ? a.k1[i] : 0ull);
}
template <int KW>
__device__ __forceinline__ void st_key(const Arr& a, uint64_t i, typename KT<KW>::T k) {
  a.k0[i] = lo64(k);
  if (KW == 2) a.k1[i] = hi64(k);
}

// ---- layout ----------------------------------------------------------------------
// Number of slots to visit and whether slot i holds a branch.
__device__ __forceinline__ uint64_t slots_of(const Arr& a, const Ctl* ctl, int slot) {
  return a.seg_cnt ? ((uint64_t)a.n_seg << a.seg_log2) : ctl->cnt[slot];
}
__device__ __forceinline__ bool slot_live(const Arr& a, uint64_t i) {
  if (!a.seg_cnt) return true;
  return (uint32_t)(i & ((1ull << a.seg_log2) - 1ull)) < a.seg_cnt[i >> a.seg_log2];
}

// Calls f(i) for every live slot: grid-stride over a dense array, or CTA per
// segment (live branches are a prefix of each segment).
// Calls f(i) for every live slot: grid-stride over a dense array, or CTA per
// segment (live branches are a prefix of each segment).
template <class F>
__device__ __forceinline__ void for_each_live(const Arr& a, uint64_t n_dense, F f) {
  if (!a.seg_cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_dense; i += stride)
      f(i);
  } else {
    for (uint32_t sg = blockIdx.x; sg < a.n_seg; sg += gridDim.x) {
      const uint32_t n = a.seg_cnt[sg];
      const uint64_t base = (uint64_t)sg << a.seg_log2;
      for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) f(base + j);
    }
  }
}

// ---- errors --------------------------------------------------------------------
__device__ __forceinline__ void raise_err(Ctl* ctl, unsigned int bit, uint32_t seq,
                                          unsigned long long need) {
  if (atomicOr(&ctl->err, bit) == 0u) ctl->err_where = seq;
  atomicMax(&ctl->need, need);
}

// ---- fused operation run ---------------------------------------------------------
// Multiply-add, multiply by a constant, divide-XOR on key fields (mod 2^w by
// set_field's truncation).
template <class K>
__device__ __forceinline__ K arith_op(const DevOp& op, K k) {
  const uint64_t d = get_field(k, op.dst_off, op.dst_w);
  uint64_t r;
  if (op.kind == OP_MUL_CONST) {
    r = d * op.constant;
  } else {
    const uint64_t a = get_field(k, op.src_off, op.src_w);
    const uint64_t b = get_field(k, op.src2_off, op.src2_w);
    r = op.kind == OP_MUL_ADD ? d + a * b : d ^ (b ? a / b : 0ull);
  }
  return set_field<K>(k, op.dst_off, op.dst_w, r);
}

// tab: the folded factors in the storage type (shared-memory copy).
template <int KW, class AT>
__device__ __forceinline__ bool apply_ops(uint32_t n_ops, const DevOp* ops, const AT* tab,
                                          typename KT<KW>::T& k, AT& a) {
  typedef typename KT<KW>::T K;
  uint32_t idx = 0;
#pragma unroll 1
  for (uint32_t o = 0; o < n_ops; ++o) {
    const DevOp& op = ops[o];
    const uint32_t kind = op.kind;
    const bool on = (k & mk<KW>(op.pmask[0], op.pmask[1])) == mk<KW>(op.pval[0], op.pval[1]);
    if (kind == OP_XOR) {
      if (on) k ^= mk<KW>(op.xmask[0], op.xmask[1]);
    } else if (kind == OP_MUL || kind == OP_MUL_XOR) {
      if (on) {
        const uint32_t one = op.sel_bit < 128 ? (uint32_t)((k >> op.sel_bit) & (K)1) : 0u;
        idx |= (1u + one) << op.shift;
        if (kind == OP_MUL_XOR) k ^= mk<KW>(op.xmask[0], op.xmask[1]);
      }
    } else if (kind == OP_ADD_REG || kind == OP_SUB_REG || kind == OP_ADD_CONST) {
      if (on) {
        const uint64_t d = get_field(k, op.dst_off, op.dst_w);
        const uint64_t s = kind == OP_ADD_CONST ? op.constant : get_field(k, op.src_off, op.src_w);
        k = set_field<K>(k, op.dst_off, op.dst_w, kind == OP_SUB_REG ? d - s : d + s);
      }
    } else if (kind == OP_TABLE) {
      if (idx) a = cmul(a, tab[op.tab_off + idx]);
      idx = 0;
    } else if (kind == OP_QRAM) {
      if (on) {
        const uint64_t addr = get_field(k, op.src_off, op.src_w);
        uint64_t d = 0;
        if (addr < op.n_entries) {
          switch ((uint32_t)op.constant) {
            case 1: d = __ldg((const uint8_t*)op.table + addr); break;
            case 2: d = __ldg((const uint16_t*)op.table + addr); break;
            case 4: d = __ldg((const uint32_t*)op.table + addr); break;
            default: d = __ldg((const unsigned long long*)op.table + addr); break;
          }
        }
        k = set_field<K>(k, op.dst_off, op.dst_w, get_field(k, op.dst_off, op.dst_w) ^ d);
      }
    } else if (kind == OP_SWAP) {
      if (on) {
        const uint64_t v1 = get_field(k, op.dst_off, op.dst_w);
        const uint64_t v2 = get_field(k, op.src_off, op.src_w);
        k = set_field<K>(set_field<K>(k, op.dst_off, op.dst_w, v2), op.src_off, op.src_w, v1);
      }
    } else if (kind == OP_PRUNE) {
      if (!keep_amp(a, op.eps, (float)op.eps, op.eps2)) return false;
    } else if (kind == OP_MUL_ADD || kind == OP_MUL_CONST || kind == OP_DIV_XOR) {
      if (on) k = arith_op(op, k);
    }
  }
  return true;
}

// The same run applied to NI branches at once, operation-major: each
// operation's descriptor is read from shared memory and dispatched once for
// the NI branches a thread carries, instead of once per branch.  Per branch
// the arithmetic and its order are those of apply_ops.  live[q] is cleared
// for a branch the run prunes; branches already dead are left alone (their
// QRAM reads are skipped).
template <int KW, class AT, int NI>
__device__ __forceinline__ void apply_ops_n(uint32_t n_ops, const DevOp* ops, const AT* tab,
                                            typename KT<KW>::T (&k)[NI], AT (&a)[NI],
                                            bool (&live)[NI]) {
  typedef typename KT<KW>::T K;
  uint32_t idx[NI];
#pragma unroll
  for (int q = 0; q < NI; ++q) idx[q] = 0;
#pragma unroll 1
  for (uint32_t o = 0; o < n_ops; ++o) {
    const DevOp& op = ops[o];
    const uint32_t kind = op.kind;
    const K pm = mk<KW>(op.pmask[0], op.pmask[1]);
    const K pv = mk<KW>(op.pval[0], op.pval[1]);
    if (kind == OP_XOR) {
      const K xm = mk<KW>(op.xmask[0], op.xmask[1]);
#pragma unroll
      for (int q = 0; q < NI; ++q)
        if ((k[q] & pm) == pv) k[q] ^= xm;
    } else if (kind == OP_MUL || kind == OP_MUL_XOR) {
      const uint32_t sel = op.sel_bit, sh = op.shift;
      const K xm = kind == OP_MUL_XOR ? mk<KW>(op.xmask[0], op.xmask[1]) : (K)0;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        if ((k[q] & pm) == pv) {
          const uint32_t one = sel < 128 ? (uint32_t)((k[q] >> sel) & (K)1) : 0u;
          idx[q] |= (1u + one) << sh;
          k[q] ^= xm;
        }
      }
    } else if (kind == OP_ADD_CONST) {
      // In place: the field's bits are added with the constant shifted to the
      // field; carries out of the field are masked off (mod 2^w).
      const K D = ((K)wmask(op.dst_w)) << op.dst_off;
      const K C = ((K)(op.constant & wmask(op.dst_w))) << op.dst_off;
#pragma unroll
      for (int q = 0; q < NI; ++q)
        if ((k[q] & pm) == pv) k[q] = (k[q] & ~D) | (((k[q] & D) + C) & D);
    } else if (kind == OP_ADD_REG || kind == OP_SUB_REG) {
      // The source field moved onto the destination's position (one shift),
      // then added or subtracted in place: ((d +- s) mod 2^w) << doff, as
      // get_field / set_field give.
      const uint32_t doff = op.dst_off, soff = op.src_off;
      const K D = ((K)wmask(op.dst_w)) << doff;
      const K S = ((K)wmask(op.src_w)) << soff;
      const bool left = doff >= soff;
      const uint32_t sh = left ? doff - soff : soff - doff;
      const bool sub = kind == OP_SUB_REG;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        if ((k[q] & pm) == pv) {
          const K t = left ? (k[q] & S) << sh : (k[q] & S) >> sh;
          const K kd = k[q] & D;
          k[q] = (k[q] & ~D) | ((sub ? kd - t : kd + t) & D);
        }
      }
    } else if (kind == OP_TABLE) {
      const uint32_t base = op.tab_off;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        if (idx[q]) a[q] = cmul(a[q], tab[base + idx[q]]);
        idx[q] = 0;
      }
    } else if (kind == OP_QRAM) {
      const uint32_t doff = op.dst_off, dw = op.dst_w, soff = op.src_off, sw = op.src_w;
      const uint64_t n_ent = op.n_entries;
      const uint32_t eb = (uint32_t)op.constant;
      const void* tbl = op.table;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        if (live[q] && (k[q] & pm) == pv) {
          const uint64_t addr = get_field(k[q], soff, sw);
          uint64_t d = 0;
          if (addr < n_ent) {
            switch (eb) {
              case 1: d = __ldg((const uint8_t*)tbl + addr); break;
              case 2: d = __ldg((const uint16_t*)tbl + addr); break;
              case 4: d = __ldg((const uint32_t*)tbl + addr); break;
              default: d = __ldg((const unsigned long long*)tbl + addr); break;
            }
          }
          k[q] = set_field<K>(k[q], doff, dw, get_field(k[q], doff, dw) ^ d);
        }
      }
    } else if (kind == OP_SWAP) {
      const uint32_t doff = op.dst_off, dw = op.dst_w, soff = op.src_off, sw = op.src_w;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        if ((k[q] & pm) == pv) {
          const uint64_t v1 = get_field(k[q], doff, dw);
          const uint64_t v2 = get_field(k[q], soff, sw);
          k[q] = set_field<K>(set_field<K>(k[q], doff, dw, v2), soff, sw, v1);
        }
      }
    } else if (kind == OP_PRUNE) {
      const double eps = op.eps, eps2 = op.eps2;
#pragma unroll
      for (int q = 0; q < NI; ++q)
        if (live[q] && !keep_amp(a[q], eps, (float)eps, eps2)) live[q] = false;
    } else if (kind == OP_MUL_ADD || kind == OP_MUL_CONST || kind == OP_DIV_XOR) {
#pragma unroll
      for (int q = 0; q < NI; ++q)
        if ((k[q] & pm) == pv) k[q] = arith_op(op, k[q]);
    }
  }
}

// Copies the launch's operations and factor table into shared memory: the
// per-branch loop then reads them with broadcast shared loads instead of
// indexed parameter-space loads.
template <class AT>
__device__ __forceinline__ void load_ops(const OpList& L, DevOp* ops, AT* tab) {
  static_assert(sizeof(DevOp) % 8 == 0, "DevOp copied as 8-byte words");
  const uint64_t* src = (const uint64_t*)L.op;
  uint64_t* dst = (uint64_t*)ops;
  const uint32_t words = L.n * (uint32_t)(sizeof(DevOp) / 8);
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  for (uint32_t i = threadIdx.x; i < L.n_tab; i += blockDim.x) to_amp(tab[i], L.tab[i]);
  __syncthreads();
}

// ---- bulk copies (TMA engine) into shared memory, completed on an mbarrier --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy: both addresses 16-byte aligned, bytes a
// multiple of 16; completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

constexpr int kStreamThreads = 256;

// ---------------------------------------------------------------------------
// The 2x2 of one merge step on a pair class: children (o0, o1) of the
// members a0 (bit 0, present when has0) and a1 (bit 1, present when has1).
// Coefficients in the storage type; products shared between the rows of a
// column when the host flagged U10 = +-U00 or U11 = +-U01.
template <class AT>
struct Coef;
template <>
struct Coef<double2> {
  typedef double S;
  __device__ static double2 c(const Gate1& g, int e) { return make_double2(g.u[2 * e], g.u[2 * e + 1]); }
  __device__ static double r(const Gate1& g, int e) { return g.u[2 * e]; }
};
template <>
struct Coef<float2> {
  typedef float S;
  __device__ static float2 c(const Gate1& g, int e) { return make_float2(g.uf[2 * e], g.uf[2 * e + 1]); }
  __device__ static float r(const Gate1& g, int e) { return g.uf[2 * e]; }
};

// ---- FP32 storage: compensated evaluation of a child ------------------------
// A child of an interference step is a short dot product, sum_i u_i a_i, of
// real coefficients u_i (matrix entries, or their real and imaginary parts)
// with FP32 amplitude components a_i.  It is evaluated as Dot2 of Ogita, Rump
// and Oishi (SIAM J. Sci. Comput. 26, 2005): every product split exactly into
// a rounded part and its error by an FMA (Dekker's two-product), the rounded
// parts summed with Knuth's error-free two-sum, and all error terms added back
// before the one final rounding.  The coefficients are carried as float-float
// pairs (h + l, the FP64 value to about 48 bits), so the result is the
// FP64-accurate sum of the FP64 coefficients times the stored amplitudes,
// rounded once to FP32: error at most half an FP32 ulp plus about 2^-46 of
// sum_i |u_i a_i|.
//
// Cancellation at storage precision.  Every stored FP32 component carries the
// rounding of its own last store, and the roundings of every operation since
// the branch split from its partner, each up to 2^-24 of its size.  A sum
// whose exact value is zero in the FP64 method (RY(t) then RY(-t) on the same
// qubit; a reflection that restores a state) therefore ends up at some units
// of 2^-24 of the terms' size, far above any pruning threshold, and would
// never leave the state.  A component whose compensated value is at most
// rho * sum_i |u_i a_i| carries no significant bit of the stored inputs: it
// is set to exactly zero, and the pruning test (keep_amp) removes the child
// when both components are zero.  rho is a per-state setting (Gate1::rho32,
// default 2^-19 = 32 units of FP32 roundoff, covering circuits where the two
// members went through a few dozen roundings since their common ancestor).
// The change to a component is at most rho * sum_i |u_i a_i|: relative to the
// terms, the same order as the storage rounding the inputs already carry.
// Single-member children are single products: no cancellation, no flush.
struct FF {
  float h, l;  // value h + l, |l| <= ulp(h) / 2
};
__device__ __forceinline__ FF ff_neg(FF u) { return FF{-u.h, -u.l}; }
// FP64 -> float-float (register-valued angles: cos / sin of the half angle).
__device__ __forceinline__ FF ff_of(double u) {
  const float h = __double2float_rn(u);
  return FF{h, __double2float_rn(u - (double)h)};
}

// Accumulates u * a into (s, c): s the running rounded sum, c the running sum
// of the error terms.
__device__ __forceinline__ void dot2_acc(FF u, float a, float& s, float& c) {
  const float p = __fmul_rn(u.h, a);
  const float e = __fmaf_rn(u.l, a, __fmaf_rn(u.h, a, -p));  // u a - p, to ~2^-48
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p - t
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}
__device__ __forceinline__ float dot2_1(FF u, float a) {
  const float p = __fmul_rn(u.h, a);
  return __fadd_rn(p, __fmaf_rn(u.l, a, __fmaf_rn(u.h, a, -p)));
}
// u0 a0 + u1 a1, with the storage-precision cancellation flush.
__device__ __forceinline__ float dot2_2(FF u0, float a0, FF u1, float a1, float rho) {
  float s = __fmul_rn(u0.h, a0);
  float c = __fmaf_rn(u0.l, a0, __fmaf_rn(u0.h, a0, -s));
  dot2_acc(u1, a1, s, c);
  const float r = __fadd_rn(s, c);
  const float size = __fmaf_rn(fabsf(u0.h), fabsf(a0), __fmul_rn(fabsf(u1.h), fabsf(a1)));
  return fabsf(r) <= __fmul_rn(rho, size) ? 0.0f : r;
}
// u0 a0 + u1 a1 + u2 a2 + u3 a3 (complex coefficients), with the flush.
__device__ __forceinline__ float dot2_4(FF u0, float a0, FF u1, float a1, FF u2, float a2, FF u3,
                                        float a3, float rho) {
  float s = __fmul_rn(u0.h, a0);
  float c = __fmaf_rn(u0.l, a0, __fmaf_rn(u0.h, a0, -s));
  dot2_acc(u1, a1, s, c);
  dot2_acc(u2, a2, s, c);
  dot2_acc(u3, a3, s, c);
  const float r = __fadd_rn(s, c);
  float size = __fmul_rn(fabsf(u0.h), fabsf(a0));
  size = __fmaf_rn(fabsf(u1.h), fabsf(a1), size);
  size = __fmaf_rn(fabsf(u2.h), fabsf(a2), size);
  size = __fmaf_rn(fabsf(u3.h), fabsf(a3), size);
  return fabsf(r) <= __fmul_rn(rho, size) ? 0.0f : r;
}
// u a (complex u, no flush: one member).
__device__ __forceinline__ float2 cdot2_1(FF ur, FF ui, float2 a) {
  float s = __fmul_rn(ur.h, a.x);
  float c = __fmaf_rn(ur.l, a.x, __fmaf_rn(ur.h, a.x, -s));
  dot2_acc(ff_neg(ui), a.y, s, c);
  float s2 = __fmul_rn(ur.h, a.y);
  float c2 = __fmaf_rn(ur.l, a.y, __fmaf_rn(ur.h, a.y, -s2));
  dot2_acc(ui, a.x, s2, c2);
  return make_float2(__fadd_rn(s, c), __fadd_rn(s2, c2));
}
// The coefficient of entry e (0: U00, 1: U01, 2: U10, 3: U11), part p (0
// real, 1 imaginary), as float-float (host-rounded pairs in Gate1).
__device__ __forceinline__ FF ff_coef(const Gate1& g, int e, int p) {
  return FF{g.uf[2 * e + p], g.ufl[2 * e + p]};
}

// cos and sin of theta / 2 for theta = scale * v + offset (mode 1).  With a
// digit table, the angle is the sum of one table angle per 16-bit digit of
// v, combined by the angle-addition formulas (four FP64 operations per digit
// after the first) instead of a full sincos per branch.
__device__ __forceinline__ void half_angle_cs(const Gate1& g, uint64_t v, double& cs,
                                              double& sn) {
  if (g.ang_tab) {
    const double2 t = __ldg(&g.ang_tab[v & 0xffffull]);
    cs = t.x;
    sn = t.y;
    for (uint32_t j = 1; j < g.ang_digits; ++j) {
      const double2 u = __ldg(&g.ang_tab[((uint64_t)j << 16) | ((v >> (16 * j)) & 0xffffull)]);
      const double c2 = __fma_rn(-sn, u.y, __dmul_rn(cs, u.x));  // cos(a + b)
      const double s2 = __fma_rn(sn, u.x, __dmul_rn(cs, u.y));   // sin(a + b)
      cs = c2;
      sn = s2;
    }
  } else {
    const double theta = g.scale * (double)v + g.offset;
    sincos(theta * 0.5, &sn, &cs);
  }
}

template <class AT>
__device__ __forceinline__ void children(const Gate1& g, uint64_t angle_value, bool has0, AT a0,
                                         bool has1, AT a1, AT& o0, AT& o1);

// FP64 storage: FP64 arithmetic, products shared between rows where the host
// flagged equal coefficients.
template <>
__device__ __forceinline__ void children<double2>(const Gate1& g, uint64_t angle_value, bool has0,
                                                  double2 a0, bool has1, double2 a1, double2& o0,
                                                  double2& o1) {
  typedef double2 AT;
  typedef typename Coef<AT>::S S;
  const bool same0 = g.reuse & 1u, neg0 = g.reuse & 4u;  // U10 = +-U00
  const bool same1 = g.reuse & 2u, neg1 = g.reuse & 8u;  // U11 = +-U01
  if (g.mode == 2 || g.mode == 1) {
    S u00, u01, u10, u11;
    if (g.mode == 1) {
      double sn, cs;
      half_angle_cs(g, angle_value, cs, sn);
      u00 = (S)cs, u01 = (S)-sn, u10 = (S)sn, u11 = (S)cs;
    } else {
      u00 = Coef<AT>::r(g, 0), u01 = Coef<AT>::r(g, 1), u10 = Coef<AT>::r(g, 2),
      u11 = Coef<AT>::r(g, 3);
    }
    if (has0 && has1) {
      const AT p01 = rmul(u01, a1);
      o0 = rfma(u00, a0, p01);
      if (same1)
        o1 = neg1 ? rfms(u10, a0, p01) : rfma(u10, a0, p01);
      else
        o1 = rfma(u10, a0, rmul(u11, a1));
    } else {
      // One member: the column of U it multiplies is selected, not branched
      // on, so lanes holding a bit-0 and a bit-1 member issue one sequence.
      const bool c1 = !has0;
      const S ua = c1 ? u01 : u00, ub = c1 ? u11 : u10;
      const bool same = c1 ? same1 : same0, neg = c1 ? neg1 : neg0;
      const AT a = c1 ? a1 : a0;
      o0 = rmul(ua, a);
      o1 = same ? (neg ? cneg(o0) : o0) : rmul(ub, a);
    }
  } else {
    const AT U00 = Coef<AT>::c(g, 0), U01 = Coef<AT>::c(g, 1);
    const AT U10 = Coef<AT>::c(g, 2), U11 = Coef<AT>::c(g, 3);
    if (has0 && has1) {
      const AT p01 = cmul(U01, a1);
      const AT p11 = same1 ? (neg1 ? cneg(p01) : p01) : cmul(U11, a1);
      o0 = cfma(U00, a0, p01);
      o1 = cfma(U10, a0, p11);
    } else {
      const bool c1 = !has0;  // one member, its column selected as above
      const AT Ua = c1 ? U01 : U00, Ub = c1 ? U11 : U10;
      const bool same = c1 ? same1 : same0, neg = c1 ? neg1 : neg0;
      const AT a = c1 ? a1 : a0;
      o0 = cmul(Ua, a);
      o1 = same ? (neg ? cneg(o0) : o0) : cmul(Ub, a);
    }
  }
}

// FP32 storage: every child by the compensated evaluation above.
template <>
__device__ __forceinline__ void children<float2>(const Gate1& g, uint64_t angle_value, bool has0,
                                                 float2 a0, bool has1, float2 a1, float2& o0,
                                                 float2& o1) {
  if (g.mode == 2 || g.mode == 1) {
    FF u00, u01, u10, u11;
    if (g.mode == 1) {
      double sn, cs;
      half_angle_cs(g, angle_value, cs, sn);
      u00 = ff_of(cs), u10 = ff_of(sn);
      u01 = ff_neg(u10), u11 = u00;
    } else {
      u00 = ff_coef(g, 0, 0), u01 = ff_coef(g, 1, 0), u10 = ff_coef(g, 2, 0),
      u11 = ff_coef(g, 3, 0);
    }
    if (has0 && has1) {
      const float rho = g.rho32;
      o0 = make_float2(dot2_2(u00, a0.x, u01, a1.x, rho), dot2_2(u00, a0.y, u01, a1.y, rho));
      o1 = make_float2(dot2_2(u10, a0.x, u11, a1.x, rho), dot2_2(u10, a0.y, u11, a1.y, rho));
    } else if (has0) {
      o0 = make_float2(dot2_1(u00, a0.x), dot2_1(u00, a0.y));
      o1 = make_float2(dot2_1(u10, a0.x), dot2_1(u10, a0.y));
    } else {
      o0 = make_float2(dot2_1(u01, a1.x), dot2_1(u01, a1.y));
      o1 = make_float2(dot2_1(u11, a1.x), dot2_1(u11, a1.y));
    }
  } else {
    if (has0 && has1) {
      // Re(U_r0 a0 + U_r1 a1) and Im(...): four real products each.
      for (int r = 0; r < 2; ++r) {
        const FF xr = ff_coef(g, 2 * r, 0), xi = ff_coef(g, 2 * r, 1);
        const FF yr = ff_coef(g, 2 * r + 1, 0), yi = ff_coef(g, 2 * r + 1, 1);
        const float2 o = make_float2(
            dot2_4(xr, a0.x, ff_neg(xi), a0.y, yr, a1.x, ff_neg(yi), a1.y, g.rho32),
            dot2_4(xr, a0.y, xi, a0.x, yr, a1.y, yi, a1.x, g.rho32));
        if (r == 0) o0 = o; else o1 = o;
      }
    } else if (has0) {
      o0 = cdot2_1(ff_coef(g, 0, 0), ff_coef(g, 0, 1), a0);
      o1 = cdot2_1(ff_coef(g, 2, 0), ff_coef(g, 2, 1), a0);
    } else {
      o0 = cdot2_1(ff_coef(g, 1, 0), ff_coef(g, 1, 1), a1);
      o1 = cdot2_1(ff_coef(g, 3, 0), ff_coef(g, 3, 1), a1);
    }
  }
}

// One child of a pair whose both members are present, real coefficients
// (mode 2): the same expression children() evaluates for it.
template <class AT>
__device__ __forceinline__ AT child_real(const Gate1& g, int r, AT a0, AT a1);
template <>
__device__ __forceinline__ double2 child_real<double2>(const Gate1& g, int r, double2 a0,
                                                       double2 a1) {
  const double u00 = g.u[0], u01 = g.u[2], u10 = g.u[4], u11 = g.u[6];
  const double2 p01 = rmul(u01, a1);
  if (r == 0) return rfma(u00, a0, p01);
  const bool same1 = g.reuse & 2u, neg1 = g.reuse & 8u;
  return same1 ? (neg1 ? rfms(u10, a0, p01) : rfma(u10, a0, p01)) : rfma(u10, a0, rmul(u11, a1));
}
template <>
__device__ __forceinline__ float2 child_real<float2>(const Gate1& g, int r, float2 a0, float2 a1) {
  const FF ur0 = ff_coef(g, 2 * r, 0), ur1 = ff_coef(g, 2 * r + 1, 0);
  return make_float2(dot2_2(ur0, a0.x, ur1, a1.x, g.rho32), dot2_2(ur0, a0.y, ur1, a1.y, g.rho32));
}

// 2 x, exactly, in integer arithmetic on the IEEE encoding (no FP64
// instruction): one more in the exponent field of a normal x; the magnitude
// bits shifted left for a zero or subnormal x (the encoding is linear across
// the subnormal range and into the first normal binade); infinity for a
// doubling out of the largest binade.
__device__ __forceinline__ double twice(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = sign_bits(x);
  const unsigned long long mag = abs_bits(x);
  const unsigned long long e = mag >> 52;
  const unsigned long long r = e == 0ull    ? (sign | (mag << 1))
                               : e < 2046ull ? b + (1ull << 52)
                                             : (sign | 0x7ff0000000000000ull);
  return __longlong_as_double((long long)r);
}

// The surviving child of a fold whose coefficients agree up to the pair's
// sign (g.fold_twice): child_real evaluates fma(u, a, round(u a)) per
// component, which is exactly 2 round(u a) -- the exact value 2 round(u a)
// - d, |d| <= ulp(round(u a)) / 2, is within a quarter ulp of 2 round(u a)
// -- so one product and an exponent increment give the same bits.  FP32
// states keep the general form (their arithmetic is not the bottleneck).
template <class AT>
__device__ __forceinline__ AT fold_child(const Gate1& g, int r, AT a0, AT a1) {
  return child_real<AT>(g, r, a0, a1);
}
template <>
__device__ __forceinline__ double2 fold_child<double2>(const Gate1& g, int r, double2 a0,
                                                       double2 a1) {
  if (!g.fold_twice) return child_real<double2>(g, r, a0, a1);
  const double u = g.u[2 * (2 * r)];
  return make_double2(twice(__dmul_rn(u, a0.x)), twice(__dmul_rn(u, a0.y)));
}

// Both components' magnitudes below the bit pattern t (FP64 storage).  For
// FP32 storage the cancelling child of a fold is u a + (-u) a evaluated
// compensated, which is exactly zero, so the test passes.
__device__ __forceinline__ bool below_bits(double2 a, uint64_t t) {
  return abs_bits(a.x) < t && abs_bits(a.y) < t;
}
__device__ __forceinline__ bool below_bits(float2, uint64_t) { return true; }


}  // namespace sqs
