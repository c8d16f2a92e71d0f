// CUDA kernels of the sparse register-level state library (sm_103a).
//
// The state is a structure of arrays: k0[] (key bits 0..63), k1[] (bits
// 64..127, two-word keys only) and amp[] (complex<double> or complex<float>),
// dense or split into fixed-capacity segments (sqs_internal.h, Arr).  Every
// kernel is a stream over those arrays; nothing is a dense contraction, so no
// tensor cores are used.  FP64 instructions are kept to the minimum the
// arithmetic needs: this GPU issues about two FP64 instructions per SM per
// clock, so a few dozen of them per branch would cost more time than moving
// the branch through HBM.
//
//  k_apply_inplace   runs of non-interference operations, fused (Sec. II.D.1)
//  k_apply_compact   the same when the run may drop branches (pruning)
//  k_partition       fused run + the first half of an interference operation:
//                    scatters every branch into a hash bucket keyed by its
//                    pair class (key with the target bit cleared), so the two
//                    members of a coherent pair (Sec. II.D.2: branches equal on
//                    every idle qubit) meet in one bucket
//  k_pair            one CTA per bucket: pairs the members in a shared-memory
//                    open-addressing table, applies the 2x2, drops |a| < eps,
//                    appends the survivors to the CTA's own output segment with
//                    warp-ballot compaction
//  k_probabilities   FP64 marginal probabilities and norm
#include <cuda_runtime.h>
#include <stdint.h>

#include "sqs_device.cuh"
#include "sqs_internal.h"

namespace sqs {

template <class AT>
__global__ void k_init(Ctl* ctl, Arr a, int slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    a.k0[0] = 0;
    if (a.k1) a.k1[0] = 0;
    to_amp(((AT*)a.amp)[0], make_double2(1.0, 0.0));
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

// Visits this CTA's units of `unit` slots of `in` -- slices of segments, or
// of the dense array -- and calls body(base, lim) with every thread for each
// unit holding live slots (lim > 0).  Units are handed out round-robin (unit
// u to CTA u mod gridDim.x), in spread order over the parts of a segment.
// For a segmented array the CTA checks blockDim.x of its candidate units at
// once, one count load per thread, and lists the non-empty ones in shared
// memory (list: blockDim.x entries): the count loads of empty units overlap
// instead of forming a chain, which matters when the segment list is sized
// for a bound far above the count (a graph's static bound).
template <class F>
__device__ __forceinline__ void for_units(const Arr& in, uint64_t n_dense, uint32_t unit,
                                          uint16_t* list, unsigned int* n_list, F&& body) {
  if (!in.seg_cnt) {
    const uint64_t units = (n_dense + unit - 1) / unit;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
      const uint64_t base = u * unit;
      body(base, (uint32_t)(n_dense - base < unit ? n_dense - base : unit));
    }
    return;
  }
  const uint32_t per_seg = ((1u << in.seg_log2) + unit - 1) / unit;
  const uint32_t l = log2_pow2(per_seg);
  const uint64_t units = (uint64_t)in.n_seg * per_seg;
  for (uint64_t k0 = 0; blockIdx.x + k0 * gridDim.x < units; k0 += blockDim.x) {
    if (threadIdx.x == 0) *n_list = 0u;
    __syncthreads();
    const uint64_t u = blockIdx.x + (k0 + threadIdx.x) * gridDim.x;
    if (u < units) {
      const uint64_t v = spread_visit(u, l);
      const uint32_t sg = (uint32_t)(v / per_seg);
      const uint32_t off = (uint32_t)(v - (uint64_t)sg * per_seg) * unit;
      if (off < in.seg_cnt[sg]) list[atomicAdd(n_list, 1u)] = (uint16_t)threadIdx.x;
    }
    __syncthreads();
    const uint32_t n = *n_list;
    for (uint32_t i = 0; i < n; ++i) {
      const uint64_t v = spread_visit(blockIdx.x + (k0 + list[i]) * gridDim.x, l);
      const uint32_t sg = (uint32_t)(v / per_seg);
      const uint32_t off = (uint32_t)(v - (uint64_t)sg * per_seg) * unit;
      const uint32_t cnt = in.seg_cnt[sg];
      body(((uint64_t)sg << in.seg_log2) + off, cnt - off < unit ? cnt - off : unit);
    }
    __syncthreads();  // the list is rebuilt for the next candidates
  }
}

// Op-major over kApplyILP branches per thread: each operation's descriptor
// is read once for four branches (the interpreter's instruction count, not
// memory, bounds a long run on a large state).
constexpr int kApplyILP = 4;

template <int KW, class AT, bool TK, bool TA>
__global__ void __launch_bounds__(kStreamThreads)
    k_apply_inplace(Ctl* ctl, Arr a, int slot, const __grid_constant__ OpList ops, uint32_t seq) {
  typedef typename KT<KW>::T K;
  __shared__ AT tab[kTabEntries];
  __shared__ DevOp sops[kMaxOps];
  if (ctl->err) return;
  load_ops(ops, sops, tab);
  const uint64_t n_dense = ctl->cnt[slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, n_dense);
  __shared__ uint16_t ulist[kStreamThreads];
  __shared__ unsigned int n_ulist;
  // Units of kApplyILP * blockDim slots: a slice of a segment, or of the
  // dense array.
  for_units(a, n_dense, kApplyILP * blockDim.x, ulist, &n_ulist, [&](uint64_t base, uint32_t lim) {
    K k[kApplyILP];
    AT v[kApplyILP];
    bool live[kApplyILP];
#pragma unroll
    for (int q = 0; q < kApplyILP; ++q) {
      const uint32_t j = q * blockDim.x + threadIdx.x;
      live[q] = j < lim;
      k[q] = 0;
      v[q].x = v[q].y = 0;
      if (live[q]) {
        k[q] = ld_key<KW>(a, base + j);
        if (TA) v[q] = ((const AT*)a.amp)[base + j];
      }
    }
    apply_ops_n<KW, AT, kApplyILP>(ops.n, sops, tab, k, v, live);
#pragma unroll
    for (int q = 0; q < kApplyILP; ++q) {
      const uint32_t j = q * blockDim.x + threadIdx.x;
      if (j < lim) {  // no operation of an in-place run drops a branch
        if (TK) st_key<KW>(a, base + j, k[q]);
        if (TA) ((AT*)a.amp)[base + j] = v[q];
      }
    }
  });
}

// Input segment (or dense chunk) c of 2^out.seg_log2 slots is compacted into
// output segment c.
template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads)
    k_apply_compact(Ctl* ctl, Arr in, int in_slot, Arr out, int out_slot,
                    const __grid_constant__ OpList ops, uint32_t seq) {
  __shared__ AT tab[kTabEntries];
  __shared__ DevOp sops[kMaxOps];
  __shared__ unsigned int seg_fill;
  if (ctl->err) return;
  load_ops(ops, sops, tab);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt[(out_slot + 1) & 3] = 0;
    atomicMax(&ctl->peak, ctl->cnt[in_slot]);
  }
  const uint64_t n_dense = ctl->cnt[in_slot];
  const uint64_t chunk = 1ull << out.seg_log2;
  const unsigned int lane = threadIdx.x & 31u;
  if (!in.seg_cnt && n_dense > ((uint64_t)out.n_seg << out.seg_log2)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_err(ctl, kErrCapacity, seq, n_dense);
    return;
  }
  // Every output segment gets its count written, including those past the
  // device-side count (the host sized them from an upper bound).
  for (uint64_t c = blockIdx.x; c < out.n_seg; c += gridDim.x) {
    if (threadIdx.x == 0) seg_fill = 0;
    __syncthreads();
    // Input segment c (any size up to the output segment's) or dense chunk c.
    const uint64_t base = c << out.seg_log2;
    const uint64_t ibase = in.seg_cnt ? (c << in.seg_log2) : base;
    uint64_t cnt;
    if (in.seg_cnt)
      cnt = c < in.n_seg ? in.seg_cnt[c] : 0;
    else
      cnt = base >= n_dense ? 0 : (n_dense - base < chunk ? n_dense - base : chunk);
    for (uint64_t r = 0; r < cnt; r += blockDim.x) {
      const uint64_t i = ibase + r + threadIdx.x;
      bool keep = false;
      typename KT<KW>::T k = 0;
      AT v;
      if (r + threadIdx.x < cnt) {
        k = ld_key<KW>(in, i);
        v = ((const AT*)in.amp)[i];
        keep = apply_ops<KW, AT>(ops.n, sops, tab, k, v);
      }
      const unsigned int ball = __ballot_sync(0xffffffffu, keep);
      unsigned int wbase = 0;
      if (lane == 0 && ball) wbase = atomicAdd(&seg_fill, (unsigned int)__popc(ball));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (keep) {
        const uint64_t pos = base + wbase + __popc(ball & ((1u << lane) - 1u));
        st_key<KW>(out, pos, k);
        ((AT*)out.amp)[pos] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      out.seg_cnt[c] = seg_fill;
      if (seg_fill) atomicAdd(&ctl->cnt[out_slot], (unsigned long long)seg_fill);
    }
  }
}

// ---------------------------------------------------------------------------
// Each thread carries kPartILP branches at once, so their loads and their
// bucket-counter atomics overlap instead of forming one long chain.
constexpr int kPartILP = 4;

template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads)
    k_partition(Ctl* ctl, Arr in, int in_slot, const __grid_constant__ OpList ops, Gate1 g,
                Arr bk, uint32_t seq, uint32_t fill_target) {
  typedef typename KT<KW>::T K;
  __shared__ AT tab[kTabEntries];
  __shared__ DevOp sops[kMaxOps];
  if (ctl->err) return;
  load_ops(ops, sops, tab);
  const uint64_t n_dense = ctl->cnt[in_slot];
  // Buckets from the device count, ceil(count / fill_target), at most the
  // host's bucket count (a bound, which may be far above the count, as
  // inside a captured graph); fill_target 0 keeps the host's count.
  uint64_t nb = fill_target ? (n_dense + fill_target - 1) / fill_target : bk.n_seg;
  if (nb < 1) nb = 1;
  if (nb > bk.n_seg) nb = bk.n_seg;
  const uint32_t n_buckets = (uint32_t)nb;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicMax(&ctl->peak, n_dense);
    ctl->buckets = n_buckets;
    ctl->pair_next = 0u;
  }
  const K bmask = bit_mask<KW>(g.t);
  const uint32_t C = 1u << bk.seg_log2;
  __shared__ uint16_t ulist[kStreamThreads];
  __shared__ unsigned int n_ulist;
  // Units of kPartILP * blockDim slots: a slice of a segment, or of the dense
  // array.
  for_units(in, n_dense, kPartILP * blockDim.x, ulist, &n_ulist, [&](uint64_t base, uint32_t lim) {
    K k[kPartILP];
    AT v[kPartILP];
    bool live[kPartILP];
#pragma unroll
    for (int q = 0; q < kPartILP; ++q) {
      const uint32_t j = q * blockDim.x + threadIdx.x;
      live[q] = j < lim;
      k[q] = 0;
      v[q].x = v[q].y = 0;
      if (live[q]) {
        k[q] = ld_key<KW>(in, base + j);
        v[q] = ((const AT*)in.amp)[base + j];
      }
    }
    apply_ops_n<KW, AT, kPartILP>(ops.n, sops, tab, k, v, live);
    unsigned int pos[kPartILP];
    uint32_t bkt[kPartILP];
#pragma unroll
    for (int q = 0; q < kPartILP; ++q) {
      if (live[q]) {
        const uint64_t h = khash(k[q] & ~bmask);
        bkt[q] = (uint32_t)(((h >> 32) * (uint64_t)n_buckets) >> 32);
        pos[q] = atomicAdd(&bk.seg_cnt[bkt[q]], 1u);
      }
    }
#pragma unroll
    for (int q = 0; q < kPartILP; ++q) {
      if (!live[q]) continue;
      if (pos[q] < C) {
        const uint64_t j = ((uint64_t)bkt[q] << bk.seg_log2) + pos[q];
        st_key<KW>(bk, j, k[q]);
        ((AT*)bk.amp)[j] = v[q];
      } else {
        raise_err(ctl, kErrBucket, seq, (unsigned long long)pos[q] + 1);
      }
    }
  });
}

// Persistent: a resident wave of CTAs takes the buckets the partition used
// (ctl->buckets, from the device count) one by one, so the launch does not
// grow with the host's bucket bound (a graph sizes it for a static bound).
// Shared memory: keys[C], amps[C] (storage type), slots[2C] (0 = empty, else
// index + 1), partner[C].
constexpr int kPairThreads = 512;

template <int KW, class AT>
__global__ void __launch_bounds__(kPairThreads, 3)
    k_pair(Ctl* ctl, Gate1 g, Arr bk, Arr out, int out_slot, uint32_t seq) {
  typedef typename KT<KW>::T K;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int fill;
  if (ctl->err) return;
  const uint32_t C = 1u << bk.seg_log2;
  const uint32_t S = 2u * C;
  K* skey = (K*)smem;
  AT* samp = (AT*)(smem + (size_t)C * sizeof(K));
  unsigned int* slot = (unsigned int*)(smem + (size_t)C * (sizeof(K) + sizeof(AT)));
  int* partner = (int*)(slot + S);

  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[(out_slot + 1) & 3] = 0;
  // Buckets the partition did not use (it sized them from the device count)
  // stay empty.
  const uint32_t nb = ctl->buckets;
  for (uint32_t b = nb + blockIdx.x * blockDim.x + threadIdx.x; b < bk.n_seg;
       b += gridDim.x * blockDim.x)
    out.seg_cnt[b] = 0u;
  // Buckets are taken one at a time from a counter (ctl->pair_next), so a CTA
  // that drew small buckets takes more of them; the next index is drawn while
  // the current bucket is processed.
  __shared__ uint32_t next_b;
  if (threadIdx.x == 0) next_b = atomicAdd(&ctl->pair_next, 1u);
  __syncthreads();
  for (uint32_t b = next_b; b < nb; b = next_b) {
    uint32_t drawn = 0u;
    if (threadIdx.x == 0) drawn = atomicAdd(&ctl->pair_next, 1u);
    const uint32_t n = bk.seg_cnt[b];
    if (n > C) {  // overflow already flagged by the partition
      __syncthreads();  // every thread has read next_b
      if (threadIdx.x == 0) next_b = drawn;
      __syncthreads();
      continue;
    }
    const uint64_t base = (uint64_t)b << bk.seg_log2;
  #pragma unroll 4
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      skey[i] = ld_key<KW>(bk, base + i);
      samp[i] = ((const AT*)bk.amp)[base + i];
      partner[i] = -1;
    }
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) slot[i] = 0u;
    if (threadIdx.x == 0) fill = 0;
    __syncthreads();
    if (threadIdx.x == 0) bk.seg_cnt[b] = 0u;  // bucket is clean for the next use

    const K bmask = bit_mask<KW>(g.t);
    const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
    const K cval = mk<KW>(g.cval[0], g.cval[1]);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const K k = skey[i];
      if ((k & cmask) != cval) continue;  // passes through unchanged
      const K p = k & ~bmask;
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

    // Emitters: branches the controls leave alone, unpaired branches and the
    // bit-0 member of each pair.  Listing them first (in the probe table, which
    // is free now) keeps every lane of the arithmetic below busy.  The pairs
    // are listed apart from the rest ([0, C) and [C, 2C) of the table), so a
    // warp evaluates one form of the 2x2 (two members, or one): mixed, it
    // would issue both FP64 sequences, each with part of its lanes.
    unsigned int* emit = slot;
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned int lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) fill = 0;
    __shared__ unsigned int n_pairs, n_rest;
    if (threadIdx.x == 0) n_pairs = n_rest = 0;
    __syncthreads();
    const uint32_t rounds_in = (n + blockDim.x - 1u) / blockDim.x;
    for (uint32_t r = 0; r < rounds_in; ++r) {
      const uint32_t i = r * blockDim.x + threadIdx.x;
      bool ep = false, er = false;
      if (i < n) {
        const K k = skey[i];
        const bool met = (k & cmask) == cval;
        const bool kt = (k & bmask) != (K)0;
        const bool paired = partner[i] >= 0;
        ep = met && !kt && paired;
        er = !met || !paired;
      }
      const unsigned int bp = __ballot_sync(0xffffffffu, ep);
      const unsigned int br = __ballot_sync(0xffffffffu, er);
      unsigned int wp = 0, wr = 0;
      if (lane == 0) {
        if (bp) wp = atomicAdd(&n_pairs, (unsigned int)__popc(bp));
        if (br) wr = atomicAdd(&n_rest, (unsigned int)__popc(br));
      }
      wp = __shfl_sync(0xffffffffu, wp, 0);
      wr = __shfl_sync(0xffffffffu, wr, 0);
      if (ep) emit[wp + __popc(bp & lt)] = i;
      if (er) emit[C + wr + __popc(br & lt)] = i;
    }
    __syncthreads();
    const uint32_t np = n_pairs;
    const uint32_t ne = np + n_rest;

    const uint64_t obase = (uint64_t)b << out.seg_log2;
    const uint32_t rounds = (ne + blockDim.x - 1u) / blockDim.x;
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t q = r * blockDim.x + threadIdx.x;
      bool keep0 = false, keep1 = false;
      K k0 = 0, k1 = 0;
      AT o0, o1;
      if (q < ne) {
        const uint32_t i = q < np ? emit[q] : emit[C + (q - np)];
        const K k = skey[i];
        const AT ai = samp[i];
        if ((k & cmask) != cval) {
          keep0 = true;  // controls not met: the branch is unchanged
          k0 = k;
          o0 = ai;
        } else {
          const bool kt = (k & bmask) != (K)0;
          const int j = partner[i];
          k0 = k & ~bmask;
          k1 = k | bmask;
          const uint64_t av = g.mode == 1 ? get_field(k0, g.ang_off, g.ang_w) : 0ull;
          if (!kt)
            children<AT>(g, av, true, ai, j >= 0, j >= 0 ? samp[j] : ai, o0, o1);
          else
            children<AT>(g, av, false, ai, true, ai, o0, o1);
          keep0 = keep_amp(o0, g.eps, g.epsf, g.eps2);
          keep1 = keep_amp(o1, g.eps, g.epsf, g.eps2);
        }
      }
      const unsigned int b0 = __ballot_sync(0xffffffffu, keep0);
      const unsigned int b1 = __ballot_sync(0xffffffffu, keep1);
      const unsigned int tot = __popc(b0) + __popc(b1);
      unsigned int wbase = 0;
      if (lane == 0 && tot) wbase = atomicAdd(&fill, tot);
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (keep0) {
        const uint64_t pos = obase + wbase + __popc(b0 & lt);
        st_key<KW>(out, pos, k0);
        ((AT*)out.amp)[pos] = o0;
      }
      if (keep1) {
        const uint64_t pos = obase + wbase + __popc(b0) + __popc(b1 & lt);
        st_key<KW>(out, pos, k1);
        ((AT*)out.amp)[pos] = o1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      out.seg_cnt[b] = fill;
      if (fill) atomicAdd(&ctl->cnt[out_slot], (unsigned long long)fill);
      next_b = drawn;
    }
    __syncthreads();  // fill, next_b and the tables are reused by the next bucket
  }
}

// ---------------------------------------------------------------------------
// Constant target bit: no branch has a partner, so each controlled branch
// expands into its two children directly (no partition, no pairing).  The
// input is walked in chunks of kExpandChunk slots (a dense range, or a slice
// of one segment).
// Copy-pair fold (g.fold_sign != 0): every controlled branch has its partner,
// holding fold_sign times its amplitude, so the bit-0 member alone emits the
// pair's two children and the bit-1 member emits nothing.  The output is
// dense: each block reserves every round's outputs with one atomic.
constexpr uint32_t kExpandChunkLog2 = 12;

// Branches per thread per round.  Two, with at most 64 registers per thread
// (four CTAs of 256 threads per SM), measured faster on the large random
// circuit than four branches at 112 registers: more warps hide the FP64 and
// shared-memory latencies of the fused run.
constexpr int kExpandILP = 2;

template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads, 4)
    k_expand(Ctl* ctl, Arr in, int in_slot, uint64_t n_chunks, Arr out, int out_slot,
             const __grid_constant__ OpList ops, Gate1 g, uint32_t seq) {
  typedef typename KT<KW>::T K;
  __shared__ AT tab[kTabEntries];
  __shared__ DevOp sops[kMaxOps];
  __shared__ unsigned int wtot[kStreamThreads / 32];
  __shared__ unsigned long long round_base;
  if (ctl->err) return;
  load_ops(ops, sops, tab);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt[(out_slot + 1) & 3] = 0;
    atomicMax(&ctl->peak, ctl->cnt[in_slot]);
  }
  const uint64_t n_dense = ctl->cnt[in_slot];
  const uint64_t chunk = 1ull << kExpandChunkLog2;
  // A dense input longer than the chunks the host sized from its bound (a
  // static bound the state outgrew) is an error, never a partial pass.
  if (!in.seg_cnt && n_dense > (n_chunks << kExpandChunkLog2)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_err(ctl, kErrCapacity, seq, n_dense);
    return;
  }
  // Chunks per input segment (segments are at least one chunk long).
  const uint32_t cps_log2 = in.seg_cnt ? in.seg_log2 - kExpandChunkLog2 : 0u;
  const K bmask = bit_mask<KW>(g.t);
  const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
  const K cval = mk<KW>(g.cval[0], g.cval[1]);
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  const uint32_t per_round = kExpandILP * blockDim.x;
  for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    uint64_t ibase, cnt;
    if (in.seg_cnt) {
      const uint64_t sg = c >> cps_log2;
      const uint64_t off = ((c ^ spread(sg, cps_log2)) & ((1ull << cps_log2) - 1ull))
                           << kExpandChunkLog2;
      const uint64_t n_sg = sg < in.n_seg ? in.seg_cnt[sg] : 0;
      ibase = (sg << in.seg_log2) + off;
      cnt = n_sg > off ? (n_sg - off < chunk ? n_sg - off : chunk) : 0;
    } else {
      ibase = c << kExpandChunkLog2;
      cnt = ibase >= n_dense ? 0 : (n_dense - ibase < chunk ? n_dense - ibase : chunk);
    }
    for (uint64_t r = 0; r < cnt; r += per_round) {
      K k[kExpandILP];
      AT v[kExpandILP];
      bool live[kExpandILP];
#pragma unroll
      for (int q = 0; q < kExpandILP; ++q) {
        const uint64_t j = r + (uint64_t)q * blockDim.x + threadIdx.x;
        live[q] = j < cnt;
        k[q] = 0;
        v[q].x = v[q].y = 0;
        if (live[q]) {
          k[q] = ld_key<KW>(in, ibase + j);
          v[q] = ((const AT*)in.amp)[ibase + j];
        }
      }
      apply_ops_n<KW, AT, kExpandILP>(ops.n, sops, tab, k, v, live);
      K k0[kExpandILP], k1[kExpandILP];
      AT o0[kExpandILP], o1[kExpandILP];
      unsigned int b0[kExpandILP], b1[kExpandILP];
      unsigned int wsum = 0;
#pragma unroll
      for (int q = 0; q < kExpandILP; ++q) {
        bool keep0 = false, keep1 = false;
        k0[q] = k1[q] = 0;
        if (live[q]) {
          if ((k[q] & cmask) != cval) {
            keep0 = true;  // controls not met: the branch is unchanged
            k0[q] = k[q];
            o0[q] = v[q];
          } else {
            const bool kt = (k[q] & bmask) != (K)0;
            k0[q] = k[q] & ~bmask;
            k1[q] = k[q] | bmask;
            const uint64_t av = g.mode == 1 ? get_field(k0[q], g.ang_off, g.ang_w) : 0ull;
            if (g.fold_sign == 0) {
              if (!kt)
                children<AT>(g, av, true, v[q], false, v[q], o0[q], o1[q]);
              else
                children<AT>(g, av, false, v[q], true, v[q], o0[q], o1[q]);
              keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
              keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
            } else if (!kt) {
              // The partner holds exactly fold_sign * v: the pair's 2x2 as the
              // merge evaluates it, without looking the partner up.
              auto fold = [&](const AT& a1) {
                if (g.fold_kill >= 0 && below_bits(v[q], g.fold_tmax)) {
                  // The cancelling child is a residue the merge would prune.
                  if (g.fold_kill == 1) {
                    o0[q] = fold_child<AT>(g, 0, v[q], a1);
                    keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
                  } else {
                    o1[q] = fold_child<AT>(g, 1, v[q], a1);
                    keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
                  }
                } else {
                  children<AT>(g, av, true, v[q], true, a1, o0[q], o1[q]);
                  keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
                  keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
                }
              };
              if (g.fold_sign > 0)
                fold(v[q]);
              else
                fold(cneg(v[q]));
            }
          }
        }
        b0[q] = __ballot_sync(0xffffffffu, keep0);
        b1[q] = __ballot_sync(0xffffffffu, keep1);
        wsum += __popc(b0[q]) + __popc(b1[q]);
      }
      // Dense output: the block reserves the round's outputs with one atomic
      // on the output count; each warp writes its items in (item, lane) order.
      if (lane == 0) wtot[warp] = wsum;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned int sum = 0;
        for (unsigned int w = 0; w < blockDim.x / 32u; ++w) {
          const unsigned int t = wtot[w];
          wtot[w] = sum;
          sum += t;
        }
        round_base = sum ? atomicAdd(&ctl->cnt[out_slot], (unsigned long long)sum) : 0ull;
        if (sum && round_base + sum > out.cap)
          raise_err(ctl, kErrCapacity, seq, round_base + sum);
      }
      __syncthreads();
      uint64_t wb = round_base + wtot[warp];
#pragma unroll
      for (int q = 0; q < kExpandILP; ++q) {
        if ((b0[q] >> lane) & 1u) {
          const uint64_t pos = wb + __popc(b0[q] & lt);
          if (pos < out.cap) {
            st_key<KW>(out, pos, k0[q]);
            ((AT*)out.amp)[pos] = o0[q];
          }
        }
        if ((b1[q] >> lane) & 1u) {
          const uint64_t pos = wb + __popc(b0[q]) + __popc(b1[q] & lt);
          if (pos < out.cap) {
            st_key<KW>(out, pos, k1[q]);
            ((AT*)out.amp)[pos] = o1[q];
          }
        }
        wb += __popc(b0[q]) + __popc(b1[q]);
      }
      __syncthreads();  // wtot and round_base are reused by the next round
    }
  }
}

// ---------------------------------------------------------------------------
// Copy-pair fold without controls: only the bit-0 member of each pair emits
// (the pair's two children), so the bit-1 members need neither their
// amplitude nor the fused run.  The run never reads or writes the target bit
// (the host drops a bit's copy-pair property as soon as an operation touches
// it), so a member's target bit is already known from its loaded key.
//
// Each CTA stages kFoldSub input slots at a time: phase 1 reads every key
// (coalesced), tests the target bit, loads the amplitudes of the bit-0
// members only and compacts those members into shared memory; phase 2 runs
// the fused run and the fold on the compacted list, so every lane of the
// FP64 sequence holds a member that emits.  The arithmetic per member is the
// fold branch of k_expand, so the state is bit-identical to it.
constexpr uint32_t kFoldSub = 2048;
constexpr int kFoldILP = 2;

template <int KW, class AT>
constexpr size_t fold_smem_bytes() {
  return (size_t)kFoldSub * (sizeof(typename KT<KW>::T) + sizeof(AT));
}

template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads, 3)
    k_fold(Ctl* ctl, Arr in, int in_slot, uint64_t n_chunks, Arr out, int out_slot,
           const __grid_constant__ OpList ops, Gate1 g, uint32_t seq) {
  typedef typename KT<KW>::T K;
  __shared__ AT tab[kTabEntries];
  __shared__ DevOp sops[kMaxOps];
  __shared__ unsigned int wtot[kStreamThreads / 32];
  __shared__ unsigned long long round_base;
  __shared__ unsigned int n_act;
  extern __shared__ __align__(16) unsigned char fold_smem[];
  K* skey = (K*)fold_smem;
  AT* samp = (AT*)(fold_smem + (size_t)kFoldSub * sizeof(K));
  if (ctl->err) return;
  load_ops(ops, sops, tab);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt[(out_slot + 1) & 3] = 0;
    atomicMax(&ctl->peak, ctl->cnt[in_slot]);
  }
  const uint64_t n_dense = ctl->cnt[in_slot];
  const uint64_t chunk = 1ull << kExpandChunkLog2;
  if (!in.seg_cnt && n_dense > (n_chunks << kExpandChunkLog2)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_err(ctl, kErrCapacity, seq, n_dense);
    return;
  }
  const uint32_t cps_log2 = in.seg_cnt ? in.seg_log2 - kExpandChunkLog2 : 0u;
  const K bmask = bit_mask<KW>(g.t);
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  constexpr int kPer = (int)(kFoldSub / kStreamThreads);
  for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    uint64_t ibase, cnt;
    if (in.seg_cnt) {
      const uint64_t sg = c >> cps_log2;
      const uint64_t off = ((c ^ spread(sg, cps_log2)) & ((1ull << cps_log2) - 1ull))
                           << kExpandChunkLog2;
      const uint64_t n_sg = sg < in.n_seg ? in.seg_cnt[sg] : 0;
      ibase = (sg << in.seg_log2) + off;
      cnt = n_sg > off ? (n_sg - off < chunk ? n_sg - off : chunk) : 0;
    } else {
      ibase = c << kExpandChunkLog2;
      cnt = ibase >= n_dense ? 0 : (n_dense - ibase < chunk ? n_dense - ibase : chunk);
    }
    for (uint64_t s0 = 0; s0 < cnt; s0 += kFoldSub) {
      const uint32_t scnt = (uint32_t)(cnt - s0 < kFoldSub ? cnt - s0 : kFoldSub);
      const uint64_t sbase = ibase + s0;
      // ---- phase 1: keys, target-bit test, bit-0 amplitudes, compaction ----
      K kk[kPer];
      AT av[kPer];
      unsigned int bal[kPer];
      unsigned int mine = 0;
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const uint32_t j = (uint32_t)r * kStreamThreads + threadIdx.x;
        bool act = false;
        kk[r] = 0;
        if (j < scnt) {
          kk[r] = ld_key<KW>(in, sbase + j);
          act = (kk[r] & bmask) == (K)0;
        }
        if (act) av[r] = ((const AT*)in.amp)[sbase + j];
        bal[r] = __ballot_sync(0xffffffffu, act);
        mine += __popc(bal[r]);
      }
      if (lane == 0) wtot[warp] = mine;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned int sum = 0;
        for (unsigned int w = 0; w < kStreamThreads / 32u; ++w) {
          const unsigned int t = wtot[w];
          wtot[w] = sum;
          sum += t;
        }
        n_act = sum;
      }
      __syncthreads();
      {
        unsigned int pos = wtot[warp];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
          if ((bal[r] >> lane) & 1u) {
            const unsigned int p = pos + __popc(bal[r] & lt);
            skey[p] = kk[r];
            samp[p] = av[r];
          }
          pos += __popc(bal[r]);
        }
      }
      __syncthreads();
      const uint32_t na = n_act;
      // ---- phase 2: fused run and fold on the compacted bit-0 members ----
      for (uint32_t r0 = 0; r0 < na; r0 += kFoldILP * kStreamThreads) {
        K k[kFoldILP];
        AT v[kFoldILP];
        bool live[kFoldILP];
#pragma unroll
        for (int q = 0; q < kFoldILP; ++q) {
          const uint32_t i = r0 + (uint32_t)q * kStreamThreads + threadIdx.x;
          live[q] = i < na;
          k[q] = 0;
          v[q].x = v[q].y = 0;
          if (live[q]) {
            k[q] = skey[i];
            v[q] = samp[i];
          }
        }
        apply_ops_n<KW, AT, kFoldILP>(ops.n, sops, tab, k, v, live);
        K k0[kFoldILP], k1[kFoldILP];
        AT o0[kFoldILP], o1[kFoldILP];
        unsigned int b0[kFoldILP], b1[kFoldILP];
        unsigned int wsum = 0;
#pragma unroll
        for (int q = 0; q < kFoldILP; ++q) {
          bool keep0 = false, keep1 = false;
          k0[q] = k[q];
          k1[q] = k[q] | bmask;
          const AT a1 = g.fold_sign > 0 ? v[q] : cneg(v[q]);
          // The cancelling child is a residue the merge would prune whenever
          // the member's magnitude is below fold_tmax (every amplitude of a
          // normalised state): then only the surviving child is evaluated.
          // The general 2x2 sits in a separate warp-uniform branch, so that
          // its FP64 products are never issued for lanes that do not need them.
          const bool kill = live[q] && g.fold_kill >= 0 && below_bits(v[q], g.fold_tmax);
          if (kill) {
            if (g.fold_kill == 1) {
              o0[q] = fold_child<AT>(g, 0, v[q], a1);
              keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
            } else {
              o1[q] = fold_child<AT>(g, 1, v[q], a1);
              keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
            }
          }
          if (__any_sync(0xffffffffu, live[q] && !kill)) {
            if (live[q] && !kill) {
              const uint64_t avv = g.mode == 1 ? get_field(k0[q], g.ang_off, g.ang_w) : 0ull;
              children<AT>(g, avv, true, v[q], true, a1, o0[q], o1[q]);
              keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
              keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
            }
          }
          b0[q] = __ballot_sync(0xffffffffu, keep0);
          b1[q] = __ballot_sync(0xffffffffu, keep1);
          wsum += __popc(b0[q]) + __popc(b1[q]);
        }
        if (lane == 0) wtot[warp] = wsum;
        __syncthreads();
        if (threadIdx.x == 0) {
          unsigned int sum = 0;
          for (unsigned int w = 0; w < kStreamThreads / 32u; ++w) {
            const unsigned int t = wtot[w];
            wtot[w] = sum;
            sum += t;
          }
          round_base = sum ? atomicAdd(&ctl->cnt[out_slot], (unsigned long long)sum) : 0ull;
          if (sum && round_base + sum > out.cap)
            raise_err(ctl, kErrCapacity, seq, round_base + sum);
        }
        __syncthreads();
        uint64_t wb = round_base + wtot[warp];
#pragma unroll
        for (int q = 0; q < kFoldILP; ++q) {
          if ((b0[q] >> lane) & 1u) {
            const uint64_t pos = wb + __popc(b0[q] & lt);
            if (pos < out.cap) {
              st_key<KW>(out, pos, k0[q]);
              ((AT*)out.amp)[pos] = o0[q];
            }
          }
          if ((b1[q] >> lane) & 1u) {
            const uint64_t pos = wb + __popc(b0[q]) + __popc(b1[q] & lt);
            if (pos < out.cap) {
              st_key<KW>(out, pos, k1[q]);
              ((AT*)out.amp)[pos] = o1[q];
            }
          }
          wb += __popc(b0[q]) + __popc(b1[q]);
        }
        __syncthreads();  // wtot and round_base are reused by the next round
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Staged input stream (TMA bulk copies, double-buffered).  The input is
// walked in units of kUnit slots: slice (G ^ spread(G >> 2, 2)) & 3 of chunk
// G >> 2 of 2^kExpandChunkLog2 slots (a dense range, or a slice of one
// segment).  A
// CTA takes units G = blockIdx.x, + gridDim.x, ...; one elected thread copies
// unit i + 2 into the stage buffer unit i has just released, with
// cp.async.bulk on that buffer's mbarrier, while every thread computes on
// unit i + 1's buffer: the loads of the next units overlap the arithmetic of
// this one and no thread stalls on a global load.
constexpr uint32_t kWaitLimit = 1u << 26;  // bounded mbarrier wait (try_wait polls)
constexpr uint32_t kUnitLog2 = 10;
constexpr uint32_t kUnit = 1u << kUnitLog2;
constexpr uint32_t kUnitsPerChunkLog2 = kExpandChunkLog2 - kUnitLog2;

struct UnitRange {
  uint64_t base;
  uint32_t cnt;
};

__device__ __forceinline__ UnitRange unit_range(const Arr& in, uint64_t n_dense, uint32_t cps_log2,
                                                uint64_t G) {
  const uint64_t c = G >> kUnitsPerChunkLog2;
  const uint64_t chunk = 1ull << kExpandChunkLog2;
  uint64_t ibase, cnt;
  if (in.seg_cnt) {
    const uint64_t sg = c >> cps_log2;
    const uint64_t off = ((c ^ spread(sg, cps_log2)) & ((1ull << cps_log2) - 1ull))
                         << kExpandChunkLog2;
    const uint64_t n_sg = sg < in.n_seg ? in.seg_cnt[sg] : 0;
    ibase = (sg << in.seg_log2) + off;
    cnt = n_sg > off ? (n_sg - off < chunk ? n_sg - off : chunk) : 0;
  } else {
    ibase = c << kExpandChunkLog2;
    cnt = ibase >= n_dense ? 0 : (n_dense - ibase < chunk ? n_dense - ibase : chunk);
  }
  const uint64_t off = ((G ^ spread(c, kUnitsPerChunkLog2)) & ((1ull << kUnitsPerChunkLog2) - 1ull))
                       << kUnitLog2;
  UnitRange r;
  r.base = ibase + off;
  r.cnt = (uint32_t)(cnt > off ? (cnt - off < kUnit ? cnt - off : kUnit) : 0);
  return r;
}

template <int KW, class AT>
struct StageBuf {
  uint64_t k0[kUnit];
  uint64_t k1[KW == 2 ? kUnit : 2];
  AT amp[kUnit];
};

template <int KW>
__device__ __forceinline__ typename KT<KW>::T stage_key(const uint64_t* k0, const uint64_t* k1,
                                                        uint32_t j) {
  return mk<KW>(k0[j], KW == 2 ? k1[j] : 0ull);
}

// Thread 0: copies unit r into buffer b, arriving on `bar` with the byte
// count.  Bulk copies need 16-byte multiples: with 8-byte elements and an odd
// count the last element is read with a plain load instead (never past the
// unit).  A unit with nothing to copy arrives with zero bytes, so every
// unit completes one phase of its barrier.
template <int KW, class AT>
__device__ __forceinline__ void stage_issue(StageBuf<KW, AT>& b, uint64_t* bar, const Arr& in,
                                            UnitRange r) {
  const uint32_t even = r.cnt & ~1u;
  const uint32_t na = sizeof(AT) == 16 ? r.cnt : even;
  const uint32_t bytes = even * 8u * (uint32_t)KW + na * (uint32_t)sizeof(AT);
  mbar_expect_tx(bar, bytes);
  if (even) {
    bulk_g2s(b.k0, in.k0 + r.base, even * 8u, bar);
    if (KW == 2) bulk_g2s(b.k1, in.k1 + r.base, even * 8u, bar);
  }
  if (na) bulk_g2s(b.amp, (const AT*)in.amp + r.base, na * (uint32_t)sizeof(AT), bar);
  if (even < r.cnt) {
    const uint64_t t = r.base + even;
    b.k0[even] = in.k0[t];
    if (KW == 2) b.k1[even] = in.k1[t];
    if (na < r.cnt) b.amp[even] = ((const AT*)in.amp)[t];
  }
}

// Bounded wait on one phase of a stage barrier (every thread polls).
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity) {
  uint32_t it = 0;
  while (!mbar_try_wait(bar, parity))
    if (++it >= kWaitLimit) return false;
  return true;
}

// Drives the staged stream over this CTA's units: waits for each unit's
// buffer, calls unit(buffer, range) -- which must end with a __syncthreads
// after its last read of the buffer -- then refills the buffer with the unit
// two steps ahead.  smem: two barriers (first 16 bytes of a 128-byte
// header), then the two buffers.  Returns false when a bounded wait ran out
// (the error is raised; copies still in flight have been waited for).
template <int KW, class AT, class F>
__device__ __forceinline__ bool staged_stream(Ctl* ctl, const Arr& in, uint64_t n_dense,
                                              uint64_t n_chunks, uint32_t seq,
                                              unsigned char* smem, unsigned int* abort_flag,
                                              F&& unit) {
  uint64_t* bar = (uint64_t*)smem;
  StageBuf<KW, AT>* stage = (StageBuf<KW, AT>*)(smem + 128);
  const uint32_t cps_log2 = in.seg_cnt ? in.seg_log2 - kExpandChunkLog2 : 0u;
  // A dense input covers only the units its device count reaches (the host
  // sized n_chunks from a bound, which may be far above it, as in a graph).
  // Whole chunks: the slices of the last chunk are visited in spread order.
  uint64_t n_units = n_chunks << kUnitsPerChunkLog2;
  if (!in.seg_cnt) {
    const uint64_t need = ((n_dense + (1ull << kExpandChunkLog2) - 1) >> kExpandChunkLog2)
                          << kUnitsPerChunkLog2;
    if (need < n_units) n_units = need;
  }
  // Units with no live slot (the tails of segments that are not full) are
  // skipped: every thread walks the same sequence of non-empty units.
  auto next_unit = [&](uint64_t G) {
    for (; G < n_units; G += gridDim.x)
      if (unit_range(in, n_dense, cps_log2, G).cnt) return G;
    return n_units;
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    *abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint64_t g_cur = next_unit(blockIdx.x);
  uint64_t g_nxt = g_cur < n_units ? next_unit(g_cur + gridDim.x) : n_units;
  if (threadIdx.x == 0) {
    if (g_cur < n_units)
      stage_issue<KW, AT>(stage[0], &bar[0], in, unit_range(in, n_dense, cps_log2, g_cur));
    if (g_nxt < n_units)
      stage_issue<KW, AT>(stage[1], &bar[1], in, unit_range(in, n_dense, cps_log2, g_nxt));
  }
  for (uint32_t i = 0; g_cur < n_units; ++i) {
    const uint32_t bi = i & 1u;
    if (!stage_wait(&bar[bi], (i >> 1) & 1u)) atomicOr(abort_flag, 1u);
    __syncthreads();
    if (*abort_flag) {
      // Copies may still be landing in this CTA's buffers: let them finish
      // (bounded again) before the CTA's shared memory is released.
      if (threadIdx.x == 0) {
        raise_err(ctl, kErrProbe, seq, 0);
        stage_wait(&bar[bi], (i >> 1) & 1u);
        if (g_nxt < n_units) stage_wait(&bar[bi ^ 1u], ((i + 1) >> 1) & 1u);
      }
      return false;
    }
    unit(stage[bi], unit_range(in, n_dense, cps_log2, g_cur));
    const uint64_t g_after = g_nxt < n_units ? next_unit(g_nxt + gridDim.x) : n_units;
    if (threadIdx.x == 0 && g_after < n_units)
      stage_issue<KW, AT>(stage[bi], &bar[bi], in, unit_range(in, n_dense, cps_log2, g_after));
    g_cur = g_nxt;
    g_nxt = g_after;
  }
  return true;
}

template <int KW, class AT>
constexpr size_t stream_smem_bytes() {
  return 128 + 2 * sizeof(StageBuf<KW, AT>);
}

// Resident CTAs per SM of a staged-stream kernel (cached per device).
template <class Kern>
static cudaError_t resident_per_sm(Kern kern, size_t smem, std::atomic<int>* per_sm_cache,
                                   int& occ) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  occ = dev < 64 ? per_sm_cache[dev].load(std::memory_order_relaxed) : 0;
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStreamThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (dev < 64) per_sm_cache[dev].store(occ, std::memory_order_relaxed);
  }
  return cudaSuccess;
}


// ---------------------------------------------------------------------------
// Staged variants of k_expand and k_fold, for launches with no fused
// operation (measured faster there: the input arrives by bulk copy while the
// previous unit computes; with a long fused run the per-unit barriers cost
// more than the loads they hide, and the register-fed kernels above win).
// They carry no operation interpreter: without its tables and registers more
// CTAs fit an SM.
// Constant target bit: no branch has a partner, so each controlled branch
// expands into its two children directly (no partition, no pairing).
// Copy-pair fold with controls (g.fold_sign != 0): every controlled branch has
// its partner, holding fold_sign times its amplitude, so the bit-0 member
// alone emits the pair's two children and the bit-1 member emits nothing;
// branches whose controls fail pass unchanged.  Input through the staged
// stream; the output is dense: each block reserves every round's outputs with
// one atomic.
template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads, 4)
    k_expand_staged(Ctl* ctl, Arr in, int in_slot, uint64_t n_chunks, Arr out, int out_slot,
                    Gate1 g, uint32_t seq) {
  typedef typename KT<KW>::T K;
  __shared__ unsigned int wtot[kStreamThreads / 32];
  __shared__ unsigned long long round_base;
  __shared__ unsigned int abort_flag;
  extern __shared__ __align__(128) unsigned char exp_smem[];
  if (ctl->err) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt[(out_slot + 1) & 3] = 0;
    atomicMax(&ctl->peak, ctl->cnt[in_slot]);
  }
  const uint64_t n_dense = ctl->cnt[in_slot];
  // A dense input longer than the chunks the host sized from its bound (a
  // static bound the state outgrew) is an error, never a partial pass.
  if (!in.seg_cnt && n_dense > (n_chunks << kExpandChunkLog2)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_err(ctl, kErrCapacity, seq, n_dense);
    return;
  }
  const K bmask = bit_mask<KW>(g.t);
  const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
  const K cval = mk<KW>(g.cval[0], g.cval[1]);
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  auto unit = [&](StageBuf<KW, AT>& sb, const UnitRange r) {
    for (uint32_t r0 = 0; r0 < r.cnt; r0 += kExpandILP * kStreamThreads) {
      K k[kExpandILP];
      AT v[kExpandILP];
      bool live[kExpandILP];
#pragma unroll
      for (int q = 0; q < kExpandILP; ++q) {
        const uint32_t j = r0 + (uint32_t)q * kStreamThreads + threadIdx.x;
        live[q] = j < r.cnt;
        k[q] = 0;
        v[q].x = v[q].y = 0;
        if (live[q]) {
          k[q] = stage_key<KW>(sb.k0, sb.k1, j);
          v[q] = sb.amp[j];
        }
      }
      K k0[kExpandILP], k1[kExpandILP];
      AT o0[kExpandILP], o1[kExpandILP];
      unsigned int b0[kExpandILP], b1[kExpandILP];
      unsigned int wsum = 0;
#pragma unroll
      for (int q = 0; q < kExpandILP; ++q) {
        bool keep0 = false, keep1 = false;
        k0[q] = k1[q] = 0;
        if (live[q]) {
          if ((k[q] & cmask) != cval) {
            keep0 = true;  // controls not met: the branch is unchanged
            k0[q] = k[q];
            o0[q] = v[q];
          } else {
            const bool kt = (k[q] & bmask) != (K)0;
            k0[q] = k[q] & ~bmask;
            k1[q] = k[q] | bmask;
            const uint64_t av = g.mode == 1 ? get_field(k0[q], g.ang_off, g.ang_w) : 0ull;
            if (g.fold_sign == 0) {
              if (!kt)
                children<AT>(g, av, true, v[q], false, v[q], o0[q], o1[q]);
              else
                children<AT>(g, av, false, v[q], true, v[q], o0[q], o1[q]);
              keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
              keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
            } else if (!kt) {
              // The partner holds exactly fold_sign * v: the pair's 2x2 as the
              // merge evaluates it, without looking the partner up.
              auto fold = [&](const AT& a1) {
                if (g.fold_kill >= 0 && below_bits(v[q], g.fold_tmax)) {
                  // The cancelling child is a residue the merge would prune.
                  if (g.fold_kill == 1) {
                    o0[q] = fold_child<AT>(g, 0, v[q], a1);
                    keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
                  } else {
                    o1[q] = fold_child<AT>(g, 1, v[q], a1);
                    keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
                  }
                } else {
                  children<AT>(g, av, true, v[q], true, a1, o0[q], o1[q]);
                  keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
                  keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
                }
              };
              if (g.fold_sign > 0)
                fold(v[q]);
              else
                fold(cneg(v[q]));
            }
          }
        }
        b0[q] = __ballot_sync(0xffffffffu, keep0);
        b1[q] = __ballot_sync(0xffffffffu, keep1);
        wsum += __popc(b0[q]) + __popc(b1[q]);
      }
      // Dense output: the block reserves the round's outputs with one atomic
      // on the output count; each warp writes its items in (item, lane) order.
      if (lane == 0) wtot[warp] = wsum;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned int sum = 0;
        for (unsigned int w = 0; w < kStreamThreads / 32u; ++w) {
          const unsigned int t = wtot[w];
          wtot[w] = sum;
          sum += t;
        }
        round_base = sum ? atomicAdd(&ctl->cnt[out_slot], (unsigned long long)sum) : 0ull;
        if (sum && round_base + sum > out.cap)
          raise_err(ctl, kErrCapacity, seq, round_base + sum);
      }
      __syncthreads();
      uint64_t wb = round_base + wtot[warp];
#pragma unroll
      for (int q = 0; q < kExpandILP; ++q) {
        if ((b0[q] >> lane) & 1u) {
          const uint64_t pos = wb + __popc(b0[q] & lt);
          if (pos < out.cap) {
            st_key<KW>(out, pos, k0[q]);
            ((AT*)out.amp)[pos] = o0[q];
          }
        }
        if ((b1[q] >> lane) & 1u) {
          const uint64_t pos = wb + __popc(b0[q]) + __popc(b1[q] & lt);
          if (pos < out.cap) {
            st_key<KW>(out, pos, k1[q]);
            ((AT*)out.amp)[pos] = o1[q];
          }
        }
        wb += __popc(b0[q]) + __popc(b1[q]);
      }
      __syncthreads();  // wtot, round_base and the buffer are reused next
    }
    __syncthreads();  // an empty unit: the buffer is released all the same
  };
  staged_stream<KW, AT>(ctl, in, n_dense, n_chunks, seq, exp_smem, &abort_flag, unit);
}

// ---------------------------------------------------------------------------
// Copy-pair fold without controls: only the bit-0 member of each pair emits
// (the pair's two children), so the bit-1 members need neither the fused run
// nor any arithmetic.  The run never reads or writes the target bit (the
// host drops a bit's copy-pair property as soon as an operation touches it),
// so a member's target bit is already known from its loaded key.
//
// Input through the staged stream above.  Per unit: the bit-0 members are
// compacted into a list (warp ballots), then the fused run and the fold run
// on the list, so every lane of the FP64 sequence holds a member that emits.
// The arithmetic per member is the fold branch of k_expand, so the state is
// bit-identical to it.
template <int KW, class AT>
constexpr size_t fold_staged_smem_bytes() {
  return stream_smem_bytes<KW, AT>() + kUnit * sizeof(uint16_t);
}

template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads, 4)
    k_fold_staged(Ctl* ctl, Arr in, int in_slot, uint64_t n_chunks, Arr out, int out_slot,
                  Gate1 g, uint32_t seq) {
  typedef typename KT<KW>::T K;
  __shared__ unsigned int wtot[kStreamThreads / 32];
  __shared__ unsigned long long round_base;
  __shared__ unsigned int n_act, abort_flag;
  extern __shared__ __align__(128) unsigned char fold_smem[];
  uint16_t* list = (uint16_t*)(fold_smem + stream_smem_bytes<KW, AT>());
  if (ctl->err) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt[(out_slot + 1) & 3] = 0;
    atomicMax(&ctl->peak, ctl->cnt[in_slot]);
  }
  const uint64_t n_dense = ctl->cnt[in_slot];
  if (!in.seg_cnt && n_dense > (n_chunks << kExpandChunkLog2)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_err(ctl, kErrCapacity, seq, n_dense);
    return;
  }
  const K bmask = bit_mask<KW>(g.t);
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  constexpr int kPer = (int)(kUnit / kStreamThreads);
  auto unit = [&](StageBuf<KW, AT>& sb, const UnitRange r) {
    // ---- compaction of the bit-0 members ----
    unsigned int bal[kPer];
    unsigned int mine = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const uint32_t j = (uint32_t)q * kStreamThreads + threadIdx.x;
      const bool act = j < r.cnt && (stage_key<KW>(sb.k0, sb.k1, j) & bmask) == (K)0;
      bal[q] = __ballot_sync(0xffffffffu, act);
      mine += __popc(bal[q]);
    }
    if (lane == 0) wtot[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int sum = 0;
      for (unsigned int w = 0; w < kStreamThreads / 32u; ++w) {
        const unsigned int t = wtot[w];
        wtot[w] = sum;
        sum += t;
      }
      n_act = sum;
    }
    __syncthreads();
    {
      unsigned int pos = wtot[warp];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        if ((bal[q] >> lane) & 1u)
          list[pos + __popc(bal[q] & lt)] = (uint16_t)((uint32_t)q * kStreamThreads + threadIdx.x);
        pos += __popc(bal[q]);
      }
    }
    __syncthreads();
    const uint32_t na = n_act;
    // ---- fused run and fold on the compacted members ----
    for (uint32_t r0 = 0; r0 < na; r0 += kFoldILP * kStreamThreads) {
      K k[kFoldILP];
      AT v[kFoldILP];
      bool live[kFoldILP];
#pragma unroll
      for (int q = 0; q < kFoldILP; ++q) {
        const uint32_t li = r0 + (uint32_t)q * kStreamThreads + threadIdx.x;
        live[q] = li < na;
        k[q] = 0;
        v[q].x = v[q].y = 0;
        if (live[q]) {
          const uint32_t j = list[li];
          k[q] = stage_key<KW>(sb.k0, sb.k1, j);
          v[q] = sb.amp[j];
        }
      }
      K k1[kFoldILP];
      AT o0[kFoldILP], o1[kFoldILP];
      unsigned int b0[kFoldILP], b1[kFoldILP];
      unsigned int wsum = 0;
#pragma unroll
      for (int q = 0; q < kFoldILP; ++q) {
        bool keep0 = false, keep1 = false;
        k1[q] = k[q] | bmask;
        const AT a1 = g.fold_sign > 0 ? v[q] : cneg(v[q]);
        // The cancelling child is a residue the merge would prune whenever
        // the member's magnitude is below fold_tmax (every amplitude of a
        // normalised state): then only the surviving child is evaluated.  The
        // general 2x2 runs in a separate, warp-uniform branch, so that its
        // FP64 products are never issued for lanes that do not need them.
        const bool kill = live[q] && g.fold_kill >= 0 && below_bits(v[q], g.fold_tmax);
        if (kill) {
          if (g.fold_kill == 1) {
            o0[q] = fold_child<AT>(g, 0, v[q], a1);
            keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
          } else {
            o1[q] = fold_child<AT>(g, 1, v[q], a1);
            keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
          }
        }
        if (__any_sync(0xffffffffu, live[q] && !kill)) {
          if (live[q] && !kill) {
            const uint64_t avv = g.mode == 1 ? get_field(k[q], g.ang_off, g.ang_w) : 0ull;
            children<AT>(g, avv, true, v[q], true, a1, o0[q], o1[q]);
            keep0 = keep_amp(o0[q], g.eps, g.epsf, g.eps2);
            keep1 = keep_amp(o1[q], g.eps, g.epsf, g.eps2);
          }
        }
        b0[q] = __ballot_sync(0xffffffffu, keep0);
        b1[q] = __ballot_sync(0xffffffffu, keep1);
        wsum += __popc(b0[q]) + __popc(b1[q]);
      }
      if (lane == 0) wtot[warp] = wsum;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned int sum = 0;
        for (unsigned int w = 0; w < kStreamThreads / 32u; ++w) {
          const unsigned int t = wtot[w];
          wtot[w] = sum;
          sum += t;
        }
        round_base = sum ? atomicAdd(&ctl->cnt[out_slot], (unsigned long long)sum) : 0ull;
        if (sum && round_base + sum > out.cap)
          raise_err(ctl, kErrCapacity, seq, round_base + sum);
      }
      __syncthreads();
      uint64_t wb = round_base + wtot[warp];
#pragma unroll
      for (int q = 0; q < kFoldILP; ++q) {
        if ((b0[q] >> lane) & 1u) {
          const uint64_t pos = wb + __popc(b0[q] & lt);
          if (pos < out.cap) {
            st_key<KW>(out, pos, k[q]);
            ((AT*)out.amp)[pos] = o0[q];
          }
        }
        if ((b1[q] >> lane) & 1u) {
          const uint64_t pos = wb + __popc(b0[q]) + __popc(b1[q] & lt);
          if (pos < out.cap) {
            st_key<KW>(out, pos, k1[q]);
            ((AT*)out.amp)[pos] = o1[q];
          }
        }
        wb += __popc(b0[q]) + __popc(b1[q]);
      }
      __syncthreads();  // wtot, round_base, the list and the buffer are reused next
    }
    // With no member the last barrier above is the compaction's: every read
    // of the buffer is done either way.
  };
  staged_stream<KW, AT>(ctl, in, n_dense, n_chunks, seq, fold_smem, &abort_flag, unit);
}

// ---------------------------------------------------------------------------
constexpr int kProbThreads = 256;
constexpr uint32_t kSmemBinsLog2 = 11;

template <int KW, class AT>
__global__ void __launch_bounds__(kProbThreads)
    k_probabilities(Ctl* ctl, Arr a, int slot, uint32_t off, uint32_t w, double* probs,
                    double* nrm) {
  __shared__ double bins[1u << kSmemBinsLog2];
  __shared__ double red[kProbThreads / 32];
  if (ctl->err) return;
  const bool smem_bins = probs != nullptr && w <= kSmemBinsLog2;
  if (smem_bins)
    for (uint32_t v = threadIdx.x; v < (1u << w); v += blockDim.x) bins[v] = 0.0;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, ctl->cnt[slot]);
  double acc = 0.0;
  for_each_live(a, ctl->cnt[slot], [&](uint64_t i) {
    const double p = norm2(((const AT*)a.amp)[i]);
    acc += p;
    if (probs) {
      const uint64_t val = get_field(ld_key<KW>(a, i), off, w);
      if (smem_bins)
        atomicAdd(&bins[val], p);
      else
        atomicAdd(&probs[val], p);
    }
  });
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31u) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kProbThreads / 32; ++q) t += red[q];
    if (nrm) atomicAdd(nrm, t);
  }
  if (smem_bins) {
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < (1u << w); v += blockDim.x)
      if (bins[v] != 0.0) atomicAdd(&probs[v], bins[v]);
  }
}

// One CTA per segment: copy it to its dense offset.
template <int KW, class AT>
__global__ void k_densify(Arr in, const uint64_t* offsets, Arr out) {
  const uint32_t s = blockIdx.x;
  const uint32_t n = in.seg_cnt[s];
  const uint64_t src = (uint64_t)s << in.seg_log2;
  const uint64_t dst = offsets[s];
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    st_key<KW>(out, dst + i, ld_key<KW>(in, src + i));
    ((AT*)out.amp)[dst + i] = ((const AT*)in.amp)[src + i];
  }
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
// Binned merge: coarse bins filled in coalesced runs, paired by a cluster.
//
// k_bin streams the state through the fused run and sorts each tile of
// kBinTile branches by bin in shared memory, so each tile reserves its place
// in a bin with one global atomic per bin it touches and writes runs, not
// single branches.  A bin holds up to kClusterCtas * kSliceCap branches.
//
// k_pair_cluster gives each bin to a cluster of kClusterCtas CTAs.  CTA r
// pulls slice r of the bin into its shared memory with one TMA bulk copy per
// array (cp.async.bulk, completion on an mbarrier), then every CTA inserts its
// branches' pair classes into one open-addressing table spread over the
// cluster's shared memory (distributed shared memory atomics), so a pair
// whose members sit in different slices still meets.  Emission is as in
// k_pair; the survivors of CTA r go to output segment (bin, r).
// ---------------------------------------------------------------------------
constexpr int kBinThreads = 512;
constexpr int kBinILP = 8;
constexpr int kBinTile = kBinThreads * kBinILP;  // 4096 branches
constexpr int kClusterCtas = 8;
constexpr int kSliceLog2 = 12;                   // 4096 branches per CTA
constexpr int kSliceCap = 1 << kSliceLog2;
constexpr int kBinLog2 = kSliceLog2 + 3;         // 32768 branches per bin
constexpr int kSlotsPerCta = 2 * kSliceCap;      // hash slots per CTA
constexpr int kPairCThreads = 512;

template <int KW, class AT>
struct BinSmem {
  typename KT<KW>::T key[kBinTile];
  AT amp[kBinTile];
  uint16_t bin[kBinTile];
  unsigned int hist[kMaxBins];
  unsigned int off[kMaxBins];
  unsigned int base[kMaxBins];
  AT tab[kTabEntries];
  DevOp ops[kMaxOps];
  unsigned int scan[kBinThreads / 32];
};

template <int KW, class AT>
__global__ void __launch_bounds__(kBinThreads)
    k_bin(Ctl* ctl, Arr in, int in_slot, const __grid_constant__ OpList ops, Gate1 g, Arr bins,
          uint32_t seq) {
  typedef typename KT<KW>::T K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BinSmem<KW, AT>& sm = *reinterpret_cast<BinSmem<KW, AT>*>(smem_raw);
  if (ctl->err) return;
  load_ops(ops, sm.ops, sm.tab);
  const uint64_t n_dense = ctl->cnt[in_slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, n_dense);
  const K bmask = bit_mask<KW>(g.t);
  const uint32_t B = bins.n_seg;
  const uint32_t cap = 1u << bins.seg_log2;
  uint32_t per_seg = 1;
  uint64_t units;
  if (in.seg_cnt) {
    per_seg = ((1u << in.seg_log2) + kBinTile - 1) / kBinTile;
    units = (uint64_t)in.n_seg * per_seg;
  } else {
    units = (n_dense + kBinTile - 1) / kBinTile;
  }
  for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) sm.hist[b] = 0u;
  __syncthreads();
  for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
    uint64_t base;
    uint32_t lim;
    if (in.seg_cnt) {
      const uint64_t v = spread_visit(u, log2_pow2(per_seg));
      const uint32_t sg = (uint32_t)(v / per_seg);
      const uint32_t o = (uint32_t)(v - (uint64_t)sg * per_seg) * kBinTile;
      const uint32_t cnt = in.seg_cnt[sg];
      lim = o >= cnt ? 0u : (cnt - o < (uint32_t)kBinTile ? cnt - o : (uint32_t)kBinTile);
      base = ((uint64_t)sg << in.seg_log2) + o;
    } else {
      base = u * kBinTile;
      lim = (uint32_t)(n_dense - base < (uint64_t)kBinTile ? n_dense - base : kBinTile);
    }
    if (lim == 0) continue;  // uniform across the CTA
    // 1. Load, apply the run, bin, rank within the tile's bin.
    K k[kBinILP];
    AT v[kBinILP];
    int bn[kBinILP];
    unsigned int rk[kBinILP];
#pragma unroll
    for (int q = 0; q < kBinILP; ++q) {
      const uint32_t j = q * blockDim.x + threadIdx.x;
      bn[q] = -1;
      if (j < lim) {
        k[q] = ld_key<KW>(in, base + j);
        v[q] = ((const AT*)in.amp)[base + j];
      }
    }
#pragma unroll
    for (int q = 0; q < kBinILP; ++q) {
      const uint32_t j = q * blockDim.x + threadIdx.x;
      if (j < lim && apply_ops<KW, AT>(ops.n, sm.ops, sm.tab, k[q], v[q])) {
        const uint64_t h = khash(k[q] & ~bmask);
        bn[q] = (int)(((h >> 32) * (uint64_t)B) >> 32);
        rk[q] = atomicAdd(&sm.hist[bn[q]], 1u);
      }
    }
    __syncthreads();
    // 2. Exclusive scan of the histogram (block-wide), global reservation.
    const uint32_t per_t = (B + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = threadIdx.x * per_t;
    uint32_t local = 0;
    for (uint32_t b = b0; b < b0 + per_t && b < B; ++b) local += sm.hist[b];
    uint32_t incl = local;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) sm.scan[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0;
    for (uint32_t w = 0; w < warp; ++w) wpre += sm.scan[w];
    uint32_t run = wpre + incl - local;
    for (uint32_t b = b0; b < b0 + per_t && b < B; ++b) {
      const uint32_t c = sm.hist[b];
      sm.off[b] = run;
      run += c;
      sm.base[b] = c ? atomicAdd(&bins.seg_cnt[b], c) : 0u;
    }
    __syncthreads();
    // 3. Stage the tile sorted by bin.
#pragma unroll
    for (int q = 0; q < kBinILP; ++q) {
      if (bn[q] >= 0) {
        const uint32_t at = sm.off[bn[q]] + rk[q];
        sm.key[at] = k[q];
        sm.amp[at] = v[q];
        sm.bin[at] = (uint16_t)bn[q];
      }
    }
    __syncthreads();
    // 4. Coalesced write-out: consecutive threads, consecutive slots of a run.
    const uint32_t total = sm.off[B - 1] + sm.hist[B - 1];
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
      const uint32_t b = sm.bin[i];
      const uint32_t pos = sm.base[b] + (i - sm.off[b]);
      if (pos < cap) {
        const uint64_t j = ((uint64_t)b << bins.seg_log2) + pos;
        st_key<KW>(bins, j, sm.key[i]);
        ((AT*)bins.amp)[j] = sm.amp[i];
      } else {
        raise_err(ctl, kErrBucket, seq, (unsigned long long)pos + 1);
      }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) sm.hist[b] = 0u;
    __syncthreads();
  }
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// Address of the same shared variable in CTA `rank` of the cluster (generic).
template <class T>
__device__ __forceinline__ T* map_rank(T* p, uint32_t rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"((uint64_t)p), "r"(rank));
  return (T*)out;
}

// Slot tag: (CTA rank << 12 | index) + 1; 0 marks an empty slot.
__device__ __forceinline__ uint32_t ctag(uint32_t r, uint32_t i) { return ((r << kSliceLog2) | i) + 1u; }


template <int KW, class AT>
size_t pair_cluster_smem_bytes_t() {
  typedef typename KT<KW>::T K;
  return 128 + (size_t)kSliceCap * (sizeof(K) + sizeof(AT) + 4) + (size_t)kSlotsPerCta * 4 + 64;
}

template <int KW, class AT>
__global__ void __launch_bounds__(kPairCThreads)
    k_pair_cluster(Ctl* ctl, Gate1 g, Arr bins, Arr out, int out_slot, uint32_t seq,
                   uint32_t wait_limit, int32_t skip_copy_rank) {
  typedef typename KT<KW>::T K;
  extern __shared__ __align__(128) unsigned char smem_pc[];
  uint64_t* bar = (uint64_t*)smem_pc;
  unsigned int* meta = (unsigned int*)(smem_pc + 16);  // [0] fill, [1] n_emit, [2] abort
  K* skey = (K*)(smem_pc + 128);
  AT* samp = (AT*)((unsigned char*)skey + (size_t)kSliceCap * sizeof(K));
  int* partner = (int*)((unsigned char*)samp + (size_t)kSliceCap * sizeof(AT));
  unsigned int* slot = (unsigned int*)((unsigned char*)partner + (size_t)kSliceCap * 4);

  const uint32_t r = cluster_rank();
  const uint32_t b = blockIdx.x / kClusterCtas;
  // Every CTA of the cluster must reach every cluster barrier: an early exit
  // is taken only after the last one.
  const bool dead = ctl->err != 0u;
  const uint32_t n_bin = dead ? 0u : bins.seg_cnt[b];
  const uint32_t lo = r * kSliceCap;
  uint32_t n = n_bin > lo ? (n_bin - lo < (uint32_t)kSliceCap ? n_bin - lo : kSliceCap) : 0u;
  const uint64_t src = ((uint64_t)b << bins.seg_log2) + lo;
  if (threadIdx.x == 0) {
    meta[0] = meta[1] = meta[2] = 0u;
    if (b == 0 && r == 0 && !dead) ctl->cnt[(out_slot + 1) & 3] = 0;
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (uint32_t i = threadIdx.x; i < kSlotsPerCta; i += blockDim.x) slot[i] = 0u;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) partner[i] = -1;
  __syncthreads();
  // Slice r of the bin -> shared memory (both arrays start 16-byte aligned:
  // slices begin at multiples of 4096 branches; sizes round up to 16 bytes
  // inside the bin's capacity).
  const uint32_t limit = wait_limit ? wait_limit : kWaitLimit;
  if (threadIdx.x == 0 && n > 0 && (int32_t)r != skip_copy_rank) {
    const uint32_t kb = (uint32_t)(((size_t)n * 8 + 15) & ~(size_t)15);
    const uint32_t ab = (uint32_t)(((size_t)n * sizeof(AT) + 15) & ~(size_t)15);
    const uint32_t total = kb * (KW == 2 ? 2u : 1u) + ab;
    mbar_expect_tx(bar, total);
    if (KW == 1) {
      bulk_g2s(skey, bins.k0 + src, kb, bar);
    } else {
      // Two-word keys are interleaved in shared memory: stage both words
      // into the partner/slot area first would cost space; load them into
      // skey as two halves and interleave below.
      bulk_g2s(skey, bins.k0 + src, kb, bar);
      bulk_g2s((unsigned char*)skey + (size_t)kSliceCap * 8, bins.k1 + src, kb, bar);
    }
    bulk_g2s(samp, (const AT*)bins.amp + src, ab, bar);
  }
  if (n > 0) {
    uint32_t it = 0;
    while (!mbar_try_wait(bar, 0) && ++it < limit) {
    }
    if (it >= limit && threadIdx.x == 0) {
      raise_err(ctl, kErrProbe, seq, 0);
      atomicOr(&meta[2], 1u);
      // Let the copies land before the CTA leaves (bounded again).
      uint32_t it2 = 0;
      while (!mbar_try_wait(bar, 0) && ++it2 < limit) {
      }
    }
  }
  __syncthreads();
  // A slice whose copies did not arrive in time takes no part: the CTA still
  // reaches every cluster barrier, with nothing to insert or emit (its keys
  // and amplitudes in shared memory are not valid).
  if (meta[2]) n = 0u;
  if (KW == 2 && n > 0) {
    // skey holds low words [0, n) and high words at byte offset 8 * kSliceCap:
    // rebuild 128-bit keys in place from the top down (each slot i reads
    // low[i] and high[i], which live at or above where key i lands only for
    // i >= n / 2; a copy through registers in two passes keeps it safe).
    uint64_t* w = (uint64_t*)skey;
    uint64_t lo_w[kSliceCap / kPairCThreads], hi_w[kSliceCap / kPairCThreads];
#pragma unroll
    for (int q = 0; q < kSliceCap / kPairCThreads; ++q) {
      const uint32_t i = q * blockDim.x + threadIdx.x;
      lo_w[q] = i < n ? w[i] : 0ull;
      hi_w[q] = i < n ? w[kSliceCap + i] : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSliceCap / kPairCThreads; ++q) {
      const uint32_t i = q * blockDim.x + threadIdx.x;
      if (i < n) skey[i] = mk<KW>(lo_w[q], hi_w[q]);
    }
  }
  cluster_sync_all();  // every slot array of the cluster is cleared and loaded

  const K bmask = bit_mask<KW>(g.t);
  const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
  const K cval = mk<KW>(g.cval[0], g.cval[1]);
  constexpr uint32_t kSlotsAll = kSlotsPerCta * kClusterCtas;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const K k = skey[i];
    if ((k & cmask) != cval) continue;  // passes through unchanged
    const K p = k & ~bmask;
    uint32_t h = (uint32_t)khash(p) & (kSlotsAll - 1u);
    const uint32_t me = ctag(r, i);
    uint32_t probe = 0;
    for (; probe < kSlotsAll; ++probe) {
      unsigned int* s = map_rank(slot, h / kSlotsPerCta) + (h % kSlotsPerCta);
      const unsigned int old = atomicCAS(s, 0u, me);
      if (old == 0u) break;
      const uint32_t orank = (old - 1u) >> kSliceLog2, oidx = (old - 1u) & (kSliceCap - 1u);
      const K ok = *map_rank(skey + oidx, orank);
      if ((ok & ~bmask) == p) {
        partner[i] = (int)old;
        *map_rank(partner + oidx, orank) = (int)me;
        break;
      }
      h = (h + 1u) & (kSlotsAll - 1u);
    }
    if (probe == kSlotsAll) raise_err(ctl, kErrProbe, seq, 0);
  }
  cluster_sync_all();  // all pairs linked

  // Emitters first (as in k_pair), then children, then warp-ballot appends
  // into this CTA's output segment.
  unsigned int* emit = slot;  // own slots are no longer read by anyone...
  // ...only after every CTA has finished reading them: the barrier above.
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned int lt = (1u << lane) - 1u;
  const uint32_t rounds_in = (n + blockDim.x - 1u) / blockDim.x;
  __syncthreads();
  for (uint32_t rr = 0; rr < rounds_in; ++rr) {
    const uint32_t i = rr * blockDim.x + threadIdx.x;
    bool e = false;
    if (i < n) {
      const K k = skey[i];
      e = (k & cmask) != cval || !((k & bmask) != (K)0 && partner[i] >= 0);
    }
    const unsigned int ball = __ballot_sync(0xffffffffu, e);
    unsigned int wb = 0;
    if (lane == 0 && ball) wb = atomicAdd(&meta[1], (unsigned int)__popc(ball));
    wb = __shfl_sync(0xffffffffu, wb, 0);
    if (e) emit[wb + __popc(ball & lt)] = i;
  }
  __syncthreads();
  const uint32_t ne = meta[1];
  const uint64_t oseg = (uint64_t)b * kClusterCtas + r;
  const uint64_t obase = oseg << out.seg_log2;
  const uint32_t rounds = (ne + blockDim.x - 1u) / blockDim.x;
  for (uint32_t rr = 0; rr < rounds; ++rr) {
    const uint32_t q = rr * blockDim.x + threadIdx.x;
    bool keep0 = false, keep1 = false;
    K k0 = 0, k1 = 0;
    AT o0, o1;
    if (q < ne) {
      const uint32_t i = emit[q];
      const K k = skey[i];
      const AT ai = samp[i];
      if ((k & cmask) != cval) {
        keep0 = true;
        k0 = k;
        o0 = ai;
      } else {
        const bool kt = (k & bmask) != (K)0;
        const int pj = partner[i];
        k0 = k & ~bmask;
        k1 = k | bmask;
        AT aj = ai;
        if (pj >= 0) {
          const uint32_t orank = ((uint32_t)pj - 1u) >> kSliceLog2;
          const uint32_t oidx = ((uint32_t)pj - 1u) & (kSliceCap - 1u);
          aj = *map_rank(samp + oidx, orank);
        }
        const uint64_t av = g.mode == 1 ? get_field(k0, g.ang_off, g.ang_w) : 0ull;
        if (!kt)
          children<AT>(g, av, true, ai, pj >= 0, aj, o0, o1);
        else
          children<AT>(g, av, false, ai, true, ai, o0, o1);
        keep0 = keep_amp(o0, g.eps, g.epsf, g.eps2);
        keep1 = keep_amp(o1, g.eps, g.epsf, g.eps2);
      }
    }
    const unsigned int b0 = __ballot_sync(0xffffffffu, keep0);
    const unsigned int b1 = __ballot_sync(0xffffffffu, keep1);
    const unsigned int tot = __popc(b0) + __popc(b1);
    unsigned int wbase = 0;
    if (lane == 0 && tot) wbase = atomicAdd(&meta[0], tot);
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (keep0) {
      const uint64_t pos = obase + wbase + __popc(b0 & lt);
      st_key<KW>(out, pos, k0);
      ((AT*)out.amp)[pos] = o0;
    }
    if (keep1) {
      const uint64_t pos = obase + wbase + __popc(b0) + __popc(b1 & lt);
      st_key<KW>(out, pos, k1);
      ((AT*)out.amp)[pos] = o1;
    }
  }
  // Partners read this CTA's keys and amplitudes remotely until every CTA is
  // past its emission: keep the shared memory alive until then.
  cluster_sync_all();
  if (threadIdx.x == 0) {
    const unsigned int fill = meta[0];
    if (!dead) {
      out.seg_cnt[oseg] = fill;
      if (fill) atomicAdd(&ctl->cnt[out_slot], (unsigned long long)fill);
      if (r == 0) bins.seg_cnt[b] = 0u;  // bin counter clean for the next use
    }
  }
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

#define SQS_DISPATCH(kw, amp32, MACRO) \
  do {                                 \
    if (kw == 1) {                     \
      if (amp32) MACRO(1, float2);     \
      else MACRO(1, double2);          \
    } else {                           \
      if (amp32) MACRO(2, float2);     \
      else MACRO(2, double2);          \
    }                                  \
  } while (0)

template <int KW, class AT>
static void apply_inplace_t(const Launch& L, Ctl* ctl, Arr a, int slot, const OpList& ops) {
  const int g = stream_grid(L, kStreamThreads);
  if (ops.touches_keys && ops.touches_amps)
    k_apply_inplace<KW, AT, true, true>
        <<<g, kStreamThreads, 0, L.stream>>>(ctl, a, slot, ops, L.seq);
  else if (ops.touches_keys)
    k_apply_inplace<KW, AT, true, false>
        <<<g, kStreamThreads, 0, L.stream>>>(ctl, a, slot, ops, L.seq);
  else
    k_apply_inplace<KW, AT, false, true>
        <<<g, kStreamThreads, 0, L.stream>>>(ctl, a, slot, ops, L.seq);
}

cudaError_t launch_apply_inplace(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 const OpList& ops) {
#define SQS_AI(KW_, AT_) apply_inplace_t<KW_, AT_>(L, ctl, a, slot, ops)
  SQS_DISPATCH(kw, amp32, SQS_AI);
#undef SQS_AI
  return cudaGetLastError();
}

cudaError_t launch_apply_compact(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                                 int in_slot, Arr out, int out_slot, const OpList& ops) {
  const uint64_t chunks = (L.n_hint + (1ull << out.seg_log2) - 1) >> out.seg_log2;
  uint64_t g = chunks < 1 ? 1 : chunks;
  if (g > (uint64_t)L.sm_count * 8) g = (uint64_t)L.sm_count * 8;
#define SQS_AC(KW_, AT_)                                                              \
  k_apply_compact<KW_, AT_>                                                           \
      <<<(int)g, kStreamThreads, 0, L.stream>>>(ctl, in, in_slot, out, out_slot, ops, \
                                                L.seq)
  SQS_DISPATCH(kw, amp32, SQS_AC);
#undef SQS_AC
  return cudaGetLastError();
}

__global__ void k_angle_table(double2* tab, uint32_t digits, double scale, double offset) {
  const uint64_t n = (uint64_t)digits << 16;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(i >> 16);
    const double d = (double)(i & 0xffffull) * ldexp(1.0, 16 * (int)j);
    const double arg = 0.5 * scale * d + (j == 0 ? 0.5 * offset : 0.0);
    double sn, cs;
    sincos(arg, &sn, &cs);
    tab[i] = make_double2(cs, sn);
  }
}

cudaError_t launch_angle_table(cudaStream_t s, double2* tab, uint32_t digits, double scale,
                               double offset) {
  k_angle_table<<<256, 256, 0, s>>>(tab, digits, scale, offset);
  return cudaGetLastError();
}

// The staged variants: one wave of resident CTAs, each streaming its units.
template <int KW, class AT>
static cudaError_t expand_staged_t(const Launch& L, Ctl* ctl, Arr in, int in_slot,
                                   uint64_t n_chunks, const Gate1& g, Arr out,
                                   int out_slot) {
  const size_t smem = stream_smem_bytes<KW, AT>();
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = ensure_smem_optin((const void*)k_expand_staged<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  static std::atomic<int> per_sm[64];
  int occ = 1;
  e = resident_per_sm(k_expand_staged<KW, AT>, smem, per_sm, occ);
  if (e != cudaSuccess) return e;
  const uint64_t units = n_chunks << kUnitsPerChunkLog2;
  uint64_t grid = (uint64_t)L.sm_count * (uint64_t)occ;
  if (grid > units) grid = units;
  if (grid < 1) grid = 1;
  k_expand_staged<KW, AT><<<(int)grid, kStreamThreads, smem, L.stream>>>(
      ctl, in, in_slot, n_chunks, out, out_slot, g, L.seq);
  return cudaGetLastError();
}

template <int KW, class AT>
static cudaError_t fold_staged_t(const Launch& L, Ctl* ctl, Arr in, int in_slot,
                                 uint64_t n_chunks, const Gate1& g, Arr out,
                                 int out_slot) {
  const size_t smem = fold_staged_smem_bytes<KW, AT>();
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = ensure_smem_optin((const void*)k_fold_staged<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  static std::atomic<int> per_sm[64];
  int occ = 1;
  e = resident_per_sm(k_fold_staged<KW, AT>, smem, per_sm, occ);
  if (e != cudaSuccess) return e;
  const uint64_t units = n_chunks << kUnitsPerChunkLog2;
  uint64_t grid = (uint64_t)L.sm_count * (uint64_t)occ;
  if (grid > units) grid = units;
  if (grid < 1) grid = 1;
  k_fold_staged<KW, AT><<<(int)grid, kStreamThreads, smem, L.stream>>>(
      ctl, in, in_slot, n_chunks, out, out_slot, g, L.seq);
  return cudaGetLastError();
}

cudaError_t launch_expand(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                          uint64_t n_chunks, const OpList& ops, const Gate1& g, Arr out,
                          int out_slot) {
  if (ops.n == 0) {
    if (kw == 1)
      return amp32 ? expand_staged_t<1, float2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot)
                   : expand_staged_t<1, double2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot);
    return amp32 ? expand_staged_t<2, float2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot)
                 : expand_staged_t<2, double2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot);
  }
  uint64_t grid = n_chunks < 1 ? 1 : n_chunks;
  if (grid > (uint64_t)L.sm_count * 8) grid = (uint64_t)L.sm_count * 8;
#define SQS_EX(KW_, AT_)                                                                  \
  k_expand<KW_, AT_><<<(int)grid, kStreamThreads, 0, L.stream>>>(ctl, in, in_slot, n_chunks, \
                                                                 out, out_slot, ops, g, L.seq)
  SQS_DISPATCH(kw, amp32, SQS_EX);
#undef SQS_EX
  return cudaGetLastError();
}

template <int KW, class AT>
static cudaError_t fold_t(const Launch& L, Ctl* ctl, Arr in, int in_slot, uint64_t n_chunks,
                          const OpList& ops, const Gate1& g, Arr out, int out_slot) {
  const size_t smem = fold_smem_bytes<KW, AT>();
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = ensure_smem_optin((const void*)k_fold<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  uint64_t grid = n_chunks < 1 ? 1 : n_chunks;
  if (grid > (uint64_t)L.sm_count * 12) grid = (uint64_t)L.sm_count * 12;
  k_fold<KW, AT><<<(int)grid, kStreamThreads, smem, L.stream>>>(ctl, in, in_slot, n_chunks, out,
                                                                out_slot, ops, g, L.seq);
  return cudaGetLastError();
}

cudaError_t launch_fold(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                        uint64_t n_chunks, const OpList& ops, const Gate1& g, Arr out,
                        int out_slot) {
  if (g.fold_sign == 0 || g.cmask[0] != 0 || g.cmask[1] != 0) return cudaErrorInvalidValue;
  if (ops.n == 0) {
    if (kw == 1)
      return amp32 ? fold_staged_t<1, float2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot)
                   : fold_staged_t<1, double2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot);
    return amp32 ? fold_staged_t<2, float2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot)
                 : fold_staged_t<2, double2>(L, ctl, in, in_slot, n_chunks, g, out, out_slot);
  }
  if (kw == 1)
    return amp32 ? fold_t<1, float2>(L, ctl, in, in_slot, n_chunks, ops, g, out, out_slot)
                 : fold_t<1, double2>(L, ctl, in, in_slot, n_chunks, ops, g, out, out_slot);
  return amp32 ? fold_t<2, float2>(L, ctl, in, in_slot, n_chunks, ops, g, out, out_slot)
               : fold_t<2, double2>(L, ctl, in, in_slot, n_chunks, ops, g, out, out_slot);
}

cudaError_t launch_partition(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                             const OpList& ops, const Gate1& g, Arr bk, uint32_t fill_target) {
  const int grid = stream_grid(L, kStreamThreads);
#define SQS_PT(KW_, AT_)                                                                \
  k_partition<KW_, AT_><<<grid, kStreamThreads, 0, L.stream>>>(ctl, in, in_slot, ops, g, \
                                                               bk, L.seq, fill_target)
  SQS_DISPATCH(kw, amp32, SQS_PT);
#undef SQS_PT
  return cudaGetLastError();
}

int pair_log2_capacity(int kw, bool amp32) {
  (void)kw;
  (void)amp32;
  return 11;  // 2048 branches per bucket
}

size_t pair_smem_bytes(int kw, bool amp32) {
  const size_t C = (size_t)1 << pair_log2_capacity(kw, amp32);
  return C * (kw == 1 ? 8 : 16) + C * (amp32 ? 8 : 16) + 2 * C * 4 + C * 4;
}

template <int KW, class AT>
static cudaError_t pair_t(const Launch& L, Ctl* ctl, const Gate1& g, Arr bk, Arr out,
                          int out_slot) {
  const size_t smem = pair_smem_bytes(KW, sizeof(AT) == 8);
  // The opt-in to more than 48 KB of dynamic shared memory is per device.
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = ensure_smem_optin((const void*)k_pair<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  // One resident wave (the kernel loops over the buckets).
  static std::atomic<int> per_sm[64];
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int occ = dev < 64 ? per_sm[dev].load(std::memory_order_relaxed) : 0;
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair<KW, AT>, kPairThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (dev < 64) per_sm[dev].store(occ, std::memory_order_relaxed);
  }
  uint64_t grid = (uint64_t)L.sm_count * (uint64_t)occ;
  if (grid > bk.n_seg) grid = bk.n_seg;
  if (grid < 1) grid = 1;
  k_pair<KW, AT><<<(int)grid, kPairThreads, smem, L.stream>>>(ctl, g, bk, out, out_slot, L.seq);
  return cudaGetLastError();
}

cudaError_t launch_pair(const Launch& L, int kw, bool amp32, Ctl* ctl, const Gate1& g, Arr bk,
                        Arr out, int out_slot) {
  if (kw == 1)
    return amp32 ? pair_t<1, float2>(L, ctl, g, bk, out, out_slot)
                 : pair_t<1, double2>(L, ctl, g, bk, out, out_slot);
  return amp32 ? pair_t<2, float2>(L, ctl, g, bk, out, out_slot)
               : pair_t<2, double2>(L, ctl, g, bk, out, out_slot);
}

cudaError_t launch_probabilities(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr a, int slot,
                                 uint32_t off, uint32_t w, double* probs, double* nrm) {
  const int g = stream_grid(L, kProbThreads);
#define SQS_PR(KW_, AT_) \
  k_probabilities<KW_, AT_><<<g, kProbThreads, 0, L.stream>>>(ctl, a, slot, off, w, probs, nrm)
  SQS_DISPATCH(kw, amp32, SQS_PR);
#undef SQS_PR
  return cudaGetLastError();
}

cudaError_t launch_densify(const Launch& L, int kw, bool amp32, Arr in, const uint64_t* offsets,
                           Arr out) {
  if (in.n_seg == 0) return cudaSuccess;
#define SQS_DN(KW_, AT_) k_densify<KW_, AT_><<<in.n_seg, 256, 0, L.stream>>>(in, offsets, out)
  SQS_DISPATCH(kw, amp32, SQS_DN);
#undef SQS_DN
  return cudaGetLastError();
}

__global__ void k_record(const Ctl* ctl, int in_slot, int out_slot, unsigned long long* rec) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    rec[0] = ctl->cnt[in_slot];
    rec[1] = ctl->cnt[out_slot];
  }
}

cudaError_t launch_record(const Launch& L, const Ctl* ctl, int in_slot, int out_slot,
                          unsigned long long* rec) {
  k_record<<<1, 32, 0, L.stream>>>(ctl, in_slot, out_slot, rec);
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


// ---- binned merge launchers -------------------------------------------------
int cluster_bin_log2() { return kBinLog2; }
int cluster_ctas() { return kClusterCtas; }
int cluster_out_seg_log2() { return kSliceLog2 + 1; }

template <int KW, class AT>
static cudaError_t bin_t(const Launch& L, Ctl* ctl, Arr in, int in_slot, const OpList& ops,
                         const Gate1& g, Arr bins) {
  const size_t smem = sizeof(BinSmem<KW, AT>);
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = ensure_smem_optin((const void*)k_bin<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  uint64_t tiles = (L.n_hint + kBinTile - 1) / kBinTile;
  if (tiles < 1) tiles = 1;
  const uint64_t cap = (uint64_t)L.sm_count * 2;
  const int grid = (int)(tiles < cap ? tiles : cap);
  k_bin<KW, AT><<<grid, kBinThreads, smem, L.stream>>>(ctl, in, in_slot, ops, g, bins, L.seq);
  return cudaGetLastError();
}

cudaError_t launch_bin(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in, int in_slot,
                       const OpList& ops, const Gate1& g, Arr bins) {
  if (bins.n_seg > (uint32_t)kMaxBins) return cudaErrorInvalidValue;
  if (kw == 1)
    return amp32 ? bin_t<1, float2>(L, ctl, in, in_slot, ops, g, bins)
                 : bin_t<1, double2>(L, ctl, in, in_slot, ops, g, bins);
  return amp32 ? bin_t<2, float2>(L, ctl, in, in_slot, ops, g, bins)
               : bin_t<2, double2>(L, ctl, in, in_slot, ops, g, bins);
}

template <int KW, class AT>
static cudaError_t pair_cluster_t(const Launch& L, Ctl* ctl, const Gate1& g, Arr bins, Arr out,
                                  int out_slot) {
  const size_t smem = pair_cluster_smem_bytes_t<KW, AT>();
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = ensure_smem_optin((const void*)k_pair_cluster<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(bins.n_seg * kClusterCtas);
  cfg.blockDim = dim3(kPairCThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pair_cluster<KW, AT>, ctl, g, bins, out, out_slot, L.seq,
                            L.wait_limit, L.skip_copy_rank);
}

cudaError_t launch_pair_cluster(const Launch& L, int kw, bool amp32, Ctl* ctl, const Gate1& g,
                                Arr bins, Arr out, int out_slot) {
  if (kw == 1)
    return amp32 ? pair_cluster_t<1, float2>(L, ctl, g, bins, out, out_slot)
                 : pair_cluster_t<1, double2>(L, ctl, g, bins, out, out_slot);
  return amp32 ? pair_cluster_t<2, float2>(L, ctl, g, bins, out, out_slot)
               : pair_cluster_t<2, double2>(L, ctl, g, bins, out, out_slot);
}

}  // namespace sqs
