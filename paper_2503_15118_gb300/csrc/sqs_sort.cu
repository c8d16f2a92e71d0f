// The sorting path of the merge (Sec. II.D.2): an interference step on
// target bit t needs the two members of each coherent pair -- branches equal
// on every bit but t -- side by side.  Here they are brought together by a
// least-significant-digit radix sort on the pair-class key (the key with bit
// t deleted), then one streaming pass combines neighbours.
//
// Each radix pass is three kernels: a per-tile digit histogram, an exclusive
// scan of the histogram in digit-major order, and a stable scatter that ranks
// a tile in shared memory (warp-ordered match_any ranking) and writes each
// digit's run contiguously.  The first pass also applies the fused run of
// non-interference operations queued before the step, reading the state
// where it lies (dense or segmented); later passes are dense.  Digits are 8
// bits wide and their windows skip key bits the host knows to be constant
// over the whole state, so a state over few varying qubits sorts in few
// passes.  The digit width is a template parameter (6, 8, 10 or 11 bits):
// wider digits mean fewer passes but larger per-tile histograms and scans; the
// host picks it (autotuned when asked).  Counts are 32-bit: the host routes
// states of 2^32 or more branches to the hash merge.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "sqs_device.cuh"
#include "sqs_internal.h"

namespace sqs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                         // branches per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 branches per tile
constexpr int kRadixBitsDefault = 8;
constexpr int kRadixBitsMax = 11;
constexpr int kScanThreads = 1024;
constexpr int kScanBlocks = 256;
constexpr uint32_t kMergeChunkLog2 = 12;  // input slots per output segment

// The pair-class key: bit t deleted, the bits above it shifted down by one.
template <class K>
__device__ __forceinline__ K drop_bit(K k, uint32_t t) {
  const K low = low_mask_bits<sizeof(K) == 16 ? 2 : 1>(t);
  return (k & low) | ((k >> 1) & ~low);
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// The digit of the sort key: the pair-class key, or (a fused run: cm set)
// the key with the run's targets cleared, whose groups the sort makes
// contiguous.
template <int RB, class K>
__device__ __forceinline__ uint32_t digit_of(K k, uint32_t t, uint32_t shift, K cm) {
  const K c = cm != (K)0 ? (k & ~cm) : drop_bit(k, t);
  return (uint32_t)(c >> shift) & ((1u << RB) - 1u);
}

// Tile `tile` of the input: a slice of one segment, or of the dense array.
// CTAs visit the tiles of segmented inputs in spread order (a permutation of
// the tiles of each segment); every tile keeps its index, so the scan over
// tile indices still ranks the input in storage order.
__device__ __forceinline__ uint64_t tile_visit(const Arr& in, uint64_t u, uint32_t per_seg) {
  return in.seg_cnt ? spread_visit(u, log2_pow2(per_seg)) : u;
}

__device__ __forceinline__ void tile_range(const Arr& in, uint64_t n_dense, uint64_t tile,
                                           uint32_t per_seg, uint64_t& base, uint32_t& lim) {
  if (in.seg_cnt) {
    const uint64_t sg = tile / per_seg;
    const uint32_t off = (uint32_t)(tile - sg * per_seg) * (uint32_t)kSortTile;
    const uint32_t cnt = sg < in.n_seg ? in.seg_cnt[sg] : 0u;
    base = (sg << in.seg_log2) + off;
    lim = cnt > off ? umin32(cnt - off, (uint32_t)kSortTile) : 0u;
  } else {
    base = tile * (uint64_t)kSortTile;
    lim = base < n_dense ? (uint32_t)umin64(n_dense - base, (uint64_t)kSortTile) : 0u;
  }
}

// Digit counts of every tile: hist[d * n_tiles + tile].
template <int KW, class AT, bool FIRST, int RB>
__global__ void __launch_bounds__(kSortThreads)
    k_rsort_hist(Ctl* ctl, Arr in, const unsigned long long* n_ptr, uint32_t per_seg,
                 const __grid_constant__ OpList ops, uint32_t t, uint32_t shift,
                 uint64_t n_tiles, unsigned int* hist, uint64_t cm0, uint64_t cm1) {
  typedef typename KT<KW>::T K;
  constexpr uint32_t R = 1u << RB;
  const K cm = mk<KW>(cm0, cm1);
  __shared__ AT tab[FIRST ? kTabEntries : 1];
  __shared__ DevOp sops[FIRST ? kMaxOps : 1];
  __shared__ unsigned int h[R];
  if (ctl->err) return;
  if (FIRST) {
    load_ops(ops, sops, tab);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ctl->peak, *n_ptr);
  }
  const uint64_t n_dense = in.seg_cnt ? 0ull : *n_ptr;
  if (n_dense > n_tiles * (uint64_t)kSortTile) {  // tiles sized from a bound the state outgrew
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->err, kErrCapacity);
    return;
  }
  for (uint64_t u = blockIdx.x; u < n_tiles; u += gridDim.x) {
    const uint64_t tile = tile_visit(in, u, per_seg);
    for (uint32_t d = threadIdx.x; d < R; d += blockDim.x) h[d] = 0u;
    uint64_t base;
    uint32_t lim;
    tile_range(in, n_dense, tile, per_seg, base, lim);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < lim; j += blockDim.x) {
      K k = ld_key<KW>(in, base + j);
      bool live = true;
      if (FIRST && ops.n) {
        AT a;
        if (ops.drops)
          a = ((const AT*)in.amp)[base + j];
        else
          a.x = a.y = 0;  // only pruning reads the amplitude
        live = apply_ops<KW, AT>(ops.n, sops, tab, k, a);
      }
      if (live) atomicAdd(&h[digit_of<RB>(k, t, shift, cm)], 1u);
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < R; d += blockDim.x) hist[(uint64_t)d * n_tiles + tile] = h[d];
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned int block_sum(unsigned int v, unsigned int* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const unsigned int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31u) == 0) red[w] = v;
  __syncthreads();
  unsigned int s = 0;
  for (unsigned int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Sum of each of gridDim.x consecutive ranges of `chunk` entries.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_reduce(const Ctl* ctl, const unsigned int* x, uint64_t m, uint64_t chunk,
                  unsigned int* part) {
  __shared__ unsigned int red[kScanThreads / 32];
  if (ctl->err) return;
  const uint64_t lo = blockIdx.x * chunk, hi = umin64(m, lo + chunk);
  unsigned int s = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Exclusive scan in place; the last block stores the grand total.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_apply(const Ctl* ctl, unsigned int* x, uint64_t m, uint64_t chunk,
                 const unsigned int* part, unsigned long long* total) {
  __shared__ unsigned int red[kScanThreads / 32];
  __shared__ unsigned int carry;
  if (ctl->err) return;
  unsigned int p = 0;
  for (unsigned int i = threadIdx.x; i < blockIdx.x; i += blockDim.x) p += part[i];
  p = block_sum(p, red);
  if (threadIdx.x == 0) carry = p;
  __syncthreads();
  const uint64_t lo = blockIdx.x * chunk, hi = umin64(m, lo + chunk);
  const unsigned int lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  for (uint64_t b = lo; b < hi; b += blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const unsigned int v = i < hi ? x[i] : 0u;
    unsigned int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned int)o) incl += y;
    }
    if (lane == 31u) red[w] = incl;
    __syncthreads();
    if (w == 0) {
      unsigned int s = lane < (kScanThreads / 32) ? red[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= (unsigned int)o) s += y;
      }
      if (lane < (kScanThreads / 32)) red[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const unsigned int before = (w ? red[w - 1] : 0u) + incl - v;
    if (i < hi) x[i] = carry + before;
    const unsigned int round = red[kScanThreads / 32 - 1];
    __syncthreads();
    if (threadIdx.x == 0) carry += round;
    __syncthreads();
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = carry;
}

// Stable scatter of one radix pass.  Warp w ranks tile items
// [w * 256, (w + 1) * 256) in order, 32 per round; ranks across warps and
// digits come from shared-memory scans; the tile is then laid out in sorted
// order in shared memory and written digit run by digit run.
template <int KW, class AT, bool FIRST, int RB>
__global__ void __launch_bounds__(kSortThreads)
    k_rsort_scatter(Ctl* ctl, Arr in, const unsigned long long* n_ptr, uint32_t per_seg,
                    const __grid_constant__ OpList ops, uint32_t t, uint32_t shift,
                    uint64_t n_tiles, const unsigned int* offs, Arr out, uint64_t cm0,
                    uint64_t cm1) {
  typedef typename KT<KW>::T K;
  constexpr uint32_t R = 1u << RB;
  // Digits each thread scans: one when R <= 256 (threads past R hold none).
  constexpr uint32_t kDpt = R > (uint32_t)kSortThreads ? R / (uint32_t)kSortThreads : 1u;
  const K cm = mk<KW>(cm0, cm1);
  extern __shared__ __align__(16) unsigned char smem[];
  K* skey = (K*)smem;
  AT* samp = (AT*)(smem + (size_t)kSortTile * sizeof(K));
  unsigned int* whist = (unsigned int*)(samp + kSortTile);  // [kSortWarps][R]
  unsigned int* tbase = whist + kSortWarps * R;
  unsigned int* gofs = tbase + R;
  uint16_t* sdig = (uint16_t*)(gofs + R);
  __shared__ AT tab[FIRST ? kTabEntries : 1];
  __shared__ DevOp sops[FIRST ? kMaxOps : 1];
  __shared__ unsigned int wsum[kSortWarps];
  __shared__ unsigned int tile_live;
  if (ctl->err) return;
  if (FIRST) load_ops(ops, sops, tab);
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  const uint64_t n_dense = in.seg_cnt ? 0ull : *n_ptr;
  for (uint64_t u = blockIdx.x; u < n_tiles; u += gridDim.x) {
    const uint64_t tile = tile_visit(in, u, per_seg);
    for (uint32_t i = threadIdx.x; i < kSortWarps * R; i += blockDim.x) whist[i] = 0u;
    uint64_t base;
    uint32_t lim;
    tile_range(in, n_dense, tile, per_seg, base, lim);
    __syncthreads();
    K k[kSortItems];
    AT a[kSortItems];
    uint32_t d[kSortItems], rk[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t j = warp * (32u * kSortItems) + (uint32_t)r * 32u + lane;
      bool live = j < lim;
      if (live) {
        k[r] = ld_key<KW>(in, base + j);
        a[r] = ((const AT*)in.amp)[base + j];
        if (FIRST) live = apply_ops<KW, AT>(ops.n, sops, tab, k[r], a[r]);
      }
      // Dead lanes get a value no live lane has, so they match only themselves.
      d[r] = live ? digit_of<RB>(k[r], t, shift, cm) : R + lane;
      const unsigned int peers = __match_any_sync(0xffffffffu, d[r]);
      unsigned int before = 0u;
      if (live) before = whist[warp * R + d[r]];
      __syncwarp();
      if (live && (peers & lt) == 0u) whist[warp * R + d[r]] = before + (unsigned int)__popc(peers);
      __syncwarp();
      rk[r] = before + (unsigned int)__popc(peers & lt);
    }
    __syncthreads();
    // Per digit (each thread kDpt consecutive digits): exclusive scan over
    // warps, then an exclusive scan of the digit totals across the block.
    {
      const uint32_t d0 = threadIdx.x * kDpt;
      unsigned int dtot[kDpt];
      unsigned int mine = 0u;
#pragma unroll
      for (uint32_t j = 0; j < kDpt; ++j) {
        const uint32_t dg = d0 + j;
        unsigned int run = 0u;
        if (dg < R) {
          for (int w = 0; w < kSortWarps; ++w) {
            const unsigned int c = whist[w * R + dg];
            whist[w * R + dg] = run;
            run += c;
          }
          gofs[dg] = offs[(uint64_t)dg * n_tiles + tile];
        }
        dtot[j] = run;
        mine += run;
      }
      unsigned int incl = mine;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned int)o) incl += y;
      }
      if (lane == 31u) wsum[warp] = incl;
      __syncthreads();
      unsigned int wb = 0u;
      for (unsigned int w = 0; w < warp; ++w) wb += wsum[w];
      unsigned int pre = wb + incl - mine;
#pragma unroll
      for (uint32_t j = 0; j < kDpt; ++j) {
        if (d0 + j < R) tbase[d0 + j] = pre;
        pre += dtot[j];
      }
      if (threadIdx.x == blockDim.x - 1u) tile_live = wb + incl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      if (d[r] < R) {
        const uint32_t lp = tbase[d[r]] + whist[warp * R + d[r]] + rk[r];
        skey[lp] = k[r];
        samp[lp] = a[r];
        sdig[lp] = (uint16_t)d[r];
      }
    }
    __syncthreads();
    const uint32_t nl = tile_live;
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) {
      const uint32_t dg = sdig[i];
      const uint64_t pos = (uint64_t)gofs[dg] + (i - tbase[dg]);
      st_key<KW>(out, pos, skey[i]);
      ((AT*)out.amp)[pos] = samp[i];
    }
    __syncthreads();
  }
}

// The merge over the sorted array: the first member of each pair class
// computes both children (Eq. of the 2x2 step, Sec. II.D.2) from itself and
// its neighbour when the neighbour shares the class; chunk c of 2^12 sorted
// branches becomes output segment c (2^13 slots).
template <int KW, class AT>
__global__ void __launch_bounds__(kStreamThreads)
    k_rsort_merge(Ctl* ctl, Arr in, const unsigned long long* n_ptr, Gate1 g, Arr out,
                  int out_slot) {
  typedef typename KT<KW>::T K;
  __shared__ unsigned int seg_fill;
  if (ctl->err) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[(out_slot + 1) & 3] = 0;
  const uint64_t n = *n_ptr;
  const uint64_t chunk = 1ull << kMergeChunkLog2;
  const K bmask = bit_mask<KW>(g.t);
  const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
  const K cval = mk<KW>(g.cval[0], g.cval[1]);
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int lt = (1u << lane) - 1u;
  for (uint64_t c = blockIdx.x; c < out.n_seg; c += gridDim.x) {
    if (threadIdx.x == 0) seg_fill = 0;
    __syncthreads();
    const uint64_t ibase = c << kMergeChunkLog2;
    const uint64_t cnt = ibase < n ? umin64(n - ibase, chunk) : 0ull;
    const uint64_t obase = c << out.seg_log2;
    for (uint64_t r = 0; r < cnt; r += blockDim.x) {
      bool keep0 = false, keep1 = false;
      K k0 = 0, k1 = 0;
      AT o0, o1;
      if (r + threadIdx.x < cnt) {
        const uint64_t i = ibase + r + threadIdx.x;
        const K k = ld_key<KW>(in, i);
        const AT ai = ((const AT*)in.amp)[i];
        if ((k & cmask) != cval) {
          keep0 = true;  // controls not met: the branch is unchanged
          k0 = k;
          o0 = ai;
        } else {
          const K p = k & ~bmask;
          const bool lead = i == 0 || (ld_key<KW>(in, i - 1) & ~bmask) != p;
          if (lead) {
            const bool has_p = i + 1 < n && (ld_key<KW>(in, i + 1) & ~bmask) == p;
            const bool kt = (k & bmask) != (K)0;
            k0 = p;
            k1 = p | bmask;
            const uint64_t av = g.mode == 1 ? get_field(k0, g.ang_off, g.ang_w) : 0ull;
            if (has_p) {
              const AT ap = ((const AT*)in.amp)[i + 1];
              if (!kt)
                children<AT>(g, av, true, ai, true, ap, o0, o1);
              else
                children<AT>(g, av, true, ap, true, ai, o0, o1);
            } else if (!kt) {
              children<AT>(g, av, true, ai, false, ai, o0, o1);
            } else {
              children<AT>(g, av, false, ai, true, ai, o0, o1);
            }
            keep0 = keep_amp(o0, g.eps, g.epsf, g.eps2);
            keep1 = keep_amp(o1, g.eps, g.epsf, g.eps2);
          }
        }
      }
      const unsigned int b0 = __ballot_sync(0xffffffffu, keep0);
      const unsigned int b1 = __ballot_sync(0xffffffffu, keep1);
      const unsigned int tot = __popc(b0) + __popc(b1);
      unsigned int wbase = 0;
      if (lane == 0 && tot) wbase = atomicAdd(&seg_fill, tot);
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
      out.seg_cnt[c] = seg_fill;
      if (seg_fill) atomicAdd(&ctl->cnt[out_slot], (unsigned long long)seg_fill);
    }
  }
}

template <int KW, class AT, int RB>
size_t scatter_smem() {
  return (size_t)kSortTile * (sizeof(typename KT<KW>::T) + sizeof(AT) + 2) +
         (size_t)4 * ((size_t)kSortWarps + 2) * ((size_t)1 << RB);
}

template <int KW, class AT, bool FIRST, int RB>
cudaError_t pass_t(const Launch& L, Ctl* ctl, Arr in, const unsigned long long* n_ptr,
                   uint32_t per_seg, uint64_t n_tiles, const OpList& ops, uint32_t t,
                   uint32_t shift, unsigned int* hist, unsigned int* part,
                   unsigned long long* n_dev, Arr out, const uint64_t* cm) {
  const uint64_t cm0 = cm ? cm[0] : 0ull, cm1 = cm ? cm[1] : 0ull;
  const int grid = (int)std::min<uint64_t>(n_tiles, (uint64_t)L.sm_count * 8);
  k_rsort_hist<KW, AT, FIRST, RB><<<grid, kSortThreads, 0, L.stream>>>(
      ctl, in, n_ptr, per_seg, ops, t, shift, n_tiles, hist, cm0, cm1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint64_t m = n_tiles << RB;
  const uint64_t blocks = std::min<uint64_t>(kScanBlocks, (m + 4095) / 4096);
  const uint64_t chunk = (m + blocks - 1) / blocks;
  k_scan_reduce<<<(int)blocks, kScanThreads, 0, L.stream>>>(ctl, hist, m, chunk, part);
  k_scan_apply<<<(int)blocks, kScanThreads, 0, L.stream>>>(ctl, hist, m, chunk, part, n_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = scatter_smem<KW, AT, RB>();
  static std::atomic<unsigned long long> configured{0};  // opt-in above 48 KB, per device
  e = ensure_smem_optin((const void*)k_rsort_scatter<KW, AT, FIRST, RB>, smem, configured);
  if (e != cudaSuccess) return e;
  const int sgrid = (int)std::min<uint64_t>(n_tiles, (uint64_t)L.sm_count * 4);
  k_rsort_scatter<KW, AT, FIRST, RB><<<sgrid, kSortThreads, smem, L.stream>>>(
      ctl, in, n_ptr, per_seg, ops, t, shift, n_tiles, hist, out, cm0, cm1);
  return cudaGetLastError();
}

}  // namespace

int sort_tile() { return kSortTile; }
int sort_radix_bits() { return kRadixBitsDefault; }
int sort_radix_bits_max() { return kRadixBitsMax; }
bool sort_radix_bits_ok(int rb) { return rb == 6 || rb == 8 || rb == 10 || rb == 11; }
uint32_t sort_merge_chunk_log2() { return kMergeChunkLog2; }
size_t sort_part_entries() { return kScanBlocks; }

#define SQS_SORT_DISPATCH(kw, amp32, M) \
  ((kw) == 1 ? ((amp32) ? M(1, float2) : M(1, double2)) : ((amp32) ? M(2, float2) : M(2, double2)))

template <int RB>
static cudaError_t pass_rb(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                           const unsigned long long* n_ptr, uint32_t per_seg, uint64_t n_tiles,
                           const OpList* first_ops, uint32_t t, uint32_t shift, unsigned int* hist,
                           unsigned int* part, unsigned long long* n_dev, Arr out,
                           const uint64_t* clear_mask) {
  if (first_ops) {
#define SQS_P1(KW_, AT_)                                                                  \
  pass_t<KW_, AT_, true, RB>(L, ctl, in, n_ptr, per_seg, n_tiles, *first_ops, t, shift, hist, \
                             part, n_dev, out, clear_mask)
    return SQS_SORT_DISPATCH(kw, amp32, SQS_P1);
#undef SQS_P1
  }
  static const OpList kNone = [] {
    OpList o;
    std::memset(&o, 0, sizeof(o));
    return o;
  }();
#define SQS_P2(KW_, AT_)                                                                 \
  pass_t<KW_, AT_, false, RB>(L, ctl, in, n_ptr, per_seg, n_tiles, kNone, t, shift, hist, \
                              part, n_dev, out, clear_mask)
  return SQS_SORT_DISPATCH(kw, amp32, SQS_P2);
#undef SQS_P2
}

cudaError_t launch_rsort_pass(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                              const unsigned long long* n_ptr, uint32_t per_seg,
                              uint64_t n_tiles, const OpList* first_ops, uint32_t t,
                              uint32_t shift, unsigned int* hist, unsigned int* part,
                              unsigned long long* n_dev, Arr out, const uint64_t* clear_mask,
                              int radix_bits) {
  if (n_tiles == 0) return cudaSuccess;
  switch (radix_bits) {
    case 6:
      return pass_rb<6>(L, kw, amp32, ctl, in, n_ptr, per_seg, n_tiles, first_ops, t, shift, hist,
                        part, n_dev, out, clear_mask);
    case 8:
      return pass_rb<8>(L, kw, amp32, ctl, in, n_ptr, per_seg, n_tiles, first_ops, t, shift, hist,
                        part, n_dev, out, clear_mask);
    case 10:
      return pass_rb<10>(L, kw, amp32, ctl, in, n_ptr, per_seg, n_tiles, first_ops, t, shift,
                         hist, part, n_dev, out, clear_mask);
    case 11:
      return pass_rb<11>(L, kw, amp32, ctl, in, n_ptr, per_seg, n_tiles, first_ops, t, shift,
                         hist, part, n_dev, out, clear_mask);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rsort_merge(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                               const unsigned long long* n_ptr, const Gate1& g, Arr out,
                               int out_slot) {
  uint64_t grid = out.n_seg < 1 ? 1 : out.n_seg;
  if (grid > (uint64_t)L.sm_count * 8) grid = (uint64_t)L.sm_count * 8;
#define SQS_M(KW_, AT_)                                                                  \
  (k_rsort_merge<KW_, AT_><<<(int)grid, kStreamThreads, 0, L.stream>>>(ctl, in, n_ptr, g, \
                                                                       out, out_slot),   \
   cudaGetLastError())
  return SQS_SORT_DISPATCH(kw, amp32, SQS_M);
#undef SQS_M
}

}  // namespace sqs
