// Fused runs of interference operations (Sec. II.D.2).  Branches that agree
// on every idle bit -- every key bit but the run's targets -- form a coherent
// group, and a run of k interference operations on distinct targets acts on
// each group independently: a group holds at most 2^k branches, indexed by
// the values of its target bits.  As in the paper, the branches are first
// sorted on their idle bits (the radix-sort passes with the targets cleared
// from the sort key), which makes every group a contiguous range; the
// operation is then applied to each group at its full dimension.  Here each
// group becomes a dense vector of 2^k amplitudes with a presence flag per
// entry, in shared memory, and the k operations are applied to it one after
// another, operation j pairing entries that differ in index bit j.  Each
// step evaluates the same 2x2 (children()) with the same presence flags and
// the same pruning test as a single merge step, so the run's result equals
// the result of the k steps applied one by one, bit for bit; what is saved
// is k - 1 sorts or partitions and k - 1 passes over the state in memory.
//
// k_group_count counts the groups (a group starts where the idle bits
// differ from the previous branch's); the host sizes the output from it (at
// most 2^k branches per group) and picks the tile length.  k_group gives
// each CTA the groups that start in its tile; the last of them may extend
// past the tile, by fewer than 2^k branches.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sqs_device.cuh"
#include "sqs_internal.h"

namespace sqs {
namespace {

constexpr int kGroupThreads = 512;
constexpr uint32_t kNoGroup = 0xffffu;

// Dense area: 2^12 amplitudes (plus one presence byte each), so that a group
// of 2^k entries, k <= kMaxRun = 12, always fits, and two CTAs share an SM.
template <class AT>
struct DenseArea {
  static constexpr uint32_t n = 1u << 12;
};

// Index of a branch inside its group: bit j = key bit g[j].t.
template <int KW>
__device__ __forceinline__ uint32_t group_index(const GroupRun& run, typename KT<KW>::T k) {
  uint32_t x = 0;
  for (uint32_t j = 0; j < run.k; ++j)
    if ((k & bit_mask<KW>(run.g[j].t)) != (typename KT<KW>::T)0) x |= 1u << j;
  return x;
}

template <int KW>
__device__ __forceinline__ typename KT<KW>::T group_key(const GroupRun& run,
                                                        typename KT<KW>::T rest, uint32_t x) {
  for (uint32_t j = 0; j < run.k; ++j)
    if ((x >> j) & 1u) rest |= bit_mask<KW>(run.g[j].t);
  return rest;
}

// One step's 2x2 on a pair of a group (children(), the merge's form).
// FP64 storage with a real U: a warp whose lanes mix pairs with both members
// and pairs with one would issue both FP64 sequences, one after the other.
// Instead, when any lane of the warp holds both members, every lane takes
// the two-member form with an absent member read as zero -- fma(u, 0, p) = p
// and fma(u, a, +-0) = round(u a) give children()'s one-member results
// exactly, up to the sign of an exact zero -- and otherwise every lane takes
// the one-member products of the member it holds.  Called by every lane of
// the warp (the vote).
template <class AT>
__device__ __forceinline__ void step_pair(const Gate1& g, uint64_t av, bool act, bool h0, AT a0,
                                          bool h1, AT a1, AT& o0, AT& o1) {
  if (act) children<AT>(g, av, h0, a0, h1, a1, o0, o1);
}
template <>
__device__ __forceinline__ void step_pair<double2>(const Gate1& g, uint64_t av, bool act, bool h0,
                                                   double2 a0, bool h1, double2 a1, double2& o0,
                                                   double2& o1) {
  if (g.mode != 2) {
    if (act) children<double2>(g, av, h0, a0, h1, a1, o0, o1);
    return;
  }
  const bool both = __any_sync(0xffffffffu, act && h0 && h1);
  if (!act) return;
  const double u00 = g.u[0], u01 = g.u[2], u10 = g.u[4], u11 = g.u[6];
  if (both) {
    if (!h0) a0 = make_double2(0.0, 0.0);
    if (!h1) a1 = make_double2(0.0, 0.0);
    const double2 p01 = rmul(u01, a1);
    o0 = rfma(u00, a0, p01);
    if (g.reuse & 2u)
      o1 = (g.reuse & 8u) ? rfms(u10, a0, p01) : rfma(u10, a0, p01);
    else
      o1 = rfma(u10, a0, rmul(u11, a1));
  } else {
    const double2 a = h0 ? a0 : a1;
    const bool same = h0 ? (g.reuse & 1u) != 0 : (g.reuse & 2u) != 0;
    const bool neg = h0 ? (g.reuse & 4u) != 0 : (g.reuse & 8u) != 0;
    o0 = rmul(h0 ? u00 : u01, a);
    o1 = same ? (neg ? cneg(o0) : o0) : rmul(h0 ? u10 : u11, a);
  }
}

template <int KW>
__device__ __forceinline__ bool starts_group(const Arr& in, uint64_t i, typename KT<KW>::T cm) {
  return i == 0 || (ld_key<KW>(in, i) & ~cm) != (ld_key<KW>(in, i - 1) & ~cm);
}

template <int KW>
__global__ void __launch_bounds__(kStreamThreads)
    k_group_count(Ctl* ctl, Arr in, const unsigned long long* n_ptr, uint64_t tm0, uint64_t tm1) {
  typedef typename KT<KW>::T K;
  __shared__ unsigned int red;
  if (ctl->err) return;
  const uint64_t n = *n_ptr;
  const K cm = mk<KW>(tm0, tm1);
  if (threadIdx.x == 0) red = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->items = n;
  __syncthreads();
  unsigned int c = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    c += starts_group<KW>(in, i, cm);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31u) == 0 && c) atomicAdd(&red, c);
  __syncthreads();
  if (threadIdx.x == 0 && red) atomicAdd(&ctl->groups, (unsigned long long)red);
}

// Shared memory of one k_group CTA:
//   dense    DenseArea amplitudes, then one presence byte each
//   skey     the tile's keys (kGroupTile)
//   gidx     u16 per tile branch: its group among the CTA's (kNoGroup: the
//            branch continues a group of an earlier tile)
//   gstart   u16 per group: first branch (tile index); one more entry for
//            the end of the last group, which may lie past the tile
template <int KW, class AT>
struct GroupSmem {
  typedef typename KT<KW>::T K;
  static constexpr size_t pres_off = (size_t)DenseArea<AT>::n * sizeof(AT);
  static constexpr size_t skey_off = pres_off + DenseArea<AT>::n;
  static constexpr size_t gidx_off = skey_off + (size_t)kGroupTile * sizeof(K);
  static constexpr size_t gstart_off = gidx_off + (size_t)kGroupTile * 2;
  static constexpr size_t bytes = gstart_off + (size_t)(kGroupTile + 8) * 2;
  static_assert(bytes <= 112u * 1024u, "two CTAs per SM");
};

template <int KW, class AT>
__global__ void __launch_bounds__(kGroupThreads, 2)
    k_group(Ctl* ctl, Arr in, const unsigned long long* n_ptr, uint32_t tile_len, Arr out,
            int out_slot, const __grid_constant__ GroupRun run, uint32_t seq) {
  typedef typename KT<KW>::T K;
  typedef GroupSmem<KW, AT> L;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int warp_sums[kGroupThreads / 32];
  __shared__ unsigned int n_groups, stage_sum, last_end;
  __shared__ unsigned long long round_base;
  if (ctl->err) return;
  AT* dense = (AT*)smem;
  unsigned char* pres = smem + L::pres_off;
  K* skey = (K*)(smem + L::skey_off);
  uint16_t* gidx = (uint16_t*)(smem + L::gidx_off);
  uint16_t* gstart = (uint16_t*)(smem + L::gstart_off);

  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[(out_slot + 1) & 3] = 0;
  const uint64_t n = *n_ptr;
  const K cm = mk<KW>(run.tmask[0], run.tmask[1]);
  const uint32_t kk = run.k;
  const uint32_t gsize = 1u << kk, half = gsize >> 1;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  const uint32_t per_batch = DenseArea<AT>::n >> kk;

  for (uint64_t c = blockIdx.x; c * tile_len < n; c += gridDim.x) {
    const uint64_t t0 = c * tile_len;
    const uint32_t m = (uint32_t)(n - t0 < tile_len ? n - t0 : tile_len);
    // 1. The tile's keys and group starts; gidx by a block scan of the
    //    start flags (4 consecutive branches per thread).
    unsigned int f[4], cnt = 0;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t i = threadIdx.x * 4u + q;
      f[q] = 0;
      if (i < m) {
        const K k = ld_key<KW>(in, t0 + i);
        skey[i] = k;
        f[q] = (t0 + i == 0 || (k & ~cm) != (ld_key<KW>(in, t0 + i - 1) & ~cm)) ? 1u : 0u;
      }
      cnt += f[q];
    }
    unsigned int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned int w = lane < kGroupThreads / 32 ? warp_sums[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= (uint32_t)o) w += y;
      }
      if (lane < kGroupThreads / 32) warp_sums[lane] = w;
      if (lane == kGroupThreads / 32 - 1) n_groups = w;
    }
    __syncthreads();
    unsigned int before = (warp ? warp_sums[warp - 1] : 0u) + incl - cnt;  // starts before mine
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t i = threadIdx.x * 4u + q;
      if (i < m) {
        if (f[q]) gstart[before] = (uint16_t)i;
        before += f[q];
        gidx[i] = before ? (uint16_t)(before - 1u) : (uint16_t)kNoGroup;
      }
    }
    __syncthreads();
    const uint32_t G = n_groups;
    // 2. The end of the last group, which may lie past the tile (by fewer
    //    than 2^k branches: keys are distinct within a group).
    if (G && warp == 0) {
      const K rest = skey[gstart[G - 1]] & ~cm;
      uint64_t end = t0 + m;
      const uint64_t lim = t0 + gstart[G - 1] + gsize < n ? t0 + gstart[G - 1] + gsize : n;
      for (uint64_t p = end; p < lim; p += 32) {
        const uint64_t q = p + lane;
        const bool same = q < lim && (ld_key<KW>(in, q) & ~cm) == rest;
        const unsigned int ball = __ballot_sync(0xffffffffu, same);
        if (ball != 0xffffffffu) {
          end = p + (uint64_t)__ffs(~ball) - 1u;
          break;
        }
        end = p + 32 < lim ? p + 32 : lim;
      }
      if (lane == 0) last_end = (uint32_t)(end - t0);
    }
    __syncthreads();
    if (G == 0) continue;  // the tile lies inside a group of an earlier tile
    if (threadIdx.x == 0) gstart[G] = (uint16_t)last_end;  // < 2048 + 4096
    __syncthreads();

    // 3. Batches of whole groups in the dense area.
    for (uint32_t g0 = 0; g0 < G; g0 += per_batch) {
      const uint32_t gn = G - g0 < per_batch ? G - g0 : per_batch;
      const uint32_t nslots = gn << kk;
      for (uint32_t s = threadIdx.x; s < nslots; s += blockDim.x) pres[s] = 0;
      __syncthreads();
      for (uint32_t i = gstart[g0] + threadIdx.x; i < gstart[g0 + gn]; i += blockDim.x) {
        const uint32_t grp = i < m ? (uint32_t)gidx[i] : G - 1u;
        const K k = i < m ? skey[i] : ld_key<KW>(in, t0 + i);
        const uint32_t s = ((grp - g0) << kk) | group_index<KW>(run, k);
        dense[s] = ((const AT*)in.amp)[t0 + i];
        pres[s] = 1;
      }
      __syncthreads();
      for (uint32_t j = 0; j < kk; ++j) {
        const Gate1& g = run.g[j];
        const K cmask = mk<KW>(g.cmask[0], g.cmask[1]);
        const K cval = mk<KW>(g.cval[0], g.cval[1]);
        const uint32_t low = (1u << j) - 1u;
        unsigned int live = 0;
        if (threadIdx.x == 0) stage_sum = 0;
        // Warp-uniform trip count: step_pair() votes across the warp.
        const uint32_t npairs = nslots >> 1;
        for (uint32_t p0 = 0; p0 < npairs; p0 += blockDim.x) {
          const uint32_t p = p0 + threadIdx.x;
          bool h0 = false, h1 = false, act = false;
          uint32_t s0 = 0, s1 = 0;
          K rest = 0;
          if (p < npairs) {
            const uint32_t grp = p >> (kk - 1u);
            const uint32_t r = p & (half - 1u);
            s0 = (grp << kk) | ((r & ~low) << 1) | (r & low);
            s1 = s0 | (1u << j);
            h0 = pres[s0] != 0;
            h1 = pres[s1] != 0;
            if (h0 || h1) {
              rest = skey[gstart[g0 + grp]] & ~cm;
              if ((rest & cmask) != cval)  // controls not met: the group is unchanged
                live += (unsigned int)h0 + (unsigned int)h1;
              else
                act = true;
            }
          }
          AT a0, a1, o0, o1;
          a0.x = a0.y = a1.x = a1.y = 0;
          if (act) {
            a0 = dense[s0];
            a1 = dense[s1];
            if (!h0) a0 = a1;  // unread for an absent member; keeps the operands defined
            if (!h1) a1 = a0;
          }
          const uint64_t av = act && g.mode == 1 ? get_field(rest, g.ang_off, g.ang_w) : 0ull;
          step_pair<AT>(g, av, act, h0, a0, h1, a1, o0, o1);
          if (act) {
            const bool k0 = keep_amp(o0, g.eps, g.epsf, g.eps2);
            const bool k1 = keep_amp(o1, g.eps, g.epsf, g.eps2);
            dense[s0] = o0;
            dense[s1] = o1;
            pres[s0] = k0;
            pres[s1] = k1;
            live += (unsigned int)k0 + (unsigned int)k1;
          }
        }
        for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
        __syncthreads();  // stage_sum reset and every pair of this step done
        if (lane == 0 && live) atomicAdd(&stage_sum, live);
        __syncthreads();
        if (threadIdx.x == 0 && stage_sum)
          atomicAdd(&ctl->stage[j], (unsigned long long)stage_sum);
      }
      // 4. Survivors to the dense output; one reservation per round.
      for (uint32_t r0 = 0; r0 < nslots; r0 += blockDim.x) {
        const uint32_t s = r0 + threadIdx.x;
        const bool keep = s < nslots && pres[s] != 0;
        const unsigned int ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_sums[warp] = __popc(ball);
        __syncthreads();
        if (threadIdx.x == 0) {
          unsigned int sum = 0;
          for (uint32_t w = 0; w < blockDim.x / 32u; ++w) {
            const unsigned int t = warp_sums[w];
            warp_sums[w] = sum;
            sum += t;
          }
          round_base = sum ? atomicAdd(&ctl->cnt[out_slot], (unsigned long long)sum) : 0ull;
          if (sum && round_base + sum > out.cap)
            raise_err(ctl, kErrCapacity, seq, round_base + sum);
        }
        __syncthreads();
        if (keep) {
          const uint64_t pos = round_base + warp_sums[warp] + __popc(ball & lt);
          if (pos < out.cap) {
            const K rest = skey[gstart[g0 + (s >> kk)]] & ~cm;
            st_key<KW>(out, pos, group_key<KW>(run, rest, s & (gsize - 1u)));
            ((AT*)out.amp)[pos] = dense[s];
          }
        }
        __syncthreads();  // warp_sums and round_base are reused
      }
    }
  }
}

__global__ void k_group_peak(Ctl* ctl, uint32_t k) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (uint32_t j = 0; j < k; ++j) atomicMax(&ctl->peak, ctl->stage[j]);
}

template <int KW, class AT>
cudaError_t group_t(const Launch& L, Ctl* ctl, Arr in, const unsigned long long* n_ptr,
                    uint32_t tile_len, uint64_t n_tiles, Arr out, int out_slot,
                    const GroupRun& run) {
  static std::atomic<unsigned long long> configured{0};  // opt-in above 48 KB, per device
  const size_t smem = GroupSmem<KW, AT>::bytes;
  cudaError_t e = ensure_smem_optin((const void*)k_group<KW, AT>, smem, configured);
  if (e != cudaSuccess) return e;
  const uint64_t grid = n_tiles < (uint64_t)L.sm_count * 64 ? n_tiles : (uint64_t)L.sm_count * 64;
  k_group<KW, AT><<<(int)(grid ? grid : 1), kGroupThreads, smem, L.stream>>>(
      ctl, in, n_ptr, tile_len, out, out_slot, run, L.seq);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_group_peak<<<1, 32, 0, L.stream>>>(ctl, run.k);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_group_count(const Launch& L, int kw, Ctl* ctl, Arr in,
                               const unsigned long long* n_ptr, const uint64_t tmask[2]) {
  const uint64_t want = (L.n_hint + kStreamThreads - 1) / kStreamThreads;
  const int grid = (int)(want < 1 ? 1 : (want > (uint64_t)L.sm_count * 8 ? L.sm_count * 8 : want));
  if (kw == 2)
    k_group_count<2><<<grid, kStreamThreads, 0, L.stream>>>(ctl, in, n_ptr, tmask[0], tmask[1]);
  else
    k_group_count<1><<<grid, kStreamThreads, 0, L.stream>>>(ctl, in, n_ptr, tmask[0], tmask[1]);
  return cudaGetLastError();
}

cudaError_t launch_group(const Launch& L, int kw, bool amp32, Ctl* ctl, Arr in,
                         const unsigned long long* n_ptr, uint32_t tile_len, uint64_t n_tiles,
                         Arr out, int out_slot, const GroupRun& run) {
  if (run.k < 2 || run.k > (uint32_t)kMaxRun || tile_len == 0 || tile_len > kGroupTile)
    return cudaErrorInvalidValue;
  if (kw == 2)
    return amp32 ? group_t<2, float2>(L, ctl, in, n_ptr, tile_len, n_tiles, out, out_slot, run)
                 : group_t<2, double2>(L, ctl, in, n_ptr, tile_len, n_tiles, out, out_slot, run);
  return amp32 ? group_t<1, float2>(L, ctl, in, n_ptr, tile_len, n_tiles, out, out_slot, run)
               : group_t<1, double2>(L, ctl, in, n_ptr, tile_len, n_tiles, out, out_slot, run);
}

}  // namespace sqs
