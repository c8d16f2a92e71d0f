// Sparse marginal probabilities of a register of any width (readout of the
// state, Table S1's measurement helpers; p(v) = sum over branches whose
// register holds v of |a|^2).
//
// Input: the state sorted by the register's field (dense, ascending field
// values, equal values contiguous).  Every run of equal values becomes one
// output pair (v, p(v)), in ascending order of v.  Work is split into tiles
// of kRunTile branches; a run may span tiles.
//   k_run_count  per tile: the runs that start in it, and the sum of its
//                leading segment (the branches that continue a run started
//                in an earlier tile), and whether that segment is the whole
//                tile;
//   k_run_scan   exclusive scan of the per-tile run counts (one CTA);
//   k_run_emit   per tile: every run that starts in it, summed over its
//                part of the tile, then over the leading segments of the
//                following tiles it covers, written at its global rank.
// Sums run in element order inside a tile and in tile order across tiles,
// so the result does not depend on scheduling (deterministic).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sqs_device.cuh"
#include "sqs_internal.h"

namespace sqs {
namespace {

constexpr uint32_t kRunTile = 2048;
constexpr int kRunThreads = 256;
constexpr int kRunScanThreads = 1024;

// Loads tile `t` of the sorted array: field values and |a|^2 into shared
// memory, and the value of the element before the tile.
template <int KW, class AT>
__device__ __forceinline__ uint32_t load_run_tile(const Arr& a, uint64_t n, uint64_t t,
                                                  uint32_t off, uint32_t w, uint64_t* sv,
                                                  double* sp, uint64_t& vprev, bool& has_prev) {
  const uint64_t base = t * (uint64_t)kRunTile;
  const uint32_t lim = base < n ? (uint32_t)(n - base < kRunTile ? n - base : kRunTile) : 0u;
  for (uint32_t j = threadIdx.x; j < lim; j += blockDim.x) {
    sv[j] = get_field(ld_key<KW>(a, base + j), off, w);
    sp[j] = norm2(((const AT*)a.amp)[base + j]);
  }
  has_prev = base > 0 && base <= n;
  vprev = has_prev ? get_field(ld_key<KW>(a, base - 1), off, w) : 0ull;
  return lim;
}

__device__ __forceinline__ bool run_head(const uint64_t* sv, uint32_t j, uint64_t vprev,
                                         bool has_prev) {
  return j == 0 ? (!has_prev || sv[0] != vprev) : sv[j] != sv[j - 1];
}

template <int KW, class AT>
__global__ void __launch_bounds__(kRunThreads)
    k_run_count(const Ctl* ctl, Arr a, const unsigned long long* n_ptr, uint32_t off, uint32_t w,
                uint64_t n_tiles, unsigned int* runs, double* lead_sum, unsigned int* lead_full) {
  __shared__ uint64_t sv[kRunTile];
  __shared__ double sp[kRunTile];
  __shared__ unsigned int cnt, first;
  if (ctl->err) return;
  const uint64_t n = *n_ptr;
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    if (threadIdx.x == 0) {
      cnt = 0u;
      first = kRunTile;
    }
    uint64_t vprev;
    bool has_prev;
    const uint32_t lim = load_run_tile<KW, AT>(a, n, t, off, w, sv, sp, vprev, has_prev);
    __syncthreads();
    unsigned int mine = 0u, mfirst = kRunTile;
    for (uint32_t j = threadIdx.x; j < lim; j += blockDim.x) {
      if (run_head(sv, j, vprev, has_prev)) {
        ++mine;
        if (j < mfirst) mfirst = j;
      }
    }
    if (mine) {
      atomicAdd(&cnt, mine);
      atomicMin(&first, mfirst);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t f = first < lim ? first : lim;
      double s = 0.0;
      for (uint32_t j = 0; j < f; ++j) s = __dadd_rn(s, sp[j]);
      runs[t] = cnt;
      lead_sum[t] = s;
      lead_full[t] = (lim > 0 && f == lim) ? 1u : 0u;
    }
    __syncthreads();
  }
}

// Exclusive scan of runs[0..n_tiles) in place (one CTA); the total goes to
// *total.
__global__ void __launch_bounds__(kRunScanThreads)
    k_run_scan(const Ctl* ctl, unsigned int* runs, uint64_t n_tiles, unsigned long long* total) {
  __shared__ unsigned long long part[kRunScanThreads];
  if (ctl->err) return;
  const uint64_t per = (n_tiles + kRunScanThreads - 1) / kRunScanThreads;
  const uint64_t lo = (uint64_t)threadIdx.x * per;
  const uint64_t hi = lo + per < n_tiles ? lo + per : n_tiles;
  unsigned long long s = 0;
  for (uint64_t i = lo; i < hi; ++i) s += runs[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < kRunScanThreads; ++i) {
      const unsigned long long c = part[i];
      part[i] = run;
      run += c;
    }
    *total = run;
  }
  __syncthreads();
  unsigned long long run = part[threadIdx.x];
  for (uint64_t i = lo; i < hi; ++i) {
    const unsigned int c = runs[i];
    runs[i] = (unsigned int)run;
    run += c;
  }
}

template <int KW, class AT>
__global__ void __launch_bounds__(kRunThreads)
    k_run_emit(const Ctl* ctl, Arr a, const unsigned long long* n_ptr, uint32_t off, uint32_t w,
               uint64_t n_tiles, const unsigned int* run_base, const double* lead_sum,
               const unsigned int* lead_full, uint64_t* values, double* probs) {
  __shared__ uint64_t sv[kRunTile];
  __shared__ double sp[kRunTile];
  __shared__ unsigned int head_rank[kRunTile];
  __shared__ unsigned int wcnt[kRunThreads / 32];
  if (ctl->err) return;
  const uint64_t n = *n_ptr;
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    uint64_t vprev;
    bool has_prev;
    const uint32_t lim = load_run_tile<KW, AT>(a, n, t, off, w, sv, sp, vprev, has_prev);
    __syncthreads();
    // Rank of each head within the tile: thread r handles the contiguous
    // slice [r * 8, r * 8 + 8), so ranks follow element order.
    constexpr uint32_t kPer = kRunTile / kRunThreads;
    const uint32_t j0 = threadIdx.x * kPer;
    unsigned int mine = 0u;
    for (uint32_t q = 0; q < kPer; ++q) {
      const uint32_t j = j0 + q;
      if (j < lim && run_head(sv, j, vprev, has_prev)) ++mine;
    }
    unsigned int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned int)o) incl += y;
    }
    if (lane == 31u) wcnt[warp] = incl;
    __syncthreads();
    unsigned int before = incl - mine;
    for (unsigned int v = 0; v < warp; ++v) before += wcnt[v];
    for (uint32_t q = 0; q < kPer; ++q) {
      const uint32_t j = j0 + q;
      if (j < lim && run_head(sv, j, vprev, has_prev)) head_rank[j] = before++;
    }
    __syncthreads();
    const uint64_t rb = run_base[t];
    for (uint32_t j = threadIdx.x; j < lim; j += blockDim.x) {
      if (!run_head(sv, j, vprev, has_prev)) continue;
      double s = sp[j];
      uint32_t e = j + 1;
      while (e < lim && sv[e] == sv[j]) {
        s = __dadd_rn(s, sp[e]);
        ++e;
      }
      if (e == lim) {
        // The run reaches the tile's end: add the leading segments of the
        // tiles it continues into, in tile order.
        for (uint64_t u = t + 1; u < n_tiles; ++u) {
          s = __dadd_rn(s, lead_sum[u]);
          if (!lead_full[u]) break;
        }
      }
      const uint64_t r = rb + head_rank[j];
      values[r] = sv[j];
      probs[r] = s;
    }
    __syncthreads();
  }
}

}  // namespace

uint64_t run_tiles(uint64_t n) { return (n + kRunTile - 1) / kRunTile; }

cudaError_t launch_sparse_marginals(const Launch& L, int kw, bool amp32, const Ctl* ctl, Arr sorted,
                                    const unsigned long long* n_ptr, uint64_t n_tiles, uint32_t off,
                                    uint32_t w, unsigned int* runs, double* lead_sum,
                                    unsigned int* lead_full, unsigned long long* total,
                                    uint64_t* values, double* probs) {
  if (n_tiles == 0) return cudaSuccess;
  const int grid = (int)(n_tiles < (uint64_t)L.sm_count * 8 ? n_tiles : (uint64_t)L.sm_count * 8);
#define SQS_RC(KW_, AT_)                                                                    \
  k_run_count<KW_, AT_><<<grid, kRunThreads, 0, L.stream>>>(ctl, sorted, n_ptr, off, w, n_tiles, \
                                                            runs, lead_sum, lead_full)
  if (kw == 1) {
    if (amp32) SQS_RC(1, float2); else SQS_RC(1, double2);
  } else {
    if (amp32) SQS_RC(2, float2); else SQS_RC(2, double2);
  }
#undef SQS_RC
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // The emit pass needs only each tile's first global rank: scan in place.
  k_run_scan<<<1, kRunScanThreads, 0, L.stream>>>(ctl, runs, n_tiles, total);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
#define SQS_RE(KW_, AT_)                                                                   \
  k_run_emit<KW_, AT_><<<grid, kRunThreads, 0, L.stream>>>(ctl, sorted, n_ptr, off, w, n_tiles, \
                                                           runs, lead_sum, lead_full, values, \
                                                           probs)
  if (kw == 1) {
    if (amp32) SQS_RE(1, float2); else SQS_RE(1, double2);
  } else {
    if (amp32) SQS_RE(2, float2); else SQS_RE(2, double2);
  }
#undef SQS_RE
  return cudaGetLastError();
}

}  // namespace sqs
