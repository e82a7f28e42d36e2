// Block-level uniform sampling of row and column index sets (Alg. 1:
// "uniformly sample row indices I and column indices J").
//
// Draw `draw` on axis `axis` of the stream `seed` is the m-subset of [0, n)
// with the m smallest keys key(i) = splitmix64(base ^ i),
// base = splitmix64(splitmix64(seed) ^ (2 draw + axis)), ties broken by the
// smaller index, returned in ascending order.  The keys are i.i.d. uniform,
// so every m-subset is equally likely (uniform sampling without replacement).
//
// One block (any multiple of 32 threads up to 1024) selects the subset in a
// few passes over the keys, each recomputed from its counter:
//   1. histogram of the next 11 key bits among keys matching the prefix found
//      so far; the bucket holding rank m becomes part of the prefix, until the
//      bucket holds at most kCap keys (one level for n up to ~2M);
//   2. the bucket's keys are collected and the exact rank of each is counted,
//      giving the m-th smallest (key, index) pair T;
//   3. an order-preserving compaction writes every i with (key, i) <= T.
#pragma once

#include "device_common.cuh"

namespace ircur {

struct SamplerSmem {
  static constexpr int kBins = 2048;  // 11 bits per histogram level
  static constexpr int kCap = 1024;   // candidates ranked exactly
  unsigned hist[kBins];
  unsigned long long ckey[kCap];
  int cidx[kCap];
  unsigned warp_tot[32];
  unsigned total;
  unsigned ccount;
  unsigned long long prefix;
  int shift;
  long long want;
  unsigned long long tkey;
  long long tidx;
};

// Exclusive scan of one count per thread across the block.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* warp_tot, unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const unsigned w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0u;
    unsigned s = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_tot[lane] = s - w;
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const unsigned r = warp_tot[wid] + x - v;
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint64_t sample_key(uint64_t base, int64_t i) { return splitmix64(base ^ (uint64_t)i); }

// Whole block: out[0..m) = the selected indices of draw (seed, draw, axis),
// 1 <= m <= n < 2^31.  With a map (n entries), map[out[a]] = index_tag(tag, a)
// for every a: the position of each selected index, tagged with its draw.
__device__ inline void sample_subset(uint64_t seed, int draw, int axis, int64_t n, int m, int* out, SamplerSmem& S,
                                     unsigned* map = nullptr, unsigned tag = 0) {
  const uint64_t base = splitmix64(splitmix64(seed) ^ (uint64_t)(2 * draw + axis));
  const int NT = blockDim.x, tid = threadIdx.x;
  if (tid == 0) {
    S.prefix = 0ull;
    S.shift = 64;
    S.want = m;
  }
  __syncthreads();
  // 1. narrow to a bucket of at most kCap keys
  for (int level = 0; level < 5; ++level) {
    const unsigned long long prefix = S.prefix;
    const int shift = S.shift;  // bits above `shift` are fixed by the prefix
    const long long want = S.want;
    for (int b = tid; b < SamplerSmem::kBins; b += NT) S.hist[b] = 0u;
    __syncthreads();
    const int nshift = shift - 11;
    for (int64_t i = tid; i < n; i += NT) {
      const uint64_t key = sample_key(base, i);
      if (shift == 64 || (key >> shift) == (prefix >> shift)) atomicAdd(&S.hist[(key >> nshift) & 2047u], 1u);
    }
    __syncthreads();
    const int per = (SamplerSmem::kBins + NT - 1) / NT;
    unsigned local = 0;
    for (int b = tid * per; b < (tid + 1) * per && b < SamplerSmem::kBins; ++b) local += S.hist[b];
    const unsigned excl = block_exclusive_scan(local, S.warp_tot, &S.total);
    if ((long long)excl < want && (long long)(excl + local) >= want) {
      long long cum = excl;
      int b = tid * per;
      while (cum + (long long)S.hist[b] < want) cum += S.hist[b++];
      S.prefix = prefix | ((unsigned long long)b << nshift);
      S.shift = nshift;
      S.want = want - cum;
      S.ccount = S.hist[b];
    }
    __syncthreads();
    if (S.ccount <= (unsigned)SamplerSmem::kCap) break;
  }
  // 2. collect the bucket and rank it exactly
  const unsigned long long prefix = S.prefix;
  const int shift = S.shift;
  const long long want = S.want;
  if (tid == 0) S.ccount = 0u;
  __syncthreads();
  for (int64_t i = tid; i < n; i += NT) {
    const uint64_t key = sample_key(base, i);
    if ((key >> shift) == (prefix >> shift)) {
      const unsigned slot = atomicAdd(&S.ccount, 1u);
      if (slot < (unsigned)SamplerSmem::kCap) {
        S.ckey[slot] = key;
        S.cidx[slot] = (int)i;
      }
    }
  }
  __syncthreads();
  const int c = (int)(S.ccount < (unsigned)SamplerSmem::kCap ? S.ccount : SamplerSmem::kCap);
  for (int u = tid; u < c; u += NT) {
    const unsigned long long ku = S.ckey[u];
    const int iu = S.cidx[u];
    long long rank = 0;
    for (int v = 0; v < c; ++v) {
      const unsigned long long kv = S.ckey[v];
      rank += (kv < ku) || (kv == ku && S.cidx[v] < iu);
    }
    if (rank == want - 1) {
      S.tkey = ku;
      S.tidx = iu;
    }
  }
  __syncthreads();
  const unsigned long long tkey = S.tkey;
  const long long tidx = S.tidx;
  // 3. order-preserving compaction of {i : (key(i), i) <= (tkey, tidx)}
  const int64_t chunk = (n + NT - 1) / NT;
  const int64_t lo = (int64_t)tid * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  unsigned cnt = 0;
  for (int64_t i = lo; i < hi; ++i) {
    const uint64_t key = sample_key(base, i);
    cnt += (key < tkey) || (key == tkey && i <= tidx);
  }
  unsigned pos = block_exclusive_scan(cnt, S.warp_tot, &S.total);
  for (int64_t i = lo; i < hi; ++i) {
    const uint64_t key = sample_key(base, i);
    if (((key < tkey) || (key == tkey && i <= tidx)) && pos < (unsigned)m) {
      out[pos] = (int)i;
      if (map) map[i] = index_tag(tag, (int)pos);
      ++pos;
    }
  }
  __syncthreads();
}

}  // namespace ircur
