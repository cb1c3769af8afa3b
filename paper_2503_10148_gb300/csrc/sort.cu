// a2 (bin) and a3 (sort): depth order, pair emission, tile radix sort, ranges.
//
// The list each tile needs is its pairs sorted by (tile, depth key, entry).
// An LSD radix sort processes the least significant digits first; here the
// depth digits are sorted before the pairs exist, on the n_entries depth keys
// (a stable sort of (key, entry) pairs from entry order, so equal keys keep
// entry order), and the pairs are then emitted in that order.  The remaining,
// most significant digits -- the tile id -- are sorted with stable passes over
// the pairs.  The result equals a stable LSD sort of the 64-bit (tile | depth)
// keys, with ties broken by component index, but the pair array (10^8
// elements at 1.5M components and 4 views) sees only ceil(tile_bits / 8)
// passes instead of ceil((32 + tile_bits) / 8).
//
// The radix sort uses a fixed grid of persistent CTAs (plan.sort_blocks),
// each owning one contiguous slice of the input, so that per-pass histograms
// are [256][blocks] and every kernel can be launched before the element count
// is known on the host (counts are read on the device; CUDA-graph friendly).
#include "common.cuh"

namespace sss {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // elements per CTA iteration
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ uint32_t load_count(const uint32_t* count_dev, uint32_t count_max) {
  return count_dev ? min(*count_dev, count_max) : count_max;
}

// Contiguous slice [begin, end) of `count` elements owned by CTA b of nb;
// slices are multiples of kTile except the last.
__device__ __forceinline__ void slice(uint32_t count, int nb, int b, uint32_t& begin, uint32_t& end) {
  const uint64_t tiles = ((uint64_t)count + kTile - 1) / kTile;
  const uint64_t per = (tiles + nb - 1) / nb;
  const uint64_t b0 = (uint64_t)b * per * kTile, b1 = (uint64_t)(b + 1) * per * kTile;
  begin = (uint32_t)(b0 < count ? b0 : (uint64_t)count);
  end = (uint32_t)(b1 < count ? b1 : (uint64_t)count);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Per-CTA digit histogram of its slice -> hist[digit * nb + cta].
__global__ void __launch_bounds__(kThreads) k_upsweep(const uint32_t* __restrict__ keys, const uint32_t* count_dev,
                                                      uint32_t count_max, int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += kThreads) sh[i] = 0;
  __syncthreads();
  uint32_t begin, end;
  slice(load_count(count_dev, count_max), gridDim.x, blockIdx.x, begin, end);
  const unsigned lane = threadIdx.x & 31;
  for (uint32_t base = begin; base < end; base += kThreads) {
    const uint32_t i = base + threadIdx.x;
    const bool ok = i < end;
    const uint32_t d = ok ? (keys[i] >> shift) & 0xffu : 0x100u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (ok && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&sh[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kThreads) hist[d * gridDim.x + blockIdx.x] = sh[d];
}

// In-place exclusive scan of n values (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_scan_exclusive(uint32_t* __restrict__ data, uint32_t n,
                                                         uint32_t* total_out) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t base = 0; base < n; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < n ? data[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= (unsigned)o) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = carry + (warp ? warp_sums[warp - 1] : 0u) + x - v;
    if (i < n) data[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

// Stable scatter of one digit.  Each CTA walks its slice in kTile chunks;
// inside a chunk warp w owns elements [w*256, w*256+256) and processes them in
// 8 rounds of 32 consecutive elements, ranking equal digits with match.any.
// vals_in == nullptr means the identity payload (element index).
__global__ void __launch_bounds__(kThreads) k_downsweep(const uint32_t* __restrict__ keys_in,
                                                        const uint32_t* __restrict__ vals_in,
                                                        uint32_t* __restrict__ keys_out,
                                                        uint32_t* __restrict__ vals_out, const uint32_t* count_dev,
                                                        uint32_t count_max, int shift,
                                                        const uint32_t* __restrict__ hist_scan) {
  __shared__ uint32_t s_off[kRadix];
  __shared__ uint32_t s_warp[kWarps][kRadix];
  uint32_t begin, end;
  slice(load_count(count_dev, count_max), gridDim.x, blockIdx.x, begin, end);
  if (begin >= end) return;
  for (int d = threadIdx.x; d < kRadix; d += kThreads) s_off[d] = hist_scan[d * gridDim.x + blockIdx.x];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  for (uint32_t t0 = begin; t0 < end; t0 += kTile) {
#pragma unroll
    for (int k = 0; k < kRadix / 32; ++k) s_warp[warp][k * 32 + lane] = 0;
    __syncwarp();
    uint32_t key[kItems], val[kItems], rank[kItems], dig[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t i = t0 + warp * (kItems * 32) + it * 32 + lane;
      const bool ok = i < end;
      key[it] = ok ? keys_in[i] : 0u;
      val[it] = ok ? (vals_in ? vals_in[i] : i) : 0u;
      dig[it] = ok ? (key[it] >> shift) & 0xffu : 0x100u;
      const unsigned peers = __match_any_sync(0xffffffffu, dig[it]);
      uint32_t basec = 0;
      if (ok) basec = s_warp[warp][dig[it]];
      rank[it] = basec + __popc(peers & lt);
      __syncwarp();
      if (ok && lane == (unsigned)(__ffs(peers) - 1)) s_warp[warp][dig[it]] = basec + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps per digit; chunk totals
    uint32_t tot = 0;
    {
      const int d = threadIdx.x;  // kThreads == kRadix
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_warp[w][d];
        s_warp[w][d] = run;
        run += c;
      }
      tot = run;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      if (dig[it] < 0x100u) {
        const uint32_t pos = s_off[dig[it]] + s_warp[warp][dig[it]] + rank[it];
        keys_out[pos] = key[it];
        vals_out[pos] = val[it];
      }
    }
    __syncthreads();
    s_off[threadIdx.x] += tot;
    __syncthreads();
  }
}

// Stable LSD sort of `count` (key, val) pairs over bits [0, bits), ping-pong
// between slot 0 and slot 1; the result lands in slot (passes & 1).
int radix_sort(uint32_t* keys0, uint32_t* keys1, uint32_t* vals0, uint32_t* vals1, const uint32_t* first_vals,
               const uint32_t* first_keys, const uint32_t* count_dev, uint32_t count_max, int bits, int nb,
               uint32_t* hist, cudaStream_t st) {
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const uint32_t* kin = (p == 0 && first_keys) ? first_keys : ((p & 1) ? keys1 : keys0);
    const uint32_t* vin = (p == 0) ? first_vals : ((p & 1) ? vals1 : vals0);
    uint32_t* kout = (p & 1) ? keys0 : keys1;
    uint32_t* vout = (p & 1) ? vals0 : vals1;
    k_upsweep<<<nb, kThreads, 0, st>>>(kin, count_dev, count_max, shift, hist);
    k_scan_exclusive<<<1, 1024, 0, st>>>(hist, (uint32_t)kRadix * nb, nullptr);
    k_downsweep<<<nb, kThreads, 0, st>>>(kin, vin, kout, vout, count_dev, count_max, shift, hist);
    SSS_LAUNCH_CHECK();
  }
  return SSS_OK;
}

__global__ void k_init_ctrl(uint32_t* ctrl, uint32_t n_entries) {
  if (threadIdx.x < 16) ctrl[threadIdx.x] = threadIdx.x == kCtrlEntries ? n_entries : 0u;
}

// Per-CTA sums of tile counts in depth order.
__global__ void __launch_bounds__(kThreads) k_count_sum(const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ ntiles, uint32_t n,
                                                        uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t ws[kWarps];
  uint32_t begin, end;
  slice(n, gridDim.x, blockIdx.x, begin, end);
  uint32_t acc = 0;
  for (uint32_t i = begin + threadIdx.x; i < end; i += kThreads) acc += ntiles[order[i]];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kWarps; ++w) t += ws[w];
    block_sums[blockIdx.x] = t;
  }
}

__global__ void k_finish_count(uint32_t* ctrl, uint32_t capacity) {
  const uint32_t need = ctrl[kCtrlPairsNeeded];
  ctrl[kCtrlPairsSorted] = min(need, capacity);
  if (need > capacity) ctrl[kCtrlStatus] |= SSS_STATUS_PAIR_OVERFLOW;
}

// Emits the pairs of every entry in depth order: CTA b scans its slice again,
// starting at block_off[b], and each entry writes (global tile, entry) for the
// tiles of its rectangle, rows in order.  Pairs at or beyond the capacity are
// dropped (the overflow bit is set by k_finish_count).
__global__ void __launch_bounds__(kThreads) k_emit(const sss_frame_plan P, const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ ntiles, const uint2* __restrict__ rect,
                                                   const uint32_t* __restrict__ block_off,
                                                   uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval) {
  __shared__ uint32_t warp_tot[kWarps];
  __shared__ uint32_t carry;
  uint32_t begin, end;
  slice(P.n_entries, gridDim.x, blockIdx.x, begin, end);
  if (threadIdx.x == 0) carry = block_off[blockIdx.x];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t cap = P.pair_capacity;
  for (uint32_t base = begin; base < end; base += kThreads) {
    const uint32_t i = base + threadIdx.x;
    uint32_t e = 0, c = 0;
    if (i < end) {
      e = order[i];
      c = ntiles[e];
    }
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint32_t before = carry;
    for (unsigned w = 0; w < warp; ++w) before += warp_tot[w];
    const uint32_t off = before + x - c;
    if (c) {
      const int j = job_of_entry(P, e);
      const sss_job_desc& J = P.jobs[j];
      const uint2 r = rect[e];
      const uint32_t tx0 = r.x & 0xffffu, tx1 = r.x >> 16, ty0 = r.y & 0xffffu, ty1 = r.y >> 16;
      uint32_t k = off;
      for (uint32_t ty = ty0; ty <= ty1; ++ty) {
        const uint32_t row = J.tile_base + ty * (uint32_t)J.tiles_x;
        for (uint32_t tx = tx0; tx <= tx1; ++tx, ++k) {
          if (k < cap) {
            pkey[k] = row + tx;
            pval[k] = e;
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == kThreads - 1) {
      uint32_t t = 0;
      for (int w = 0; w < kWarps; ++w) t += warp_tot[w];
      carry += t;
    }
    __syncthreads();
  }
}

// [start, end) of every tile from the sorted tile keys.
__global__ void k_ranges(const uint32_t* __restrict__ keys, const uint32_t* count_dev, uint2* __restrict__ ranges) {
  const uint32_t n = *count_dev;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i + 1 == n || keys[i + 1] != t) ranges[t].y = i + 1;
  }
}

}  // namespace
}  // namespace sss

using namespace sss;

extern "C" int sss_bin(const sss_frame_plan* plan, void* ws, sss_stream_t stream) {
  if (!plan || !ws) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* ctrl = ws_ptr<uint32_t>(ws, P.ws_off_ctrl);
  k_init_ctrl<<<1, 32, 0, st>>>(ctrl, P.n_entries);
  SSS_LAUNCH_CHECK();
  const uint32_t n = P.n_entries;
  if (n == 0) return SSS_OK;
  const int nb = P.sort_blocks;
  uint32_t* order = ws_ptr<uint32_t>(ws, P.ws_off_order);
  uint32_t* okey = ws_ptr<uint32_t>(ws, P.ws_off_okey);
  uint32_t* hist = ws_ptr<uint32_t>(ws, P.ws_off_hist);
  // depth digits: 4 passes over the n entries, sorted result in slot 0
  int rc = radix_sort(okey, okey + n, order, order + n, nullptr, ws_ptr<uint32_t>(ws, P.ws_off_dkey), nullptr, n,
                      32, nb, hist, st);
  if (rc != SSS_OK) return rc;
  uint32_t* block_sums = hist;  // reused: nb words
  k_count_sum<<<nb, kThreads, 0, st>>>(order, ws_ptr<uint32_t>(ws, P.ws_off_ntiles), n, block_sums);
  k_scan_exclusive<<<1, 1024, 0, st>>>(block_sums, nb, ctrl + kCtrlPairsNeeded);
  k_finish_count<<<1, 1, 0, st>>>(ctrl, P.pair_capacity);
  k_emit<<<nb, kThreads, 0, st>>>(P, order, ws_ptr<uint32_t>(ws, P.ws_off_ntiles), ws_ptr<uint2>(ws, P.ws_off_rect),
                                  block_sums, ws_ptr<uint32_t>(ws, P.ws_off_pkey),
                                  ws_ptr<uint32_t>(ws, P.ws_off_pval));
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

extern "C" int sss_sort(const sss_frame_plan* plan, void* ws, sss_stream_t stream) {
  if (!plan || !ws) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* ctrl = ws_ptr<uint32_t>(ws, P.ws_off_ctrl);
  uint2* ranges = ws_ptr<uint2>(ws, P.ws_off_ranges);
  if (cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)P.n_tiles, st) != cudaSuccess) return SSS_ERR_CUDA;
  if (P.n_entries == 0) return SSS_OK;
  uint32_t* pkey = ws_ptr<uint32_t>(ws, P.ws_off_pkey);
  uint32_t* pval = ws_ptr<uint32_t>(ws, P.ws_off_pval);
  const uint32_t cap = P.pair_capacity;
  int rc = radix_sort(pkey, pkey + cap, pval, pval + cap, pval, nullptr, ctrl + kCtrlPairsSorted, cap, P.tile_bits,
                      P.sort_blocks, ws_ptr<uint32_t>(ws, P.ws_off_hist), st);
  if (rc != SSS_OK) return rc;
  const uint32_t* skeys = pkey + (size_t)P.pair_slot * cap;
  k_ranges<<<4 * kNumSMs, 256, 0, st>>>(skeys, ctrl + kCtrlPairsSorted, ranges);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
