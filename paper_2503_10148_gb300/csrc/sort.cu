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
// A pass is reduce-then-scan: per-CTA digit histograms (upsweep), a scan of
// every digit's row in parallel (one CTA per digit), then the scatter
// (downsweep).  The scatter ranks a 4096-element tile in shared memory and
// writes it out in digit order, so consecutive threads write consecutive
// addresses of a digit's run instead of 4-byte scattered stores.  The last
// pass of the pair sort also records every tile's [start, end) with
// atomicMin/atomicMax of the run ends it writes (order independent).
#include <algorithm>

#include "common.cuh"

namespace sss {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // elements per CTA iteration
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpSpan = kItems * 32;  // elements of a tile owned by one warp
// entries per CTA of the pair count and the emission: four 256-entry chunks,
// so that a frame's entries spread over many CTAs (their gathers are
// latency-bound)
constexpr uint32_t kEmitSlice = 4 * 256;
static_assert(kThreads == kRadix, "one thread per digit");

__device__ __forceinline__ uint32_t load_count(const uint32_t* count_dev, uint32_t count_max) {
  return count_dev ? min(*count_dev, count_max) : count_max;
}

// Contiguous slice [begin, end) of `count` elements owned by CTA b of nb;
// slices are multiples of UNIT (kTile for the radix passes) except the last.
template <uint32_t UNIT = kTile>
__device__ __forceinline__ void slice(uint32_t count, int nb, int b, uint32_t& begin, uint32_t& end) {
  const uint64_t tiles = ((uint64_t)count + UNIT - 1) / UNIT;
  const uint64_t per = (tiles + nb - 1) / nb;
  const uint64_t b0 = (uint64_t)b * per * UNIT, b1 = (uint64_t)(b + 1) * per * UNIT;
  begin = (uint32_t)(b0 < count ? b0 : (uint64_t)count);
  end = (uint32_t)(b1 < count ? b1 : (uint64_t)count);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lanes of the warp whose DB-bit digit equals this lane's, among the lanes
// in `valid` (a match.any built from DB ballots: two lanes match when they
// agree on every bit).  Ballots are plain vote instructions, where
// match.any goes through the MIO pipe and its latency dominated the passes.
template <int DB>
__device__ __forceinline__ unsigned digit_peers(uint32_t d, unsigned valid) {
  unsigned peers = valid;
#pragma unroll
  for (int b = 0; b < DB; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned m = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? m : ~m;
  }
  return peers;
}

// Inclusive scan of one value per thread over a CTA of kThreads threads;
// `total` = the sum over the CTA.  Contains two barriers (s_w is reusable on
// return).
__device__ __forceinline__ uint32_t block_scan_incl(uint32_t v, uint32_t* s_w, uint32_t& total) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint32_t before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t s = s_w[w];
    before += (unsigned)w < warp ? s : 0u;
    tot += s;
  }
  __syncthreads();
  total = tot;
  return before + x;
}

// Per-CTA digit histogram of its slice -> hist[digit * nb + cta].  A
// histogram needs no order, so each warp counts into its own sub-histogram
// with shared-memory atomics (the eight are summed at the end).
__global__ void __launch_bounds__(kThreads) k_upsweep(const uint32_t* __restrict__ keys, const uint32_t* count_dev,
                                                      uint32_t count_max, int shift, uint32_t mask,
                                                      uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[kWarps][kRadix];
  const unsigned warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) sh[w][threadIdx.x] = 0;
  __syncthreads();
  uint32_t begin, end;
  slice(load_count(count_dev, count_max), gridDim.x, blockIdx.x, begin, end);
  uint32_t* my = sh[warp];
  for (uint32_t t0 = begin; t0 < end; t0 += kTile) {
    uint32_t d[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t i = t0 + it * kThreads + threadIdx.x;
      d[it] = i < end ? (__ldg(keys + i) >> shift) & mask : 0xffffffffu;
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it)
      if (d[it] != 0xffffffffu) atomicAdd(my + d[it], 1u);
  }
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) tot += sh[w][threadIdx.x];
  hist[threadIdx.x * gridDim.x + blockIdx.x] = tot;
}

// Exclusive scan, in place, of each row of `rows` (one CTA per row of n
// values); the row's sum goes to totals[row].
__global__ void __launch_bounds__(kThreads) k_scan_rows(uint32_t* __restrict__ data, uint32_t n,
                                                        uint32_t* __restrict__ totals) {
  __shared__ uint32_t s_w[kWarps];
  uint32_t* row = data + (size_t)blockIdx.x * n;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < n; base += kThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < n ? row[i] : 0u;
    uint32_t tot;
    const uint32_t incl = block_scan_incl(v, s_w, tot);
    if (i < n) row[i] = carry + incl - v;
    carry += tot;
  }
  if (threadIdx.x == 0 && totals) totals[blockIdx.x] = carry;
}

// 4-byte asynchronous global -> shared copies (no registers held while the
// loads are in flight).
__device__ __forceinline__ void cp_async4(uint32_t* smem, const uint32_t* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Shared memory of k_downsweep (dynamic, 73 KB: three CTAs per SM).
struct DownsweepSmem {
  uint32_t kin[kTile], vin[kTile];    // chunk in input order
  uint32_t key[kTile], val[kTile];    // chunk in digit order
  uint32_t warp_cnt[kWarps][kRadix];  // per-warp digit counters, then offsets
  uint32_t base[kRadix];              // global position of chunk position 0 of digit d's run
  uint32_t w[kWarps];
};

// Stable scatter of one digit.  Each CTA walks its slice in kTile chunks,
// copied to shared memory in input order.  Ranking: warp w owns elements
// [w*512, w*512+512) of the chunk and ranks them in 16 rounds of 32
// consecutive elements with match.any against its own per-digit counters; an
// exclusive scan over the warps per digit and one over the digits give every
// element its position in the digit-ordered chunk.  Write-out: thread t takes
// chunk positions t, t+256, ...; position i of digit d goes to
// (CTA's next slot of d) + (i - chunk start of d), so a digit's run is
// written by consecutive threads.  vals_in == nullptr means the identity
// payload (element index).  With `ranges`, runs of equal keys report their
// global ends (keys are the tile ids and this is the last pass).
template <int DB>
__global__ void __launch_bounds__(kThreads, 3)
    k_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const uint32_t* count_dev,
                uint32_t count_max, int shift, const uint32_t* __restrict__ hist_scan,
                const uint32_t* __restrict__ totals, uint2* __restrict__ ranges) {
  constexpr uint32_t kDMask = (1u << DB) - 1u;  // digit bits of this pass
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DownsweepSmem& S = *reinterpret_cast<DownsweepSmem*>(smem_raw);
  uint32_t begin, end;
  slice(load_count(count_dev, count_max), gridDim.x, blockIdx.x, begin, end);
  if (begin >= end) return;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const uint32_t dme = threadIdx.x;  // the digit this thread keeps the counters of
  uint32_t next;                     // global position of this CTA's next element of digit dme
  {
    const uint32_t v = totals[dme];
    uint32_t tot;
    next = block_scan_incl(v, S.w, tot) - v + hist_scan[dme * gridDim.x + blockIdx.x];
  }
  // chunk loads are asynchronous: chunk c + 1 is requested once chunk c has
  // been ranked and moved to the digit-ordered buffers, so it arrives while
  // chunk c is written out
  // 16-byte copies when both input arrays are 16-byte aligned (chunk starts
  // are multiples of kTile elements), else 4-byte copies
  const bool vec = ((reinterpret_cast<uintptr_t>(keys_in) | reinterpret_cast<uintptr_t>(vals_in)) & 15u) == 0;
  auto request = [&](uint32_t t0) {
    const uint32_t n = min(end - t0, (uint32_t)kTile);
    if (vec) {
#pragma unroll
      for (int j = 0; j < kItems / 4; ++j) {
        const uint32_t i = 4 * (j * kThreads + threadIdx.x);
        if (i + 4 <= n) {
          cp_async16(&S.kin[i], keys_in + t0 + i);
          if (vals_in) cp_async16(&S.vin[i], vals_in + t0 + i);
        } else {
          for (uint32_t e = i; e < n; ++e) {
            cp_async4(&S.kin[e], keys_in + t0 + e);
            if (vals_in) cp_async4(&S.vin[e], vals_in + t0 + e);
          }
        }
        if (!vals_in) {
#pragma unroll
          for (uint32_t r = 0; r < 4; ++r)
            if (i + r < n) S.vin[i + r] = t0 + i + r;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const uint32_t i = j * kThreads + threadIdx.x;
        if (i < n) {
          cp_async4(&S.kin[i], keys_in + t0 + i);
          if (vals_in) cp_async4(&S.vin[i], vals_in + t0 + i);
          else S.vin[i] = t0 + i;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kRadix / 32; ++k) S.warp_cnt[warp][k * 32 + lane] = 0;
  };
  request(begin);
  for (uint32_t t0 = begin; t0 < end; t0 += kTile) {
    const uint32_t n_here = min(end - t0, (uint32_t)kTile);
    cp_async_wait_all();
    __syncthreads();
    const uint32_t wloc = warp * kWarpSpan;  // chunk position of this warp's first element
    // ranking: the 16 rounds' digit matches first (independent, so their
    // votes interleave), then the chain through the warp's digit counters
    uint32_t dg[kItems], rk[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t i = wloc + it * 32 + lane;
      const bool ok = i < n_here;
      dg[it] = ok ? (S.kin[i] >> shift) & kDMask : 0u;
      rk[it] = digit_peers<DB>(dg[it], __ballot_sync(0xffffffffu, ok));  // peers for now
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const bool ok = wloc + it * 32 + lane < n_here;
      const unsigned peers = rk[it];
      const uint32_t c = ok ? S.warp_cnt[warp][dg[it]] : 0u;
      rk[it] = c + __popc(peers & lt);
      __syncwarp();
      if (ok && (peers & lt) == 0u) S.warp_cnt[warp][dg[it]] = c + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // digit dme: exclusive scan over warps, then over digits
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = S.warp_cnt[w][dme];
      S.warp_cnt[w][dme] = cnt;
      cnt += c;
    }
    uint32_t chunk_total;
    const uint32_t start = block_scan_incl(cnt, S.w, chunk_total) - cnt;  // barriers inside
#pragma unroll
    for (int w = 0; w < kWarps; ++w) S.warp_cnt[w][dme] += start;
    S.base[dme] = next - start;
    next += cnt;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t i = wloc + it * 32 + lane;
      if (i < n_here) {
        const uint32_t k = S.kin[i];
        const uint32_t loc = S.warp_cnt[warp][(k >> shift) & kDMask] + rk[it];
        S.key[loc] = k;
        S.val[loc] = S.vin[i];
      }
    }
    __syncthreads();
    // the input buffers and counters are free: request the next chunk
    if (t0 + kTile < end) request(t0 + kTile);
#pragma unroll 4
    for (int j = 0; j < kItems; ++j) {
      const uint32_t i = j * kThreads + threadIdx.x;
      if (i < n_here) {
        const uint32_t k = S.key[i];
        const uint32_t g = S.base[(k >> shift) & kDMask] + i;
        keys_out[g] = k;
        vals_out[g] = S.val[i];
        if (ranges) {
          if (i == 0 || S.key[i - 1] != k) atomicMin(&ranges[k].x, g);
          if (i + 1 == n_here || S.key[i + 1] != k) atomicMax(&ranges[k].y, g + 1);
        }
      }
    }
    // S.key, S.val and S.base are rewritten only after the next chunk's
    // first barrier, which every thread reaches after its write-out
  }
  cp_async_wait_all();
}

template <int DB>
int downsweep_optin_one() {
  return cudaFuncSetAttribute(k_downsweep<DB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(DownsweepSmem)) == cudaSuccess
             ? SSS_OK
             : SSS_ERR_CUDA;
}

// Opt-in to the dynamic shared memory of k_downsweep, once per device.
int downsweep_smem_optin() {
  static int done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SSS_ERR_CUDA;
  if (!done[dev]) {
    if (downsweep_optin_one<1>() || downsweep_optin_one<2>() || downsweep_optin_one<3>() ||
        downsweep_optin_one<4>() || downsweep_optin_one<5>() || downsweep_optin_one<6>() ||
        downsweep_optin_one<7>() || downsweep_optin_one<8>()) {
      (void)cudaGetLastError();
      return SSS_ERR_CUDA;
    }
    done[dev] = 1;
  }
  return SSS_OK;
}

template <int DB>
void launch_downsweep(int nb, cudaStream_t st, const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                      uint32_t* vout, const uint32_t* count_dev, uint32_t count_max, int shift, const uint32_t* hist,
                      const uint32_t* totals, uint2* ranges) {
  k_downsweep<DB><<<nb, kThreads, sizeof(DownsweepSmem), st>>>(kin, vin, kout, vout, count_dev, count_max, shift, hist,
                                                               totals, ranges);
}

// Stable LSD sort of `count` (key, val) pairs over bits [0, bits), ping-pong
// between slot 0 and slot 1; the result lands in slot (passes & 1).  `hist`
// holds [256][nb] counts followed by 256 digit totals.  Passes take 8 bits,
// the last one the remaining 1..8 (the ballot match of the downsweep costs
// one vote per digit bit).  With `ranges`, the last pass records the
// [start, end) of every key (which must be < the ranges array's length).
int radix_sort(uint32_t* keys0, uint32_t* keys1, uint32_t* vals0, uint32_t* vals1, const uint32_t* first_vals,
               const uint32_t* first_keys, const uint32_t* count_dev, uint32_t count_max, int bits, int nb,
               uint32_t* hist, uint2* ranges, cudaStream_t st) {
  const int passes = (bits + 7) / 8;
  uint32_t* totals = hist + (size_t)kRadix * nb;
  if (int rc = downsweep_smem_optin()) return rc;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const int db = std::min(8, bits - shift);
    const uint32_t* kin = (p == 0 && first_keys) ? first_keys : ((p & 1) ? keys1 : keys0);
    const uint32_t* vin = (p == 0) ? first_vals : ((p & 1) ? vals1 : vals0);
    uint32_t* kout = (p & 1) ? keys0 : keys1;
    uint32_t* vout = (p & 1) ? vals0 : vals1;
    uint2* rg = p + 1 == passes ? ranges : nullptr;
    k_upsweep<<<nb, kThreads, 0, st>>>(kin, count_dev, count_max, shift, (1u << db) - 1u, hist);
    k_scan_rows<<<kRadix, kThreads, 0, st>>>(hist, (uint32_t)nb, totals);
    switch (db) {
      case 1: launch_downsweep<1>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      case 2: launch_downsweep<2>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      case 3: launch_downsweep<3>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      case 4: launch_downsweep<4>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      case 5: launch_downsweep<5>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      case 6: launch_downsweep<6>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      case 7: launch_downsweep<7>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
      default: launch_downsweep<8>(nb, st, kin, vin, kout, vout, count_dev, count_max, shift, hist, totals, rg); break;
    }
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
  slice<kEmitSlice>(n, gridDim.x, blockIdx.x, begin, end);
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

// Emits the pairs of every entry in depth order.  CTA b takes its slice of
// the depth order again, starting at output position block_off[b], in chunks
// of 256 entries: a CTA scan of the chunk's tile counts places each entry's
// pairs, and the threads then walk the chunk's output positions k = t,
// t+256, ... (coalesced stores, no per-entry loop): the entry is the last one
// whose start is <= k (binary search over the 256 starts) and the tile is
// the (k - start)-th of its rectangle, rows in order.  Pairs at or beyond the
// capacity are dropped (the overflow bit is set by k_finish_count).
__global__ void __launch_bounds__(kThreads) k_emit(const sss_frame_plan P, const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ ntiles, const uint2* __restrict__ rect,
                                                   const uint32_t* __restrict__ block_off,
                                                   uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval) {
  __shared__ uint32_t s_start[kThreads];  // first output position of each entry of the chunk
  __shared__ uint32_t s_t0[kThreads];     // global tile id of the rectangle's first tile
  __shared__ uint32_t s_wx[kThreads];     // rectangle width (tiles)
  __shared__ uint32_t s_stride[kThreads]; // tiles per row of the entry's view
  __shared__ uint32_t s_e[kThreads];
  __shared__ uint32_t s_w[kWarps];
  uint32_t begin, end;
  slice<kEmitSlice>(P.n_entries, gridDim.x, blockIdx.x, begin, end);
  uint32_t carry = block_off[blockIdx.x];
  const uint32_t cap = P.pair_capacity;
  // software pipeline over the 256-entry chunks: the entry id of chunk k + 2
  // and the count and rectangle of chunk k + 1 are loaded while chunk k's
  // pairs are written, so the dependent gathers (depth order -> entry ->
  // count, rectangle) overlap the scan and the stores
  auto entry_at = [&](uint32_t base) -> uint32_t {
    const uint32_t i = base + threadIdx.x;
    return i < end ? order[i] : 0xffffffffu;
  };
  uint32_t e_cur = entry_at(begin), e_nxt = entry_at(begin + kThreads);
  uint32_t c_cur = e_cur != 0xffffffffu ? ntiles[e_cur] : 0u;
  uint2 r_cur = c_cur ? rect[e_cur] : make_uint2(0u, 0u);
  for (uint32_t base = begin; base < end; base += kThreads) {
    const uint32_t c_nxt = e_nxt != 0xffffffffu ? ntiles[e_nxt] : 0u;
    const uint2 r_nxt = c_nxt ? rect[e_nxt] : make_uint2(0u, 0u);
    const uint32_t e_nn = entry_at(base + 2 * kThreads);
    const uint32_t c = c_cur;
    uint32_t t0 = 0, wx = 1, stride = 0;
    if (c) {
      const sss_job_desc& J = P.jobs[job_of_entry(P, e_cur)];
      const uint32_t tx0 = r_cur.x & 0xffffu, tx1 = r_cur.x >> 16, ty0 = r_cur.y & 0xffffu;
      stride = (uint32_t)J.tiles_x;
      t0 = J.tile_base + ty0 * stride + tx0;
      wx = tx1 - tx0 + 1;
    }
    uint32_t total;
    const uint32_t incl = block_scan_incl(c, s_w, total);
    s_start[threadIdx.x] = incl - c;
    s_t0[threadIdx.x] = t0;
    s_wx[threadIdx.x] = wx;
    s_stride[threadIdx.x] = stride;
    s_e[threadIdx.x] = e_cur;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < total; k += kThreads) {
      uint32_t j = 0;
#pragma unroll
      for (uint32_t step = kThreads / 2; step; step >>= 1)
        if (s_start[j + step] <= k) j += step;
      const uint32_t local = k - s_start[j], w = s_wx[j];
      const uint32_t row = local / w, col = local - row * w;
      const uint32_t g = carry + k;
      if (g < cap) {
        pkey[g] = s_t0[j] + row * s_stride[j] + col;
        pval[g] = s_e[j];
      }
    }
    carry += total;
    e_cur = e_nxt;
    c_cur = c_nxt;
    r_cur = r_nxt;
    e_nxt = e_nn;
    __syncthreads();
  }
}

// Tile ranges start as (~0, 0) so that the last sort pass can take the
// minimum start and maximum end of the runs it writes ...
__global__ void k_ranges_init(uint2* __restrict__ ranges, uint32_t n_tiles) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
    ranges[t] = make_uint2(0xffffffffu, 0u);
}
// ... and tiles that received no pair end as (0, 0).
__global__ void k_ranges_fix(uint2* __restrict__ ranges, uint32_t n_tiles) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
    if (ranges[t].x == 0xffffffffu) ranges[t].x = 0u;
}

}  // namespace

int radix_sort_pairs(uint32_t* keys0, uint32_t* keys1, uint32_t* vals0, uint32_t* vals1, const uint32_t* first_vals,
                     const uint32_t* first_keys, const uint32_t* count_dev, uint32_t count_max, int bits, int nb,
                     uint32_t* hist, cudaStream_t st) {
  return radix_sort(keys0, keys1, vals0, vals1, first_vals, first_keys, count_dev, count_max, bits, nb, hist, nullptr,
                    st);
}

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
  const uint32_t n4 = (n + 3) & ~3u;  // slot stride (16-byte aligned slot 1)
  int rc = radix_sort(okey, okey + n4, order, order + n4, nullptr, ws_ptr<uint32_t>(ws, P.ws_off_dkey), nullptr, n,
                      32, nb, hist, nullptr, st);
  if (rc != SSS_OK) return rc;
  uint32_t* block_sums = hist;  // reused: nb words
  // emission: one kEmitSlice slice of the depth order per CTA (many CTAs
  // hide the latency of the dependent order -> count / rectangle gathers);
  // the block sums fit in the histogram scratch (256 nb + 256 words)
  const unsigned nbe = (unsigned)std::min<size_t>(ceil_div(n, kEmitSlice), (size_t)kRadix * nb);
  k_count_sum<<<nbe, kThreads, 0, st>>>(order, ws_ptr<uint32_t>(ws, P.ws_off_ntiles), n, block_sums);
  k_scan_rows<<<1, kThreads, 0, st>>>(block_sums, nbe, ctrl + kCtrlPairsNeeded);
  k_finish_count<<<1, 1, 0, st>>>(ctrl, P.pair_capacity);
  k_emit<<<nbe, kThreads, 0, st>>>(P, order, ws_ptr<uint32_t>(ws, P.ws_off_ntiles), ws_ptr<uint2>(ws, P.ws_off_rect),
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
  if (P.n_entries == 0) {
    if (cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)P.n_tiles, st) != cudaSuccess) return SSS_ERR_CUDA;
    return SSS_OK;
  }
  const unsigned rgrid = min(ceil_div(P.n_tiles, 256), 4u * (unsigned)device_sm_count());
  k_ranges_init<<<rgrid, 256, 0, st>>>(ranges, P.n_tiles);
  uint32_t* pkey = ws_ptr<uint32_t>(ws, P.ws_off_pkey);
  uint32_t* pval = ws_ptr<uint32_t>(ws, P.ws_off_pval);
  const uint32_t cap = P.pair_capacity;
  int rc = radix_sort(pkey, pkey + cap, pval, pval + cap, pval, nullptr, ctrl + kCtrlPairsSorted, cap, P.tile_bits,
                      P.sort_blocks, ws_ptr<uint32_t>(ws, P.ws_off_hist), ranges, st);
  if (rc != SSS_OK) return rc;
  k_ranges_fix<<<rgrid, 256, 0, st>>>(ranges, P.n_tiles);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
