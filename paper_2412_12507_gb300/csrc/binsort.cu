// binsort.cu — duplicate (tile | depth) keys, sort them, find per-tile ranges
// (Sec. 4.3; the Duplicate and Sort phases of Table 2).
//
// The result equals a stable sort of key = (tile << 32) | bits(depth) over the entries
// emitted per particle in index order and per tile in row-major order, but it is computed
// in cheaper steps:
//   1. a stable LSD radix sort of the N particle depths (bits(depth), index);
//   2. emission, in that depth order, of one entry per (particle, tile column) it covers,
//      and a stable radix sort of those entries by global tile column;
//   3. expansion, in that (column, depth) order, of every column entry into its tile rows,
//      stably ordered by global tile row: scattered straight to the final positions (the row
//      scatter below) when every view has at most 512 tile rows and the batch at most 16384
//      tile columns, else emitted and sorted by one more radix pass per 8 row bits.
// A stable order by row of a sequence ordered by (column, depth) is ordered by
// (row, column, depth) = (tile, depth), so the outputs are identical, while the K entries
// are written once (row scatter) or pass through one 8-bit radix pass per ceil(log2 rows / 8)
// instead of ceil(log2 tiles / 8) passes, and only the shorter column list (one entry per
// covered column, not per tile) pays for the column order.
//
// The radix sort is the project's own: per 8-bit digit pass an upsweep (per-warp shared
// histograms fed by uint4 key loads), a digit-major exclusive scan (per-chunk totals, then a
// down-sweep whose blocks add up the totals before their chunk), and a downsweep that
// ranks keys stably in shared memory (same-digit lanes found with 8 ballots per 32-key group,
// per-warp running digit counters) and writes them out digit-grouped for coalescing.
// No kernel waits on another block, so nothing in here can spin.
#include "ut3d_debug.cuh"
#include "ut3d_device.cuh"
#include "ut3d_internal.h"

namespace ut3d {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIPT = 16;
constexpr int kTile = kThreads * kIPT;  // keys per scan tile
constexpr int kRIPT = 8;                 // keys per thread in a radix tile
constexpr int kRTile = kThreads * kRIPT; // keys per radix tile (upsweep and downsweep agree)
constexpr int kRadixBits = 8;

typedef unsigned long long u64;

// Element count of a pass: a host constant, or a device total that is honoured only if it
// and the optional guard total (the call's K) fit the caller's capacity (0 otherwise, so an
// overflowing call writes nothing).
struct Count {
  const u64 *dev;
  u64 cap;
  uint32_t host;
  const u64 *guard = nullptr;
  __device__ __forceinline__ uint32_t get() const {
    if (!dev) return host;
    if (guard && *guard > cap) return 0u;
    u64 v = *dev;
    return v <= cap ? (uint32_t)v : 0u;
  }
};

// Length of the digit-major spine: nd digits x number of radix tiles.
struct SpineLen {
  Count c;
  int nd;
  __device__ __forceinline__ uint32_t get() const {
    uint32_t k = c.get();
    return (uint32_t)nd * ((k + kRTile - 1) / kRTile);
  }
};

__device__ __forceinline__ u64 warp_incl_scan_u64(u64 x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive block scan of one u64 per thread (kThreads threads); returns the block total.
__device__ __forceinline__ u64 block_excl_scan_u64(u64 x, u64 *s_warp, u64 &excl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 inc = warp_incl_scan_u64(x, lane);
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    u64 w = lane < kWarps ? s_warp[lane] : 0;
    u64 wi = warp_incl_scan_u64(w, lane);
    if (lane < kWarps) s_warp[lane] = wi - w;
    if (lane == kWarps - 1) s_warp[kWarps] = wi;
  }
  __syncthreads();
  excl = s_warp[warp] + inc - x;
  u64 total = s_warp[kWarps];
  __syncthreads();
  return total;
}

// ---------------------------------------------------------------- exclusive scan (u32 -> u32, u64 total)

// Input transforms of the scans: the value itself, or the upper 16 bits (the tile height a
// column key carries).
struct Ident {
  __device__ __forceinline__ uint32_t operator()(uint32_t v) const { return v; }
};
struct High16 {
  __device__ __forceinline__ uint32_t operator()(uint32_t v) const { return v >> 16; }
};

template <class L, class X = Ident>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t *__restrict__ in, L len,
                                                          u64 *__restrict__ chunk) {
  __shared__ u64 s_warp[kWarps + 1];
  const uint32_t n = len.get();
  const uint32_t nchunks = (n + kTile - 1) / kTile;
  for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    u64 s = 0;
    uint32_t base = c * kTile;
#pragma unroll 4
    for (int i = 0; i < kIPT; ++i) {
      uint32_t p = base + i * kThreads + threadIdx.x;
      if (p < n) s += X()(in[p]);
    }
    u64 ex;
    u64 tot = block_excl_scan_u64(s, s_warp, ex);
    if (threadIdx.x == 0) chunk[c] = tot;
  }
}

template <class L>
__global__ void __launch_bounds__(1024) k_scan_spine(u64 *__restrict__ chunk, L len, u64 *__restrict__ total) {
  __shared__ u64 s_warp[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n = len.get();
  const uint32_t nchunks = (n + kTile - 1) / kTile;
  u64 carry = 0;
  for (uint32_t base = 0; base < nchunks; base += 1024) {
    uint32_t c = base + threadIdx.x;
    u64 x = c < nchunks ? chunk[c] : 0;
    u64 inc = warp_incl_scan_u64(x, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      u64 w = s_warp[lane];
      u64 wi = warp_incl_scan_u64(w, lane);
      s_warp[lane] = wi - w;
      if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    if (c < nchunks) chunk[c] = carry + s_warp[warp] + inc - x;
    carry += s_warp[32];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// skewed shared-memory index: conflict-free for both coalesced loads and per-thread runs
__device__ __forceinline__ int skew(int p) { return p + (p >> 5); }

template <class L, class X = Ident>
__global__ void __launch_bounds__(kThreads) k_scan_down(const uint32_t *in, uint32_t *out, L len,
                                                        const u64 *__restrict__ chunk) {
  __shared__ uint32_t s_v[kTile + kTile / 32];
  __shared__ u64 s_warp[kWarps + 1];
  const uint32_t n = len.get();
  const uint32_t nchunks = (n + kTile - 1) / kTile;
  for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    uint32_t base = c * kTile;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      int q = i * kThreads + threadIdx.x;
      uint32_t p = base + q;
      s_v[skew(q)] = p < n ? X()(in[p]) : 0u;
    }
    __syncthreads();
    uint32_t v[kIPT];
    u64 s = 0;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      v[i] = s_v[skew(threadIdx.x * kIPT + i)];
      s += v[i];
    }
    u64 ex;
    block_excl_scan_u64(s, s_warp, ex);
    u64 run = chunk[c] + ex;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      s_v[skew(threadIdx.x * kIPT + i)] = (uint32_t)run;
      run += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      int q = i * kThreads + threadIdx.x;
      uint32_t p = base + q;
      if (p < n) out[p] = s_v[skew(q)];
    }
    __syncthreads();
  }
}

// k_scan_down for chunk lists of up to kSelfPrefixChunks: `chunk` holds each chunk's raw
// total (from k_scan_reduce) and every block sums the totals before its chunk itself, so no
// separate spine pass is needed; block 0 writes the grand total when `total` is given.
constexpr uint32_t kSelfPrefixChunks = 65536;  // also keeps the launch sequence independent of the capacity

template <class L, class X = Ident>
__global__ void __launch_bounds__(kThreads) k_scan_down_self(const uint32_t *in, uint32_t *out, L len,
                                                             const u64 *__restrict__ chunk, u64 *__restrict__ total) {
  __shared__ uint32_t s_v[kTile + kTile / 32];
  __shared__ u64 s_warp[kWarps + 1];
  const uint32_t n = len.get();
  const uint32_t nchunks = (n + kTile - 1) / kTile;
  if (blockIdx.x == 0 && total) {
    u64 a = 0;
    for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) a += chunk[c];
    u64 ex;
    const u64 t = block_excl_scan_u64(a, s_warp, ex);
    if (threadIdx.x == 0) *total = t;
  }
  for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    u64 a = 0;
    for (uint32_t cc = threadIdx.x; cc < c; cc += blockDim.x) a += chunk[cc];
    u64 ex;
    const u64 prefix = block_excl_scan_u64(a, s_warp, ex);
    uint32_t base = c * kTile;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      int q = i * kThreads + threadIdx.x;
      uint32_t p = base + q;
      s_v[skew(q)] = p < n ? X()(in[p]) : 0u;
    }
    __syncthreads();
    uint32_t v[kIPT];
    u64 sum = 0;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      v[i] = s_v[skew(threadIdx.x * kIPT + i)];
      sum += v[i];
    }
    block_excl_scan_u64(sum, s_warp, ex);
    u64 run = prefix + ex;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      s_v[skew(threadIdx.x * kIPT + i)] = (uint32_t)run;
      run += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
      int q = i * kThreads + threadIdx.x;
      uint32_t p = base + q;
      if (p < n) out[p] = s_v[skew(q)];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- radix sort passes


// Lanes of this warp whose 8-bit digit equals mine, from 8 ballots (one per digit bit).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int bit = 0; bit < 8; ++bit) {
    const bool one = (d >> bit) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, one);
    peers &= one ? bal : ~bal;
  }
  return peers;
}

// Per radix tile, the count of each digit (digit-major layout counts[d * nb + b]).  Keys are
// read as uint4 (the next tile's while the current one is counted into the warps' shared
// histograms and totalled).
__global__ void __launch_bounds__(kThreads) k_radix_upsweep(const uint32_t *__restrict__ keys, Count cnt, int shift,
                                                            uint32_t mask, uint32_t *__restrict__ counts) {
  __shared__ uint32_t s_wh[kWarps][256];
  const uint32_t n = cnt.get();
  const uint32_t nb = (n + kRTile - 1) / kRTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *wh = s_wh[warp];
  constexpr int kQ = kRIPT / 4;
  uint32_t b = blockIdx.x;
  if (b >= nb) return;
  uint4 q[kQ];
  auto load = [&](uint32_t t) {
    const uint32_t base = t * kRTile;
    if (base + kRTile <= n) {
      const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
      for (int i = 0; i < kQ; ++i) q[i] = k4[i * kThreads + threadIdx.x];
    } else {  // ragged last tile: element loads, 0xffffffff marks "no key"
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const uint32_t p = base + 4 * (i * kThreads + threadIdx.x);
        q[i].x = p < n ? keys[p] : 0xffffffffu;
        q[i].y = p + 1 < n ? keys[p + 1] : 0xffffffffu;
        q[i].z = p + 2 < n ? keys[p + 2] : 0xffffffffu;
        q[i].w = p + 3 < n ? keys[p + 3] : 0xffffffffu;
      }
    }
  };
  load(b);
  for (; b < nb; b += gridDim.x) {
    for (int d = lane; d < 256; d += 32) wh[d] = 0;
    __syncwarp();
    const uint32_t base = b * kRTile;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const uint32_t p = base + 4 * (i * kThreads + threadIdx.x);
      if (p < n) atomicAdd(&wh[(q[i].x >> shift) & mask], 1u);
      if (p + 1 < n) atomicAdd(&wh[(q[i].y >> shift) & mask], 1u);
      if (p + 2 < n) atomicAdd(&wh[(q[i].z >> shift) & mask], 1u);
      if (p + 3 < n) atomicAdd(&wh[(q[i].w >> shift) & mask], 1u);
    }
    if (b + gridDim.x < nb) load(b + gridDim.x);
    __syncthreads();
    if (threadIdx.x <= mask) {
      uint32_t s = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += s_wh[w][threadIdx.x];
      counts[(size_t)threadIdx.x * nb + b] = s;
    }
    __syncthreads();
  }
}

// Keys and values of radix tile b (kRIPT per thread, warp-contiguous segments; past n: keys
// 0xffffffff, which sort last and are never written out).
__device__ __forceinline__ void load_radix_tile(const uint32_t *__restrict__ keys_in,
                                                const uint32_t *__restrict__ vals_in, uint32_t n, uint32_t b,
                                                uint32_t (&k)[kRIPT], uint32_t (&v)[kRIPT]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t base = b * kRTile + warp * (kRIPT * 32) + lane;
#pragma unroll
  for (int i = 0; i < kRIPT; ++i) {
    const uint32_t p = base + i * 32;
    const bool valid = p < n;
    k[i] = valid ? keys_in[p] : 0xffffffffu;
    v[i] = valid ? vals_in[p] : 0u;
  }
}

// Stable scatter of one digit pass.  Per radix tile: every key's rank among the same-digit
// keys of its warp segment (leader lane bumps the warp's digit counter, the old value is
// broadcast), digit starts from the per-warp counts and a block scan, a scatter into shared
// memory in digit order, and a write-out grouped by digit (coalesced runs).  The next tile's
// keys, values and global digit offsets are loaded while the current tile is written out.
// SELF (lists of at most kSelfRadixTiles tiles): `offsets` holds the upsweep's raw digit-major
// counts and every block derives its own offsets from them (the digit totals' exclusive scan
// plus the counts of its digit in the tiles before it), which saves the two scan launches.
constexpr uint32_t kSelfRadixTiles = 128;

template <bool SELF>
__global__ void __launch_bounds__(kThreads) k_radix_downsweep(const uint32_t *__restrict__ keys_in,
                                                              const uint32_t *__restrict__ vals_in,
                                                              uint32_t *__restrict__ keys_out,
                                                              uint32_t *__restrict__ vals_out, Count cnt, int shift,
                                                              uint32_t mask, const uint32_t *__restrict__ offsets) {
  __shared__ uint32_t s_k[kRTile];
  __shared__ uint32_t s_v[kRTile];
  __shared__ uint32_t s_whist[kWarps][256];
  __shared__ uint32_t s_dstart[256];
  __shared__ uint32_t s_goff[256];
  __shared__ u64 s_warp[kWarps + 1];
  const uint32_t n = cnt.get();
  const uint32_t nb = (n + kRTile - 1) / kRTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int nd = (int)mask + 1;
  uint32_t b = blockIdx.x;
  if (b >= nb) return;
  __shared__ uint32_t s_dbase[SELF ? 256 : 1];
  if (SELF) {  // exclusive scan of the digit totals
    uint32_t t = 0;
    if (threadIdx.x < nd)
      for (uint32_t bb = 0; bb < nb; ++bb) t += offsets[(size_t)threadIdx.x * nb + bb];
    u64 ex;
    block_excl_scan_u64(t, s_warp, ex);
    if (threadIdx.x < nd) s_dbase[threadIdx.x] = (uint32_t)ex;
    __syncthreads();
  }
  // global start of this thread's digit in tile bb
  auto offset_of = [&](uint32_t bb) -> uint32_t {
    if (threadIdx.x >= nd) return 0u;
    if (!SELF) return offsets[(size_t)threadIdx.x * nb + bb];
    uint32_t o = s_dbase[SELF ? threadIdx.x : 0];
    for (uint32_t b2 = 0; b2 < bb; ++b2) o += offsets[(size_t)threadIdx.x * nb + b2];
    return o;
  };
  uint32_t k[kRIPT], v[kRIPT];
  load_radix_tile(keys_in, vals_in, n, b, k, v);
  uint32_t goff = offset_of(b);
  for (; b < nb; b += gridDim.x) {
    for (int d = lane; d < nd; d += 32) s_whist[warp][d] = 0;
    __syncwarp();
    // stable rank of every key among the same-digit keys of this warp's segment
    uint32_t rank[kRIPT];
#pragma unroll
    for (int i = 0; i < kRIPT; ++i) {
      const uint32_t d = (k[i] >> shift) & mask;
      const uint32_t peers = digit_peers(d);
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (lane == leader) before = atomicAdd(&s_whist[warp][d], (uint32_t)__popc(peers));
      before = __shfl_sync(0xffffffffu, before, leader);
      rank[i] = before + (uint32_t)__popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: offsets of each warp's run, block totals, and the digit starts in the tile
    uint32_t tot = 0;
    if (threadIdx.x < nd) {
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        uint32_t c = s_whist[w][threadIdx.x];
        s_whist[w][threadIdx.x] = tot;
        tot += c;
      }
      s_goff[threadIdx.x] = goff;
    }
    u64 ex;
    block_excl_scan_u64(tot, s_warp, ex);
    if (threadIdx.x < nd) s_dstart[threadIdx.x] = (uint32_t)ex;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRIPT; ++i) {
      uint32_t d = (k[i] >> shift) & mask;
      uint32_t pos = s_dstart[d] + s_whist[warp][d] + rank[i];
      s_k[pos] = k[i];
      s_v[pos] = v[i];
    }
    const uint32_t bn = b + gridDim.x;
    if (bn < nb) {  // prefetch the next tile into the now free registers
      load_radix_tile(keys_in, vals_in, n, bn, k, v);
      goff = offset_of(bn);
    }
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kRTile, n - b * kRTile);
    for (uint32_t j = threadIdx.x; j < nvalid; j += kThreads) {
      uint32_t kk = s_k[j];
      uint32_t d = (kk >> shift) & mask;
      uint32_t g = s_goff[d] + j - s_dstart[d];
      keys_out[g] = kk;
      vals_out[g] = s_v[j];
    }
    // the next tile's first write to shared memory that the write-out reads (s_goff, s_dstart,
    // s_k, s_v) comes after its first __syncthreads, so no barrier is needed here
  }
}

// ---------------------------------------------------------------- binning kernels

// Depth keys (culled particles last) and the particle indices, and K = sum of ntiles added to
// *ksum (zeroed beforehand) with one atomic per block.
__global__ void __launch_bounds__(kThreads) k_depth_init(int n, const float *__restrict__ depth,
                                                         const uint32_t *__restrict__ ntiles,
                                                         uint32_t *__restrict__ dk, uint32_t *__restrict__ dv,
                                                         u64 *__restrict__ ksum) {
  __shared__ u64 s_warp[kWarps + 1];
  u64 k = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = ntiles[i];
    dk[i] = t > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
    dv[i] = (uint32_t)i;
    k += t;
  }
  u64 ex;
  const u64 tot = block_excl_scan_u64(k, s_warp, ex);
  if (threadIdx.x == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long *>(ksum), (unsigned long long)tot);
}

// Depth order -> number of tile columns each particle covers (0 if culled).
__global__ void k_gather_widths(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ ntiles,
                                const short4 *__restrict__ rect, int tile_w, uint32_t *__restrict__ cnt) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t g = order[j];
    uint32_t w = 0;
    if (ntiles[g]) {
      const short4 r = rect[g];
      w = (uint32_t)(r.z / tile_w - r.x / tile_w + 1);
    }
    cnt[j] = w;
  }
}

__global__ void k_write_kout(const u64 *__restrict__ total, int64_t *__restrict__ k_out) { *k_out = (int64_t)*total; }

// Lane owning output position p among the warp's 32 consecutive runs (run l starts at
// start_l; starts are non-decreasing, lanes past the items hold 0xffffffff): the last lane
// whose run starts at or before p.  Every lane of the warp must call it.
__device__ __forceinline__ int run_owner(uint32_t start, uint32_t p) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t s = __shfl_sync(0xffffffffu, start, (lo + step) & 31);
    if (lo + step < 32 && s <= p) lo += step;
  }
  return lo;
}

// Column entries, one warp per 32 particles of the depth order.  The particles' runs are
// consecutive in the output, so the warp writes their union [start_0, end_31) with all lanes,
// each lane finding the run of its position.  Key = (tile rows covered << 16) | global tile
// column, or with PACK global tile column | first tile row << 14 | (rows - 1) << 23 (the sort
// uses the column bits only; the rest rides along for the row stage), value = flattened
// particle index.
template <bool PACK>
__global__ void __launch_bounds__(kThreads) k_emit_cols(const __grid_constant__ BatchDesc bd, int n,
                                                        const uint32_t *__restrict__ order,
                                                        const uint32_t *__restrict__ offs,
                                                        const uint32_t *__restrict__ widths,
                                                        const short4 *__restrict__ rect, Count total, int tile_w,
                                                        int tile_h, uint32_t *__restrict__ ckeys,
                                                        uint32_t *__restrict__ cvals) {
  if (total.get() == 0) return;  // nothing to emit, or more than the capacity
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int j0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < n; j0 += nw * 32) {
    const int j = j0 + lane;
    uint32_t start = 0xffffffffu, end = 0, g = 0, key0 = 0;
    if (j < n) {
      start = offs[j];
      const uint32_t w = widths[j];
      end = start + w;
      if (w) {
        g = order[j];
        const short4 r = rect[g];
        const uint32_t h = (uint32_t)(r.w / tile_h - r.y / tile_h + 1);
        const uint32_t col = (uint32_t)(bd.v[view_of_particle(bd, (int)g)].col_off + r.x / tile_w);
        key0 = PACK ? (col | ((uint32_t)(r.y / tile_h) << 14) | ((h - 1u) << 23)) : ((h << 16) | col);
      }
    }
    const uint32_t S = __shfl_sync(0xffffffffu, start, 0);
    const uint32_t E = __shfl_sync(0xffffffffu, end, min(31, n - 1 - j0));
    for (uint32_t b = S; b < E; b += 32) {
      const uint32_t p = b + lane;
      const int l = run_owner(start, p);
      const uint32_t s0 = __shfl_sync(0xffffffffu, start, l);
      const uint32_t k0 = __shfl_sync(0xffffffffu, key0, l);
      const uint32_t g0 = __shfl_sync(0xffffffffu, g, l);
      if (p < E) {
        UT_DBG_CHECK(p < total.cap, UT_DBG_KEY_INDEX, p, total.cap, 0);
        ckeys[p] = k0 + (p - s0);
        cvals[p] = g0;
      }
    }
  }
}

// Row entries, one warp per 32 column entries (in column order), written like k_emit_cols:
// each column entry expands into its particle's tile rows, ascending.  Key = (global tile
// row << col_bits) | column within the view, value = particle index within its scene.
__global__ void __launch_bounds__(kThreads) k_emit_rows(const __grid_constant__ BatchDesc bd, Count ccount,
                                                        const uint32_t *__restrict__ ckeys,
                                                        const uint32_t *__restrict__ cvals,
                                                        const uint32_t *__restrict__ offs,
                                                        const short4 *__restrict__ rect, Count total, int tile_h,
                                                        uint32_t *__restrict__ rkeys, uint32_t *__restrict__ rvals) {
  if (total.get() == 0) return;
  const uint32_t m = ccount.get();
  const int lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; i0 < m; i0 += nw * 32) {
    const uint32_t i = i0 + lane;
    uint32_t start = 0xffffffffu, end = 0, local = 0, key0 = 0;
    if (i < m) {
      const uint32_t ck = ckeys[i];
      start = offs[i];
      end = start + (ck >> 16);
      const uint32_t g = cvals[i];
      const DevView &view = bd.v[view_of_particle(bd, (int)g)];
      local = g - (uint32_t)view.part_off;
      const uint32_t tx = (ck & 0xffffu) - (uint32_t)view.col_off;
      key0 = ((uint32_t)(view.row_off + rect[g].y / tile_h) << bd.col_bits) | tx;
    }
    const uint32_t S = __shfl_sync(0xffffffffu, start, 0);
    const uint32_t E = __shfl_sync(0xffffffffu, end, (int)min(31u, m - 1 - i0));
    for (uint32_t b = S; b < E; b += 32) {
      const uint32_t p = b + lane;
      const int l = run_owner(start, p);
      const uint32_t s0 = __shfl_sync(0xffffffffu, start, l);
      const uint32_t k0 = __shfl_sync(0xffffffffu, key0, l);
      const uint32_t l0 = __shfl_sync(0xffffffffu, local, l);
      if (p < E) {
        UT_DBG_CHECK(p < total.cap, UT_DBG_KEY_INDEX, p, total.cap, 1);
        rkeys[p] = k0 + ((p - s0) << bd.col_bits);
        rvals[p] = l0;
      }
    }
  }
}

// Global tile id of a sorted (row << col_bits | column) key.
__device__ __forceinline__ uint32_t tile_of_key(const BatchDesc &bd, uint32_t key) {
  const int row = (int)(key >> bd.col_bits);
  const DevView &v = bd.v[view_of_row(bd, row)];
  return (uint32_t)(v.tile_off + (row - v.row_off) * v.tiles_x) + (key & ((1u << bd.col_bits) - 1u));
}

// Tile ranges from the sorted keys: four keys per thread (uint4) and their neighbours (equal
// keys <=> equal tiles).
__global__ void k_ranges(const __grid_constant__ BatchDesc bd, const uint32_t *__restrict__ tkeys,
                         const uint32_t *__restrict__ vals, Count cnt, const float *__restrict__ depth,
                         uint32_t *__restrict__ ranges, uint64_t *__restrict__ keys) {
  const uint32_t K = cnt.get();
  const uint32_t nq = (K + 3) / 4;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t p0 = 4 * q;
    uint32_t t[6];  // t[0] = key before p0, t[1..4] = keys p0..p0+3, t[5] = key after
    if (p0 + 4 <= K) {
      const uint4 v = reinterpret_cast<const uint4 *>(tkeys)[q];
      t[1] = v.x; t[2] = v.y; t[3] = v.z; t[4] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) t[1 + i] = p0 + i < K ? tkeys[p0 + i] : 0xffffffffu;
    }
    t[0] = p0 > 0 ? tkeys[p0 - 1] : 0xffffffffu;
    t[5] = p0 + 4 < K ? tkeys[p0 + 4] : 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t p = p0 + i;
      if (p >= K) break;
      const uint32_t cur = t[1 + i];
      const bool first = t[i] != cur, last = t[2 + i] != cur;
      if (!(first || last || keys)) continue;
      const uint32_t tile = tile_of_key(bd, cur);
      UT_DBG_CHECK(tile < (uint32_t)bd.total_tiles, UT_DBG_TILE_ID, tile, bd.total_tiles, 0);
      if (first) ranges[2 * tile] = p;
      if (last) ranges[2 * tile + 1] = p + 1;
      if (keys) {
        const int v = view_of_tile(bd, (int)tile);
        keys[p] = ((uint64_t)tile << 32) | (uint64_t)__float_as_uint(depth[bd.v[v].part_off + vals[p]]);
      }
    }
  }
}

// ---------------------------------------------------------------- row scatter
//
// The row stage without materialising the row entries.  The column keys carry each entry's
// first tile row a and row count h next to the column; the column-sorted list is split into
// CH chunks per tile column, one warp per chunk.  k_row_count counts every chunk's entries per
// tile row; one exclusive scan over the (tile, chunk) counts in tile order gives each chunk's
// first position in each tile's run (and the tile ranges); k_row_scatter then walks the chunk
// 32 entries at a time (lanes in entry order): a lane's rank in row r among the 32 is the
// number of lower lanes covering r, read off the group's lane mask of r, so every (entry, row)
// pair lands at its (tile, depth) position.

constexpr int kScatterMaxRows = 512;       // tile rows per view handled by the scatter
constexpr int kScatterMaxCols = 1 << 14;   // tile columns per batch handled by the scatter
constexpr int kPackColBits = 14, kPackRowBits = 9;

// Packed column key: global tile column | a << 14 | (h - 1) << 23.
__device__ __forceinline__ uint32_t pk_col(uint32_t key) { return key & ((1u << kPackColBits) - 1u); }
__device__ __forceinline__ uint32_t pk_a(uint32_t key) { return (key >> kPackColBits) & ((1u << kPackRowBits) - 1u); }
__device__ __forceinline__ uint32_t pk_h(uint32_t key) { return (key >> (kPackColBits + kPackRowBits)) + 1u; }

// Chunk plan of the row stage (device scratch, written by k_chunk_plan): the column list is
// cut into about kChunkWarps chunks of similar length (a column of m entries gets
// ceil(m / target) chunks, target = max(32, ceil(M / kChunkWarps))), one warp each.  The
// (tile, chunk) counts are laid out in tile order: view v's part starts at voff[v], then per
// tile row the view's columns in order, each with its chunks, so that position of chunk k of
// column c in row r = voff[v] + r * vch[v] + (co[c] - co[col_off_v]) + k.
constexpr int kChunkWarps = 8192;

struct ChunkPlan {
  uint32_t *ch;         // [cols] chunks of each column
  uint32_t *co;         // [cols + 1] exclusive prefix of ch
  uint32_t *chunk_col;  // [kChunkWarps + cols] column of every chunk
  uint32_t *voff, *vch; // [kMaxViews] spine offset and chunks per tile row of every view
  u64 *len;             // [2] spine length, number of chunks
};

inline size_t plan_spine_words(int max_rows, int tiles, int cols) {
  return (size_t)(max_rows > 0 ? max_rows : 1) * (size_t)kChunkWarps + (size_t)(tiles > 0 ? tiles : 1) +
         (size_t)(cols > 0 ? cols : 1);
}

__device__ __forceinline__ uint32_t spine_pos(const ChunkPlan &pl, const DevView &v, int vi, int c, uint32_t r) {
  return pl.voff[vi] + r * pl.vch[vi] + (pl.co[c] - pl.co[v.col_off]);
}

// Entry range of chunk k of global tile column c (colb: first / end entry of each column).
__device__ __forceinline__ void chunk_range(const uint32_t *colb, int c, uint32_t k, uint32_t ch, uint32_t &lo,
                                            uint32_t &hi) {
  const uint32_t a = colb[2 * c], e = colb[2 * c + 1];
  const u64 m = e - a;
  lo = a + (uint32_t)(m * (u64)k / (u64)ch);
  hi = a + (uint32_t)(m * (u64)(k + 1) / (u64)ch);
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// First and end entry of every global tile column in the sorted packed column keys (columns
// left at {0, 0} when empty); four keys per thread and their neighbours.
__global__ void k_col_bounds(const uint32_t *__restrict__ ckeys, Count cc, uint32_t *__restrict__ colb) {
  const uint32_t M = cc.get();
  const uint32_t nq = (M + 3) / 4;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint32_t p0 = 4 * q;
    uint32_t t[6];  // columns of entries p0 - 1 .. p0 + 4 (0xffffffff outside the list)
    if (p0 + 4 <= M) {
      const uint4 v = reinterpret_cast<const uint4 *>(ckeys)[q];
      t[1] = pk_col(v.x); t[2] = pk_col(v.y); t[3] = pk_col(v.z); t[4] = pk_col(v.w);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) t[1 + i] = p0 + i < M ? pk_col(ckeys[p0 + i]) : 0xffffffffu;
    }
    t[0] = p0 > 0 ? pk_col(ckeys[p0 - 1]) : 0xffffffffu;
    t[5] = p0 + 4 < M ? pk_col(ckeys[p0 + 4]) : 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t p = p0 + i;
      if (p >= M) break;
      if (t[i] != t[1 + i]) colb[2 * t[1 + i]] = p;
      if (t[2 + i] != t[1 + i]) colb[2 * t[1 + i] + 1] = p + 1;
    }
  }
}

// The chunk plan from the column bounds (one block of 1024 threads).  With dspine, the column
// order came from one radix pass over all column bits, and the bounds are read off its scanned
// digit-major counts instead (column c starts at dspine[c * tiles], tiles = radix tiles of the
// M column entries) and written to colb here; with raw, dspine holds the pass's unscanned
// counts (the short pass derived its offsets itself) and the bounds come from the exclusive
// scan of the per-column totals.
__global__ void __launch_bounds__(1024) k_chunk_plan(const __grid_constant__ BatchDesc bd, uint32_t *__restrict__ colb,
                                                     ChunkPlan pl, const uint32_t *__restrict__ dspine, int ndigits,
                                                     Count mcnt, int raw) {
  __shared__ u64 s_w[33];
  __shared__ u64 s_tot;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, cols = bd.total_cols;
  if (dspine && !raw) {
    const uint32_t M = mcnt.get(), nt = (M + kRTile - 1) / kRTile;
    for (int c = t; c < cols; c += 1024) {
      const uint32_t a = M ? dspine[(size_t)c * nt] : 0u;
      const uint32_t e = !M ? 0u : (c + 1 < ndigits ? dspine[(size_t)(c + 1) * nt] : M);
      colb[2 * c] = a;
      colb[2 * c + 1] = e;
    }
    __syncthreads();
  } else if (dspine) {
    const uint32_t M = mcnt.get(), nt = (M + kRTile - 1) / kRTile;
    u64 carry = 0;
    for (int c0 = 0; c0 < cols; c0 += 1024) {
      const int c = c0 + t;
      uint32_t tot = 0;
      if (c < cols)
        for (uint32_t tt = 0; tt < nt; ++tt) tot += dspine[(size_t)c * nt + tt];
      const u64 inc = warp_incl_scan_u64((u64)tot, lane);
      if (lane == 31) s_w[warp] = inc;
      __syncthreads();
      if (warp == 0) {
        const u64 w = s_w[lane];
        const u64 wi = warp_incl_scan_u64(w, lane);
        s_w[lane] = wi - w;
        if (lane == 31) s_w[32] = wi;
      }
      __syncthreads();
      if (c < cols) {
        const uint32_t a = (uint32_t)(carry + s_w[warp] + inc - tot);
        colb[2 * c] = a;
        colb[2 * c + 1] = a + tot;
      }
      carry += s_w[32];
      __syncthreads();
    }
  }
  auto block_sum = [&](u64 x) -> u64 {
    x = warp_incl_scan_u64(x, lane);
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (t == 0) {
      u64 a = 0;
      for (int w = 0; w < 32; ++w) a += s_w[w];
      s_tot = a;
    }
    __syncthreads();
    const u64 r = s_tot;
    __syncthreads();
    return r;
  };
  u64 m = 0;
  for (int c = t; c < cols; c += 1024) m += colb[2 * c + 1] - colb[2 * c];
  const u64 M = block_sum(m);
  const u64 target = M / kChunkWarps + 1 > 32 ? M / kChunkWarps + 1 : 32;
  // chunks per column and their exclusive prefix
  u64 carry = 0;
  for (int c0 = 0; c0 < cols; c0 += 1024) {
    const int c = c0 + t;
    uint32_t n = 0;
    if (c < cols) {
      const u64 mc = colb[2 * c + 1] - colb[2 * c];
      n = (uint32_t)((mc + target - 1) / target);
      pl.ch[c] = n;
    }
    u64 inc = warp_incl_scan_u64((u64)n, lane);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const u64 w = s_w[lane];
      const u64 wi = warp_incl_scan_u64(w, lane);
      s_w[lane] = wi - w;
      if (lane == 31) s_w[32] = wi;
    }
    __syncthreads();
    if (c < cols) pl.co[c] = (uint32_t)(carry + s_w[warp] + inc - n);
    carry += s_w[32];
    __syncthreads();
  }
  if (t == 0) pl.co[cols] = (uint32_t)carry;
  __syncthreads();
  if (t == 0) {
    u64 off = 0;
    for (int v = 0; v < bd.nv; ++v) {
      const uint32_t chv = pl.co[bd.v[v].col_off + bd.v[v].tiles_x] - pl.co[bd.v[v].col_off];
      pl.voff[v] = (uint32_t)off;
      pl.vch[v] = chv;
      off += (u64)chv * (u64)bd.v[v].tiles_y;
    }
    pl.len[0] = off;
    pl.len[1] = carry;
  }
  for (int c = t; c < cols; c += 1024) {
    const uint32_t o = pl.co[c], n = pl.ch[c];
    for (uint32_t k = 0; k < n; ++k) pl.chunk_col[o + k] = (uint32_t)c;
  }
}

// Entries of every chunk in every tile of its column, at the chunk's spine positions (one warp
// per chunk; dynamic shared memory kWarps x (max rows + 1) words).
__global__ void __launch_bounds__(kThreads) k_row_count(const __grid_constant__ BatchDesc bd,
                                                        const uint32_t *__restrict__ ck,
                                                        const uint32_t *__restrict__ colb, ChunkPlan pl,
                                                        int max_rows, uint32_t *__restrict__ spine) {
  extern __shared__ uint32_t s_mem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wid = blockIdx.x * kWarps + warp;
  if (wid >= (uint32_t)pl.len[1]) return;
  const int c = (int)pl.chunk_col[wid];
  const uint32_t k = wid - pl.co[c];
  const int vi = view_of_col(bd, c);
  const DevView &v = bd.v[vi];
  const int rows = v.tiles_y;
  uint32_t *D = s_mem + (size_t)warp * (max_rows + 1);
  for (int r = lane; r <= rows; r += 32) D[r] = 0;
  __syncwarp();
  uint32_t lo, hi;
  chunk_range(colb, c, k, pl.ch[c], lo, hi);
  for (uint32_t i = lo + lane; i < hi; i += 32) {
    const uint32_t key = ck[i], a = pk_a(key);
    atomicAdd(&D[a], 1u);
    atomicAdd(&D[a + pk_h(key)], 0xffffffffu);
  }
  __syncwarp();
  const uint32_t base = spine_pos(pl, v, vi, c, 0) + k;
  uint32_t carry = 0;
  for (int r0 = 0; r0 < rows; r0 += 32) {
    const int r = r0 + lane;
    const uint32_t x = warp_incl_scan_u32(r < rows ? D[r] : 0u, lane) + carry;
    if (r < rows) spine[base + (uint32_t)r * pl.vch[vi]] = x;
    carry = __shfl_sync(0xffffffffu, x, 31);
  }
}

// Stable expansion of a warp's run of entries [lo, hi) — each covering the bins [a, b) — into
// (entry, bin) outputs at each bin's next output position G[bin] (the row scatter's core).  The
// warp takes windows of consecutive 32-entry groups whose outputs fit kStage: it counts the
// window's outputs per bin, then per group each lane marks its bins in the group's lane masks
// and places each of its bins at the bin's next staging slot plus its rank among the group's
// lanes covering the bin; the staged window, bin-major, then goes out in contiguous runs (a
// group that alone exceeds kStage is written directly).  Per-warp shared memory: D (bins + 1)
// window counts, G (bins) next global positions, OW (bins) {next slot, group lane mask}, st
// (kStage) staged outputs.  The policy P supplies load(e, a, b, x, y) (bins and two payload
// words of entry e), stage(x, y, a, bin) (the staged form of one output), bin_of(staged) and
// emit(pos, staged).
constexpr int kStage = 512;

__host__ __device__ inline size_t scatter_words(int bins) {
  return ((2 * (size_t)bins + 2) & ~(size_t)1) + 2 * (size_t)bins + 2 * (size_t)kStage;
}

struct ScatterSmem {
  uint32_t *D, *G;
  uint2 *OW, *st;
  __device__ ScatterSmem(uint32_t *base, int bins) {
    D = base;
    G = D + bins + 1;
    OW = reinterpret_cast<uint2 *>(D + ((2 * (size_t)bins + 2) & ~(size_t)1));  // 8-byte aligned
    st = OW + bins;
  }
};

template <class P>
__device__ __forceinline__ void scatter_windows(const P &pol, uint32_t lo, uint32_t hi, int nbins, const ScatterSmem &m,
                                                int lane) {
  const uint32_t full = 0xffffffffu, bit = 1u << lane, lt = bit - 1u;
  uint32_t *D = m.D, *G = m.G;
  uint2 *OW = m.OW, *st = m.st;
  uint32_t i = lo;
  while (i < hi) {
    // the window [i, j): outputs per bin (difference array in D), their total, bins [bmin, bend)
    uint32_t j = i, tot = 0;
    int bmin = nbins, bend = 0;
    while (j < hi) {
      uint32_t a = 0, b = 0, x, y;
      if (j + lane < hi) pol.load(j + lane, a, b, x, y);
      const uint32_t gs = __reduce_add_sync(full, b - a);
      if (tot > 0 && tot + gs > (uint32_t)kStage) break;
      if (b > a) {
        atomicAdd(&D[a], 1u);
        atomicAdd(&D[b], 0xffffffffu);
      }
      bmin = min(bmin, (int)__reduce_min_sync(full, b > a ? a : (uint32_t)nbins));
      bend = max(bend, (int)__reduce_max_sync(full, b));
      tot += gs;
      j = hi - j > 32u ? j + 32u : hi;
      if (tot > (uint32_t)kStage) break;
    }
    __syncwarp();
    const bool direct = tot > (uint32_t)kStage;
    {  // counts (D) and each bin's first slot (bin-major staging offsets, or G when direct)
      uint32_t carry = 0, run = 0;
      for (int r0 = bmin; r0 < bend; r0 += 32) {
        const int r = r0 + lane;
        const uint32_t cnt = warp_incl_scan_u32(r < bend ? D[r] : 0u, lane) + carry;
        const uint32_t ci = warp_incl_scan_u32(r < bend ? cnt : 0u, lane);
        if (r < bend) {
          D[r] = cnt;
          OW[r].x = direct ? G[r] : run + ci - cnt;
        }
        carry = __shfl_sync(full, cnt, 31);
        run += __shfl_sync(full, ci, 31);
      }
      __syncwarp();
      if (lane == 0) D[bend] = 0;
      __syncwarp();
    }
    for (uint32_t g0 = i; g0 < j; g0 += 32) {
      uint32_t a = 0, b = 0, x = 0, y = 0;  // bins [a, b) of this lane's entry
      if (g0 + lane < j) pol.load(g0 + lane, a, b, x, y);
      for (uint32_t r = a; r < b; ++r) atomicOr(&OW[r].y, bit);
      __syncwarp();
      for (uint32_t r = a; r < b; ++r) {
        const uint2 ow = OW[r];
        const uint32_t q = ow.x + (uint32_t)__popc(ow.y & lt);
        if (direct) pol.emit(q, pol.stage(x, y, a, r));
        else if (q < (uint32_t)kStage) st[q] = pol.stage(x, y, a, r);
      }
      __syncwarp();
      for (int r = bmin + lane; r < bend; r += 32) {
        const uint2 ow = OW[r];
        if (ow.y) OW[r] = make_uint2(ow.x + (uint32_t)__popc(ow.y), 0u);
      }
      __syncwarp();
    }
    if (!direct) {
      // bin r's slots [first, first + D[r]) go to G[r]...: shift = G[r] - first slot
      for (int r = bmin + lane; r < bend; r += 32) OW[r].x = G[r] - (OW[r].x - D[r]);
      __syncwarp();
      for (uint32_t q = lane; q < tot; q += 32) {
        const uint2 e = st[q];
        pol.emit(OW[pol.bin_of(e)].x + q, e);
      }
      __syncwarp();
    }
    for (int r = bmin + lane; r < bend; r += 32) {
      G[r] += D[r];
      D[r] = 0;
      OW[r] = make_uint2(0u, 0u);
    }
    __syncwarp();
    i = j;
  }
}

// Row stage: entries = column entries (packed keys ck, flattened particle cv), bins = the
// view's tile rows, output = the particle's index within its scene (and the optional key).
struct RowPolicy {
  const uint32_t *ck, *cv;
  uint32_t *vals;
  uint64_t *keys;
  const float *depth;
  uint32_t part_off, tile0, tiles_x, kmax;
  __device__ void load(uint32_t e, uint32_t &a, uint32_t &b, uint32_t &x, uint32_t &y) const {
    const uint32_t key = ck[e];
    x = cv[e];
    y = 0;
    a = pk_a(key);
    b = a + pk_h(key);
  }
  __device__ uint2 stage(uint32_t x, uint32_t, uint32_t, uint32_t r) const { return make_uint2(x, r); }
  __device__ uint32_t bin_of(uint2 s) const { return s.y; }
  __device__ void emit(uint32_t pos, uint2 s) const {
    UT_DBG_CHECK(pos < kmax, UT_DBG_KEY_INDEX, pos, kmax, 2);
    if (pos >= kmax) return;  // every position is below K; the tests only guard the stores
    vals[pos] = s.x - part_off;
    if (keys) keys[pos] = ((u64)(tile0 + s.y * tiles_x) << 32) | (u64)__float_as_uint(depth[s.x]);
  }
};

// Writes every row entry of every chunk at its sorted position (one warp per chunk, as
// k_row_count); chunk 0 of each column also writes the column's tile ranges.
inline size_t row_scatter_smem(int max_rows) { return sizeof(uint32_t) * (size_t)kWarps * scatter_words(max_rows); }

__global__ void __launch_bounds__(kThreads) k_row_scatter(const __grid_constant__ BatchDesc bd,
                                                          const uint32_t *__restrict__ ck,
                                                          const uint32_t *__restrict__ cv,
                                                          const uint32_t *__restrict__ colb, ChunkPlan pl,
                                                          int max_rows, const uint32_t *__restrict__ spine,
                                                          Count kcnt, const float *__restrict__ depth,
                                                          uint32_t *__restrict__ vals, uint32_t *__restrict__ ranges,
                                                          uint64_t *__restrict__ keys, const u64 *__restrict__ ktotal,
                                                          int64_t *__restrict__ k_out) {
  extern __shared__ uint2 s_mem2[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wid = blockIdx.x * kWarps + warp;
  if (wid == 0 && lane == 0) *k_out = (int64_t)*ktotal;  // K, also when it exceeds the capacity
  if (wid >= (uint32_t)pl.len[1]) return;
  const int c = (int)pl.chunk_col[wid];
  const uint32_t k = wid - pl.co[c], nch = pl.ch[c];
  const int vi = view_of_col(bd, c);
  const DevView &v = bd.v[vi];
  const int rows = v.tiles_y;
  const ScatterSmem m(reinterpret_cast<uint32_t *>(s_mem2) + (size_t)warp * scatter_words(max_rows), max_rows);
  const uint32_t tile0 = (uint32_t)v.tile_off + (uint32_t)(c - v.col_off);
  const uint32_t kmax = kcnt.get();
  const uint32_t base = spine_pos(pl, v, vi, c, 0), rstride = pl.vch[vi];
  const uint32_t slen = (uint32_t)pl.len[0];
  for (int r = lane; r <= rows; r += 32) {
    m.D[r] = 0;
    if (r == rows) break;
    m.OW[r] = make_uint2(0u, 0u);
    const uint32_t sp = base + (uint32_t)r * rstride;
    m.G[r] = spine[sp + k];
    if (k == 0) {  // the tile's run ends where the next tile's (the next spine position's) begins
      const uint32_t tile = tile0 + (uint32_t)r * v.tiles_x;
      const uint32_t start = spine[sp];
      const uint32_t end = sp + nch < slen ? spine[sp + nch] : kmax;
      if (start < end) {
        UT_DBG_CHECK(tile < (uint32_t)bd.total_tiles, UT_DBG_TILE_ID, tile, bd.total_tiles, 1);
        ranges[2 * tile] = start;
        ranges[2 * tile + 1] = end;
      }
    }
  }
  __syncwarp();
  uint32_t lo, hi;
  chunk_range(colb, c, k, nch, lo, hi);
  const RowPolicy pol{ck, cv, vals, keys, depth, (uint32_t)v.part_off, tile0, (uint32_t)v.tiles_x, kmax};
  scatter_windows(pol, lo, hi, rows, m, lane);
}

// ---------------------------------------------------------------- host orchestration

// Guard bytes after every sub-buffer of a debug build's binning workspace (their offsets).
constexpr int kMaxGuards = 48;
#ifdef UT_DEBUG
constexpr uint32_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xa5;
#endif
struct GuardList {
  int n = 0;
  uint32_t off[kMaxGuards];
};

struct Arena {
  char *p;
  size_t off;
  GuardList *guards = nullptr;
  template <class T>
  T *take(size_t count) {
    T *r = reinterpret_cast<T *>(p ? p + off : nullptr);
    off += align256(count * sizeof(T));
#ifdef UT_DEBUG
    if (guards && guards->n < kMaxGuards) guards->off[guards->n++] = (uint32_t)off;
    off += kGuardBytes;
#endif
    return r;
  }
};

#ifdef UT_DEBUG
// Debug build: every guard byte still kGuardByte, else UT_DBG_CANARY (guard, offset, byte).
__global__ void k_check_guards(const unsigned char *__restrict__ ws, GuardList g) {
  for (int i = 0; i < g.n; ++i)
    for (uint32_t b = threadIdx.x; b < kGuardBytes; b += blockDim.x) {
      const unsigned char v = ws[(size_t)g.off[i] + b];
      UT_DBG_CHECK(v == kGuardByte, UT_DBG_CANARY, i, b, v);
    }
}
#endif

inline uint32_t ceil_div(u64 a, u64 b) { return (uint32_t)((a + b - 1) / b); }

struct Buffers {
  GuardList guards;
  uint32_t *dk[2], *dv[2], *cnt, *offs, *x[3], *spine;
  uint32_t *colb, *tspine;  // row scatter: column bounds [2 x cols], (tile, chunk) counts
  ChunkPlan plan;
  u64 *chunk, *total;       // total[0] = column entries, total[1] = K
};

// Workspace layout; with ws == nullptr only the size is accumulated.
Buffers carve(void *ws, int n, int64_t cap, int tiles, int cols, int max_rows, size_t *bytes = nullptr) {
  Buffers b;
  Arena a{static_cast<char *>(ws), 0, &b.guards};
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t cc = (size_t)(cap > 0 ? cap : 1);
  size_t maxc = nn > cc ? nn : cc;
  for (int i = 0; i < 2; ++i) b.dk[i] = a.take<uint32_t>(nn);
  for (int i = 0; i < 2; ++i) b.dv[i] = a.take<uint32_t>(nn);
  b.cnt = a.take<uint32_t>(maxc);   // widths per particle, then heights per column entry
  b.offs = a.take<uint32_t>(maxc);  // their exclusive scans
  for (int i = 0; i < 3; ++i) b.x[i] = a.take<uint32_t>(cc);
  size_t spine = 256 * (size_t)ceil_div(maxc, kRTile);
  b.spine = a.take<uint32_t>(spine);
  const size_t ncol = (size_t)(cols > 0 ? cols : 1);
  const size_t tsp = plan_spine_words(max_rows, tiles, cols);
  b.colb = a.take<uint32_t>(2 * ncol);
  b.tspine = a.take<uint32_t>(tsp);
  b.plan.ch = a.take<uint32_t>(ncol);
  b.plan.co = a.take<uint32_t>(ncol + 1);
  b.plan.chunk_col = a.take<uint32_t>(kChunkWarps + ncol);
  b.plan.voff = a.take<uint32_t>(kMaxViews);
  b.plan.vch = a.take<uint32_t>(kMaxViews);
  b.plan.len = a.take<u64>(2);
  size_t maxlen = spine > maxc ? spine : maxc;
  if (tsp > maxlen) maxlen = tsp;
  b.chunk = a.take<u64>(ceil_div(maxlen, kTile) + 1);
  b.total = a.take<u64>(2);
  if (bytes) *bytes = a.off;
  return b;
}

size_t carve_bytes(int n, int64_t cap, int tiles, int cols, int max_rows) {
  size_t bytes = 0;
  carve(nullptr, n, cap, tiles, cols, max_rows, &bytes);
  return bytes;
}

int grid_for(u64 items, int per_block) {
  u64 need = (items + per_block - 1) / per_block;
  u64 cap = (u64)device_sm_count() * 8;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

template <class L, class X = Ident>
void scan(const uint32_t *in, uint32_t *out, L len, u64 max_len, u64 *chunk, u64 *total, cudaStream_t s) {
  int g = grid_for(max_len, kTile);
  k_scan_reduce<L, X><<<g, kThreads, 0, s>>>(in, len, chunk);
  if (ceil_div(max_len, kTile) <= kSelfPrefixChunks) {  // short chunk lists: no spine pass
    k_scan_down_self<L, X><<<g, kThreads, 0, s>>>(in, out, len, chunk, total);
    count_launches(2);
    return;
  }
  k_scan_spine<L><<<1, 1024, 0, s>>>(chunk, len, total);
  k_scan_down<L, X><<<g, kThreads, 0, s>>>(in, out, len, chunk);
  count_launches(3);
}

// Sorts (keys, vals) in place across the two buffers; returns the buffer index holding the result.
// Bits [shift0, shift0 + bits) of the keys are sorted.  With self_offsets, lists of at most
// kSelfRadixTiles radix tiles skip the spine scan (the downsweep derives its offsets; the spine
// is then left unscanned, so callers that read it afterwards pass false).
int radix_sort(uint32_t *keys[2], uint32_t *vals[2], Count cnt, u64 max_count, int shift0, int bits,
               uint32_t *spine, u64 *chunk, cudaStream_t s, bool self_offsets = false) {
  int cur = 0;
  int g = grid_for(max_count, kRTile);
  const bool self = self_offsets && ceil_div(max_count, kRTile) <= kSelfRadixTiles;
  for (int shift = shift0; shift < shift0 + bits; shift += kRadixBits) {
    int db = shift0 + bits - shift < kRadixBits ? shift0 + bits - shift : kRadixBits;
    uint32_t mask = (1u << db) - 1u;
    k_radix_upsweep<<<g, kThreads, 0, s>>>(keys[cur], cnt, shift, mask, spine);
    if (self) {
      k_radix_downsweep<true><<<g, kThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], cnt, shift,
                                                    mask, spine);
    } else {
      SpineLen sl{cnt, (int)mask + 1};
      scan(spine, spine, sl, (u64)(mask + 1) * ceil_div(max_count, kRTile), chunk, nullptr, s);
      k_radix_downsweep<false><<<g, kThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], cnt,
                                                     shift, mask, spine);
    }
    count_launches(2);
    cur ^= 1;
  }
  return cur;
}

int bits_for(int tiles) {
  int b = 0;
  while ((1ll << b) < (long long)tiles) ++b;
  return b;
}

}  // namespace

size_t bin_workspace_bytes(int n, int64_t cap, int tiles, int cols, int max_rows) {
  return carve_bytes(n, cap, tiles, cols, max_rows);
}

ut_status launch_bin(const BatchDesc &bd, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                     const DevOpts &op, void *ws, int64_t cap, uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                     int64_t *k_out, cudaStream_t s, bool short_sort) {
  const int n = bd.total_particles;
  const int tiles = bd.total_tiles;
  const short4 *r4 = reinterpret_cast<const short4 *>(rect);
  int max_rows = 0;
  for (int v = 0; v < bd.nv; ++v) max_rows = bd.v[v].tiles_y > max_rows ? bd.v[v].tiles_y : max_rows;
  Buffers b = carve(ws, n, cap, tiles, bd.total_cols, max_rows);
#ifdef UT_DEBUG
  for (int i = 0; i < b.guards.n; ++i)
    if (cudaMemsetAsync(static_cast<char *>(ws) + b.guards.off[i], kGuardByte, kGuardBytes, s) != cudaSuccess)
      return UT_ERR_CUDA;
  struct GuardCheck {  // checks the guards when launch_bin returns
    const Buffers &b;
    void *ws;
    cudaStream_t s;
    ~GuardCheck() { k_check_guards<<<1, 256, 0, s>>>(static_cast<const unsigned char *>(ws), b.guards); }
  } guard_check{b, ws, s};
#endif
  if (cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles, s) != cudaSuccess) return UT_ERR_CUDA;
  if (cudaMemsetAsync(b.total, 0, 2 * sizeof(u64), s) != cudaSuccess) return UT_ERR_CUDA;
  if (n > 0) {
    const int g = grid_for(n, kThreads);
    const Count cn{nullptr, 0, (uint32_t)n};
    // depth keys, and K = sum of ntiles (reported even when it exceeds the capacity)
    k_depth_init<<<g, kThreads, 0, s>>>(n, depth, ntiles, b.dk[0], b.dv[0], b.total + 1);
    count_launches(1);
    const int r = radix_sort(b.dk, b.dv, cn, (u64)n, 0, 32, b.spine, b.chunk, s, short_sort);
    // buffer plan: column keys ping-pong in x[0] / x[1]; values (column, then row) over x[2]
    // and the caller's vals, arranged so that the row stage lands in vals: the row scatter
    // reads the column values from x[2]; the row radix passes end in vals
    const bool scatter = max_rows <= kScatterMaxRows && bd.total_cols <= kScatterMaxCols;
    const int cbits = bits_for(bd.total_cols), rbits = bits_for(bd.total_rows);
    const int cp = (cbits + kRadixBits - 1) / kRadixBits, rp = (rbits + kRadixBits - 1) / kRadixBits;
    uint32_t *r0 = (scatter || (rp & 1)) ? b.x[2] : vals;  // row values start here ...
    uint32_t *r1 = r0 == vals ? b.x[2] : vals;               // ... and end in vals
    uint32_t *cv[2], *ck[2] = {b.x[0], b.x[1]};
    cv[0] = (cp & 1) ? (scatter ? r1 : r0) : (scatter ? r0 : r1);  // column values end in x[2] / r1
    cv[1] = cv[0] == r0 ? r1 : r0;
    // 2. column entries in depth order, sorted by global tile column
    k_gather_widths<<<g, kThreads, 0, s>>>(n, b.dv[r], ntiles, r4, op.tile_w, b.cnt);
    count_launches(1);
    scan(b.cnt, b.offs, cn, (u64)n, b.chunk, b.total, s);
    const Count cc{b.total, (u64)cap, 0, b.total + 1};  // nothing is written unless K fits
    const int eg = (int)std::min<u64>((u64)(n + kThreads - 1) / kThreads, (u64)device_sm_count() * 16);
    if (scatter)
      k_emit_cols<true><<<eg, kThreads, 0, s>>>(bd, n, b.dv[r], b.offs, b.cnt, r4, cc, op.tile_w, op.tile_h, ck[0],
                                                cv[0]);
    else
      k_emit_cols<false><<<eg, kThreads, 0, s>>>(bd, n, b.dv[r], b.offs, b.cnt, r4, cc, op.tile_w, op.tile_h, ck[0],
                                                 cv[0]);
    count_launches(1);
    // the short pass leaves the spine unscanned: only the single-pass scatter path reads it, raw
    const bool col_short = short_sort && scatter && cp == 1 && ceil_div((u64)cap, kRTile) <= kSelfRadixTiles;
    const int rc = radix_sort(ck, cv, cc, (u64)cap, 0, cbits, b.spine, b.chunk, s, col_short);
    const Count ck2{b.total + 1, (u64)cap, 0};
    if (scatter) {
      // 3. row entries scattered straight into (tile, depth) order
      const uint32_t *ckc = ck[rc], *cvc = cv[rc];
      const int blocks = (kChunkWarps + bd.total_cols + kWarps - 1) / kWarps;
      if (cp == 1) {  // bounds from the single column pass's digit counts
        k_chunk_plan<<<1, 1024, 0, s>>>(bd, b.colb, b.plan, b.spine, 1 << cbits, cc, col_short ? 1 : 0);
      } else {
        if (cudaMemsetAsync(b.colb, 0, sizeof(uint32_t) * 2 * (size_t)bd.total_cols, s) != cudaSuccess)
          return UT_ERR_CUDA;
        k_col_bounds<<<grid_for((u64)cap, kThreads * 4), kThreads, 0, s>>>(ckc, cc, b.colb);
        k_chunk_plan<<<1, 1024, 0, s>>>(bd, b.colb, b.plan, nullptr, 0, cc, 0);
        count_launches(1);
      }
      k_row_count<<<blocks, kThreads, sizeof(uint32_t) * kWarps * (max_rows + 1), s>>>(bd, ckc, b.colb, b.plan,
                                                                                       max_rows, b.tspine);
      count_launches(2);
      const u64 tmax = plan_spine_words(max_rows, tiles, bd.total_cols);
      scan(b.tspine, b.tspine, Count{b.plan.len, tmax, 0}, tmax, b.chunk, nullptr, s);
      const size_t smem = row_scatter_smem(max_rows);
      if (cudaFuncSetAttribute(k_row_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return UT_ERR_CUDA;
      k_row_scatter<<<blocks, kThreads, smem, s>>>(bd, ckc, cvc, b.colb, b.plan, max_rows, b.tspine, ck2, depth,
                                                   vals, ranges, keys, b.total + 1, k_out);
      count_launches(1);
      return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
    }
    // 3. row entries in (column, depth) order, sorted by global tile row; the run lengths are
    //    the heights carried in the column keys
    scan<Count, High16>(ck[rc], b.offs, cc, (u64)cap, b.chunk, nullptr, s);
    uint32_t *rk[2] = {ck[rc ^ 1], ck[rc]}, *rv[2] = {r0, r1};
    const int rg = (int)std::min<u64>(((u64)cap + kThreads - 1) / kThreads, (u64)device_sm_count() * 16);
    k_emit_rows<<<rg, kThreads, 0, s>>>(bd, cc, ck[rc], cv[rc], b.offs, r4, ck2, op.tile_h, rk[0], rv[0]);
    count_launches(1);
    const int rr = radix_sort(rk, rv, ck2, (u64)cap, bd.col_bits, rbits, b.spine, b.chunk, s);
    k_ranges<<<grid_for((u64)cap, kThreads * 4), kThreads, 0, s>>>(bd, rk[rr], rv[rr], ck2, depth, ranges, keys);
    count_launches(1);
  }
  k_write_kout<<<1, 1, 0, s>>>(b.total + 1, k_out);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

UT_DBG_READER(dbg_read_binsort)

ut_status dbg_check_bin_guards(const void *ws, int n, int64_t cap, int tiles, int cols, int max_rows,
                               cudaStream_t stream) {
#ifdef UT_DEBUG
  const Buffers b = carve(const_cast<void *>(ws), n, cap, tiles, cols, max_rows);
  k_check_guards<<<1, 256, 0, stream>>>(static_cast<const unsigned char *>(ws), b.guards);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
#else
  (void)ws; (void)n; (void)cap; (void)tiles; (void)cols; (void)max_rows; (void)stream;
  return UT_ERR_UNSUPPORTED;
#endif
}

}  // namespace ut3d
