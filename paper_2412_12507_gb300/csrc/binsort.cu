// binsort.cu — duplicate (tile | depth) keys, sort them, find per-tile ranges
// (Sec. 4.3; the Duplicate and Sort phases of Table 2).
//
// The result equals a stable sort of key = (tile << 32) | bits(depth) over the entries
// emitted per particle in index order and per tile in row-major order, but it is
// computed in two cheaper steps:
//   1. a stable LSD radix sort of the N particle depths (bits(depth), index);
//   2. emission of the K (tile, particle) entries in that depth order, then a stable
//      LSD radix sort on the tile id alone (ceil(log2 T) bits instead of 32 + log2 T).
// Both orders are (tile, bits(depth), particle index), so the outputs are identical,
// while step 2 moves 8 bytes per entry per pass over ceil(log2 T / 8) passes instead of
// 12 bytes over ceil((32 + log2 T) / 8) passes.
//
// The radix sort is the project's own: per 8-bit digit pass an upsweep (per-warp shared
// histograms fed by uint4 key loads), a digit-major exclusive scan, and a downsweep that
// ranks keys stably in shared memory (same-digit lanes found with 8 ballots per 32-key group,
// per-warp running digit counters) and writes them out digit-grouped for coalescing.
// No kernel waits on another block, so nothing in here can spin.
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

// Element count of a pass: a host constant, or a device total that is honoured only if
// it fits the caller's capacity (0 otherwise, so an overflowing call writes nothing).
struct Count {
  const u64 *dev;
  u64 cap;
  uint32_t host;
  __device__ __forceinline__ uint32_t get() const {
    if (!dev) return host;
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

template <class L>
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
      if (p < n) s += in[p];
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

template <class L>
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
      s_v[skew(q)] = p < n ? in[p] : 0u;
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
// read as uint4; every warp counts into its own shared histogram.
__global__ void __launch_bounds__(kThreads) k_radix_upsweep(const uint32_t *__restrict__ keys, Count cnt, int shift,
                                                            uint32_t mask, uint32_t *__restrict__ counts) {
  __shared__ uint32_t s_wh[kWarps][256];
  const uint32_t n = cnt.get();
  const uint32_t nb = (n + kRTile - 1) / kRTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *wh = s_wh[warp];
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    for (int d = lane; d < 256; d += 32) wh[d] = 0;
    __syncwarp();
    const uint32_t base = b * kRTile;
    if (base + kRTile <= n) {
      const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
      for (int i = 0; i < kRIPT / 4; ++i) {
        uint4 q = k4[i * kThreads + threadIdx.x];
        atomicAdd(&wh[(q.x >> shift) & mask], 1u);
        atomicAdd(&wh[(q.y >> shift) & mask], 1u);
        atomicAdd(&wh[(q.z >> shift) & mask], 1u);
        atomicAdd(&wh[(q.w >> shift) & mask], 1u);
      }
    } else {
      for (uint32_t p = base + threadIdx.x; p < n; p += kThreads) atomicAdd(&wh[(keys[p] >> shift) & mask], 1u);
    }
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
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint32_t base = b * kRTile;
    uint32_t k[kRIPT], v[kRIPT], rank[kRIPT];
#pragma unroll
    for (int i = 0; i < kRIPT; ++i) {
      uint32_t p = base + warp * (kRIPT * 32) + i * 32 + lane;
      bool valid = p < n;
      k[i] = valid ? keys_in[p] : 0xffffffffu;
      v[i] = valid ? vals_in[p] : 0u;
    }
    for (int d = lane; d < nd; d += 32) s_whist[warp][d] = 0;
    __syncwarp();
    // stable rank of every key among the same-digit keys of this warp's segment
#pragma unroll
    for (int i = 0; i < kRIPT; ++i) {
      const uint32_t d = (k[i] >> shift) & mask;
      const uint32_t peers = digit_peers(d);
      const uint32_t before = s_whist[warp][d];
      rank[i] = before + (uint32_t)__popc(peers & lt_mask);
      __syncwarp();
      if (lane == __ffs(peers) - 1) s_whist[warp][d] = before + (uint32_t)__popc(peers);
      __syncwarp();
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
      s_goff[threadIdx.x] = offsets[(size_t)threadIdx.x * nb + b];
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
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kRTile, n - base);
    for (uint32_t j = threadIdx.x; j < nvalid; j += kThreads) {
      uint32_t kk = s_k[j];
      uint32_t d = (kk >> shift) & mask;
      uint32_t g = s_goff[d] + j - s_dstart[d];
      keys_out[g] = kk;
      vals_out[g] = s_v[j];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- binning kernels

__global__ void k_depth_init(int n, const float *__restrict__ depth, const uint32_t *__restrict__ ntiles,
                             uint32_t *__restrict__ dk, uint32_t *__restrict__ dv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    dk[i] = ntiles[i] > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
    dv[i] = (uint32_t)i;
  }
}

__global__ void k_gather_counts(int n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ ntiles,
                                uint32_t *__restrict__ cnt) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) cnt[j] = ntiles[order[j]];
}

__global__ void k_write_kout(const u64 *__restrict__ total, int64_t *__restrict__ k_out) { *k_out = (int64_t)*total; }

// One warp per particle of the depth order: the warp fills the particle's contiguous run of
// entries [offs[j], offs[j+1]) with consecutive lanes (coalesced), tiles in row-major order.
// Entries of a batch: `order` holds flattened (view, particle) indices; the emitted key is
// the global tile id (view's tile offset + row-major tile in the view) and the value is the
// particle index within its scene.
__global__ void __launch_bounds__(kThreads) k_emit(const __grid_constant__ BatchDesc bd, int n,
                                                   const uint32_t *__restrict__ order,
                                                   const uint32_t *__restrict__ offs, const short4 *__restrict__ rect,
                                                   const u64 *__restrict__ total, u64 cap, int tile_w, int tile_h,
                                                   uint32_t *__restrict__ tkeys, uint32_t *__restrict__ vals) {
  const u64 K = *total;
  if (K > cap) return;
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int j0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; j0 < n; j0 += nw * 32) {
    // every lane fetches one of the 32 particles (independent loads in flight together)
    const int j = j0 + lane;
    uint32_t start = 0, cnt = 0, local = 0;
    int base = 0, w = 1, tiles_x = 0;
    if (j < n) {
      start = offs[j];
      const uint32_t end = (j + 1 < n) ? offs[j + 1] : (uint32_t)K;
      cnt = end - start;
      if (cnt) {
        const uint32_t g = order[j];
        const short4 r = rect[g];
        const DevView &view = bd.v[view_of_particle(bd, (int)g)];
        local = g - (uint32_t)view.part_off;
        const int tx0 = r.x / tile_w, tx1 = r.z / tile_w, ty0 = r.y / tile_h;
        w = tx1 - tx0 + 1;
        tiles_x = view.tiles_x;
        base = view.tile_off + ty0 * tiles_x + tx0;
      }
    }
    // then the warp writes the particles' runs one after the other, lanes over the run
    uint32_t todo = __ballot_sync(0xffffffffu, cnt > 0);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t s0 = __shfl_sync(0xffffffffu, start, src);
      const uint32_t c0 = __shfl_sync(0xffffffffu, cnt, src);
      const uint32_t l0 = __shfl_sync(0xffffffffu, local, src);
      const int b0 = __shfl_sync(0xffffffffu, base, src);
      const int w0 = __shfl_sync(0xffffffffu, w, src);
      const int tx_0 = __shfl_sync(0xffffffffu, tiles_x, src);
      const float inv_w = 1.f / (float)w0;
      for (uint32_t q = lane; q < c0; q += 32) {
        // row / column of the q-th tile of the rect: a float estimate, corrected to the exact quotient
        int ty = (int)(((float)q + 0.5f) * inv_w);
        if (ty * w0 > (int)q) --ty;
        else if ((ty + 1) * w0 <= (int)q) ++ty;
        const int tx = (int)q - ty * w0;
        tkeys[s0 + q] = (uint32_t)(b0 + ty * tx_0 + tx);
        vals[s0 + q] = l0;
      }
    }
  }
}

// Tile ranges from the sorted tile keys: four keys per thread (uint4) and their neighbours.
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
      if (t[i] != cur) ranges[2 * cur] = p;
      if (t[2 + i] != cur) ranges[2 * cur + 1] = p + 1;
      if (keys) {
        const int v = view_of_tile(bd, (int)cur);
        keys[p] = ((uint64_t)cur << 32) | (uint64_t)__float_as_uint(depth[bd.v[v].part_off + vals[p]]);
      }
    }
  }
}

// ---------------------------------------------------------------- host orchestration

struct Arena {
  char *p;
  size_t off;
  template <class T>
  T *take(size_t count) {
    T *r = reinterpret_cast<T *>(p ? p + off : nullptr);
    off += align256(count * sizeof(T));
    return r;
  }
};

inline uint32_t ceil_div(u64 a, u64 b) { return (uint32_t)((a + b - 1) / b); }

struct Buffers {
  uint32_t *dk[2], *dv[2], *cnt, *offs, *tk[2], *valt, *spine;
  u64 *chunk, *total;
};

Buffers carve(void *ws, int n, int64_t cap) {
  Arena a{static_cast<char *>(ws), 0};
  Buffers b;
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t cc = (size_t)(cap > 0 ? cap : 1);
  for (int i = 0; i < 2; ++i) b.dk[i] = a.take<uint32_t>(nn);
  for (int i = 0; i < 2; ++i) b.dv[i] = a.take<uint32_t>(nn);
  b.cnt = a.take<uint32_t>(nn);
  b.offs = a.take<uint32_t>(nn);
  for (int i = 0; i < 2; ++i) b.tk[i] = a.take<uint32_t>(cc);
  b.valt = a.take<uint32_t>(cc);
  size_t maxc = nn > cc ? nn : cc;
  size_t spine = 256 * (size_t)ceil_div(maxc, kRTile);
  b.spine = a.take<uint32_t>(spine);
  size_t maxlen = spine > maxc ? spine : maxc;
  b.chunk = a.take<u64>(ceil_div(maxlen, kTile) + 1);
  b.total = a.take<u64>(2);
  return b;
}

size_t carve_bytes(int n, int64_t cap) {
  Arena a{nullptr, 0};
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t cc = (size_t)(cap > 0 ? cap : 1);
  a.take<uint32_t>(nn); a.take<uint32_t>(nn); a.take<uint32_t>(nn); a.take<uint32_t>(nn);
  a.take<uint32_t>(nn); a.take<uint32_t>(nn);
  a.take<uint32_t>(cc); a.take<uint32_t>(cc); a.take<uint32_t>(cc);
  size_t maxc = nn > cc ? nn : cc;
  size_t spine = 256 * (size_t)ceil_div(maxc, kRTile);
  a.take<uint32_t>(spine);
  size_t maxlen = spine > maxc ? spine : maxc;
  a.take<u64>(ceil_div(maxlen, kTile) + 1);
  a.take<u64>(2);
  return a.off;
}

int grid_for(u64 items, int per_block) {
  u64 need = (items + per_block - 1) / per_block;
  u64 cap = (u64)device_sm_count() * 8;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

template <class L>
void scan(const uint32_t *in, uint32_t *out, L len, u64 max_len, u64 *chunk, u64 *total, cudaStream_t s) {
  int g = grid_for(max_len, kTile);
  k_scan_reduce<L><<<g, kThreads, 0, s>>>(in, len, chunk);
  k_scan_spine<L><<<1, 1024, 0, s>>>(chunk, len, total);
  k_scan_down<L><<<g, kThreads, 0, s>>>(in, out, len, chunk);
  count_launches(3);
}

// Sorts (keys, vals) in place across the two buffers; returns the buffer index holding the result.
int radix_sort(uint32_t *keys[2], uint32_t *vals[2], Count cnt, u64 max_count, int bits, uint32_t *spine, u64 *chunk,
               cudaStream_t s) {
  int cur = 0;
  int g = grid_for(max_count, kRTile);
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    int db = bits - shift < kRadixBits ? bits - shift : kRadixBits;
    uint32_t mask = (1u << db) - 1u;
    k_radix_upsweep<<<g, kThreads, 0, s>>>(keys[cur], cnt, shift, mask, spine);
    SpineLen sl{cnt, (int)mask + 1};
    scan(spine, spine, sl, (u64)(mask + 1) * ceil_div(max_count, kRTile), chunk, nullptr, s);
    k_radix_downsweep<<<g, kThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], cnt, shift, mask,
                                            spine);
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

size_t bin_workspace_bytes(int n, int64_t cap, int /*tiles*/) { return carve_bytes(n, cap); }

ut_status launch_bin(const BatchDesc &bd, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                     const DevOpts &op, void *ws, int64_t cap, uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                     int64_t *k_out, cudaStream_t s) {
  const int n = bd.total_particles;
  const int tiles = bd.total_tiles;
  Buffers b = carve(ws, n, cap);
  if (cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles, s) != cudaSuccess) return UT_ERR_CUDA;
  if (cudaMemsetAsync(b.total, 0, sizeof(u64), s) != cudaSuccess) return UT_ERR_CUDA;
  if (n > 0) {
    int g = grid_for(n, kThreads);
    k_depth_init<<<g, kThreads, 0, s>>>(n, depth, ntiles, b.dk[0], b.dv[0]);
    count_launches(1);
    Count cn{nullptr, 0, (uint32_t)n};
    int r = radix_sort(b.dk, b.dv, cn, (u64)n, 32, b.spine, b.chunk, s);
    k_gather_counts<<<g, kThreads, 0, s>>>(n, b.dv[r], ntiles, b.cnt);
    count_launches(1);
    scan(b.cnt, b.offs, cn, (u64)n, b.chunk, b.total, s);
    // tile sort: the final pass must land in the caller's vals buffer
    int tb = bits_for(tiles);
    int passes = (tb + kRadixBits - 1) / kRadixBits;
    uint32_t *tv[2];
    tv[passes & 1] = vals;
    tv[(passes & 1) ^ 1] = b.valt;
    const int eg = (int)std::min<u64>((u64)(n + kThreads - 1) / kThreads, (u64)device_sm_count() * 16);
    k_emit<<<eg, kThreads, 0, s>>>(bd, n, b.dv[r], b.offs,
                                                              reinterpret_cast<const short4 *>(rect), b.total,
                                                              (u64)cap, op.tile_w, op.tile_h, b.tk[0], tv[0]);
    count_launches(1);
    Count ck{b.total, (u64)cap, 0};
    int rr = radix_sort(b.tk, tv, ck, (u64)cap, tb, b.spine, b.chunk, s);
    k_ranges<<<grid_for((u64)cap, kThreads * 4), kThreads, 0, s>>>(bd, b.tk[rr], tv[rr], ck, depth, ranges, keys);
    count_launches(1);
  }
  k_write_kout<<<1, 1, 0, s>>>(b.total, k_out);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

}  // namespace ut3d
