// composite_bwd.cu — hand-written backward of the compositing (supplementary Sec. B) for a
// batch of views.
//
// The backward replays the forward IN FORWARD ORDER: the stored rgb and T_final give the
// suffix sums S_i = C - sum_{j<=i} c_j alpha_j T_j without dividing transmittances,
// and n_used tells each pixel where the forward stopped.  Per (particle, warp) the 13
// geometry partials are reduced with a transposing reduce-scatter and the 3 x (deg+1)^2 SH
// partials with a tensor-core contraction over the warp's pixels; both are accumulated
// across warps in shared memory and pushed to global memory with one atomic per value per
// (tile, particle).  A final per-particle kernel maps the accumulated dL/dM, dL/dmu,
// dL/dsigma onto log-scales, quaternions and logits.  Tiles run heaviest replay first.
#include <cuda_bf16.h>

#include "composite_common.cuh"

namespace ut3d {
namespace {

// Reduce-scatter of 16 per-lane values over the 32 lanes: afterwards lanes 2i and 2i+1 hold
// the warp total of value i.
__device__ __forceinline__ void warp_reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 16, L = 8; L >= 1; o >>= 1, L >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      float send = up ? v[j] : v[j + L];
      float keep = up ? v[j + L] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Two floats as bf16 pairs hi + lo (x = hi + lo to about 2^-17): the three-term products
// hi*hi + hi*lo + lo*hi keep FP32-level accuracy on the BF16 tensor-core path.
__device__ __forceinline__ void split_bf16x2(float x, float y, uint32_t &hi, uint32_t &lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  float2 hf = __bfloat1622float2(h);
  __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
  hi = *reinterpret_cast<uint32_t *>(&h);
  lo = *reinterpret_cast<uint32_t *>(&l);
}

// D += A B for one m16n8k16 BF16 tile (FP32 accumulate).
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kSlots = 8;     // particle columns of one tensor-core flush (the MMA's N)

// Float index of (row, col) in a warp's 32-column W tile: columns are XOR-swizzled by the row so
// that the fragment loads of four rows (8-byte pairs, 16 lanes per phase) hit distinct banks
// without padding.
__device__ __forceinline__ int wtile(int row, int col) { return row * 32 + (col ^ ((row & 3) << 3)); }

// Shared-memory layout of the backward kernel (dynamic; bytes for a block of `warps` warps).
// PP: per-particle colour mode (no SH coefficients staged, no W tiles).
template <int DEG, bool PP>
struct BwdSmem {
  static constexpr int NSH = (DEG + 1) * (DEG + 1);
  static constexpr int NC = NSH * 3;
  static constexpr int NST = PP ? 4 : NC;                   // staged colour floats per particle
  static constexpr int ACC = PP ? 17 : (16 + NC) | 1;      // accumulators per particle (odd: rows spread over banks)
  static __host__ __device__ size_t geo() { return 0; }
  static __host__ __device__ size_t aux() { return geo() + sizeof(float4) * 4 * kBatch; }
  static __host__ __device__ size_t sh() { return aux() + sizeof(float4) * kBatch; }
  static __host__ __device__ size_t acc() { return sh() + sizeof(float) * ((kBatch * NST + 3) / 4 * 4); }
  static __host__ __device__ size_t wmat() { return acc() + sizeof(float) * kBatch * ACC; }
  // per warp: 3 channels x kSlots rows of W (the first 16 rows double as the staging area of
  // Y), then the A fragments (uint4 [4][32]: hi/lo of both k-steps, lane-minor)
  static constexpr int kWRows = PP ? 0 : (3 * kSlots > 16 ? 3 * kSlots : 16);
  static constexpr int kWarpFloats = PP ? 0 : kWRows * 32 + 4 * 4 * 32;
  static __host__ __device__ size_t idx(int warps) { return wmat() + sizeof(float) * warps * kWarpFloats; }
  static __host__ __device__ size_t any(int warps) { return idx(warps) + sizeof(uint32_t) * kBatch; }
  static __host__ __device__ size_t bytes(int warps) { return any(warps) + sizeof(int) * kBatch; }
};

// Backward of k_composite_fwd for one tile.  Per (pixel, particle) pair the partials are
// dL/dbeta_k,c = w_c Y_k (w_c = dL/dc_c alpha T where the colour is not clamped), the 9
// products v x^T for dL/dM, v for dL/dmu and dL/dsigma.
//
// The SH part is a dense contraction over the warp's 32 pixels, D[k][j] = sum_p Y_k(p) W_c(p, j),
// run on the tensor cores (m16n8k16, BF16 hi/lo split with the three cross terms, FP32
// accumulate): A = Y^T (basis x pixels) is fixed for the tile and its fragments are parked in
// shared memory; B = W (pixels x particles) collects, column by column, only particles that
// reach at least one pixel of the warp, and is contracted once kSlots columns are full (and at
// the end of each staged batch).  The 13 geometry partials are summed with a 16-value
// reduce-scatter.  Both land in per-particle shared accumulators that are added to global
// memory once per (tile, particle).
// PP (per-particle colour mode): the colour gradient dL/dc is one 3-vector per particle, summed
// in the three spare slots of the reduce-scatter; at the per-(tile, particle) flush it becomes
// dL/dbeta = dL/dc Y(dir) and the mean's gradient through the view direction.
// SMALL: tiles of at most 256 pixels, compiled for three resident blocks per SM (80 registers).
template <int DEG, bool RS, bool SMALL, bool PP, bool GEN>
__global__ void __launch_bounds__(SMALL ? 256 : 512, SMALL ? 3 : 1)
    k_composite_bwd(const __grid_constant__ BatchDesc bd, DevOpts op,
                                                       const short4 *__restrict__ rect,
                                                       const uint32_t *__restrict__ vals,
                                                       const uint2 *__restrict__ ranges, TileSched ts) {
  using L = BwdSmem<DEG, PP>;
  constexpr int NSH = L::NSH;
  constexpr int NC = L::NC;
  constexpr int PDEG = PP ? 0 : DEG;  // per-pixel SH basis only when colours are per pixel
  constexpr int ACC = L::ACC;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warps = blockDim.x >> 5;
  float4(*s_geo)[4] = reinterpret_cast<float4(*)[4]>(smem + L::geo());
  float4 *s_aux = reinterpret_cast<float4 *>(smem + L::aux());
  float *s_sh = reinterpret_cast<float *>(smem + L::sh());
  float *s_acc = reinterpret_cast<float *>(smem + L::acc());
  uint32_t *s_idx = reinterpret_cast<uint32_t *>(smem + L::idx(warps));
  int *s_any = reinterpret_cast<int *>(smem + L::any(warps));

  // tiles in the order k_tile_order gave them (most list entries to replay first)
  if (blockIdx.x >= *ts.n_work) return;
  const int tile = (int)ts.order[blockIdx.x];
  UT_DBG_CHECK(tile < bd.total_tiles, UT_DBG_TILE_ID, tile, bd.total_tiles, 3);
  const DevView &view = bd.v[view_of_tile(bd, tile)];
  const DevScene &sc = bd.s[view.scene];
  const DevCam &cam = view.cam;
  const int lt = tile - view.tile_off;
  const int tx = lt % view.tiles_x, ty = lt / view.tiles_x;
  int lx, ly;
  tile_pixel(op, (int)threadIdx.x, lx, ly);
  const int px = tx * op.tile_w + lx;
  const int py = ty * op.tile_h + ly;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;
  float *s_W = reinterpret_cast<float *>(smem + L::wmat()) + (size_t)warp * L::kWarpFloats;
  uint4 *s_Af = reinterpret_cast<uint4 *>(s_W + L::kWRows * 32);
  const bool inside = px < cam.W && py < cam.H;
  float3 o, d;
  float Y[(PDEG + 1) * (PDEG + 1)];
  bool valid;
  pixel_setup<PDEG>(cam, op, px, py, inside, o, d, Y, valid);

  if constexpr (!PP) {
  // A operand (basis x pixels), fixed for the whole tile: the warp's Y transposed through
  // its W tile (row k = basis function k, column = lane), split into hi + lo fragments and
  // parked in shared memory (s_Af[2 ks + 0] = hi, s_Af[2 ks + 1] = lo)
#pragma unroll
  for (int k = 0; k < 16; ++k) s_W[wtile(k, lane)] = k < NSH ? Y[k < NSH ? k : 0] : 0.f;
  __syncwarp();
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const int c0 = 16 * ks + 2 * t4;
    uint4 hi, lo;
    split_bf16x2(s_W[wtile(g8, c0)], s_W[wtile(g8, c0 + 1)], hi.x, lo.x);
    split_bf16x2(s_W[wtile(g8 + 8, c0)], s_W[wtile(g8 + 8, c0 + 1)], hi.y, lo.y);
    split_bf16x2(s_W[wtile(g8, c0 + 8)], s_W[wtile(g8, c0 + 9)], hi.z, lo.z);
    split_bf16x2(s_W[wtile(g8 + 8, c0 + 8)], s_W[wtile(g8 + 8, c0 + 9)], hi.w, lo.w);
    s_Af[(2 * ks) * 32 + lane] = hi;
    s_Af[(2 * ks + 1) * 32 + lane] = lo;
  }
  __syncwarp();
  // W starts finite: unused columns of a partial flush only feed their own (discarded) outputs
#pragma unroll
  for (int r = 0; r < 3 * kSlots; ++r) s_W[wtile(r, lane)] = 0.f;
  }

  const uint2 rg = ranges[tile];
  uint32_t my_end = 0;
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, gAT = 0.f, Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f;  // gAT = dL/dalpha T_final
  if (valid) {
    size_t pix = (size_t)py * cam.W + px;
    size_t plane = (size_t)cam.W * cam.H;
    my_end = view.n_used[pix];
    g0 = view.d_rgb[pix]; g1 = view.d_rgb[plane + pix]; g2 = view.d_rgb[2 * plane + pix];
    gAT = view.d_alpha[pix] * view.tfinal[pix];
    Cf0 = view.rgb[pix]; Cf1 = view.rgb[plane + pix]; Cf2 = view.rgb[2 * plane + pix];
  }
  const uint32_t block_end = rg.x + ts.work[tile];
  uint32_t warp_end = my_end;  // no pixel of this warp blends a particle at or after warp_end
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) warp_end = max(warp_end, __shfl_xor_sync(0xffffffffu, warp_end, o));

  // Contracts the first `cols` columns of W with Y and adds them to the particles' SH
  // accumulators; lane s < kSlots holds in slot_b the batch index of column s.
  int slot_b = 0;
  auto flush = [&](int cols) {
    __syncwarp();
    float acc[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint4 h4 = s_Af[(2 * ks) * 32 + lane], l4 = s_Af[(2 * ks + 1) * 32 + lane];
      const uint32_t ahi[4] = {h4.x, h4.y, h4.z, h4.w}, alo[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int row = c * kSlots + g8, c0 = 16 * ks + 2 * t4;
        const float2 x0 = *reinterpret_cast<const float2 *>(s_W + wtile(row, c0));
        const float2 x1 = *reinterpret_cast<const float2 *>(s_W + wtile(row, c0 + 8));
        uint32_t bhi0, blo0, bhi1, blo1;
        split_bf16x2(x0.x, x0.y, bhi0, blo0);
        split_bf16x2(x1.x, x1.y, bhi1, blo1);
        mma_bf16(acc[c], ahi, bhi0, bhi1);
        mma_bf16(acc[c], ahi, blo0, blo1);
        mma_bf16(acc[c], alo, bhi0, bhi1);
      }
    }
    // acc[c][r]: basis g8 (+8 for r >= 2), column 2 t4 (+1 for odd r)
    const int bA = __shfl_sync(0xffffffffu, slot_b, 2 * t4), bB = __shfl_sync(0xffffffffu, slot_b, 2 * t4 + 1);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = g8 + (r >= 2 ? 8 : 0), col = 2 * t4 + (r & 1);
      if (k < NSH && col < cols) {
        float *dst = s_acc + (r & 1 ? bB : bA) * ACC + 16 + 3 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (acc[c][r] != 0.f) atomicAdd(dst + c, acc[c][r]);
      }
    }
    __syncwarp();
  };

  float T = 1.f, A0 = 0.f, A1 = 0.f, A2 = 0.f;  // running prefix of the composited colour
  for (uint32_t start = rg.x; start < block_end; start += kBatch) {
    const int nb = min((uint32_t)kBatch, block_end - start);
    __syncthreads();
    if (threadIdx.x < nb) s_idx[threadIdx.x] = vals[start + threadIdx.x];
    for (int f = threadIdx.x; f < kBatch * ACC; f += blockDim.x) s_acc[f] = 0.f;
    if (threadIdx.x < kBatch) s_any[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x < nb) {
      uint32_t idx = s_idx[threadIdx.x];
      stage_particle<RS>(sc, cam, op, rect[view.part_off + idx], idx, s_geo[threadIdx.x], &s_aux[threadIdx.x]);
      if (PP) reinterpret_cast<float4 *>(s_sh)[threadIdx.x] = particle_colour<DEG, RS>(sc, cam, op, idx);
    }
    if (!PP) stage_sh<NC>(sc, s_idx, nb, s_sh);
    __syncthreads();
    // particles of this batch any pixel of the warp can still blend (warp-uniform)
    const int nw = (int)min((uint32_t)nb, warp_end > start ? warp_end - start : 0u);
    int cols = 0;
    for (int b = 0; b < nw; ++b) {
      bool contrib = false;
      float vv[3] = {0.f, 0.f, 0.f}, xx[3] = {0.f, 0.f, 0.f}, wc[3] = {0.f, 0.f, 0.f}, dsig = 0.f;
      float3 og, dg;
      float dd, a;
      if (start + b < my_end && eval_response<RS, GEN>(s_geo[b], px, py, o, d, og, dg, dd, a, op)) {
        contrib = true;
        float al = fminf(a, op.alpha_max);
        float r0, r1, r2;
        if (PP) {
          const float4 cr = reinterpret_cast<const float4 *>(s_sh)[b];
          r0 = cr.x; r1 = cr.y; r2 = cr.z;
        } else {
          sh_colour<NSH>(s_sh + b * NC, Y, r0, r1, r2);
        }
        float c0 = fmaxf(r0, 0.f), c1 = fmaxf(r1, 0.f), c2 = fmaxf(r2, 0.f);
        float w = al * T;
        A0 = fmaf(c0, w, A0);
        A1 = fmaf(c1, w, A1);
        A2 = fmaf(c2, w, A2);
        const float inv = __fdividef(1.f, 1.f - al);  // 1 - al >= 1 - alpha_max > 0
        // dL/dalpha = sum_c g_c (c T - S_c / (1 - alpha)) + g_A T_final / (1 - alpha)
        float dal = g0 * fmaf(-(Cf0 - A0), inv, c0 * T) + g1 * fmaf(-(Cf1 - A1), inv, c1 * T) +
                    g2 * fmaf(-(Cf2 - A2), inv, c2 * T) + gAT * inv;
        wc[0] = r0 > 0.f ? g0 * w : 0.f;
        wc[1] = r1 > 0.f ? g1 * w : 0.f;
        wc[2] = r2 > 0.f ? g2 * w : 0.f;
        T = T * (1.f - al);
        float da = a > op.alpha_max ? 0.f : dal;
        float sigma = s_geo[b][3].x;
        dsig = da * __fdividef(a, sigma);
        float dw2 = dresponse<GEN>(op, a, og, dg, dd) * da;
        float tau = -__fdividef(dot3(og, dg), dd);
        float3 pp = make_float3(fmaf(tau, dg.x, og.x), fmaf(tau, dg.y, og.y), fmaf(tau, dg.z, og.z));
        vv[0] = 2.f * dw2 * pp.x;
        vv[1] = 2.f * dw2 * pp.y;
        vv[2] = 2.f * dw2 * pp.z;
        float4 ax = s_aux[b];
        if (RS) {
          xx[0] = fmaf(tau, d.x, o.x - ax.x);
          xx[1] = fmaf(tau, d.y, o.y - ax.y);
          xx[2] = fmaf(tau, d.z, o.z - ax.z);
        } else {
          xx[0] = fmaf(tau, d.x, ax.x);
          xx[1] = fmaf(tau, d.y, ax.y);
          xx[2] = fmaf(tau, d.z, ax.z);
        }
      }
      if (!__any_sync(0xffffffffu, contrib)) continue;
      if (!PP) {
        // SH weights into the next free column of W (row = channel x column, entry = pixel)
#pragma unroll
        for (int c = 0; c < 3; ++c) s_W[wtile(c * kSlots + cols, lane)] = wc[c];
        if (lane == cols) slot_b = b;
      }
      float v[16];
      v[0] = vv[0]; v[1] = vv[1]; v[2] = vv[2];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[3 + 3 * r + c] = vv[r] * xx[c];
      v[12] = dsig;
      v[13] = PP ? wc[0] : 0.f;
      v[14] = PP ? wc[1] : 0.f;
      v[15] = PP ? wc[2] : 0.f;
      warp_reduce_scatter16(v, lane);
      const int vi = (lane >> 1) & 15;
      if (!(lane & 1) && vi < (PP ? 16 : 13)) atomicAdd(&s_acc[b * ACC + vi], v[0]);
      if (lane == 0) s_any[b] = 1;
      if (!PP && ++cols == kSlots) {
        flush(kSlots);
        cols = 0;
      }
    }
    if (!PP && cols > 0) flush(cols);
    __syncthreads();
    for (int f = threadIdx.x; f < nb * ACC; f += blockDim.x) {
      int b = f / ACC, j = f - b * ACC;
      if (!s_any[b]) continue;
      uint32_t idx = s_idx[b];
      float v = s_acc[f];
      if (j < 13) atomicAdd(&sc.gacc[(size_t)idx * 16 + j], v);
      else if (!PP && j >= 16 && j < 16 + NC) atomicAdd(&sc.d_sh[(size_t)idx * NC + (j - 16)], v);
    }
    if (PP) {
      // dL/dc of this tile's pixels -> dL/dbeta_k,ch = dL/dc_ch Y_k(dir) and the mean's gradient
      // through dir = (mu - c) / |mu - c|: (I - dir dir^T) / |mu - c| sum_ch dL/dc_ch grad c_ch
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        if (!s_any[b]) continue;
        const float g0c = s_acc[b * ACC + 13], g1c = s_acc[b * ACC + 14], g2c = s_acc[b * ACC + 15];
        if (g0c == 0.f && g1c == 0.f && g2c == 0.f) continue;
        const uint32_t idx = s_idx[b];
        const float3 mu = make_float3(sc.means[3 * idx], sc.means[3 * idx + 1], sc.means[3 * idx + 2]);
        float il;
        const float3 dir = particle_dir<RS>(cam, op, mu, il);
        float Yp[NSH], a[NSH];
        sh_basis<DEG>(dir.x, dir.y, dir.z, Yp);
        const float *beta = sc.sh + (size_t)idx * NC;
        float *dsh = sc.d_sh + (size_t)idx * NC;
#pragma unroll
        for (int k = 0; k < NSH; ++k) {
          a[k] = fmaf(g0c, beta[3 * k], fmaf(g1c, beta[3 * k + 1], g2c * beta[3 * k + 2]));
          if (g0c != 0.f) atomicAdd(&dsh[3 * k], g0c * Yp[k]);
          if (g1c != 0.f) atomicAdd(&dsh[3 * k + 1], g1c * Yp[k]);
          if (g2c != 0.f) atomicAdd(&dsh[3 * k + 2], g2c * Yp[k]);
        }
        const float3 G = sh_poly_grad<DEG>(dir.x, dir.y, dir.z, a);
        const float gd = dot3(G, dir);
        atomicAdd(&sc.gacc[(size_t)idx * 16 + 13], (G.x - gd * dir.x) * il);
        atomicAdd(&sc.gacc[(size_t)idx * 16 + 14], (G.y - gd * dir.y) * il);
        atomicAdd(&sc.gacc[(size_t)idx * 16 + 15], (G.z - gd * dir.z) * il);
      }
    }
  }
}

// One warp per tile: work = list entries the backward replays (up to one past the last
// particle any of the tile's pixels blended, from n_used), and a histogram of the buckets.
__global__ void k_tile_work(const __grid_constant__ BatchDesc bd, DevOpts op, const uint2 *__restrict__ ranges,
                            TileSched ts) {
  const int tile = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (tile >= bd.total_tiles) return;
  const DevView &view = bd.v[view_of_tile(bd, tile)];
  const int lt = tile - view.tile_off;
  const int x0 = (lt % view.tiles_x) * op.tile_w, y0 = (lt / view.tiles_x) * op.tile_h;
  const int W = view.cam.W, H = view.cam.H;
  uint32_t m = 0;
  for (int i = lane; i < op.tile_w * op.tile_h; i += 32) {
    const int px = x0 + i % op.tile_w, py = y0 + i / op.tile_w;
    if (px < W && py < H) m = max(m, view.n_used[(size_t)py * W + px]);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    const uint2 rg = ranges[tile];
    const uint32_t w = m > rg.x ? min(m, rg.y) - rg.x : 0u;
    ts.work[tile] = w;
    if (w) atomicAdd(&ts.hist[work_bucket(w)], 1u);
  }
}

// d(rotation matrix)/d(unit quaternion) contracted with G = dL/dR (row-major).
__device__ __forceinline__ void rot_grad(const float *q, const float *G, float *gq) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  gq[0] = 2.f * (x * (G[7] - G[5]) + y * (G[2] - G[6]) + z * (G[3] - G[1]));
  gq[1] = 2.f * (-2.f * x * (G[4] + G[8]) + y * (G[1] + G[3]) + z * (G[2] + G[6]) + w * (G[7] - G[5]));
  gq[2] = 2.f * (x * (G[1] + G[3]) - 2.f * y * (G[0] + G[8]) + z * (G[5] + G[7]) + w * (G[2] - G[6]));
  gq[3] = 2.f * (x * (G[2] + G[6]) + y * (G[5] + G[7]) - 2.f * z * (G[0] + G[4]) + w * (G[3] - G[1]));
}

// Per particle of every scene in the batch: dL/dM, sum v, dL/dsigma -> parameter gradients.
__global__ void k_finalize(const __grid_constant__ BatchDesc bd, int total) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const DevScene &sc = bd.s[scene_of_grad(bd, g)];
    const int i = g - sc.grad_off;
    float3 mu = make_float3(sc.means[3 * i], sc.means[3 * i + 1], sc.means[3 * i + 2]);
    float3 ls = make_float3(sc.log_scales[3 * i], sc.log_scales[3 * i + 1], sc.log_scales[3 * i + 2]);
    Particle p;
    bool ok = activate(mu, ls, sc.quats[i], sc.logits[i], p);
    // the particle's 16 accumulators as four 16-byte loads (rows are 64-byte aligned)
    const float4 *A4 = reinterpret_cast<const float4 *>(sc.gacc + (size_t)i * 16);
    const float4 a0 = A4[0], a1 = A4[1], a2 = A4[2], a3 = A4[3];
    const float A[16] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x, a3.y, a3.z, a3.w};
    float out_m[3] = {0.f, 0.f, 0.f}, out_s[3] = {0.f, 0.f, 0.f}, out_q[4] = {0.f, 0.f, 0.f, 0.f}, out_l = 0.f;
    if (ok) {
      float v0 = A[0], v1 = A[1], v2 = A[2];
      // slots 13..15: the mean's gradient through the per-particle view direction (zero in
      // the per-pixel colour mode)
      for (int j = 0; j < 3; ++j) out_m[j] = A[13 + j] - (p.M[j] * v0 + p.M[3 + j] * v1 + p.M[6 + j] * v2);
      float G[9];
      for (int k = 0; k < 3; ++k) {
        float acc = 0.f;
        const float is = 1.f / p.s[k];
        for (int j = 0; j < 3; ++j) {
          float dm = A[3 + 3 * k + j];
          acc = fmaf(dm, p.M[3 * k + j], acc);
          G[3 * j + k] = dm * is;
        }
        out_s[k] = -acc;
      }
      float gq[4];
      rot_grad(p.q, G, gq);
      float dot = gq[0] * p.q[0] + gq[1] * p.q[1] + gq[2] * p.q[2] + gq[3] * p.q[3];
      const float iqn = 1.f / p.qn;
      for (int j = 0; j < 4; ++j) out_q[j] = (gq[j] - p.q[j] * dot) * iqn;
      out_l = A[12] * p.sigma * (1.f - p.sigma);
    }
    for (int j = 0; j < 3; ++j) {
      sc.d_means[3 * i + j] = out_m[j];
      sc.d_log_scales[3 * i + j] = out_s[j];
    }
    for (int j = 0; j < 4; ++j) sc.d_quats[4 * i + j] = out_q[j];
    sc.d_logits[i] = out_l;
  }
}

template <int DEG, bool RS, bool SMALL, bool PP, bool GEN>
void bwd_launch_k(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                  const uint32_t *ranges, const TileSched &ts, cudaStream_t s) {
  const int blocks = bd.total_tiles, threads = op.tile_w * op.tile_h;
  const size_t smem = BwdSmem<DEG, PP>::bytes(threads / 32);
  cudaFuncSetAttribute(k_composite_bwd<DEG, RS, SMALL, PP, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_composite_bwd<DEG, RS, SMALL, PP, GEN><<<blocks, threads, smem, s>>>(
      bd, op, reinterpret_cast<const short4 *>(rect), vals, reinterpret_cast<const uint2 *>(ranges), ts);
}

template <int DEG, bool RS, bool PP, bool GEN>
void bwd_launch_pp(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                   const uint32_t *ranges, const TileSched &ts, cudaStream_t s) {
  if (op.tile_w * op.tile_h <= 256) bwd_launch_k<DEG, RS, true, PP, GEN>(bd, op, rect, vals, ranges, ts, s);
  else bwd_launch_k<DEG, RS, false, PP, GEN>(bd, op, rect, vals, ranges, ts, s);
}

// Degree 0 colours do not depend on the direction: both colour modes run the per-pixel kernel.
// The degree-n kernels run with per-pixel colours (make_opts rejects the combination with
// per-particle colours).
template <int DEG, bool RS>
void bwd_launch(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                const uint32_t *ranges, const TileSched &ts, cudaStream_t s) {
  if (op.kernel_degree != 2) {
    bwd_launch_pp<DEG, RS, false, true>(bd, op, rect, vals, ranges, ts, s);
    return;
  }
  if constexpr (DEG > 0) {
    if (op.colour_mode == UT_COLOUR_PER_PARTICLE) {
      bwd_launch_pp<DEG, RS, true, false>(bd, op, rect, vals, ranges, ts, s);
      return;
    }
  }
  bwd_launch_pp<DEG, RS, false, false>(bd, op, rect, vals, ranges, ts, s);
}

}  // namespace

size_t backward_workspace_bytes(int n, bool kbuffer) {
  const size_t part = align256(sizeof(float) * 16 * (size_t)(n > 0 ? n : 1));
  return kbuffer ? 2 * part : part;
}

size_t tile_sched_bytes(int tiles) {
  const size_t t = (size_t)(tiles > 0 ? tiles : 1);
  return 2 * align256(sizeof(uint32_t) * t) + align256(sizeof(uint32_t) * (2 * kOrderBuckets + 1));
}


// Clears the scenes' accumulators and d_sh, orders the tiles by replay length, runs the
// backward over every tile with work, then finalize.
ut_status launch_composite_bwd(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                               const uint32_t *ranges, void *sched, cudaStream_t s) {
  int total = 0;
  for (int k = 0; k < bd.ns; ++k) {
    const DevScene &sc = bd.s[k];
    if (sc.n <= 0) continue;
    const size_t nc = 3 * (size_t)(sc.deg + 1) * (sc.deg + 1);
    if (cudaMemsetAsync(sc.gacc, 0, sizeof(float) * 16 * (size_t)sc.n, s) != cudaSuccess) return UT_ERR_CUDA;
    if (cudaMemsetAsync(sc.d_sh, 0, sizeof(float) * nc * sc.n, s) != cudaSuccess) return UT_ERR_CUDA;
    total = sc.grad_off + sc.n > total ? sc.grad_off + sc.n : total;
  }
  if (op.kbuffer > 0) {  // "Ours (sorted)": its own replay of the per-ray k-buffer
    const ut_status st = launch_composite_bwd_kbuffer(bd, op, rect, vals, ranges, s);
    if (st != UT_OK) return st;
  } else if (bd.total_tiles > 0) {
    const TileSched ts = carve_tile_sched(sched, bd.total_tiles);
    if (cudaMemsetAsync(ts.hist, 0, sizeof(uint32_t) * (2 * kOrderBuckets + 1), s) != cudaSuccess) return UT_ERR_CUDA;
    const auto *rg = reinterpret_cast<const uint2 *>(ranges);
    k_tile_work<<<(bd.total_tiles + 7) / 8, 256, 0, s>>>(bd, op, rg, ts);
    const int ob = (bd.total_tiles + kOrderBuckets - 1) / kOrderBuckets, cap = device_sm_count();
    k_tile_order<<<ob < cap ? ob : cap, kOrderBuckets, 0, s>>>(bd.total_tiles, ts);
    count_launches(2);
    const bool rs = any_rs(bd);
#define UT3D_BWD(D)                                                  \
  (rs ? bwd_launch<D, true>(bd, op, rect, vals, ranges, ts, s) \
      : bwd_launch<D, false>(bd, op, rect, vals, ranges, ts, s))
    switch (bd.s[0].deg) {
      case 0: UT3D_BWD(0); break;
      case 1: UT3D_BWD(1); break;
      case 2: UT3D_BWD(2); break;
      default: UT3D_BWD(3); break;
    }
#undef UT3D_BWD
    count_launches(1);
  }
  if (total > 0) {
    int g = (total + 255) / 256;
    int cap = device_sm_count() * 8;
    k_finalize<<<g < cap ? g : cap, 256, 0, s>>>(bd, total);
    count_launches(1);
  }
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

UT_DBG_READER(dbg_read_bwd)

}  // namespace ut3d
