// composite_fwd.cu — tile-based front-to-back compositing with 3D particle evaluation
// (Sec. 4.2, eq. GaussianMaxResponse; eq. QuadratureVolumeRendering) for a batch of views.
// Each block leaves its tile's list as soon as every pixel's transmittance has dropped below
// t_min; tiles run longest predicted walk first (k_fwd_predict + k_tile_order).
#include "composite_common.cuh"

namespace ut3d {
namespace {

// PP: per-particle colour mode (the colour of each staged particle is evaluated once, at its
// view direction, while staging; pixels read it from shared memory).
template <int DEG, bool RS, bool STATS, bool PP, bool GEN>
__global__ void __launch_bounds__(512) k_composite_fwd(const __grid_constant__ BatchDesc bd, DevOpts op,
                                                       const short4 *__restrict__ rect,
                                                       const uint32_t *__restrict__ vals,
                                                       const uint2 *__restrict__ ranges,
                                                       unsigned long long *__restrict__ stats, TileSched ts) {
  constexpr int NSH = (DEG + 1) * (DEG + 1);
  constexpr int NC = NSH * 3;
  constexpr int PDEG = PP ? 0 : DEG;        // per-pixel SH basis only when colours are per pixel
  constexpr int NST = PP ? 4 : NC;          // staged colour floats per particle
  __shared__ float4 s_geo[kBatchF][4];
  __shared__ __align__(16) float s_sh[kBatchF * NST];
  __shared__ uint32_t s_idx[kBatchF];

  // tiles in the order k_tile_order gave them (longest predicted walk first); every tile is
  // in the order, so every pixel is written
  if (blockIdx.x >= *ts.n_work) return;
  const int tile = (int)ts.order[blockIdx.x];
  UT_DBG_CHECK(tile < bd.total_tiles, UT_DBG_TILE_ID, tile, bd.total_tiles, 2);
  const DevView &view = bd.v[view_of_tile(bd, tile)];
  const DevScene &sc = bd.s[view.scene];
  const DevCam &cam = view.cam;
  const int lt = tile - view.tile_off;
  const int tx = lt % view.tiles_x, ty = lt / view.tiles_x;
  int lx, ly;
  tile_pixel(op, (int)threadIdx.x, lx, ly);
  const int px = tx * op.tile_w + lx;
  const int py = ty * op.tile_h + ly;
  const bool inside = px < cam.W && py < cam.H;
  float3 o, d;
  float Y[(PDEG + 1) * (PDEG + 1)];
  bool valid;
  pixel_setup<PDEG>(cam, op, px, py, inside, o, d, Y, valid);

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0;
  unsigned long long n_eval = 0, n_blend = 0;
  bool done = !valid;
  const uint2 rg = ranges[tile];
  for (uint32_t start = rg.x; start < rg.y; start += kBatchF) {
    if (__syncthreads_count(!done) == 0) break;
    const int nb = min((uint32_t)kBatchF, rg.y - start);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s_idx[t] = vals[start + t];
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      uint32_t idx = s_idx[t];
      stage_particle<RS>(sc, cam, op, rect[view.part_off + idx], idx, s_geo[t], nullptr);
      if (PP) reinterpret_cast<float4 *>(s_sh)[t] = particle_colour<DEG, RS>(sc, cam, op, idx);
    }
    if (!PP) stage_sh<NC>(sc, s_idx, nb, s_sh);
    __syncthreads();
    if (done) continue;
    for (int b = 0; b < nb; ++b) {
      float3 og, dg;
      float dd, a;
      if (STATS) {
        int r0 = __float_as_int(s_geo[b][3].z), r1 = __float_as_int(s_geo[b][3].w);
        n_eval += !(px < (r0 & 0xffff) || px > (r1 & 0xffff) || py < (r0 >> 16) || py > (r1 >> 16));
      }
      if (!eval_response<RS, GEN>(s_geo[b], px, py, o, d, og, dg, dd, a, op)) continue;
      float al = fminf(a, op.alpha_max);
      float Tn = T * (1.f - al);
      if (Tn < op.t_min) {
        done = true;
        break;
      }
      if (STATS) ++n_blend;
      float r0, r1, r2;
      if (PP) {
        const float4 c = reinterpret_cast<const float4 *>(s_sh)[b];
        r0 = c.x; r1 = c.y; r2 = c.z;
      } else {
        sh_colour<NSH>(s_sh + b * NC, Y, r0, r1, r2);
      }
      float w = al * T;
      C0 = fmaf(fmaxf(r0, 0.f), w, C0);
      C1 = fmaf(fmaxf(r1, 0.f), w, C1);
      C2 = fmaf(fmaxf(r2, 0.f), w, C2);
      T = Tn;
      last = start + b + 1;
    }
  }
  if (inside) {
    size_t pix = (size_t)py * cam.W + px;
    size_t plane = (size_t)cam.W * cam.H;
    view.rgb[pix] = C0;
    view.rgb[plane + pix] = C1;
    view.rgb[2 * plane + pix] = C2;
    view.alpha[pix] = valid ? 1.f - T : 0.f;
    if (view.tfinal) view.tfinal[pix] = T;
    if (view.n_used) view.n_used[pix] = last;
  }
  if (STATS) {
    for (int s = 16; s >= 1; s >>= 1) {
      n_eval += __shfl_xor_sync(0xffffffffu, n_eval, s);
      n_blend += __shfl_xor_sync(0xffffffffu, n_blend, s);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], n_eval);
      atomicAdd(&stats[1], n_blend);
    }
  }
}

// "Ours (sorted)" (Sec. 4.4): compositing through a per-ray k-buffer (multi-layer alpha
// blending).  Hits (sigma rho >= alpha_min) met in the tile's depth order enter a buffer of at
// most k = op.kbuffer entries kept in shared memory (tau_max, alpha, rgb and the hit's position
// in the tile's list per entry); when a hit meets a full buffer, the closest of the buffered
// hits and the new one by tau_max -- the earlier arrival, i.e. the smaller list position, on
// equal tau_max -- is blended front to back (stop rule as in k_composite_fwd) and the new hit
// takes its slot unless it was itself the closest; at the end of the list the rest are blended
// in ascending (tau_max, arrival).
// n_used is written as 0 (the backward does not replay this variant).
template <int DEG, bool RS>
__global__ void __launch_bounds__(512, 1) k_composite_fwd_kbuffer(const __grid_constant__ BatchDesc bd, DevOpts op,
                                                               const short4 *__restrict__ rect,
                                                               const uint32_t *__restrict__ vals,
                                                               const uint2 *__restrict__ ranges, TileSched ts) {
  constexpr int NSH = (DEG + 1) * (DEG + 1);
  constexpr int NC = NSH * 3;
  __shared__ float4 s_geo[kBatchK][4];
  __shared__ __align__(16) float s_sh[kBatchK * NC];
  __shared__ uint32_t s_idx[kBatchK];
  extern __shared__ float s_kb[];  // [6][k][threads]: tau, alpha, r, g, b, list position of each hit

  if (blockIdx.x >= *ts.n_work) return;
  const int tile = (int)ts.order[blockIdx.x];
  UT_DBG_CHECK(tile < bd.total_tiles, UT_DBG_TILE_ID, tile, bd.total_tiles, 2);
  const DevView &view = bd.v[view_of_tile(bd, tile)];
  const DevScene &sc = bd.s[view.scene];
  const DevCam &cam = view.cam;
  const int lt = tile - view.tile_off;
  const int tx = lt % view.tiles_x, ty = lt / view.tiles_x;
  int lx, ly;
  tile_pixel(op, (int)threadIdx.x, lx, ly);
  const int px = tx * op.tile_w + lx;
  const int py = ty * op.tile_h + ly;
  const bool inside = px < cam.W && py < cam.H;
  const int K = op.kbuffer, nt = blockDim.x;
  float *kb_tau = s_kb + threadIdx.x, *kb_a = kb_tau + K * nt, *kb_r = kb_a + K * nt, *kb_g = kb_r + K * nt,
        *kb_b = kb_g + K * nt;  // entry j of this thread at [j * nt]
  uint32_t *kb_p = reinterpret_cast<uint32_t *>(kb_b + K * nt);
  float3 o, d;
  float Y[NSH];
  bool valid;
  pixel_setup<DEG>(cam, op, px, py, inside, o, d, Y, valid);

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int nbuf = 0;
  bool done = !valid;
  auto blend = [&](float al, float r, float g, float b) {
    const float Tn = T * (1.f - al);
    if (Tn < op.t_min) {
      done = true;
      return;
    }
    const float w = al * T;
    C0 = fmaf(r, w, C0);
    C1 = fmaf(g, w, C1);
    C2 = fmaf(b, w, C2);
    T = Tn;
  };
  const uint2 rg = ranges[tile];
  for (uint32_t start = rg.x; start < rg.y; start += kBatchK) {
    if (__syncthreads_count(!done) == 0) break;
    const int nb = min((uint32_t)kBatchK, rg.y - start);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s_idx[t] = vals[start + t];
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      uint32_t idx = s_idx[t];
      stage_particle<RS>(sc, cam, op, rect[view.part_off + idx], idx, s_geo[t], nullptr);
    }
    stage_sh<NC>(sc, s_idx, nb, s_sh);
    __syncthreads();
    if (done) continue;
    for (int b = 0; b < nb && !done; ++b) {
      float3 og, dg;
      float dd, a;
      if (!eval_response<RS, false>(s_geo[b], px, py, o, d, og, dg, dd, a, op)) continue;
      const float tau = -__fdividef(dot3(og, dg), dd);
      const float al = fminf(a, op.alpha_max);
      float r0, r1, r2;
      sh_colour<NSH>(s_sh + b * NC, Y, r0, r1, r2);
      r0 = fmaxf(r0, 0.f); r1 = fmaxf(r1, 0.f); r2 = fmaxf(r2, 0.f);
      const uint32_t pos = start + b;
      if (nbuf < K) {
        kb_tau[nbuf * nt] = tau; kb_a[nbuf * nt] = al;
        kb_r[nbuf * nt] = r0; kb_g[nbuf * nt] = r1; kb_b[nbuf * nt] = r2; kb_p[nbuf * nt] = pos;
        ++nbuf;
        continue;
      }
      // closest of the buffer and the new hit (the new hit arrived last: it wins only with a
      // strictly smaller tau_max)
      const int bi = kb_select(kb_tau, kb_p, nt, K, tau, true);
      if (bi < 0) {
        blend(al, r0, r1, r2);
      } else {
        blend(kb_a[bi * nt], kb_r[bi * nt], kb_g[bi * nt], kb_b[bi * nt]);
        kb_tau[bi * nt] = tau; kb_a[bi * nt] = al;
        kb_r[bi * nt] = r0; kb_g[bi * nt] = r1; kb_b[bi * nt] = r2; kb_p[bi * nt] = pos;
      }
    }
  }
  // end of the list: the remaining hits in ascending (tau_max, arrival)
  while (!done && nbuf > 0) {
    const int bi = kb_select(kb_tau, kb_p, nt, nbuf, 0.f, false);
    blend(kb_a[bi * nt], kb_r[bi * nt], kb_g[bi * nt], kb_b[bi * nt]);
    --nbuf;
    kb_tau[bi * nt] = kb_tau[nbuf * nt]; kb_a[bi * nt] = kb_a[nbuf * nt];
    kb_r[bi * nt] = kb_r[nbuf * nt]; kb_g[bi * nt] = kb_g[nbuf * nt]; kb_b[bi * nt] = kb_b[nbuf * nt];
    kb_p[bi * nt] = kb_p[nbuf * nt];
  }
  if (inside) {
    size_t pix = (size_t)py * cam.W + px;
    size_t plane = (size_t)cam.W * cam.H;
    view.rgb[pix] = C0;
    view.rgb[plane + pix] = C1;
    view.rgb[2 * plane + pix] = C2;
    view.alpha[pix] = valid ? 1.f - T : 0.f;
    if (view.tfinal) view.tfinal[pix] = T;
    if (view.n_used) view.n_used[pix] = 0;
  }
}

// Forward schedule estimate, one warp per tile.  A heuristic that only orders the tiles (no
// result depends on it): a tile's pixels saturate after roughly a fixed optical depth of
// particles that cover the whole tile, so the estimate is the list position where
// sum -ln(1 - 0.3 sigma) over particles whose rect contains the tile's pixels reaches
// kFwdDepth, or the end of the first kFwdCap entries.  Every tile gets work >= 1 so that
// every tile, even an empty one, is scheduled (its pixels must still be written).
constexpr int kFwdCap = 512;
constexpr float kFwdDepth = 40.f;

__global__ void k_fwd_predict(const __grid_constant__ BatchDesc bd, DevOpts op, const short4 *__restrict__ rect,
                              const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges, TileSched ts) {
  const int tile = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (tile >= bd.total_tiles) return;
  const DevView &view = bd.v[view_of_tile(bd, tile)];
  const float *logits = bd.s[view.scene].logits;
  const int lt = tile - view.tile_off;
  const int x0 = (lt % view.tiles_x) * op.tile_w, y0 = (lt / view.tiles_x) * op.tile_h;
  const int x1 = min(x0 + op.tile_w, view.cam.W) - 1, y1 = min(y0 + op.tile_h, view.cam.H) - 1;
  const uint2 rg = ranges[tile];
  const uint32_t end = min(rg.y, rg.x + (uint32_t)kFwdCap);
  uint32_t pred = end - rg.x;
  float tau = 0.f;
  bool found = false;
  for (uint32_t base = rg.x; base < end && !found; base += 128) {
    float c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // four chunks of 32 entries in flight per step
      const uint32_t k = base + 32 * j + lane;
      c[j] = 0.f;
      if (k < end) {
        const uint32_t idx = vals[k];
        const short4 r = rect[view.part_off + idx];
        if (r.x <= x0 && r.y <= y0 && r.z >= x1 && r.w >= y1) {
          const float sg = 1.f / (1.f + __expf(-logits[idx]));
          c[j] = -__logf(1.f - fminf(0.3f * sg, 0.99f));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float incl = c[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, !found && tau + incl >= kFwdDepth);
      if (hit) {
        pred = base + 32 * j + (__ffs(hit) - 1) + 1 - rg.x;
        found = true;
      }
      tau += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (lane == 0) {
    const uint32_t w = (rg.y > rg.x ? pred : 0u) + 1u;
    ts.work[tile] = w;
    atomicAdd(&ts.hist[work_bucket(w)], 1u);
  }
}

template <int DEG, bool RS, bool PP, bool GEN>
void fwd_launch_k(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                  const uint32_t *ranges, unsigned long long *stats, const TileSched &ts, cudaStream_t s) {
  const int blocks = bd.total_tiles, threads = op.tile_w * op.tile_h;
  const short4 *r4 = reinterpret_cast<const short4 *>(rect);
  const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
  if (stats)
    k_composite_fwd<DEG, RS, true, PP, GEN><<<blocks, threads, 0, s>>>(bd, op, r4, vals, rg, stats, ts);
  else
    k_composite_fwd<DEG, RS, false, PP, GEN><<<blocks, threads, 0, s>>>(bd, op, r4, vals, rg, nullptr, ts);
}

// Degree 0 colours do not depend on the direction: both colour modes run the per-pixel kernel.
// The degree-n kernels and the k-buffer run with per-pixel colours (make_opts rejects the
// other combinations).
template <int DEG, bool RS>
void fwd_launch(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                const uint32_t *ranges, unsigned long long *stats, const TileSched &ts, cudaStream_t s) {
  if (op.kbuffer > 0) {
    const int threads = op.tile_w * op.tile_h;
    const size_t smem = sizeof(float) * 6 * (size_t)op.kbuffer * threads;
    cudaFuncSetAttribute(k_composite_fwd_kbuffer<DEG, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_composite_fwd_kbuffer<DEG, RS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    k_composite_fwd_kbuffer<DEG, RS><<<bd.total_tiles, threads, smem, s>>>(
        bd, op, reinterpret_cast<const short4 *>(rect), vals, reinterpret_cast<const uint2 *>(ranges), ts);
    return;
  }
  if (op.kernel_degree != 2) {
    fwd_launch_k<DEG, RS, false, true>(bd, op, rect, vals, ranges, stats, ts, s);
    return;
  }
  if constexpr (DEG > 0) {
    if (op.colour_mode == UT_COLOUR_PER_PARTICLE) {
      fwd_launch_k<DEG, RS, true, false>(bd, op, rect, vals, ranges, stats, ts, s);
      return;
    }
  }
  fwd_launch_k<DEG, RS, false, false>(bd, op, rect, vals, ranges, stats, ts, s);
}

}  // namespace

// Predicts each tile's walk, orders the tiles longest first, then composites them in that order.
ut_status launch_composite_fwd(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                               const uint32_t *ranges, unsigned long long *stats, void *sched, cudaStream_t s) {
  if (op.kbuffer > 0 && stats) return UT_ERR_UNSUPPORTED;
  if (bd.total_tiles == 0) return UT_OK;
  const TileSched ts = carve_tile_sched(sched, bd.total_tiles);
  if (cudaMemsetAsync(ts.hist, 0, sizeof(uint32_t) * (2 * kOrderBuckets + 1), s) != cudaSuccess) return UT_ERR_CUDA;
  k_fwd_predict<<<(bd.total_tiles + 7) / 8, 256, 0, s>>>(bd, op, reinterpret_cast<const short4 *>(rect), vals,
                                                         reinterpret_cast<const uint2 *>(ranges), ts);
  const int ob = (bd.total_tiles + kOrderBuckets - 1) / kOrderBuckets, cap = device_sm_count();
  k_tile_order<<<ob < cap ? ob : cap, kOrderBuckets, 0, s>>>(bd.total_tiles, ts);
  count_launches(2);
  const bool rs = any_rs(bd);
#define UT3D_FWD(D)                                                     \
  (rs ? fwd_launch<D, true>(bd, op, rect, vals, ranges, stats, ts, s) \
      : fwd_launch<D, false>(bd, op, rect, vals, ranges, stats, ts, s))
  switch (bd.s[0].deg) {
    case 0: UT3D_FWD(0); break;
    case 1: UT3D_FWD(1); break;
    case 2: UT3D_FWD(2); break;
    default: UT3D_FWD(3); break;
  }
#undef UT3D_FWD
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

UT_DBG_READER(dbg_read_fwd)

}  // namespace ut3d
