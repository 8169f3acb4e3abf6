// composite_bwd_kbuffer.cu — backward of the "Ours (sorted)" compositing (Sec. 4.4): per-ray
// k-buffer (multi-layer alpha blending) with per-pixel SH colour and the Gaussian kernel.
//
// The blending order of a k-buffer ray is decided per pixel (the closest buffered hit by tau_max,
// the earlier arrival on equal tau_max, leaves when a new hit meets a full buffer, the rest leave
// in that order at the end), so a particle is often blended after its batch has left shared
// memory.  The kernel replays the forward kernel's buffer logic exactly (same staging, same FP32
// decisions), and at each blend it takes the gradient of that (pixel, particle) pair in the
// forward order, as the tile-order backward does: the stored final colour gives the colour still
// to come, S = C_final - A after the pair's own contribution, so
// dL/dalpha = sum_c g_c (c_c T - S_c / (1 - alpha)) + g_A T_final / (1 - alpha).  The pair's
// canonical ray (o_g, d_g) is recomputed from the particle's parameters in global memory, and
// its contributions (the 13 geometry partials of k_finalize's layout, and dL/dbeta for the
// unclamped channels) go to the particle's accumulators with one global atomic each (a window of
// per-list-position accumulators in shared memory was measured 5x slower: the lanes of a warp
// blend the same particle at nearly the same time, and shared-memory atomics on one address
// serialise, while the L2's reductions absorb them).
// Selection by tau_max is piecewise constant and carries no gradient.
#include "composite_common.cuh"

namespace ut3d {
namespace {

template <int DEG, bool RS>
__global__ void __launch_bounds__(512, 1) k_composite_bwd_kbuffer(const __grid_constant__ BatchDesc bd, DevOpts op,
                                                               const short4 *__restrict__ rect,
                                                               const uint32_t *__restrict__ vals,
                                                               const uint2 *__restrict__ ranges) {
  constexpr int NSH = (DEG + 1) * (DEG + 1);
  constexpr int NC = NSH * 3;
  __shared__ float4 s_geo[kBatchK][4];
  __shared__ __align__(16) float s_sh[kBatchK * NC];
  __shared__ uint32_t s_idx[kBatchK];
  extern __shared__ float s_kb[];  // [6][k][threads]: tau, alpha, r, g, b, list position

  const int tile = blockIdx.x;
  const DevView &view = bd.v[view_of_tile(bd, tile)];
  const DevScene &sc = bd.s[view.scene];
  const DevCam &cam = view.cam;
  const int lt = tile - view.tile_off;
  const int tx = lt % view.tiles_x, ty = lt / view.tiles_x;
  const int px = tx * op.tile_w + (int)threadIdx.x % op.tile_w;
  const int py = ty * op.tile_h + (int)threadIdx.x / op.tile_w;
  const bool inside = px < cam.W && py < cam.H;
  const int K = op.kbuffer, nt = blockDim.x;
  float *kb_tau = s_kb + threadIdx.x, *kb_a = kb_tau + K * nt, *kb_r = kb_a + K * nt, *kb_g = kb_r + K * nt,
        *kb_b = kb_g + K * nt;
  uint32_t *kb_p = reinterpret_cast<uint32_t *>(kb_b + K * nt);  // entry j of this thread at [j * nt]
  float3 o, d;
  float Y[NSH];
  bool valid;
  pixel_setup<DEG>(cam, op, px, py, inside, o, d, Y, valid);

  float g0 = 0.f, g1 = 0.f, g2 = 0.f, gAT = 0.f, Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f;  // gAT = dL/dalpha T_final
  if (valid) {
    const size_t pix = (size_t)py * cam.W + px, plane = (size_t)cam.W * cam.H;
    g0 = view.d_rgb[pix]; g1 = view.d_rgb[plane + pix]; g2 = view.d_rgb[2 * plane + pix];
    gAT = view.d_alpha[pix] * view.tfinal[pix];
    Cf0 = view.rgb[pix]; Cf1 = view.rgb[plane + pix]; Cf2 = view.rgb[2 * plane + pix];
  }
  float T = 1.f, A0 = 0.f, A1 = 0.f, A2 = 0.f;  // running prefix of the composited colour
  int nbuf = 0;
  bool done = !valid;

  // blends the pair (the particle at list position pos, alpha al, clamped colour c) at
  // transmittance T, with the stop rule of the forward, and adds its gradient contributions
  auto blend = [&](float al, float c0, float c1, float c2, uint32_t pos) {
    const float Tn = T * (1.f - al);
    if (Tn < op.t_min) {
      done = true;
      return;
    }
    const float w = al * T;
    A0 = fmaf(c0, w, A0);
    A1 = fmaf(c1, w, A1);
    A2 = fmaf(c2, w, A2);
    const float inv = 1.f / (1.f - al);
    const float dal = g0 * fmaf(-(Cf0 - A0), inv, c0 * T) + g1 * fmaf(-(Cf1 - A1), inv, c1 * T) +
                      g2 * fmaf(-(Cf2 - A2), inv, c2 * T) + gAT * inv;
    T = Tn;
    const uint32_t idx = vals[pos];
    UT_DBG_CHECK(idx < (uint32_t)sc.n, UT_DBG_PARTICLE, idx, sc.n, 1);
    if (idx >= (uint32_t)sc.n) return;  // every index is a particle of the scene; the test only guards
    // SH coefficients: dL/dbeta_k,ch = g_ch w Y_k where the colour's clamp is inactive
    const float gc[3] = {c0 > 0.f ? g0 * w : 0.f, c1 > 0.f ? g1 * w : 0.f, c2 > 0.f ? g2 * w : 0.f};
    float *dsh = sc.d_sh + (size_t)idx * NC;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      if (gc[ch] == 0.f) continue;
#pragma unroll
      for (int k = 0; k < NSH; ++k) atomicAdd(&dsh[3 * k + ch], gc[ch] * Y[k]);
    }
    // geometry: the pair's canonical ray from the particle's parameters
    const float3 mu = make_float3(sc.means[3 * idx], sc.means[3 * idx + 1], sc.means[3 * idx + 2]);
    const float3 ls = make_float3(sc.log_scales[3 * idx], sc.log_scales[3 * idx + 1], sc.log_scales[3 * idx + 2]);
    Particle p;
    activate(mu, ls, sc.quats[idx], sc.logits[idx], p);
    const float3 om = make_float3(o.x - mu.x, o.y - mu.y, o.z - mu.z);
    const float3 og = mat3_mul(p.M, om), dg = mat3_mul(p.M, d);
    const float3 cr = cross3(og, dg);
    const float cc = dot3(cr, cr), dd = dot3(dg, dg);
    const float a = p.sigma * __expf(-0.5f * __fdividef(cc, dd));
    const float da = a > op.alpha_max ? 0.f : dal;
    const float dsig = da * a / p.sigma;
    const float dw2 = -0.5f * a * da;
    const float tau = -dot3(og, dg) / dd;
    const float3 pp = make_float3(fmaf(tau, dg.x, og.x), fmaf(tau, dg.y, og.y), fmaf(tau, dg.z, og.z));
    const float vv[3] = {2.f * dw2 * pp.x, 2.f * dw2 * pp.y, 2.f * dw2 * pp.z};
    const float xx[3] = {fmaf(tau, d.x, om.x), fmaf(tau, d.y, om.y), fmaf(tau, d.z, om.z)};
    float *acc = sc.gacc + (size_t)idx * 16;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      atomicAdd(&acc[r], vv[r]);
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(&acc[3 + 3 * r + c], vv[r] * xx[c]);
    }
    atomicAdd(&acc[12], dsig);
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
      // closest of the buffer and the new hit (the forward kernel's choice)
      const int bi = kb_select(kb_tau, kb_p, nt, K, tau, true);
      if (bi < 0) {
        blend(al, r0, r1, r2, pos);
      } else {
        blend(kb_a[bi * nt], kb_r[bi * nt], kb_g[bi * nt], kb_b[bi * nt], kb_p[bi * nt]);
        kb_tau[bi * nt] = tau; kb_a[bi * nt] = al;
        kb_r[bi * nt] = r0; kb_g[bi * nt] = r1; kb_b[bi * nt] = r2; kb_p[bi * nt] = pos;
      }
    }
  }
  // end of the list: the remaining hits in ascending (tau_max, arrival)
  while (!done && nbuf > 0) {
    const int bi = kb_select(kb_tau, kb_p, nt, nbuf, 0.f, false);
    blend(kb_a[bi * nt], kb_r[bi * nt], kb_g[bi * nt], kb_b[bi * nt], kb_p[bi * nt]);
    --nbuf;
    kb_tau[bi * nt] = kb_tau[nbuf * nt]; kb_a[bi * nt] = kb_a[nbuf * nt];
    kb_r[bi * nt] = kb_r[nbuf * nt]; kb_g[bi * nt] = kb_g[nbuf * nt]; kb_b[bi * nt] = kb_b[nbuf * nt];
    kb_p[bi * nt] = kb_p[nbuf * nt];
  }
}

template <int DEG, bool RS>
ut_status launch_k(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                   const uint32_t *ranges, cudaStream_t s) {
  const int threads = op.tile_w * op.tile_h;
  const size_t smem = sizeof(float) * 6 * (size_t)op.kbuffer * threads;
  constexpr size_t kStatic = sizeof(float4) * kBatchK * 4 + sizeof(float) * kBatchK * 3 * (DEG + 1) * (DEG + 1) +
                             sizeof(uint32_t) * kBatchK;
  if (smem + kStatic > 227 * 1024) return UT_ERR_UNSUPPORTED;  // the buffer does not fit one block
  if (cudaFuncSetAttribute(k_composite_bwd_kbuffer<DEG, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_composite_bwd_kbuffer<DEG, RS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return UT_ERR_CUDA;
  k_composite_bwd_kbuffer<DEG, RS><<<bd.total_tiles, threads, smem, s>>>(
      bd, op, reinterpret_cast<const short4 *>(rect), vals, reinterpret_cast<const uint2 *>(ranges));
  count_launches(1);
  return UT_OK;
}

}  // namespace

// The k-buffer backward over every tile of the batch (accumulators cleared by the caller).
ut_status launch_composite_bwd_kbuffer(const BatchDesc &bd, const DevOpts &op, const int16_t *rect,
                                       const uint32_t *vals, const uint32_t *ranges, cudaStream_t s) {
  if (bd.total_tiles == 0) return UT_OK;
  const bool rs = any_rs(bd);
  switch (bd.s[0].deg) {
    case 0: return rs ? launch_k<0, true>(bd, op, rect, vals, ranges, s) : launch_k<0, false>(bd, op, rect, vals, ranges, s);
    case 1: return rs ? launch_k<1, true>(bd, op, rect, vals, ranges, s) : launch_k<1, false>(bd, op, rect, vals, ranges, s);
    case 2: return rs ? launch_k<2, true>(bd, op, rect, vals, ranges, s) : launch_k<2, false>(bd, op, rect, vals, ranges, s);
    default: return rs ? launch_k<3, true>(bd, op, rect, vals, ranges, s) : launch_k<3, false>(bd, op, rect, vals, ranges, s);
  }
}

UT_DBG_READER(dbg_read_kbuffer)

}  // namespace ut3d
