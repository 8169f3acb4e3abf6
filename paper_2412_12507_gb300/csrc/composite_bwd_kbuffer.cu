// composite_bwd_kbuffer.cu — backward of the "Ours (sorted)" compositing (Sec. 4.4): per-ray
// k-buffer (multi-layer alpha blending) with per-pixel SH colour and the Gaussian kernel.
//
// The blending order of a k-buffer ray is decided per pixel (the closest buffered hit by tau_max,
// the earlier arrival on equal tau_max, leaves when a new hit meets a full buffer, the rest leave
// in that order at the end), so a particle is often blended after its batch has left shared
// memory.  The kernel replays the forward kernel's buffer logic exactly (the same FP32 decisions
// and tie-aware search), and at each blend it takes the gradient of that (pixel, particle) pair in the
// forward order, as the tile-order backward does: the stored final colour gives the colour still
// to come, S = C_final - A after the pair's own contribution, so
// dL/dalpha = sum_c g_c (c_c T - S_c / (1 - alpha)) + g_A T_final / (1 - alpha).  The pair's
// canonical ray (o_g, d_g) is recomputed from the particle's staged record while its batch is in
// shared memory (about 70% of the blends at k = 16), else from the call's per-particle record
// table (k_kb_records: M, M mu, mu, sigma), and its contributions (the 13 geometry partials of k_finalize's layout, and dL/dbeta for the
// unclamped channels) go to the particle's accumulators.  The lanes of a warp blend in step (one
// blend event per lane per staged particle, and per step of the final drain), and the events of a
// step are grouped by particle: neighbouring pixels' buffers evolve alike, so a step's 20 or so
// events name three or four particles.  A group of four or more lanes sums its contributions with
// reduce-scatters over the warp and adds each value with one atomic; the lanes of smaller groups
// add their own, one global atomic per value (a window of
// per-list-position accumulators in shared memory was measured 5x slower: the lanes of a warp
// blend the same particle at nearly the same time, and shared-memory atomics on one address
// serialise, while the L2's reductions absorb them).
// Selection by tau_max is piecewise constant and carries no gradient.
#include "composite_common.cuh"

namespace ut3d {
namespace {

constexpr int kBatchKB = 48;  // particles staged per block step: two blocks of 256 fit an SM at k = 16

// Reduce-scatter of 16 per-lane values over the 32 lanes: afterwards lanes 2i and 2i+1 hold the
// warp total of value i.
__device__ __forceinline__ void kb_reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 16, L = 8; L >= 1; o >>= 1, L >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const float send = up ? v[j] : v[j + L];
      const float keep = up ? v[j + L] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// The record table of the scene's particles: M (row-major, 9), M mu, mu and sigma, 16 floats.
__global__ void k_kb_records(const DevScene sc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sc.n; i += gridDim.x * blockDim.x) {
    const float3 mu = make_float3(sc.means[3 * i], sc.means[3 * i + 1], sc.means[3 * i + 2]);
    const float3 ls = make_float3(sc.log_scales[3 * i], sc.log_scales[3 * i + 1], sc.log_scales[3 * i + 2]);
    Particle p;
    activate(mu, ls, sc.quats[i], sc.logits[i], p);
    const float3 a = mat3_mul(p.M, mu);
    float4 *rec = sc.kbrec + 4 * (size_t)i;
    rec[0] = make_float4(p.M[0], p.M[1], p.M[2], p.M[3]);
    rec[1] = make_float4(p.M[4], p.M[5], p.M[6], p.M[7]);
    rec[2] = make_float4(p.M[8], a.x, a.y, a.z);
    rec[3] = make_float4(mu.x, mu.y, mu.z, p.sigma);
  }
}

template <int DEG, bool RS>
__global__ void __launch_bounds__(512, 1) k_composite_bwd_kbuffer(const __grid_constant__ BatchDesc bd, DevOpts op,
                                                               const short4 *__restrict__ rect,
                                                               const uint32_t *__restrict__ vals,
                                                               const uint2 *__restrict__ ranges) {
  constexpr int NSH = (DEG + 1) * (DEG + 1);
  constexpr int NC = NSH * 3;
  __shared__ float4 s_geo[kBatchKB][4];
  __shared__ float4 s_aux[kBatchKB];
  __shared__ __align__(16) float s_sh[kBatchKB * NC];
  __shared__ uint32_t s_idx[kBatchKB];
  extern __shared__ float s_kb[];  // [6][k][threads]: tau, alpha, r, g, b, list position

  const int tile = blockIdx.x;
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
  uint32_t sb = 0;  // list position of the batch staged in shared memory
  int snb = 0;      // and its length
  // this lane's blend event of the current step: particle, SH weights g_c w, the geometry partial
  // v = 2 dL/domega^2 (o_g + tau d_g), x = o - mu + tau d, and dL/dsigma
  bool has_ev = false;
  uint32_t ev_idx = 0;
  float ev_gc[3] = {0.f, 0.f, 0.f}, ev_v[3] = {0.f, 0.f, 0.f}, ev_x[3] = {0.f, 0.f, 0.f}, ev_dsig = 0.f;

  // blends the pair (the particle at list position pos, alpha al, clamped colour c) at
  // transmittance T, with the stop rule of the forward, and records its gradient contributions
  // as this lane's event of the step (emit adds them to the particle's accumulators)
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
    const float inv = __fdividef(1.f, 1.f - al);  // 1 - al >= 1 - alpha_max > 0
    const float dal = g0 * fmaf(-(Cf0 - A0), inv, c0 * T) + g1 * fmaf(-(Cf1 - A1), inv, c1 * T) +
                      g2 * fmaf(-(Cf2 - A2), inv, c2 * T) + gAT * inv;
    T = Tn;
    // a particle of the staged batch is read from shared memory (its staged record and o - mu or
    // mu), an older one from the call's record table (M, M mu, mu, sigma)
    const bool staged = pos >= sb && pos < sb + (uint32_t)snb;
    const uint32_t idx = staged ? s_idx[pos - sb] : vals[pos];
    UT_DBG_CHECK(idx < (uint32_t)sc.n, UT_DBG_PARTICLE, idx, sc.n, 1);
    if (idx >= (uint32_t)sc.n) return;  // every index is a particle of the scene; the test only guards
    // SH coefficients: dL/dbeta_k,ch = g_ch w Y_k where the colour's clamp is inactive
    ev_gc[0] = c0 > 0.f ? g0 * w : 0.f;
    ev_gc[1] = c1 > 0.f ? g1 * w : 0.f;
    ev_gc[2] = c2 > 0.f ? g2 * w : 0.f;
    // geometry: the pair's canonical ray
    float4 q0, q1, q2, q3;  // M row-major in q0, q1, q2.x; then M mu (or M (o - mu)), mu (or o - mu), sigma
    if (staged) {
      const float4 *g = s_geo[pos - sb];
      q0 = g[0]; q1 = g[1]; q2 = g[2];
      q3 = s_aux[pos - sb];
      q3.w = g[3].x;
    } else {
      const float4 *rec = sc.kbrec + 4 * (size_t)idx;
      q0 = __ldg(rec); q1 = __ldg(rec + 1); q2 = __ldg(rec + 2); q3 = __ldg(rec + 3);
    }
    const float3 dg = make_float3(fmaf(q0.x, d.x, fmaf(q0.y, d.y, q0.z * d.z)),
                                  fmaf(q0.w, d.x, fmaf(q1.x, d.y, q1.y * d.z)),
                                  fmaf(q1.z, d.x, fmaf(q1.w, d.y, q2.x * d.z)));
    float3 og, om;
    if (RS || !staged) {  // the record holds M mu and mu
      og = make_float3(fmaf(q0.x, o.x, fmaf(q0.y, o.y, q0.z * o.z)) - q2.y,
                       fmaf(q0.w, o.x, fmaf(q1.x, o.y, q1.y * o.z)) - q2.z,
                       fmaf(q1.z, o.x, fmaf(q1.w, o.y, q2.x * o.z)) - q2.w);
      om = make_float3(o.x - q3.x, o.y - q3.y, o.z - q3.z);
    } else {  // the staged record of a global-shutter view holds M (o - mu) and o - mu
      og = make_float3(q2.y, q2.z, q2.w);
      om = make_float3(q3.x, q3.y, q3.z);
    }
    const float sigma = q3.w;
    const float3 cr = cross3(og, dg);
    const float cc = dot3(cr, cr), dd = dot3(dg, dg);
    const float a = sigma * __expf(-0.5f * __fdividef(cc, dd));
    const float da = a > op.alpha_max ? 0.f : dal;
    ev_dsig = da * __fdividef(a, sigma);
    const float dw2 = -0.5f * a * da;
    const float tau = -__fdividef(dot3(og, dg), dd);
    const float3 pp = make_float3(fmaf(tau, dg.x, og.x), fmaf(tau, dg.y, og.y), fmaf(tau, dg.z, og.z));
    ev_v[0] = 2.f * dw2 * pp.x;
    ev_v[1] = 2.f * dw2 * pp.y;
    ev_v[2] = 2.f * dw2 * pp.z;
    ev_x[0] = fmaf(tau, d.x, om.x);
    ev_x[1] = fmaf(tau, d.y, om.y);
    ev_x[2] = fmaf(tau, d.z, om.z);
    ev_idx = idx;
    has_ev = true;
  };

  // adds this step's blend events to the particles' accumulators; every lane of the warp calls it
  const int lane = threadIdx.x & 31;
  auto emit = [&]() {
    const unsigned act = __ballot_sync(0xffffffffu, has_ev);
    if (!act) return;
    const unsigned grp = __match_any_sync(0xffffffffu, has_ev ? ev_idx : 0xffffffffu);
    unsigned big = __ballot_sync(0xffffffffu, has_ev && (int)(__ffs(grp) - 1) == lane && __popc(grp) >= 4);
    const int vi = lane >> 1;
    while (big) {
      const int l = __ffs(big) - 1;
      big &= big - 1;
      const unsigned gm = __shfl_sync(0xffffffffu, grp, l);
      const uint32_t p0 = __shfl_sync(0xffffffffu, ev_idx, l);
      const bool in = (gm >> lane) & 1u;
      float v[16];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        v[r] = in ? ev_v[r] : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[3 + 3 * r + c] = in ? ev_v[r] * ev_x[c] : 0.f;
      }
      v[12] = in ? ev_dsig : 0.f;
      v[13] = v[14] = v[15] = 0.f;
      kb_reduce_scatter16(v, lane);
      if (!(lane & 1) && vi < 13) atomicAdd(&sc.gacc[(size_t)p0 * 16 + vi], v[0]);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        if (!__any_sync(0xffffffffu, in && ev_gc[ch] != 0.f)) continue;
        float u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = (in && k < NSH) ? ev_gc[ch] * Y[k < NSH ? k : 0] : 0.f;
        kb_reduce_scatter16(u, lane);
        if (!(lane & 1) && vi < NSH && u[0] != 0.f) atomicAdd(&sc.d_sh[(size_t)p0 * NC + 3 * vi + ch], u[0]);
      }
    }
    if (has_ev && __popc(grp) < 4) {
      float *dsh = sc.d_sh + (size_t)ev_idx * NC;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        if (ev_gc[ch] == 0.f) continue;
#pragma unroll
        for (int k = 0; k < NSH; ++k) atomicAdd(&dsh[3 * k + ch], ev_gc[ch] * Y[k]);
      }
      float *acc = sc.gacc + (size_t)ev_idx * 16;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        atomicAdd(&acc[r], ev_v[r]);
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(&acc[3 + 3 * r + c], ev_v[r] * ev_x[c]);
      }
      atomicAdd(&acc[12], ev_dsig);
    }
    has_ev = false;
  };

  const uint2 rg = ranges[tile];
  for (uint32_t start = rg.x; start < rg.y; start += kBatchKB) {
    if (__syncthreads_count(!done) == 0) break;
    const int nb = (int)min((uint32_t)kBatchKB, rg.y - start);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s_idx[t] = vals[start + t];
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      uint32_t idx = s_idx[t];
      stage_particle<RS>(sc, cam, op, rect[view.part_off + idx], idx, s_geo[t], &s_aux[t]);
    }
    stage_sh<NC>(sc, s_idx, nb, s_sh);
    __syncthreads();
    sb = start;
    snb = nb;
    if (__all_sync(0xffffffffu, done)) continue;
    // every lane of the warp walks every staged particle (the emit steps are warp-wide)
    for (int b = 0; b < nb; ++b) {
      float3 og, dg;
      float dd, a;
      bool leave = false;
      float l_a = 0.f, l_r = 0.f, l_g = 0.f, l_b = 0.f;
      uint32_t l_p = 0;
      if (!done && eval_response<RS, false>(s_geo[b], px, py, o, d, og, dg, dd, a, op)) {
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
        } else {
          // closest of the buffer and the new hit (the forward kernel's choice) leaves
          const int bi = kb_select(kb_tau, kb_p, nt, K, tau, true);
          leave = true;
          if (bi < 0) {
            l_a = al; l_r = r0; l_g = r1; l_b = r2; l_p = pos;
          } else {
            l_a = kb_a[bi * nt]; l_r = kb_r[bi * nt]; l_g = kb_g[bi * nt]; l_b = kb_b[bi * nt]; l_p = kb_p[bi * nt];
            kb_tau[bi * nt] = tau; kb_a[bi * nt] = al;
            kb_r[bi * nt] = r0; kb_g[bi * nt] = r1; kb_b[bi * nt] = r2; kb_p[bi * nt] = pos;
          }
        }
      }
      // one blend site for the warp, whichever way its lanes' hits went
      if (leave) blend(l_a, l_r, l_g, l_b, l_p);
      emit();
      if (__all_sync(0xffffffffu, done)) break;
    }
  }
  // end of the list: the remaining hits in ascending (tau_max, arrival), the warp in step
  while (__any_sync(0xffffffffu, !done && nbuf > 0)) {
    if (!done && nbuf > 0) {
      const int bi = kb_select(kb_tau, kb_p, nt, nbuf, 0.f, false);
      blend(kb_a[bi * nt], kb_r[bi * nt], kb_g[bi * nt], kb_b[bi * nt], kb_p[bi * nt]);
      --nbuf;
      kb_tau[bi * nt] = kb_tau[nbuf * nt]; kb_a[bi * nt] = kb_a[nbuf * nt];
      kb_r[bi * nt] = kb_r[nbuf * nt]; kb_g[bi * nt] = kb_g[nbuf * nt]; kb_b[bi * nt] = kb_b[nbuf * nt];
      kb_p[bi * nt] = kb_p[nbuf * nt];
    }
    emit();
  }
}

template <int DEG, bool RS>
ut_status launch_k(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                   const uint32_t *ranges, cudaStream_t s) {
  const int threads = op.tile_w * op.tile_h;
  const size_t smem = sizeof(float) * 6 * (size_t)op.kbuffer * threads;
  constexpr size_t kStatic = sizeof(float4) * kBatchKB * 5 + sizeof(float) * kBatchKB * 3 * (DEG + 1) * (DEG + 1) +
                             sizeof(uint32_t) * kBatchKB;
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
  for (int k = 0; k < bd.ns; ++k) {
    const DevScene &sc = bd.s[k];
    if (sc.n <= 0) continue;
    if (!sc.kbrec) return UT_ERR_INVALID_ARG;
    const int g = (sc.n + 255) / 256, cap = device_sm_count() * 8;
    k_kb_records<<<g < cap ? g : cap, 256, 0, s>>>(sc);
    count_launches(1);
  }
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
