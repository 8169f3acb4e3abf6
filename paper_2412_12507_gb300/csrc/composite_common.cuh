// composite_common.cuh — pieces shared by the compositing forward (composite_fwd.cu) and
// backward (composite_bwd.cu): particle staging, the 3D response at the maximum along a pixel
// ray (Sec. 4.2, eq. GaussianMaxResponse) for the Gaussian and the degree-n kernels
// (supplementary Sec. A), SH colour (per pixel or per particle), pixel setup, and the tile
// schedule both passes use (a counting sort of the tiles by their expected walk, longest first).
//
// One thread block per image tile (global tile ids over all views of the batch), one thread
// per pixel.  The tile's depth-sorted particle list is consumed in batches: the block gathers
// each batch's parameters once, activates them (M = S^-1 R^T, sigma, the alpha_min test
// threshold, packed rect) into shared memory together with their colour data, and every pixel
// then walks the batch from shared memory.
//
// Template RS selects the general ray-origin path (per-pixel origin, needed when any view
// has a rolling shutter); without it the origin is the camera centre of the view.
#pragma once

#include "ut3d_debug.cuh"
#include "ut3d_device.cuh"
#include "ut3d_internal.h"

namespace ut3d {
namespace {

constexpr int kBatch = 64;    // particles staged per block step (backward)
constexpr int kBatchF = 128;  // particles staged per block step (forward)
constexpr int kBatchK = 64;   // particles staged per block step (k-buffer): two blocks of 256 fit an SM
constexpr int kOrderBuckets = 1024;  // log buckets of the backward's tile schedule

// Tile schedule of the backward (device scratch): per-tile replay length, the tiles with work
// ordered by decreasing length, the bucket histogram and scatter cursors, and the count.
struct TileSched {
  uint32_t *work, *order, *hist, *cursor, *n_work;
};

TileSched carve_tile_sched(void *p, int tiles) {
  const size_t t = (size_t)(tiles > 0 ? tiles : 1);
  char *c = static_cast<char *>(p);
  TileSched ts;
  ts.work = reinterpret_cast<uint32_t *>(c);
  ts.order = reinterpret_cast<uint32_t *>(c + align256(sizeof(uint32_t) * t));
  ts.hist = reinterpret_cast<uint32_t *>(c + 2 * align256(sizeof(uint32_t) * t));
  ts.cursor = ts.hist + kOrderBuckets;
  ts.n_work = ts.cursor + kOrderBuckets;
  return ts;
}

// Staged particle record (4 x float4):
//   g0 = M00 M01 M02 M10   g1 = M11 M12 M20 M21   g2 = M22 a.x a.y a.z
//   g3 = sigma, thr = 2 ln(sigma / alpha_min), rect (x0 | y0 << 16), rect (x1 | y1 << 16)
// where a = M (o - mu) with o the camera centre (RS = false) or a = M mu (RS = true).
// aux (backward only) = o - mu (RS = false) or mu (RS = true).
template <bool RS>
__device__ __forceinline__ void stage_particle(const DevScene &sc, const DevCam &cam, const DevOpts &op, short4 r,
                                               uint32_t idx, float4 *g, float4 *aux) {
  // debug build: a listed particle belongs to the scene and its rectangle lies in the image
  UT_DBG_CHECK(idx < (uint32_t)sc.n, UT_DBG_PARTICLE, idx, sc.n, 0);
  UT_DBG_CHECK(r.x >= 0 && r.y >= 0 && r.x <= r.z && r.y <= r.w && r.z < cam.W && r.w < cam.H, UT_DBG_RECT, idx,
               (uint16_t)r.x | ((uint32_t)(uint16_t)r.y << 16), (uint16_t)r.z | ((uint32_t)(uint16_t)r.w << 16));
  float3 mu = make_float3(sc.means[3 * idx], sc.means[3 * idx + 1], sc.means[3 * idx + 2]);
  float3 ls = make_float3(sc.log_scales[3 * idx], sc.log_scales[3 * idx + 1], sc.log_scales[3 * idx + 2]);
  Particle p;
  activate(mu, ls, sc.quats[idx], sc.logits[idx], p);
  float3 a;
  float3 om = make_float3(cam.cen[0] - mu.x, cam.cen[1] - mu.y, cam.cen[2] - mu.z);
  if (RS) a = mat3_mul(p.M, mu);
  else a = mat3_mul(p.M, om);
  // bound on omega^2 where sigma rho >= alpha_min: 2 ln(sigma / alpha_min) for the Gaussian,
  // (ln(sigma / alpha_min) / lambda)^(2/n) for the degree-n kernel exp(-lambda d^n)
  const float lnr = logf(p.sigma / op.alpha_min);
  float thr = op.kernel_degree == 2 ? 2.f * lnr : powf(lnr / op.kernel_lambda, 2.f / op.kernel_degree);
  g[0] = make_float4(p.M[0], p.M[1], p.M[2], p.M[3]);
  g[1] = make_float4(p.M[4], p.M[5], p.M[6], p.M[7]);
  g[2] = make_float4(p.M[8], a.x, a.y, a.z);
  int r0 = ((int)(unsigned short)r.x) | ((int)r.y << 16);
  int r1 = ((int)(unsigned short)r.z) | ((int)r.w << 16);
  g[3] = make_float4(p.sigma, thr, __int_as_float(r0), __int_as_float(r1));
  if (aux) *aux = RS ? make_float4(mu.x, mu.y, mu.z, 0.f) : make_float4(om.x, om.y, om.z, 0.f);
}

// SH coefficients of the batch's particles into shared memory (float4 when aligned).
template <int NC>
__device__ __forceinline__ void stage_sh(const DevScene &sc, const uint32_t *s_idx, int nb, float *s_sh) {
  if constexpr (NC % 4 == 0) {
    if (!sc.sh_vec) {
      for (int f = threadIdx.x; f < nb * NC; f += blockDim.x) {
        int b = f / NC;
        s_sh[f] = sc.sh[(size_t)s_idx[b] * NC + (f - b * NC)];
      }
      return;
    }
    constexpr int N4 = NC / 4;
    const float4 *src = reinterpret_cast<const float4 *>(sc.sh);
    float4 *dst = reinterpret_cast<float4 *>(s_sh);
    for (int f = threadIdx.x; f < nb * N4; f += blockDim.x) {
      int b = f / N4;
      dst[f] = src[(size_t)s_idx[b] * N4 + (f - b * N4)];
    }
  } else {
    for (int f = threadIdx.x; f < nb * NC; f += blockDim.x) {
      int b = f / NC;
      s_sh[f] = sc.sh[(size_t)s_idx[b] * NC + (f - b * NC)];
    }
  }
}

// Raw colour sum_k beta_k,ch Y_k + 1/2 of one staged particle (before the clamp at 0).
template <int NSH>
__device__ __forceinline__ void sh_colour(const float *shb, const float *Y, float &r0, float &r1, float &r2) {
  constexpr int NC = NSH * 3;
  r0 = 0.5f; r1 = 0.5f; r2 = 0.5f;
  if constexpr (NC % 4 == 0) {
    const float4 *s4 = reinterpret_cast<const float4 *>(shb);
#pragma unroll
    for (int j = 0; j < NC / 4; ++j) {
      float4 c = s4[j];
      const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = 4 * j + e, k = idx / 3, ch = idx % 3;
        if (ch == 0) r0 = fmaf(cv[e], Y[k], r0);
        else if (ch == 1) r1 = fmaf(cv[e], Y[k], r1);
        else r2 = fmaf(cv[e], Y[k], r2);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NSH; ++k) {
      r0 = fmaf(shb[3 * k], Y[k], r0);
      r1 = fmaf(shb[3 * k + 1], Y[k], r1);
      r2 = fmaf(shb[3 * k + 2], Y[k], r2);
    }
  }
}

// x^(m/2) for an integer m >= 0: repeated products (and a square root for odd m).
__device__ __forceinline__ float pow_half(float x, int m) {
  float p = (m & 1) ? sqrtf(x) : 1.f;
  for (int i = 0; i < (m >> 1); ++i) p *= x;
  return p;
}

// Response of a staged particle for the ray (o, d) of pixel (px, py).  Returns false if the
// pixel is outside the particle's rect or sigma rho < alpha_min (tested as
// |o_g x d_g|^2 > thr |d_g|^2).  Otherwise returns a = sigma rho(omega^2) — exp(-omega^2/2), or
// exp(-lambda (omega^2)^(n/2)) for a kernel of degree n — and the canonical-space ray (o_g, d_g)
// with |d_g|^2.
// GEN: the degree-n kernel (op.kernel_degree != 2), a separate instantiation so that the
// Gaussian path carries no test for it.
template <bool RS, bool GEN>
__device__ __forceinline__ bool eval_response(const float4 *g, int px, int py, float3 o, float3 d, float3 &og,
                                              float3 &dg, float &dd, float &a, const DevOpts &op) {
  float4 g3 = g[3];
  int r0 = __float_as_int(g3.z), r1 = __float_as_int(g3.w);
  if (px < (r0 & 0xffff) || px > (r1 & 0xffff) || py < (r0 >> 16) || py > (r1 >> 16)) return false;
  float4 g0 = g[0], g1 = g[1], g2 = g[2];
  dg = make_float3(fmaf(g0.x, d.x, fmaf(g0.y, d.y, g0.z * d.z)), fmaf(g0.w, d.x, fmaf(g1.x, d.y, g1.y * d.z)),
                   fmaf(g1.z, d.x, fmaf(g1.w, d.y, g2.x * d.z)));
  if (RS) {
    og = make_float3(fmaf(g0.x, o.x, fmaf(g0.y, o.y, g0.z * o.z)) - g2.y,
                     fmaf(g0.w, o.x, fmaf(g1.x, o.y, g1.y * o.z)) - g2.z,
                     fmaf(g1.z, o.x, fmaf(g1.w, o.y, g2.x * o.z)) - g2.w);
  } else {
    og = make_float3(g2.y, g2.z, g2.w);
  }
  float3 c = cross3(og, dg);
  float cc = fmaf(c.x, c.x, fmaf(c.y, c.y, c.z * c.z));
  dd = fmaf(dg.x, dg.x, fmaf(dg.y, dg.y, dg.z * dg.z));
  if (!(cc <= g3.y * dd)) return false;
  if (!GEN) a = g3.x * __expf(-0.5f * __fdividef(cc, dd));
  else a = g3.x * __expf(-op.kernel_lambda * pow_half(__fdividef(cc, dd), op.kernel_degree));
  return true;
}

// d rho / d omega^2 times sigma, from a = sigma rho at the response's omega^2.
template <bool GEN>
__device__ __forceinline__ float dresponse(const DevOpts &op, float a, float3 og, float3 dg, float dd) {
  if (!GEN) return -0.5f * a;
  const float3 c = cross3(og, dg);
  const float w2 = __fdividef(fmaf(c.x, c.x, fmaf(c.y, c.y, c.z * c.z)), dd);
  return -op.kernel_lambda * 0.5f * (float)op.kernel_degree * pow_half(w2, op.kernel_degree - 2) * a;
}

// Per-particle colour mode: unit view direction of a particle, from the camera centre at the
// mean's shutter time (the rolling-shutter fixed point; t = 0 for a global shutter) to the
// mean, and 1 / the distance.
template <bool RS>
__device__ __forceinline__ float3 particle_dir(const DevCam &cam, const DevOpts &op, float3 mu, float &inv_len) {
  float3 c = make_float3(cam.cen[0], cam.cen[1], cam.cen[2]);
  if (RS && cam.rs) {
    float2 uv;
    float t;
    project_world(cam, op.rs_iters, mat3_mul(cam.R0, mu), uv, t);
    // centre -R(t)^T T(t) with R(t) = Rot(ax, t phi) R0
    const float3 Tt = make_float3(fmaf(t, cam.dT[0], cam.T0[0]), fmaf(t, cam.dT[1], cam.T0[1]),
                                  fmaf(t, cam.dT[2], cam.T0[2]));
    c = mat3_tmul(cam.R0, rotate_axis(cam.ax, make_float3(-Tt.x, -Tt.y, -Tt.z), -t * cam.phi));
  }
  const float3 v = make_float3(mu.x - c.x, mu.y - c.y, mu.z - c.z);
  inv_len = rsqrtf(dot3(v, v));
  return make_float3(v.x * inv_len, v.y * inv_len, v.z * inv_len);
}

// Per-particle colour mode: raw colour sum_k beta_k,ch Y_k(dir) + 1/2 of particle idx.
template <int DEG, bool RS>
__device__ __forceinline__ float4 particle_colour(const DevScene &sc, const DevCam &cam, const DevOpts &op,
                                                  uint32_t idx) {
  constexpr int NSH = (DEG + 1) * (DEG + 1);
  const float3 mu = make_float3(sc.means[3 * idx], sc.means[3 * idx + 1], sc.means[3 * idx + 2]);
  float il;
  const float3 dir = particle_dir<RS>(cam, op, mu, il);
  float Y[NSH];
  sh_basis<DEG>(dir.x, dir.y, dir.z, Y);
  const float *beta = sc.sh + (size_t)idx * NSH * 3;
  float r0 = 0.5f, r1 = 0.5f, r2 = 0.5f;
#pragma unroll
  for (int k = 0; k < NSH; ++k) {
    r0 = fmaf(beta[3 * k], Y[k], r0);
    r1 = fmaf(beta[3 * k + 1], Y[k], r1);
    r2 = fmaf(beta[3 * k + 2], Y[k], r2);
  }
  return make_float4(r0, r1, r2, 0.f);
}

// sum_k a_k grad p_k(x, y, z) for the polynomials p_k that sh_basis evaluates on the unit sphere
// (differentiated as polynomials in x, y, z; callers project onto the tangent plane).
template <int DEG>
__device__ __forceinline__ float3 sh_poly_grad(float x, float y, float z, const float *a) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (DEG >= 1) {
    const float c1 = 0.4886025119029199f;
    gy -= c1 * a[1];
    gz += c1 * a[2];
    gx -= c1 * a[3];
  }
  if (DEG >= 2) {
    const float c4 = 1.0925484305920792f, c6 = 0.31539156525252005f, c8 = 0.5462742152960396f;
    gx += c4 * y * a[4];
    gy += c4 * x * a[4];
    gy -= c4 * z * a[5];
    gz -= c4 * y * a[5];
    gx -= 2.f * c6 * x * a[6];
    gy -= 2.f * c6 * y * a[6];
    gz += 4.f * c6 * z * a[6];
    gx -= c4 * z * a[7];
    gz -= c4 * x * a[7];
    gx += 2.f * c8 * x * a[8];
    gy -= 2.f * c8 * y * a[8];
  }
  if (DEG >= 3) {
    const float c9 = 0.5900435899266435f, c10 = 2.890611442640554f, c11 = 0.4570457994644658f,
                c12 = 0.3731763325901154f, c14 = 1.445305721320277f;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx -= 6.f * c9 * x * y * a[9];
    gy -= 3.f * c9 * (xx - yy) * a[9];
    gx += c10 * y * z * a[10];
    gy += c10 * x * z * a[10];
    gz += c10 * x * y * a[10];
    gx += 2.f * c11 * x * y * a[11];
    gy -= c11 * (4.f * zz - xx - 3.f * yy) * a[11];
    gz -= 8.f * c11 * y * z * a[11];
    gx -= 6.f * c12 * x * z * a[12];
    gy -= 6.f * c12 * y * z * a[12];
    gz += c12 * (6.f * zz - 3.f * xx - 3.f * yy) * a[12];
    gx -= c11 * (4.f * zz - 3.f * xx - yy) * a[13];
    gy += 2.f * c11 * x * y * a[13];
    gz -= 8.f * c11 * x * z * a[13];
    gx += 2.f * c14 * x * z * a[14];
    gy -= 2.f * c14 * y * z * a[14];
    gz += c14 * (xx - yy) * a[14];
    gx -= 3.f * c9 * (xx - yy) * a[15];
    gy += 6.f * c9 * x * y * a[15];
  }
  return make_float3(gx, gy, gz);
}

// Pixel (lx, ly) of thread t within its tile: each warp takes an 8 x 4 block of the tile when
// the tile is made of such blocks (a compact footprint meets fewer distinct particles than a
// 16 x 2 or 32 x 1 strip, so more of the warp's lanes work on each staged particle), else the
// tile is row-major.  Results do not depend on the mapping: every pixel's walk is its own.
__device__ __forceinline__ void tile_pixel(const DevOpts &op, int t, int &lx, int &ly) {
  if (op.tile_w % 8 == 0 && op.tile_h % 4 == 0) {
    const int lane = t & 31, warp = t >> 5, bx = op.tile_w / 8;
    lx = (warp % bx) * 8 + (lane & 7);
    ly = (warp / bx) * 4 + (lane >> 3);
  } else {
    lx = t % op.tile_w;
    ly = t / op.tile_w;
  }
}

template <int DEG>
__device__ __forceinline__ void pixel_setup(const DevCam &cam, const DevOpts &op, int px, int py, bool inside,
                                            float3 &o, float3 &d, float *Y, bool &valid) {
  valid = inside && pixel_ray(cam, px, py, op.newton_iters, o, d);
  if (valid) {
    float in = rsqrtf(dot3(d, d));
    sh_basis<DEG>(d.x * in, d.y * in, d.z * in, Y);
  } else {
    o = d = make_float3(0.f, 0.f, 1.f);
#pragma unroll
    for (int k = 0; k < (DEG + 1) * (DEG + 1); ++k) Y[k] = 0.f;
  }
}

// Log-spaced bucket (about 1.5 % wide) of a tile's replay length.
__device__ __forceinline__ int work_bucket(uint32_t w) {
  return min((int)(48.f * __log2f(1.f + (float)w)), kOrderBuckets - 1);
}

// Counting sort of the tiles with work by descending bucket (heaviest first, so the longest
// replays start in the first wave instead of trailing at the end).  1024 threads per block;
// every block scans the histogram itself and scatters its share of the tiles.
__global__ void __launch_bounds__(kOrderBuckets) k_tile_order(int total_tiles, TileSched ts) {
  __shared__ uint32_t s_off[kOrderBuckets];
  __shared__ uint32_t s_warp[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t h = ts.hist[kOrderBuckets - 1 - t];  // rank t in descending bucket order
  uint32_t incl = h;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = s_warp[lane], x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_warp[lane] = x - v;
  }
  __syncthreads();
  incl += s_warp[warp];
  s_off[kOrderBuckets - 1 - t] = incl - h;
  if (blockIdx.x == 0 && t == kOrderBuckets - 1) *ts.n_work = incl;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + t; i < total_tiles; i += gridDim.x * blockDim.x) {
    const uint32_t w = ts.work[i];
    if (!w) continue;
    const int b = work_bucket(w);
    ts.order[s_off[b] + atomicAdd(&ts.cursor[b], 1u)] = (uint32_t)i;
  }
}

// The k-buffer's closest hit among entries [0, n) of a thread's buffer (tau_max at tau[j * nt],
// list position at pos[j * nt]) and, with with_new, a new hit of tau_max tau0 that arrived last:
// the smallest tau_max, the earlier arrival (smaller list position) on equal tau_max.  Returns
// -1 for the new hit, else the entry.  One pass over tau_max finds the minimum and whether it is
// tied; only a tie (rare: equal FP32 values) takes a second pass over the list positions.
__device__ __forceinline__ int kb_select(const float *tau, const uint32_t *pos, int nt, int n, float tau0,
                                         bool with_new) {
  float bt = with_new ? tau0 : tau[0];
  int bi = with_new ? -1 : 0;
  bool tie = false;
  for (int j = with_new ? 0 : 1; j < n; ++j) {
    const float tj = tau[j * nt];
    tie = tj == bt ? true : (tj < bt ? false : tie);
    if (tj < bt) {
      bt = tj;
      bi = j;
    }
  }
  if (tie) {  // the new hit (arrived last) loses every tie
    uint32_t bp = 0xffffffffu;
    for (int j = 0; j < n; ++j) {
      const uint32_t pj = pos[j * nt];
      if (tau[j * nt] == bt && pj < bp) {
        bp = pj;
        bi = j;
      }
    }
  }
  return bi;
}

bool any_rs(const BatchDesc &bd) {
  for (int v = 0; v < bd.nv; ++v)
    if (bd.v[v].cam.rs) return true;
  return false;
}

}  // namespace
}  // namespace ut3d
