// a3 / a5: front-to-back alpha blending per 16x16 tile and its reverse replay.
//
// One CTA per (unit, tile), one thread per pixel; each warp owns a BW x (32/BW)
// pixel block of the 16x16 tile (BW = 8, 16 or 4: the tunable variant) and walks the tile's list
// independently of the other warps (no block barriers: warps whose block few
// splats reach do not wait for the busy ones).  A record is blended by a warp
// only if the bounding box of the ellipse where its alpha can reach 1/255
// meets the warp's block; this skips only (pixel, record) pairs that the
// per-pixel alpha test would reject anyway, so results are unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

__device__ __forceinline__ void atomic_add2(float* p, float a, float b) {
#if __CUDA_ARCH__ >= 900
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(a, b));
#else
  atomicAdd(p, a); atomicAdd(p + 1, b);
#endif
}
__device__ __forceinline__ void atomic_add4(float* p, float a, float b, float c, float d) {
#if __CUDA_ARCH__ >= 900
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
#else
  atomicAdd(p, a); atomicAdd(p + 1, b); atomicAdd(p + 2, c); atomicAdd(p + 3, d);
#endif
}

// Bounding box (xmin, xmax, ymin, ymax) of {d : o exp(-d^T Q d / 2) >= 1/255},
// i.e. d^T Q d <= 2 ln(255 o), half-widths sqrt(2 ln(255 o) Sigma_xx) with
// Sigma = Q^-1; inflated so float rounding can never cull a passing pixel.
// An empty box (xmin > xmax) when o < 1/255.  Also returns the power below
// which alpha < 1/255 for certain (used to skip the exponential).
__device__ __forceinline__ float4 alpha_box(float2 m, float4 co, float& pmin) {
  float tau = logf(255.f * co.w) + 1e-3f;  // >= ln(255 o) with margin
  float det = co.x * co.z - co.y * co.y;
  if (!(tau > 0.f) || !(det > 0.f)) {
    pmin = 0.f;
    return make_float4(1.f, -1.f, 1.f, -1.f);
  }
  float sxx = co.z / det, syy = co.x / det;
  float ex = sqrtf(2.f * tau * sxx) * 1.001f + 0.01f;
  float ey = sqrtf(2.f * tau * syy) * 1.001f + 0.01f;
  pmin = -tau * 1.001f - 1e-3f;
  return make_float4(m.x - ex, m.x + ex, m.y - ey, m.y + ey);
}

__device__ __forceinline__ bool box_misses(float4 b, float x0, float x1, float y0, float y1) {
  return b.y < x0 || b.x > x1 || b.w < y0 || b.z > y1;
}

// Forward.  Each warp walks its tile's list on its own, 32 records per round
// (one per lane): a lane loads a record and tests its alpha box against the
// warp's 8x4 pixel block; the records that hit are taken in list order and
// broadcast with shuffles.  The next round's loads are issued before the
// current round is blended.
template <int BW>
__global__ void __launch_bounds__(TILE_PIX) k_render_fwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ vals,
                                                         const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_op,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         int n_tiles, float bg0, float bg1, float bg2,
                                                         float* __restrict__ img, float* __restrict__ final_T,
                                                         uint32_t* __restrict__ n_contrib) {
  const unsigned FULL = 0xffffffffu;
  int tile = blockIdx.x, u = blockIdx.y;
  int tx = tile % TX, ty = tile / TX;
  constexpr int BH = 32 / BW, NWX = TILE / BW;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float wx0 = (float)(tx * TILE + (w % NWX) * BW), wy0 = (float)(ty * TILE + (w / NWX) * BH);
  float wx1 = wx0 + (float)(BW - 1), wy1 = wy0 + (float)(BH - 1);
  int px = (int)wx0 + (lane % BW), py = (int)wy0 + (lane / BW);
  bool inside = px < W && py < H;
  uint2 rg = ranges[(int64_t)u * n_tiles + tile];
  int n = (int)(rg.y - rg.x);
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  int last = 0;
  bool done = !inside;
  float fx = (float)px, fy = (float)py;
  // prefetch of the first round
  uint32_t p_n = 0;
  float2 m_n = make_float2(0.f, 0.f);
  float4 co_n = make_float4(0.f, 0.f, 0.f, 0.f);
  if (lane < n) { p_n = vals[rg.x + lane]; m_n = xy[p_n]; co_n = conic_op[p_n]; }
  for (int base = 0; base < n; base += 32) {
    if (__all_sync(FULL, done)) break;
    uint32_t p = p_n;
    float2 m = m_n;
    float4 co = co_n;
    bool valid = base + lane < n;
    int kn = base + 32 + lane;
    if (kn < n) { p_n = vals[rg.x + kn]; m_n = xy[p_n]; co_n = conic_op[p_n]; }
    float pmin = 0.f;
    bool hit = false;
    if (valid) {
      float4 b = alpha_box(m, co, pmin);
      hit = !box_misses(b, wx0, wx1, wy0, wy1);
    }
    unsigned mask = __ballot_sync(FULL, hit);
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (hit) c = rgb[p];
    while (mask) {
      int j = __ffs(mask) - 1;
      mask &= mask - 1;
      float ex = __shfl_sync(FULL, m.x, j), ey = __shfl_sync(FULL, m.y, j);
      float A = __shfl_sync(FULL, co.x, j), B = __shfl_sync(FULL, co.y, j);
      float Cc = __shfl_sync(FULL, co.z, j), op = __shfl_sync(FULL, co.w, j);
      float pm = __shfl_sync(FULL, pmin, j);
      float r = __shfl_sync(FULL, c.x, j), gg = __shfl_sync(FULL, c.y, j), bb = __shfl_sync(FULL, c.z, j);
      if (done) continue;
      float power = splat_power(A, B, Cc, ex - fx, ey - fy);
      if (power > 0.f || power < pm) continue;
      float alpha = fminf(ALPHA_MAX, op * __expf(power));
      if (alpha < ALPHA_MIN) continue;
      float tT = T * (1.f - alpha);
      if (tT < T_MIN) { done = true; continue; }
      float wgt = alpha * T;
      c0 += r * wgt; c1 += gg * wgt; c2 += bb * wgt;
      T = tT;
      last = base + j + 1;
    }
  }
  if (inside) {
    int64_t plane = (int64_t)W * H;
    int64_t pix = (int64_t)py * W + px;
    float* im = img + (int64_t)u * 3 * plane;
    im[pix] = c0 + T * bg0;
    im[plane + pix] = c1 + T * bg1;
    im[2 * plane + pix] = c2 + T * bg2;
    final_T[(int64_t)u * plane + pix] = T;
    n_contrib[(int64_t)u * plane + pix] = (uint32_t)last;
  }
}

// Backward.  Each warp replays its tile's list back to front from the largest
// n_contrib among its pixels, in rounds of 32 records; hits are taken in
// reverse list order.  The 9 gradient values of a record are summed over the
// warp with xor shuffles (only if some lane contributed); the lane that loaded
// the record keeps the sum and issues the global vector atomics at the end of
// the round.
template <int BW>
__global__ void __launch_bounds__(TILE_PIX) k_render_bwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ vals,
                                                         const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_op,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         int n_tiles, float bg0, float bg1, float bg2,
                                                         const float* __restrict__ final_T,
                                                         const uint32_t* __restrict__ n_contrib,
                                                         const float* __restrict__ dimg, float* __restrict__ dxy,
                                                         float* __restrict__ dco, float* __restrict__ drgb) {
  const unsigned FULL = 0xffffffffu;
  int tile = blockIdx.x, u = blockIdx.y;
  int tx = tile % TX, ty = tile / TX;
  constexpr int BH = 32 / BW, NWX = TILE / BW;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float wx0 = (float)(tx * TILE + (w % NWX) * BW), wy0 = (float)(ty * TILE + (w / NWX) * BH);
  float wx1 = wx0 + (float)(BW - 1), wy1 = wy0 + (float)(BH - 1);
  int px = (int)wx0 + (lane % BW), py = (int)wy0 + (lane / BW);
  bool inside = px < W && py < H;
  uint2 rg = ranges[(int64_t)u * n_tiles + tile];
  int64_t plane = (int64_t)W * H;
  int64_t pix = (int64_t)py * W + px;
  float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  int last = 0;
  if (inside) {
    T = final_T[(int64_t)u * plane + pix];
    last = (int)n_contrib[(int64_t)u * plane + pix];
    const float* d = dimg + (int64_t)u * 3 * plane;
    g0 = d[pix]; g1 = d[plane + pix]; g2 = d[2 * plane + pix];
  }
  int n = min(__reduce_max_sync(FULL, last), (int)(rg.y - rg.x));
  float S0 = bg0, S1 = bg1, S2 = bg2;  // colour behind the current entry
  float fx = (float)px, fy = (float)py;
  for (int top = n; top > 0; top -= 32) {
    int base = top - 32;
    int k = base + lane;
    bool valid = k >= 0;
    uint32_t p = 0;
    float2 m = make_float2(0.f, 0.f);
    float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
    bool hit = false;
    if (valid) {
      p = vals[rg.x + k];
      m = xy[p];
      co = conic_op[p];
      float pm;
      float4 b = alpha_box(m, co, pm);
      hit = !box_misses(b, wx0, wx1, wy0, wy1);
    }
    unsigned mask = __ballot_sync(FULL, hit);
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (hit) c = rgb[p];
    float acc[9];
    #pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.f;
    bool mine = false;  // this lane's record received a contribution
    while (mask) {
      int j = 31 - __clz(mask);
      mask &= ~(1u << j);
      float ex = __shfl_sync(FULL, m.x, j), ey = __shfl_sync(FULL, m.y, j);
      float A = __shfl_sync(FULL, co.x, j), B = __shfl_sync(FULL, co.y, j);
      float Cc = __shfl_sync(FULL, co.z, j), op = __shfl_sync(FULL, co.w, j);
      float cr = __shfl_sync(FULL, c.x, j), cg = __shfl_sync(FULL, c.y, j), cb = __shfl_sync(FULL, c.z, j);
      int pos = base + j;
      float v[9];
      #pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = 0.f;
      bool contrib = false;
      if (pos < last) {
        float dx = ex - fx, dy = ey - fy;
        float power = splat_power(A, B, Cc, dx, dy);
        if (power <= 0.f) {
          float G = __expf(power);
          float araw = op * G;
          bool clamped = araw > ALPHA_MAX;
          float alpha = clamped ? ALPHA_MAX : araw;
          if (alpha >= ALPHA_MIN) {
            contrib = true;
            T = __fdividef(T, 1.f - alpha);  // transmittance in front of this entry
            float wgt = alpha * T;
            v[6] = wgt * g0; v[7] = wgt * g1; v[8] = wgt * g2;
            float dalpha = T * ((cr - S0) * g0 + (cg - S1) * g1 + (cb - S2) * g2);
            S0 = alpha * cr + (1.f - alpha) * S0;
            S1 = alpha * cg + (1.f - alpha) * S1;
            S2 = alpha * cb + (1.f - alpha) * S2;
            if (!clamped) {
              v[5] = G * dalpha;
              float dp = araw * dalpha;
              v[2] = -0.5f * dx * dx * dp;
              v[3] = -dx * dy * dp;
              v[4] = -0.5f * dy * dy * dp;
              v[0] = -(A * dx + B * dy) * dp;
              v[1] = -(Cc * dy + B * dx) * dp;
            }
          }
        }
      }
      if (__ballot_sync(FULL, contrib)) {
        #pragma unroll
        for (int q = 0; q < 9; ++q) {
          float x = v[q];
          x += __shfl_xor_sync(FULL, x, 16);
          x += __shfl_xor_sync(FULL, x, 8);
          x += __shfl_xor_sync(FULL, x, 4);
          x += __shfl_xor_sync(FULL, x, 2);
          x += __shfl_xor_sync(FULL, x, 1);
          if (lane == j) acc[q] = x;
        }
        if (lane == j) mine = true;
      }
    }
    if (mine) {
      atomic_add2(dxy + 2 * (int64_t)p, acc[0], acc[1]);
      atomic_add4(dco + 4 * (int64_t)p, acc[2], acc[3], acc[4], acc[5]);
      atomic_add4(drgb + 4 * (int64_t)p, acc[6], acc[7], acc[8], 0.f);
    }
  }
}

// Number of blended (pixel, record) pairs: records before n_contrib whose
// alpha reaches 1/255 (the work any implementation of the blend must do).
__global__ void __launch_bounds__(TILE_PIX) k_blend_pairs(const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ vals,
                                                          const float2* __restrict__ xy,
                                                          const float4* __restrict__ conic_op, int W, int H, int TX,
                                                          int n_tiles, const uint32_t* __restrict__ n_contrib,
                                                          unsigned long long* __restrict__ count) {
  int tile = blockIdx.x, u = blockIdx.y;
  int tx = tile % TX, ty = tile / TX;
  int px = tx * TILE + (threadIdx.x & 15), py = ty * TILE + (threadIdx.x >> 4);
  unsigned long long c = 0;
  if (px < W && py < H) {
    uint2 rg = ranges[(int64_t)u * n_tiles + tile];
    int last = (int)n_contrib[(int64_t)u * W * H + (int64_t)py * W + px];
    for (int j = 0; j < last; ++j) {
      uint32_t p = vals[rg.x + j];
      float2 m = xy[p];
      float4 co = conic_op[p];
      float power = splat_power(co.x, co.y, co.z, m.x - (float)px, m.y - (float)py);
      if (power > 0.f) continue;
      float alpha = fminf(ALPHA_MAX, co.w * __expf(power));
      if (alpha >= ALPHA_MIN) ++c;
    }
  }
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

int gs_render_fwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                       int width, int height, const float* bg, float* img, float* final_T, uint32_t* n_contrib,
                       int variant, cudaStream_t s) {
  if (!proj || !proj->xy || !proj->conic_op || !proj->rgb || !sorted_vals || !ranges || !bg || !img ||
      !final_T || !n_contrib || n_units < 1 || n_units > GS_MAX_UNITS || width <= 0 || height <= 0 ||
      variant < 0 || variant > 2)
    return GS_ERR_INVALID;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  dim3 grid(TX * TY, n_units);
#define GS_FWD(BW)                                                                                                \
  k_render_fwd<BW><<<grid, TILE_PIX, 0, s>>>((const uint2*)ranges, sorted_vals, (const float2*)proj->xy,          \
                                             (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height, \
                                             TX, TX * TY, bg[0], bg[1], bg[2], img, final_T, n_contrib)
  if (variant == 0) GS_FWD(8); else if (variant == 1) GS_FWD(16); else GS_FWD(4);
#undef GS_FWD
  return gs_check_launch();
}

GS_API int gs_render_fwd(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                         int width, int height, const float* bg, float* img, float* final_T, uint32_t* n_contrib,
                         int variant, gs_stream_t stream) {
  return gs_render_fwd_impl(proj, sorted_vals, ranges, n_units, width, height, bg, img, final_T, n_contrib, variant,
                            (cudaStream_t)stream);
}

int gs_blend_bwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                      int width, int height, const float* bg, const float* final_T, const uint32_t* n_contrib,
                      const float* dL_dimg, const gs_grad2d* g2d, int64_t n_proj, int variant, cudaStream_t s) {
  if (!proj || !proj->xy || !proj->conic_op || !proj->rgb || !sorted_vals || !ranges || !bg || !final_T ||
      !n_contrib || !dL_dimg || !g2d || !g2d->dxy || !g2d->dconic_op || !g2d->drgb || n_units < 1 ||
      n_units > GS_MAX_UNITS || width <= 0 || height <= 0 || n_proj < 0 || variant < 0 || variant > 2)
    return GS_ERR_INVALID;
  if (cudaMemsetAsync(g2d->dxy, 0, sizeof(float) * 2 * (size_t)n_proj, s) != cudaSuccess ||
      cudaMemsetAsync(g2d->dconic_op, 0, sizeof(float) * 4 * (size_t)n_proj, s) != cudaSuccess ||
      cudaMemsetAsync(g2d->drgb, 0, sizeof(float) * 4 * (size_t)n_proj, s) != cudaSuccess)
    return GS_ERR_CUDA;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  dim3 grid(TX * TY, n_units);
#define GS_BWD(BW)                                                                                                   \
  k_render_bwd<BW><<<grid, TILE_PIX, 0, s>>>((const uint2*)ranges, sorted_vals, (const float2*)proj->xy,             \
                                             (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height,    \
                                             TX, TX * TY, bg[0], bg[1], bg[2], final_T, n_contrib, dL_dimg, g2d->dxy, \
                                             g2d->dconic_op, g2d->drgb)
  if (variant == 0) GS_BWD(8); else if (variant == 1) GS_BWD(16); else GS_BWD(4);
#undef GS_BWD
  return gs_check_launch();
}

GS_API int gs_blend_pairs(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                          int width, int height, const uint32_t* n_contrib, unsigned long long* d_count,
                          gs_stream_t stream) {
  if (!proj || !proj->xy || !proj->conic_op || !sorted_vals || !ranges || !n_contrib || !d_count || n_units < 1 ||
      n_units > GS_MAX_UNITS || width <= 0 || height <= 0)
    return GS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s) != cudaSuccess) return GS_ERR_CUDA;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  k_blend_pairs<<<dim3(TX * TY, n_units), TILE_PIX, 0, s>>>((const uint2*)ranges, sorted_vals, (const float2*)proj->xy,
                                                            (const float4*)proj->conic_op, width, height, TX, TX * TY,
                                                            n_contrib, d_count);
  return gs_check_launch();
}
