// a3 / a5: front-to-back alpha blending per 16x16 tile and its reverse replay.
//
// One CTA per (unit, tile), one thread per pixel.  The tile's sorted list is
// consumed in batches of BATCH records staged in shared memory (each thread
// gathers one record: its projected index, mean, conic/opacity and colour).
// The backward replays the same list back to front, recovering each
// transmittance by division, reduces the per-record gradients of a warp with
// shuffles (only when some lane contributed), accumulates the 8 warps in
// shared memory and issues one set of global vector atomics per
// (tile, record).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

constexpr int BATCH = 256;

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

__global__ void __launch_bounds__(TILE_PIX) k_render_fwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ vals,
                                                         const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_op,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         int n_tiles, float bg0, float bg1, float bg2,
                                                         float* __restrict__ img, float* __restrict__ final_T,
                                                         uint32_t* __restrict__ n_contrib) {
  __shared__ float2 s_xy[BATCH];
  __shared__ float4 s_co[BATCH];
  __shared__ float4 s_rgb[BATCH];
  int tile = blockIdx.x, u = blockIdx.y;
  int tx = tile % TX, ty = tile / TX;
  int px = tx * TILE + (threadIdx.x & (TILE - 1));
  int py = ty * TILE + (threadIdx.x / TILE);
  bool inside = px < W && py < H;
  uint2 rg = ranges[(int64_t)u * n_tiles + tile];
  int n = (int)(rg.y - rg.x);
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  int last = 0;
  bool done = !inside;
  float fx = (float)px, fy = (float)py;
  for (int b0 = 0; b0 < n; b0 += BATCH) {
    if (__syncthreads_count(!done) == 0) break;
    int k = b0 + threadIdx.x;
    if (k < n) {
      uint32_t p = vals[rg.x + k];
      s_xy[threadIdx.x] = xy[p];
      s_co[threadIdx.x] = conic_op[p];
      s_rgb[threadIdx.x] = rgb[p];
    }
    __syncthreads();
    int m = min(BATCH, n - b0);
    for (int j = 0; !done && j < m; ++j) {
      float2 mxy = s_xy[j];
      float4 co = s_co[j];
      float power = splat_power(co.x, co.y, co.z, mxy.x - fx, mxy.y - fy);
      if (power > 0.f) continue;
      float alpha = fminf(ALPHA_MAX, co.w * __expf(power));
      if (alpha < ALPHA_MIN) continue;
      float tT = T * (1.f - alpha);
      if (tT < T_MIN) { done = true; break; }
      float4 c = s_rgb[j];
      float wgt = alpha * T;
      c0 += c.x * wgt; c1 += c.y * wgt; c2 += c.z * wgt;
      T = tT;
      last = b0 + j + 1;
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
  __shared__ float2 s_xy[BATCH];
  __shared__ float4 s_co[BATCH];
  __shared__ float4 s_rgb[BATCH];
  __shared__ uint32_t s_p[BATCH];
  __shared__ float s_acc[BATCH][9];
  __shared__ int s_max[TILE_PIX / 32];
  int tile = blockIdx.x, u = blockIdx.y;
  int tx = tile % TX, ty = tile / TX;
  int px = tx * TILE + (threadIdx.x & (TILE - 1));
  int py = ty * TILE + (threadIdx.x / TILE);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
  int wm = __reduce_max_sync(0xffffffffu, last);
  if (lane == 0) s_max[w] = wm;
  __syncthreads();
  int n = 0;
  #pragma unroll
  for (int q = 0; q < TILE_PIX / 32; ++q) n = max(n, s_max[q]);
  n = min(n, (int)(rg.y - rg.x));
  float S0 = bg0, S1 = bg1, S2 = bg2;  // colour behind the current entry
  float fx = (float)px, fy = (float)py;
  for (int bend = n; bend > 0; bend -= BATCH) {
    int bstart = max(0, bend - BATCH);
    int m = bend - bstart;
    __syncthreads();
    if ((int)threadIdx.x < m) {
      uint32_t p = vals[rg.x + bstart + threadIdx.x];
      s_p[threadIdx.x] = p;
      s_xy[threadIdx.x] = xy[p];
      s_co[threadIdx.x] = conic_op[p];
      s_rgb[threadIdx.x] = rgb[p];
      #pragma unroll
      for (int q = 0; q < 9; ++q) s_acc[threadIdx.x][q] = 0.f;
    }
    __syncthreads();
    for (int j = m - 1; j >= 0; --j) {
      int pos = bstart + j;
      float v[9];
      #pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = 0.f;
      bool contrib = false;
      if (pos < last) {
        float2 mxy = s_xy[j];
        float4 co = s_co[j];
        float dx = mxy.x - fx, dy = mxy.y - fy;
        float power = splat_power(co.x, co.y, co.z, dx, dy);
        if (power <= 0.f) {
          float G = __expf(power);
          float araw = co.w * G;
          bool clamped = araw > ALPHA_MAX;
          float alpha = clamped ? ALPHA_MAX : araw;
          if (alpha >= ALPHA_MIN) {
            contrib = true;
            T = T / (1.f - alpha);  // transmittance in front of this entry
            float4 c = s_rgb[j];
            float wgt = alpha * T;
            v[6] = wgt * g0; v[7] = wgt * g1; v[8] = wgt * g2;
            float dalpha = T * ((c.x - S0) * g0 + (c.y - S1) * g1 + (c.z - S2) * g2);
            S0 = alpha * c.x + (1.f - alpha) * S0;
            S1 = alpha * c.y + (1.f - alpha) * S1;
            S2 = alpha * c.z + (1.f - alpha) * S2;
            if (!clamped) {
              v[5] = G * dalpha;
              float dp = araw * dalpha;
              v[2] = -0.5f * dx * dx * dp;
              v[3] = -dx * dy * dp;
              v[4] = -0.5f * dy * dy * dp;
              v[0] = -(co.x * dx + co.y * dy) * dp;
              v[1] = -(co.z * dy + co.y * dx) * dp;
            }
          }
        }
      }
      if (__ballot_sync(0xffffffffu, contrib)) {
        #pragma unroll
        for (int q = 0; q < 9; ++q) {
          float x = v[q];
          x += __shfl_xor_sync(0xffffffffu, x, 16);
          x += __shfl_xor_sync(0xffffffffu, x, 8);
          x += __shfl_xor_sync(0xffffffffu, x, 4);
          x += __shfl_xor_sync(0xffffffffu, x, 2);
          x += __shfl_xor_sync(0xffffffffu, x, 1);
          v[q] = x;
        }
        if (lane == 0) {
          #pragma unroll
          for (int q = 0; q < 9; ++q) atomicAdd(&s_acc[j][q], v[q]);
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < m) {
      const float* a = s_acc[threadIdx.x];
      bool nz = false;
      #pragma unroll
      for (int q = 0; q < 9; ++q) nz |= a[q] != 0.f;
      if (nz) {
        uint32_t p = s_p[threadIdx.x];
        atomic_add2(dxy + 2 * (int64_t)p, a[0], a[1]);
        atomic_add4(dco + 4 * (int64_t)p, a[2], a[3], a[4], a[5]);
        atomic_add4(drgb + 4 * (int64_t)p, a[6], a[7], a[8], 0.f);
      }
    }
  }
}

}  // namespace

GS_API int gs_render_fwd(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                         int width, int height, const float* bg, float* img, float* final_T, uint32_t* n_contrib,
                         gs_stream_t stream) {
  if (!proj || !proj->xy || !proj->conic_op || !proj->rgb || !sorted_vals || !ranges || !bg || !img ||
      !final_T || !n_contrib || n_units < 1 || n_units > GS_MAX_UNITS || width <= 0 || height <= 0)
    return GS_ERR_INVALID;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  dim3 grid(TX * TY, n_units);
  k_render_fwd<<<grid, TILE_PIX, 0, (cudaStream_t)stream>>>(
      (const uint2*)ranges, sorted_vals, (const float2*)proj->xy, (const float4*)proj->conic_op,
      (const float4*)proj->rgb, width, height, TX, TX * TY, bg[0], bg[1], bg[2], img, final_T, n_contrib);
  return gs_check_launch();
}

int gs_blend_bwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                      int width, int height, const float* bg, const float* final_T, const uint32_t* n_contrib,
                      const float* dL_dimg, const gs_grad2d* g2d, int64_t n_proj, cudaStream_t s) {
  if (!proj || !proj->xy || !proj->conic_op || !proj->rgb || !sorted_vals || !ranges || !bg || !final_T ||
      !n_contrib || !dL_dimg || !g2d || !g2d->dxy || !g2d->dconic_op || !g2d->drgb || n_units < 1 ||
      n_units > GS_MAX_UNITS || width <= 0 || height <= 0 || n_proj < 0)
    return GS_ERR_INVALID;
  if (cudaMemsetAsync(g2d->dxy, 0, sizeof(float) * 2 * (size_t)n_proj, s) != cudaSuccess ||
      cudaMemsetAsync(g2d->dconic_op, 0, sizeof(float) * 4 * (size_t)n_proj, s) != cudaSuccess ||
      cudaMemsetAsync(g2d->drgb, 0, sizeof(float) * 4 * (size_t)n_proj, s) != cudaSuccess)
    return GS_ERR_CUDA;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  dim3 grid(TX * TY, n_units);
  k_render_bwd<<<grid, TILE_PIX, 0, s>>>((const uint2*)ranges, sorted_vals, (const float2*)proj->xy,
                                         (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height, TX,
                                         TX * TY, bg[0], bg[1], bg[2], final_T, n_contrib, dL_dimg, g2d->dxy,
                                         g2d->dconic_op, g2d->drgb);
  return gs_check_launch();
}
