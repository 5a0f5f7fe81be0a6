// a4: masked L1 + SSIM photometric loss and its image gradient.
//
// The mask restricts the loss to the pixels a partition owns (paper Sec. II,
// "Image Rendering and Masking").  SSIM uses the 11x11 Gaussian window
// (sigma 1.5) as a separable, zero-padded "same" convolution; each 16x16
// output tile stages its (16+10)^2 input halo in shared memory.  The SSIM
// gradient w.r.t. the rendered image is the adjoint convolution of three
// per-pixel factor maps (dS/dmu_x, dS/dE[x^2], dS/dE[xy] times the mask
// weight), again separable and zero padded.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

constexpr int LT = 16;           // output tile edge
constexpr int R = 5;             // window radius
constexpr int HT = LT + 2 * R;   // halo tile edge (26)
constexpr float C1 = 0.01f * 0.01f;
constexpr float C2 = 0.03f * 0.03f;

// Normalised 11-tap Gaussian window (sigma 1.5), computed by each block.
__device__ __forceinline__ void load_window(float* w) {
  if (threadIdx.x < 11) {
    float s = 0.f;
    for (int t = 0; t < 11; ++t) s += expf(-(t - 5.f) * (t - 5.f) / (2.f * 1.5f * 1.5f));
    float d = threadIdx.x - 5.f;
    w[threadIdx.x] = expf(-d * d / (2.f * 1.5f * 1.5f)) / s;
  }
}

__host__ __device__ inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct LossWs {
  size_t msum, l1, ss, fac, total;
};
LossWs loss_ws(int U, int W, int H) {
  LossWs L;
  size_t o = 0;
  L.msum = o; o += a256(sizeof(uint32_t) * U);
  L.l1 = o; o += a256(sizeof(double) * U);
  L.ss = o; o += a256(sizeof(double) * U);
  L.fac = o; o += a256(sizeof(float) * 3 * 3 * (size_t)U * W * H);
  L.total = o;
  return L;
}

__device__ __forceinline__ float block_sum(float v, float* s) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s[w] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s[q];
  return t;  // valid in thread 0
}

__global__ void k_mask_count(const uint8_t* __restrict__ mask, int64_t plane, uint32_t* msum) {
  __shared__ float s[32];
  int u = blockIdx.y;
  uint32_t c = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < plane; k += (int64_t)gridDim.x * blockDim.x)
    c += mask[(int64_t)u * plane + k] ? 1u : 0u;
  float t = block_sum((float)c, s);
  if (threadIdx.x == 0 && t > 0.f) atomicAdd(&msum[u], (uint32_t)t);
}

// L1 part only (lambda = 0): gradient and loss sums
__global__ void k_l1(const float* __restrict__ img, const float* __restrict__ gt, const uint8_t* __restrict__ mask,
                     int64_t plane, const uint32_t* __restrict__ msum, float w1, float invU, double* l1sum,
                     float* __restrict__ dimg) {
  __shared__ float s[32];
  int u = blockIdx.y;
  float acc = 0.f;
  float nm = (float)msum[u];
  float scale = nm > 0.f ? w1 * invU / (3.f * nm) : 0.f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < plane; k += (int64_t)gridDim.x * blockDim.x) {
    bool in = mask[(int64_t)u * plane + k] != 0;
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
      int64_t q = ((int64_t)u * 3 + c) * plane + k;
      float d = img[q] - gt[q];
      float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      dimg[q] = in ? scale * sg : 0.f;
      if (in) acc += fabsf(d);
    }
  }
  float t = block_sum(acc, s);
  if (threadIdx.x == 0 && t != 0.f) atomicAdd(&l1sum[u], (double)t);
}

// Separable 11-tap window over a (HT x HT) halo tile of NQ quantities held in
// shared memory; result for output pixel (ly, lx) of each quantity.
template <int NQ>
__device__ __forceinline__ void conv_tile(float (*in)[HT][HT], float (*tmp)[HT][LT], float* out, int lx, int ly,
                                          const float* c_win) {
  // horizontal: rows 0..HT-1, output columns 0..LT-1
  for (int k = threadIdx.x; k < HT * LT; k += blockDim.x) {
    int r = k / LT, cx = k % LT;
    #pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float a = 0.f;
      #pragma unroll
      for (int t = 0; t < 11; ++t) a += c_win[t] * in[q][r][cx + t];
      tmp[q][r][cx] = a;
    }
  }
  __syncthreads();
  #pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float a = 0.f;
    #pragma unroll
    for (int t = 0; t < 11; ++t) a += c_win[t] * tmp[q][ly + t][lx];
    out[q] = a;
  }
}

// SSIM statistics, loss sums and the three factor maps.
__global__ void __launch_bounds__(256) k_ssim_stats(const float* __restrict__ img, const float* __restrict__ gt,
                                                    const uint8_t* __restrict__ mask, int W, int H,
                                                    const uint32_t* __restrict__ msum, float lam, float invU,
                                                    double* l1sum, double* ssum, float* __restrict__ fac) {
  __shared__ float s_in[5][HT][HT];
  __shared__ float s_tmp[5][HT][LT];
  __shared__ float s_red[32];
  __shared__ float s_win[11];
  int tiles_x = (W + LT - 1) / LT;
  int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  int c = blockIdx.y, u = blockIdx.z;
  int64_t plane = (int64_t)W * H;
  {
    // a tile without mask pixels adds nothing to the loss and has no factor map entries
    int qx = bx * LT + (int)(threadIdx.x % LT), qy = by * LT + (int)(threadIdx.x / LT);
    bool m = qx < W && qy < H && mask[(int64_t)u * plane + (int64_t)qy * W + qx] != 0;
    if (!__syncthreads_or(m)) return;
  }
  load_window(s_win);
  const float* X = img + ((int64_t)u * 3 + c) * plane;
  const float* Y = gt + ((int64_t)u * 3 + c) * plane;
  int x0 = bx * LT - R, y0 = by * LT - R;
  for (int k = threadIdx.x; k < HT * HT; k += blockDim.x) {
    int r = k / HT, q = k % HT;
    int gx = x0 + q, gy = y0 + r;
    float a = 0.f, b = 0.f;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) { a = X[(int64_t)gy * W + gx]; b = Y[(int64_t)gy * W + gx]; }
    s_in[0][r][q] = a; s_in[1][r][q] = b; s_in[2][r][q] = a * a; s_in[3][r][q] = b * b; s_in[4][r][q] = a * b;
  }
  __syncthreads();
  int lx = threadIdx.x % LT, ly = threadIdx.x / LT;
  float st[5];
  conv_tile<5>(s_in, s_tmp, st, lx, ly, s_win);
  int px = bx * LT + lx, py = by * LT + ly;
  float nm = (float)msum[u];
  float sacc = 0.f, lacc = 0.f;
  if (px < W && py < H) {
    int64_t pix = (int64_t)py * W + px;
    bool in = mask[(int64_t)u * plane + pix] != 0;
    float fmu = 0.f, fxx = 0.f, fxy = 0.f;
    if (in && nm > 0.f) {
      float ux = st[0], uy = st[1];
      float vx = st[2] - ux * ux, vy = st[3] - uy * uy, cxy = st[4] - ux * uy;
      float A1 = 2.f * ux * uy + C1, A2 = 2.f * cxy + C2;
      float B1 = ux * ux + uy * uy + C1, B2 = vx + vy + C2;
      float S = (A1 * A2) / (B1 * B2);
      sacc = S;
      lacc = fabsf(X[pix] - Y[pix]);
      float wp = -lam * invU / (3.f * nm);  // d loss / d S_p
      fmu = wp * S * (2.f * uy / A1 - 2.f * ux / B1 - 2.f * uy / A2 + 2.f * ux / B2);
      fxx = wp * S * (-1.f / B2);
      fxy = wp * S * (2.f / A2);
    }
    if (in) {  // the factor maps are zero off the mask; only mask pixels are stored and read
      int64_t base = ((int64_t)u * 3 + c) * plane + pix;
      int64_t fs = (int64_t)3 * plane * gridDim.z;  // stride between the three factor maps
      fac[base] = fmu;
      fac[fs + base] = fxx;
      fac[2 * fs + base] = fxy;
    }
  }
  float ts = block_sum(sacc, s_red);
  if (threadIdx.x == 0 && ts != 0.f) atomicAdd(&ssum[u], (double)ts);
  float tl = block_sum(lacc, s_red);
  if (threadIdx.x == 0 && tl != 0.f) atomicAdd(&l1sum[u], (double)tl);
}

// dL/dimg = L1 part + conv(fmu) + 2 x conv(fxx) + y conv(fxy)
__global__ void __launch_bounds__(256) k_ssim_grad(const float* __restrict__ img, const float* __restrict__ gt,
                                                   const uint8_t* __restrict__ mask, int W, int H,
                                                   const uint32_t* __restrict__ msum, float w1, float invU,
                                                   const float* __restrict__ fac, float* __restrict__ dimg) {
  __shared__ float s_in[3][HT][HT];
  __shared__ float s_tmp[3][HT][LT];
  __shared__ float s_win[11];
  int tiles_x = (W + LT - 1) / LT;
  int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  int c = blockIdx.y, u = blockIdx.z;
  int64_t plane = (int64_t)W * H;
  int64_t off = ((int64_t)u * 3 + c) * plane;
  int64_t fs = (int64_t)3 * plane * gridDim.z;
  int x0 = bx * LT - R, y0 = by * LT - R;
  // factor maps are nonzero only at mask pixels: read them there, zero elsewhere
  bool any = false;
  for (int k = threadIdx.x; k < HT * HT; k += blockDim.x) {
    int r = k / HT, q = k % HT;
    int gx = x0 + q, gy = y0 + r;
    float a = 0.f, b = 0.f, d = 0.f;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H && mask[(int64_t)u * plane + (int64_t)gy * W + gx] != 0) {
      int64_t pix = off + (int64_t)gy * W + gx;
      a = fac[pix]; b = fac[fs + pix]; d = fac[2 * fs + pix];
      any = true;
    }
    s_in[0][r][q] = a; s_in[1][r][q] = b; s_in[2][r][q] = d;
  }
  if (!__syncthreads_or(any)) {
    // no mask pixel within the window's reach: both gradient terms vanish
    int px = bx * LT + (int)(threadIdx.x % LT), py = by * LT + (int)(threadIdx.x / LT);
    if (px < W && py < H) dimg[off + (int64_t)py * W + px] = 0.f;
    return;
  }
  load_window(s_win);
  __syncthreads();
  int lx = threadIdx.x % LT, ly = threadIdx.x / LT;
  float cv[3];
  conv_tile<3>(s_in, s_tmp, cv, lx, ly, s_win);
  int px = bx * LT + lx, py = by * LT + ly;
  if (px < W && py < H) {
    int64_t pix = (int64_t)py * W + px;
    float x = img[off + pix], y = gt[off + pix];
    float nm = (float)msum[u];
    bool in = mask[(int64_t)u * plane + pix] != 0;
    float d = x - y;
    float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    float gl1 = (in && nm > 0.f) ? w1 * invU / (3.f * nm) * sg : 0.f;
    dimg[off + pix] = gl1 + cv[0] + 2.f * x * cv[1] + y * cv[2];
  }
}

__global__ void k_loss_final(const uint32_t* msum, const double* l1sum, const double* ssum, int U, float lam,
                             float* out) {
  double acc = 0.0;
  for (int u = 0; u < U; ++u) {
    double nm = (double)msum[u];
    if (nm <= 0.0) continue;
    double l1 = l1sum[u] / (3.0 * nm);
    double v = (1.0 - lam) * l1;
    if (lam > 0.f) v += lam * (1.0 - ssum[u] / (3.0 * nm));
    acc += v;
  }
  *out = (float)(acc / U);
}

// Background-opacity penalty (variant of the mask): per unit, the number of pixels outside the mask
// and the sum of their rendered opacity 1 - T_final (one atomic per warp).
__global__ void __launch_bounds__(256) k_bg_sum(const float* __restrict__ final_T, const uint8_t* __restrict__ mask,
                                                int64_t plane, unsigned long long* __restrict__ cnt,
                                                double* __restrict__ sum) {
  int u = blockIdx.y;
  const float* T = final_T + (int64_t)u * plane;
  const uint8_t* m = mask + (int64_t)u * plane;
  unsigned c = 0;
  double a = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < plane; k += (int64_t)gridDim.x * blockDim.x)
    if (m[k] == 0) { ++c; a += (double)(1.f - T[k]); }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    a += __shfl_down_sync(0xffffffffu, a, o);
  }
  if ((threadIdx.x & 31) == 0 && c) {
    atomicAdd(&cnt[u], (unsigned long long)c);
    atomicAdd(&sum[u], a);
  }
}

// dpenalty/dT_final: -lambda / (U n_bg) at the unit's background pixels, 0 at mask pixels
__global__ void __launch_bounds__(256) k_bg_grad(const uint8_t* __restrict__ mask, int64_t plane,
                                                 const unsigned long long* __restrict__ cnt, float lam, float invU,
                                                 float* __restrict__ dLdT) {
  int u = blockIdx.y;
  unsigned long long n = cnt[u];
  float g = n ? -lam * invU / (float)n : 0.f;
  const uint8_t* m = mask + (int64_t)u * plane;
  float* d = dLdT + (int64_t)u * plane;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < plane; k += (int64_t)gridDim.x * blockDim.x)
    d[k] = m[k] == 0 ? g : 0.f;
}

__global__ void k_bg_final(const unsigned long long* cnt, const double* sum, int U, float lam, float* out) {
  double acc = 0.0;
  for (int u = 0; u < U; ++u)
    if (cnt[u]) acc += sum[u] / (double)cnt[u];
  *out += (float)(lam * acc / U);
}

}  // namespace

GS_API size_t gs_bg_penalty_workspace_size(int n_units) {
  if (n_units < 1) return 0;
  return a256(sizeof(unsigned long long) * (size_t)n_units) + a256(sizeof(double) * (size_t)n_units);
}

GS_API int gs_bg_penalty(const float* final_T, const uint8_t* mask, int n_units, int width, int height,
                         float lambda_bg, void* workspace, size_t workspace_bytes, float* d_loss, float* dL_dT,
                         gs_stream_t stream) {
  GS_RANGE("gs_bg_penalty");
  if (!final_T || !mask || !d_loss || !dL_dT || !workspace || n_units < 1 || n_units > GS_MAX_UNITS || width <= 0 ||
      height <= 0 || !(lambda_bg >= 0.f) || !isfinite(lambda_bg))
    return GS_ERR_INVALID;
  size_t need = gs_bg_penalty_workspace_size(n_units);
  if (workspace_bytes < need || ((uintptr_t)workspace & 255u)) return GS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* cnt = (unsigned long long*)workspace;
  double* sum = (double*)((char*)workspace + a256(sizeof(unsigned long long) * (size_t)n_units));
  if (cudaMemsetAsync(workspace, 0, need, s) != cudaSuccess) return GS_ERR_CUDA;
  int64_t plane = (int64_t)width * height;
  int gx = (int)((plane + 255) / 256);
  if (gx > 1024) gx = 1024;
  k_bg_sum<<<dim3(gx, n_units), 256, 0, s>>>(final_T, mask, plane, cnt, sum);
  k_bg_grad<<<dim3(gx, n_units), 256, 0, s>>>(mask, plane, cnt, lambda_bg, 1.f / n_units, dL_dT);
  k_bg_final<<<1, 1, 0, s>>>(cnt, sum, n_units, lambda_bg, d_loss);
  return gs_check_launch();
}

GS_API size_t gs_loss_workspace_size(int n_units, int width, int height) {
  if (n_units < 1 || width <= 0 || height <= 0) return 0;
  return loss_ws(n_units, width, height).total;
}

GS_API int gs_loss(const float* img, const float* gt, const uint8_t* mask, int n_units, int width, int height,
                   float lambda_ssim, void* workspace, size_t workspace_bytes, float* d_loss, float* dL_dimg,
                   gs_stream_t stream) {
  GS_RANGE("gs_loss");
  if (!img || !gt || !mask || !d_loss || !dL_dimg || !workspace || n_units < 1 || width <= 0 || height <= 0 ||
      !(lambda_ssim >= 0.f && lambda_ssim <= 1.f))
    return GS_ERR_INVALID;
  LossWs L = loss_ws(n_units, width, height);
  if (workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) return GS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  uint32_t* msum = (uint32_t*)(ws + L.msum);
  double* l1 = (double*)(ws + L.l1);
  double* ss = (double*)(ws + L.ss);
  float* fac = (float*)(ws + L.fac);
  if (cudaMemsetAsync(ws, 0, L.fac, s) != cudaSuccess) return GS_ERR_CUDA;
  int64_t plane = (int64_t)width * height;
  float invU = 1.f / n_units;
  int gx = (int)((plane + 255) / 256);
  if (gx > 1024) gx = 1024;
  k_mask_count<<<dim3(gx, n_units), 256, 0, s>>>(mask, plane, msum);
  if (lambda_ssim == 0.f) {
    k_l1<<<dim3(gx, n_units), 256, 0, s>>>(img, gt, mask, plane, msum, 1.f, invU, l1, dL_dimg);
  } else {
    int tiles = ((width + LT - 1) / LT) * ((height + LT - 1) / LT);
    dim3 grid(tiles, 3, n_units);
    k_ssim_stats<<<grid, 256, 0, s>>>(img, gt, mask, width, height, msum, lambda_ssim, invU, l1, ss, fac);
    k_ssim_grad<<<grid, 256, 0, s>>>(img, gt, mask, width, height, msum, 1.f - lambda_ssim, invU, fac, dL_dimg);
  }
  k_loss_final<<<1, 1, 0, s>>>(msum, l1, ss, n_units, lambda_ssim, d_loss);
  return gs_check_launch();
}

// ---- backward entry points (blend + projection)
int gs_blend_bwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                      int width, int height, const float* bg, const float* final_T, const uint32_t* n_contrib,
                      const float* dL_dimg, const float* dL_dT, const gs_grad2d* g2d, int64_t n_proj, int variant,
                      const gs_schedule* sched, const float* img, cudaStream_t s);

GS_API int gs_blend_bwd(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                        int width, int height, const float* bg, const float* img, const float* final_T,
                        const uint32_t* n_contrib, const float* dL_dimg, const float* dL_dT, const gs_grad2d* g2d,
                        int64_t n_proj, int variant, const gs_schedule* sched, gs_stream_t stream) {
  GS_RANGE("gs_blend_bwd");
  return gs_blend_bwd_impl(proj, sorted_vals, ranges, n_units, width, height, bg, final_T, n_contrib, dL_dimg,
                           dL_dT, g2d, n_proj, variant, sched, img, (cudaStream_t)stream);
}

GS_API int gs_render_bwd(const float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                         const gs_camera* cams, const gs_proj* proj, const uint32_t* sorted_vals,
                         const uint32_t* ranges, int width, int height, const float* bg, const float* img,
                         const float* final_T, const uint32_t* n_contrib, const float* dL_dimg,
                         const float* dL_dT, const gs_grad2d* g2d, float* grads, int variant,
                         const gs_schedule* sched, gs_stream_t stream) {
  GS_RANGE("gs_render_bwd");
  UnitTable U;
  int64_t P = 0;
  if (gs_fill_units(units, U, &P) != GS_OK) return GS_ERR_INVALID;
  int r = gs_blend_bwd_impl(proj, sorted_vals, ranges, U.n, width, height, bg, final_T, n_contrib, dL_dimg, dL_dT,
                            g2d, P, variant, sched, img, (cudaStream_t)stream);
  if (r != GS_OK) return r;
  return gs_project_bwd(params, n_gauss, sh_degree, units, cams, proj, g2d, grads, stream);
}
