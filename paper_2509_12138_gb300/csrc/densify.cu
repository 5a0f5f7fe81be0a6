// Adaptive density control of 3D Gaussian Splatting, the optimisation each
// partition is trained with (Sec. II, "Parallel Training"): per-view
// statistics of the projected-position gradient, the clone / split / prune
// plan with its compaction into new parameter planes, and the opacity reset.
//
// Plan: each Gaussian's action (prune, keep, keep + clone, split) is decided
// from its statistics; three counts (kept, cloned, split) are scanned on the
// device.  The caller reads the counts, allocates planes for
// kept + cloned + 2 split Gaussians and applies: kept sources in index order,
// then the copies, then two children per split source (mean + R (s * z),
// scales / 1.6), with zero Adam moments for every new Gaussian.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

__host__ __device__ inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct DensifyWs {
  size_t keep, clone, split, scan, total;
};
DensifyWs densify_ws(int64_t n) {
  DensifyWs L;
  size_t o = 0;
  size_t cnt = sizeof(uint32_t) * (size_t)(n + 1);
  L.keep = o; o += a256(cnt);
  L.clone = o; o += a256(cnt);
  L.split = o; o += a256(cnt);
  L.scan = o; o += a256(gs_scan_ws_bytes(n > 0 ? n : 1));
  L.total = o;
  return L;
}

__global__ void k_densify_stats(UnitTable U, const int* __restrict__ radius, const float2* __restrict__ dxy, int W,
                                int H, float* __restrict__ grad_accum, float* __restrict__ denom,
                                float* __restrict__ max_radius) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= U.proj_base[U.n]) return;
  int r = radius[p];
  if (r <= 0) return;
  int u = unit_of(U, p);
  int64_t i = U.gauss_begin[u] + (p - U.proj_base[u]);
  float2 g = dxy[p];
  atomicAdd(grad_accum + i, hypotf(g.x * (0.5f * W), g.y * (0.5f * H)));
  atomicAdd(denom + i, 1.f);
  // non-negative floats order like their bit patterns
  atomicMax(reinterpret_cast<int*>(max_radius + i), __float_as_int((float)r));
}

__global__ void k_densify_mark(const float4* __restrict__ params, int64_t N, const float* __restrict__ grad_accum,
                               const float* __restrict__ denom, const float* __restrict__ max_radius,
                               gs_densify_cfg c, uint32_t* __restrict__ keep, uint32_t* __restrict__ clone,
                               uint32_t* __restrict__ split) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float4 so = params[N + i];  // log scales, logit opacity
  float smax = expf(fmaxf(so.x, fmaxf(so.y, so.z)));
  float op = 1.f / (1.f + expf(-so.w));
  float avg = denom[i] > 0.f ? grad_accum[i] / denom[i] : 0.f;
  bool prune = op < c.min_opacity ||
               (c.step > c.reset_interval && (max_radius[i] > c.max_screen || smax > 0.1f * c.extent));
  bool dense = !prune && avg >= c.grad_threshold;
  bool sp = dense && smax > c.percent_dense * c.extent;
  keep[i] = (!prune && !sp) ? 1u : 0u;
  clone[i] = (dense && !sp) ? 1u : 0u;
  split[i] = sp ? 1u : 0u;
}

__global__ void k_densify_apply(const float4* __restrict__ params, const float4* __restrict__ m,
                                const float4* __restrict__ v, int64_t N, int npl, const float* __restrict__ z,
                                const uint32_t* __restrict__ keep, const uint32_t* __restrict__ clone,
                                const uint32_t* __restrict__ split, float shrink_log, float4* __restrict__ op,
                                float4* __restrict__ om, float4* __restrict__ ov, int64_t n_out,
                                int* __restrict__ d_status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  // exclusive prefixes with the totals at [N]
  uint32_t nk = keep[N], nc = clone[N];
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (keep[i + 1] != keep[i]) {
    int64_t d = keep[i];
    if (d < n_out) {
      for (int k = 0; k < npl; ++k) {
        op[k * n_out + d] = params[k * N + i];
        om[k * n_out + d] = m[k * N + i];
        ov[k * n_out + d] = v[k * N + i];
      }
    } else if (d_status) {
      atomicOr(d_status, GS_ERR_CAPACITY);
    }
  }
  if (clone[i + 1] != clone[i]) {
    int64_t d = (int64_t)nk + clone[i];
    if (d < n_out) {
      for (int k = 0; k < npl; ++k) {
        op[k * n_out + d] = params[k * N + i];
        om[k * n_out + d] = zero;
        ov[k * n_out + d] = zero;
      }
    } else if (d_status) {
      atomicOr(d_status, GS_ERR_CAPACITY);
    }
  }
  if (split[i + 1] != split[i]) {
    float4 mean = params[i], so = params[N + i], q = params[2 * N + i];
    float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float w = q.x * qn, x = q.y * qn, y = q.z * qn, zq = q.w * qn;
    float R[9] = {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq), 2.f * (x * zq + w * y),
                  2.f * (x * y + w * zq), 1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x),
                  2.f * (x * zq - w * y), 2.f * (y * zq + w * x), 1.f - 2.f * (x * x + y * y)};
    float s[3] = {expf(so.x), expf(so.y), expf(so.z)};
    for (int c = 0; c < 2; ++c) {
      int64_t d = (int64_t)nk + nc + 2 * (int64_t)split[i] + c;
      if (d >= n_out) {
        if (d_status) atomicOr(d_status, GS_ERR_CAPACITY);
        continue;
      }
      const float* zz = z + (i * 2 + c) * 3;
      float off[3];
      #pragma unroll
      for (int a = 0; a < 3; ++a) off[a] = R[3 * a] * (s[0] * zz[0]) + R[3 * a + 1] * (s[1] * zz[1]) + R[3 * a + 2] * (s[2] * zz[2]);
      op[d] = make_float4(mean.x + off[0], mean.y + off[1], mean.z + off[2], mean.w);
      op[n_out + d] = make_float4(so.x - shrink_log, so.y - shrink_log, so.z - shrink_log, so.w);
      for (int k = 2; k < npl; ++k) op[k * n_out + d] = params[k * N + i];
      for (int k = 0; k < npl; ++k) {
        om[k * n_out + d] = zero;
        ov[k * n_out + d] = zero;
      }
    }
  }
}

__global__ void k_opacity_reset(float4* __restrict__ params, float4* __restrict__ m, float4* __restrict__ v,
                                int64_t N, float logit_max) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float4 so = params[N + i];
  so.w = fminf(so.w, logit_max);
  params[N + i] = so;
  m[N + i].w = 0.f;
  v[N + i].w = 0.f;
}

}  // namespace

GS_API size_t gs_densify_workspace_size(int64_t n_gauss) {
  if (n_gauss < 0) return 0;
  return densify_ws(n_gauss).total;
}

GS_API int gs_densify_stats(const gs_proj* proj, const gs_grad2d* g2d, const gs_units* units, int width, int height,
                            float* grad_accum, float* denom, float* max_radius, gs_stream_t stream) {
  GS_RANGE("gs_densify_stats");
  UnitTable U;
  int64_t P = 0;
  if (!proj || !proj->radius || !g2d || !g2d->dxy || !grad_accum || !denom || !max_radius || width <= 0 ||
      height <= 0 || gs_fill_units(units, U, &P) != GS_OK)
    return GS_ERR_INVALID;
  if (P == 0) return GS_OK;
  k_densify_stats<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      U, proj->radius, (const float2*)g2d->dxy, width, height, grad_accum, denom, max_radius);
  return gs_check_launch();
}

GS_API int gs_densify_plan(const float* params, int64_t n_gauss, const float* grad_accum, const float* denom,
                           const float* max_radius, const gs_densify_cfg* cfg, void* workspace,
                           size_t workspace_bytes, uint32_t* d_counts, gs_stream_t stream) {
  GS_RANGE("gs_densify_plan");
  if (!params || n_gauss < 1 || !grad_accum || !denom || !max_radius || !cfg || !workspace || !d_counts ||
      ((uintptr_t)workspace & 255u) || !(cfg->extent > 0.f))
    return GS_ERR_INVALID;
  DensifyWs L = densify_ws(n_gauss);
  if (workspace_bytes < L.total) return GS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  uint32_t* keep = (uint32_t*)(ws + L.keep);
  uint32_t* clone = (uint32_t*)(ws + L.clone);
  uint32_t* split = (uint32_t*)(ws + L.split);
  unsigned nb = (unsigned)((n_gauss + 255) / 256);
  k_densify_mark<<<nb, 256, 0, s>>>((const float4*)params, n_gauss, grad_accum, denom, max_radius, *cfg, keep, clone,
                                    split);
  int r = gs_scan_u32(keep, keep, n_gauss, ws + L.scan, keep + n_gauss, s);
  if (r == GS_OK) r = gs_scan_u32(clone, clone, n_gauss, ws + L.scan, clone + n_gauss, s);
  if (r == GS_OK) r = gs_scan_u32(split, split, n_gauss, ws + L.scan, split + n_gauss, s);
  if (r != GS_OK) return r;
  if (cudaMemcpyAsync(d_counts, keep + n_gauss, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_counts + 1, clone + n_gauss, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_counts + 2, split + n_gauss, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GS_ERR_CUDA;
  return gs_check_launch();
}

GS_API int gs_densify_apply(const float* params, const float* m, const float* v, int64_t n_gauss, int sh_degree,
                            const float* z, const void* workspace, size_t workspace_bytes, float* out_params,
                            float* out_m, float* out_v, int64_t n_out, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_densify_apply");
  int npl = param_planes(sh_degree);
  if (!params || !m || !v || n_gauss < 1 || npl < 0 || !z || !workspace || !out_params || !out_m || !out_v ||
      n_out < 0 || ((uintptr_t)workspace & 255u))
    return GS_ERR_INVALID;
  DensifyWs L = densify_ws(n_gauss);
  if (workspace_bytes < L.total) return GS_ERR_INVALID;
  const char* ws = (const char*)workspace;
  k_densify_apply<<<(unsigned)((n_gauss + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const float4*)params, (const float4*)m, (const float4*)v, n_gauss, npl, z, (const uint32_t*)(ws + L.keep),
      (const uint32_t*)(ws + L.clone), (const uint32_t*)(ws + L.split), logf(1.6f), (float4*)out_params,
      (float4*)out_m, (float4*)out_v, n_out, d_status);
  return gs_check_launch();
}

GS_API int gs_opacity_reset(float* params, float* m, float* v, int64_t n_gauss, float max_opacity,
                            gs_stream_t stream) {
  GS_RANGE("gs_opacity_reset");
  if (!params || !m || !v || n_gauss < 0 || !(max_opacity > 0.f && max_opacity < 1.f)) return GS_ERR_INVALID;
  if (n_gauss == 0) return GS_OK;
  k_opacity_reset<<<(unsigned)((n_gauss + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (float4*)params, (float4*)m, (float4*)v, n_gauss, logf(max_opacity / (1.f - max_opacity)));
  return gs_check_launch();
}
