// a1 projection (EWA splatting), the projection backward and Adam: the
// per-Gaussian, HBM-bound kernels of libgs.
//
// Parameters are float4 planes (mean, scale/opacity, rotation, SH...), so one
// thread issues coalesced 16-byte loads per plane.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

using namespace gs;

namespace {

// ---------------------------------------------------------------- real SH
// Real spherical harmonics of degree <= 3 (Condon-Shortley phase, m = -l..l)
// as polynomials of the unit direction.  Normalisation constants:
//   Y_00 = 1/(2 sqrt(pi)),          l=1: sqrt(3/(4 pi)),
//   l=2: 1/2 sqrt(15/pi), 1/4 sqrt(5/pi), 1/4 sqrt(15/pi),
//   l=3: 1/4 sqrt(35/(2 pi)), 1/2 sqrt(105/pi), 1/4 sqrt(21/(2 pi)),
//        1/4 sqrt(7/pi), 1/4 sqrt(105/pi).
constexpr float SH_C0 = 0.28209479177387814f;
constexpr float SH_C1 = 0.4886025119029199f;
constexpr float SH_C2a = 1.0925484305920792f;
constexpr float SH_C2b = 0.31539156525252005f;
constexpr float SH_C2c = 0.5462742152960396f;
constexpr float SH_C3a = 0.5900435899266435f;
constexpr float SH_C3b = 2.890611442640554f;
constexpr float SH_C3c = 0.4570457994644658f;
constexpr float SH_C3d = 0.3731763325901154f;
constexpr float SH_C3e = 1.445305721320277f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = SH_C0;
  if (DEG >= 1) {
    Y[1] = -SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = -SH_C1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_C2a * x * y;
    Y[5] = -SH_C2a * y * z;
    Y[6] = SH_C2b * (2.f * zz - xx - yy);
    Y[7] = -SH_C2a * x * z;
    Y[8] = SH_C2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -SH_C3a * y * (3.f * xx - yy);
      Y[10] = SH_C3b * x * y * z;
      Y[11] = -SH_C3c * y * (4.f * zz - xx - yy);
      Y[12] = SH_C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -SH_C3c * x * (4.f * zz - xx - yy);
      Y[14] = SH_C3e * z * (xx - yy);
      Y[15] = -SH_C3a * x * (xx - 3.f * yy);
    }
  }
}

// sum_k w_k grad Y_k(x, y, z) (Cartesian gradient of the polynomials above)
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float* w, float& gx, float& gy,
                                        float& gz) {
  gx = gy = gz = 0.f;
  if (DEG >= 1) {
    gy += -SH_C1 * w[1];
    gz += SH_C1 * w[2];
    gx += -SH_C1 * w[3];
  }
  if (DEG >= 2) {
    gx += SH_C2a * y * w[4];
    gy += SH_C2a * x * w[4];
    gy += -SH_C2a * z * w[5];
    gz += -SH_C2a * y * w[5];
    gx += -2.f * SH_C2b * x * w[6];
    gy += -2.f * SH_C2b * y * w[6];
    gz += 4.f * SH_C2b * z * w[6];
    gx += -SH_C2a * z * w[7];
    gz += -SH_C2a * x * w[7];
    gx += 2.f * SH_C2c * x * w[8];
    gy += -2.f * SH_C2c * y * w[8];
    if (DEG >= 3) {
      float xx = x * x, yy = y * y, zz = z * z;
      gx += -6.f * SH_C3a * x * y * w[9];
      gy += -3.f * SH_C3a * (xx - yy) * w[9];
      gx += SH_C3b * y * z * w[10];
      gy += SH_C3b * x * z * w[10];
      gz += SH_C3b * x * y * w[10];
      gx += 2.f * SH_C3c * x * y * w[11];
      gy += -SH_C3c * (4.f * zz - xx - 3.f * yy) * w[11];
      gz += -8.f * SH_C3c * y * z * w[11];
      gx += -6.f * SH_C3d * x * z * w[12];
      gy += -6.f * SH_C3d * y * z * w[12];
      gz += SH_C3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
      gx += -SH_C3c * (4.f * zz - 3.f * xx - yy) * w[13];
      gy += 2.f * SH_C3c * x * y * w[13];
      gz += -8.f * SH_C3c * x * z * w[13];
      gx += 2.f * SH_C3e * x * z * w[14];
      gy += -2.f * SH_C3e * y * z * w[14];
      gz += SH_C3e * (xx - yy) * w[14];
      gx += -3.f * SH_C3a * (xx - yy) * w[15];
      gy += 6.f * SH_C3a * x * y * w[15];
    }
  }
}

template <int DEG>
struct ShCount { static constexpr int NC = (DEG + 1) * (DEG + 1); static constexpr int NP = (3 * NC + 3) / 4; };

template <int DEG>
__device__ __forceinline__ void load_sh(const float4* __restrict__ params, int64_t N, int64_t i, float* c) {
  constexpr int NP = ShCount<DEG>::NP;
  #pragma unroll
  for (int k = 0; k < NP; ++k) {
    float4 q = __ldg(params + (3 + k) * N + i);
    c[4 * k] = q.x; c[4 * k + 1] = q.y; c[4 * k + 2] = q.z; c[4 * k + 3] = q.w;
  }
}

// Quantities of the forward projection that the backward recomputes.
struct Geo {
  float t[3];
  float Rq[9];
  float s[3];
  float Sig[6];  // xx xy xz yy yz zz
  float T2[6];   // rows of J W
  float a, b, c, det;
  bool clx, cly;
  float xzc, yzc;
};

// One row of the view transform, r0 x + r1 y + r2 z + t, as a float pair
// (h, l) with h the value rounded once to float32.  Each product is split
// exactly by TwoProduct, the products are summed with TwoSum, which returns
// every addition's rounding error, and the collected error terms are added at
// the end; h + l then equals the exact value up to about 2^-44 of the terms'
// magnitude, so h is the correctly rounded value unless the exact one lies
// that close to a rounding boundary.  The explicitly rounded intrinsics keep
// the compiler from contracting the steps.
__device__ __forceinline__ void view_row(const float* r, float4 m, float& h, float& l) {
  float p0, e0, p1, e1, p2, e2;
  two_prod(r[0], m.x, p0, e0);
  two_prod(r[1], m.y, p1, e1);
  two_prod(r[2], m.z, p2, e2);
  float lo = __fadd_rn(__fadd_rn(e0, e1), e2);
  float s, e;
  two_sum(r[3], p0, s, e);
  lo = __fadd_rn(lo, e);
  two_sum(s, p1, s, e);
  lo = __fadd_rn(lo, e);
  two_sum(s, p2, s, e);
  lo = __fadd_rn(lo, e);
  two_sum(s, lo, h, l);
}

// Camera-space z rounded to float32: the depth sort key (row 2 of viewmat).
__device__ __forceinline__ float cam_z(const float* V, float4 m) {
  float h, l;
  view_row(V + 8, m, h, l);
  return h;
}

// Pixel coordinate f t / z + c of camera-space (t, z), both float pairs, as a
// float pair (h, l): the quotient's remainder t_h - q_h z_h is exact by one
// fused multiply-add, the product f q by TwoProduct, the sum with c by TwoSum.
__device__ __forceinline__ void pixel_pair(float th, float tl, float zh, float zl, float f, float c, float& h,
                                           float& l) {
  float qh = __fdiv_rn(th, zh);
  float r = __fmaf_rn(-qh, zh, th);
  r = __fadd_rn(r, __fsub_rn(tl, __fmul_rn(qh, zl)));
  float ql = __fdiv_rn(r, zh);
  float ph, pe;
  two_prod(f, qh, ph, pe);
  pe = __fmaf_rn(f, ql, pe);
  float sh, se;
  two_sum(ph, c, sh, se);
  two_sum(sh, __fadd_rn(se, pe), h, l);
}

__device__ __forceinline__ void quat_rot(float4 q, float* R, float* qn_out) {
  float inv = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
  if (qn_out) { qn_out[0] = w; qn_out[1] = x; qn_out[2] = y; qn_out[3] = z; qn_out[4] = inv; }
}

__device__ __forceinline__ void geometry(const gs_camera& cam, float4 mean, float4 sop, float4 quat, Geo& g,
                                         float* qn) {
  const float* V = cam.viewmat;
  g.t[0] = V[0] * mean.x + V[1] * mean.y + V[2] * mean.z + V[3];
  g.t[1] = V[4] * mean.x + V[5] * mean.y + V[6] * mean.z + V[7];
  g.t[2] = cam_z(V, mean);
  quat_rot(quat, g.Rq, qn);
  g.s[0] = expf(sop.x); g.s[1] = expf(sop.y); g.s[2] = expf(sop.z);
  float M[9];
  #pragma unroll
  for (int i = 0; i < 3; ++i)
    #pragma unroll
    for (int j = 0; j < 3; ++j) M[3 * i + j] = g.Rq[3 * i + j] * g.s[j];
  g.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  g.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  g.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  g.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  g.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  g.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  float tz = g.t[2];
  float limx = JCLAMP * cam.tan_fovx, limy = JCLAMP * cam.tan_fovy;
  float xz = g.t[0] / tz, yz = g.t[1] / tz;
  g.clx = (xz < -limx) || (xz > limx);
  g.cly = (yz < -limy) || (yz > limy);
  g.xzc = fminf(fmaxf(xz, -limx), limx);
  g.yzc = fminf(fmaxf(yz, -limy), limy);
  float J00 = cam.fx / tz, J02 = -cam.fx * g.xzc / tz;
  float J11 = cam.fy / tz, J12 = -cam.fy * g.yzc / tz;
  #pragma unroll
  for (int j = 0; j < 3; ++j) {
    g.T2[j] = J00 * V[4 * 0 + j] + J02 * V[4 * 2 + j];
    g.T2[3 + j] = J11 * V[4 * 1 + j] + J12 * V[4 * 2 + j];
  }
  // cov = T2 Sig T2^T
  const float* S = g.Sig;
  float v0[3], v1[3];
  #pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float* T = g.T2 + 3 * r;
    float* v = r == 0 ? v0 : v1;
    v[0] = S[0] * T[0] + S[1] * T[1] + S[2] * T[2];
    v[1] = S[1] * T[0] + S[3] * T[1] + S[4] * T[2];
    v[2] = S[2] * T[0] + S[4] * T[1] + S[5] * T[2];
  }
  g.a = g.T2[0] * v0[0] + g.T2[1] * v0[1] + g.T2[2] * v0[2] + DILATION;
  g.b = g.T2[0] * v1[0] + g.T2[1] * v1[1] + g.T2[2] * v1[2];
  g.c = g.T2[3] * v1[0] + g.T2[4] * v1[1] + g.T2[5] * v1[2] + DILATION;
  g.det = g.a * g.c - g.b * g.b;
}

__device__ __forceinline__ bool owned_keep(const OwnedTable& O, int64_t i, float4 mean) {
  if (O.n == 0) return true;
  int k = part_of(O, i);
  const float* b = O.box[k];
  float x[3] = {mean.x, mean.y, mean.z};
  bool in = true;
  #pragma unroll
  for (int a = 0; a < 3; ++a) {
    bool hi = (O.closed_hi[k] >> a) & 1 ? (x[a] <= b[3 + a]) : (x[a] < b[3 + a]);
    in = in && (x[a] >= b[a]) && hi;
  }
  return in;
}

// One projected record (a1) of a Gaussian for one camera: depth always;
// position pair, conic and opacity, colour and power floor when it is
// visible; radius and tile count (0 when culled).  keep: the Gaussian passes
// the caller's ownership filter.  The SH planes are read (only for a visible
// record) from sh[k * sh_stride], k < NP: global memory for k_preprocess,
// shared memory for the fused projection backward + Adam, which projects the
// updated Gaussian for the next step's camera.  Not inlined, so that both
// callers run one compiled body: the compiler cannot contract the covariance,
// conic or colour arithmetic differently in the two kernels, and their
// records are bit-identical for equal inputs.
template <int DEG>
__device__ __noinline__ void project_record(const gs_camera& cam, float4 mean, float4 sop, float4 quat, int W, int H,
                                            bool keep, const float4* sh, int64_t sh_stride, float4* xy,
                                            float4* conic_op, float4* rgb, float* depth, int* radius,
                                            uint32_t* tiles, int* status) {
  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  int r_out = 0;
  uint32_t tiles_out = 0;
  const float* V = cam.viewmat;
  float tz, tzl;
  view_row(V + 8, mean, tz, tzl);  // tz: the correctly rounded camera-space z (the sort key)
  *depth = tz;
  if (tz > cam.znear && keep) {
    Geo g;
    geometry(cam, mean, sop, quat, g, nullptr);
    if (g.det > 0.f) {
      float idet = 1.0f / g.det;
      float mid = 0.5f * (g.a + g.c);
      float lam = mid + sqrtf(fmaxf(LAMBDA_FLOOR, mid * mid - g.det));
      int r = (int)ceilf(3.0f * sqrtf(lam));
      // pixel position as float pairs (x + x_lo, y + y_lo), from the view rows in pairs
      float t0h, t0l, t1h, t1l;
      view_row(V, mean, t0h, t0l);
      view_row(V + 4, mean, t1h, t1l);
      float4 pxy;
      pixel_pair(t0h, t0l, tz, tzl, cam.fx, cam.cx, pxy.x, pxy.z);
      pixel_pair(t1h, t1l, tz, tzl, cam.fy, cam.cy, pxy.y, pxy.w);
      float px = pxy.x, py = pxy.y;
      int x0, y0, x1, y1;
      tile_rect(pxy, r, TX, TY, x0, y0, x1, y1);
      uint32_t nt = (uint32_t)((x1 - x0) * (y1 - y0));
      if (r > 0 && nt > 0) {
        // colour
        float dx = mean.x - cam.campos[0], dy = mean.y - cam.campos[1], dz = mean.z - cam.campos[2];
        float il = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        float Y[16];
        sh_basis<DEG>(dx, dy, dz, Y);
        float c[4 * ShCount<DEG>::NP];
        #pragma unroll
        for (int k = 0; k < ShCount<DEG>::NP; ++k) {
          float4 q = sh[k * sh_stride];
          c[4 * k] = q.x; c[4 * k + 1] = q.y; c[4 * k + 2] = q.z; c[4 * k + 3] = q.w;
        }
        float col[3];
        #pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          float acc = 0.5f;
          #pragma unroll
          for (int k = 0; k < ShCount<DEG>::NC; ++k) acc += Y[k] * c[3 * k + ch];
          col[ch] = fmaxf(acc, 0.f);
        }
        float op = 1.0f / (1.0f + expf(-sop.w));
        *xy = pxy;
        *conic_op = make_float4(g.c * idet, -g.b * idet, g.a * idet, op);
        *rgb = make_float4(col[0], col[1], col[2], power_floor(op));
        r_out = r;
        tiles_out = nt;
        if (!(isfinite(px) && isfinite(py) && isfinite(col[0] + col[1] + col[2]) &&
              isfinite(g.c * idet + g.b * idet + g.a * idet) && isfinite(op))) {
          set_status(status, GS_ERR_NONFINITE);
          r_out = 0;
          tiles_out = 0;
        }
      }
    }
  }
  *radius = r_out;
  *tiles = tiles_out;
}

template <int DEG>
__global__ void __launch_bounds__(256) k_preprocess(const float4* __restrict__ params, int64_t N,
                                                    UnitTable U, OwnedTable O,
                                                    const gs_camera* __restrict__ cams, int W, int H,
                                                    float4* __restrict__ xy, float4* __restrict__ conic_op,
                                                    float4* __restrict__ rgb, float* __restrict__ depth,
                                                    int* __restrict__ radius, uint32_t* __restrict__ tiles,
                                                    int* status) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= U.proj_base[U.n]) return;
  int u = unit_of(U, p);
  int64_t i = U.gauss_begin[u] + (p - U.proj_base[u]);
  float4 mean = __ldg(params + i);
  float4 sop = __ldg(params + N + i);
  float4 quat = __ldg(params + 2 * N + i);
  project_record<DEG>(cams[u], mean, sop, quat, W, H, owned_keep(O, i, mean), params + 3 * N + i, N, xy + p,
                      conic_op + p, rgb + p, depth + p, radius + p, tiles + p, status);
}

// Projection backward: chain rule of k_preprocess for every parameter of
// Gaussian i, summed over the units that contain it.  c holds the SH
// coefficients (loaded by the caller); the results go to dmean, dls, dq,
// dlogit and dsh (SH gradients, same packing as c).
template <int DEG>
__device__ __forceinline__ void project_grads(int64_t i, float4 mean, float4 sop, float4 quat, const float* c,
                                              const UnitTable& U, const gs_camera* __restrict__ cams,
                                              const int* __restrict__ radius, const float2* __restrict__ gxy,
                                              const float4* __restrict__ gco, const float4* __restrict__ grgb,
                                              float* dmean, float* dls, float* dq, float& dlogit, float* dsh) {
  constexpr int NC = ShCount<DEG>::NC;
  constexpr int NP = ShCount<DEG>::NP;
  dmean[0] = dmean[1] = dmean[2] = 0.f;
  dls[0] = dls[1] = dls[2] = 0.f;
  dq[0] = dq[1] = dq[2] = dq[3] = 0.f;
  dlogit = 0.f;
  #pragma unroll
  for (int k = 0; k < 4 * NP; ++k) dsh[k] = 0.f;
  for (int u = 0; u < U.n; ++u) {
    int64_t cnt = U.proj_base[u + 1] - U.proj_base[u];
    int64_t l = i - U.gauss_begin[u];
    if (l < 0 || l >= cnt) continue;
    int64_t p = U.proj_base[u] + l;
    if (__ldg(radius + p) <= 0) continue;
    const gs_camera& cam = cams[u];
    float2 g_xy = gxy[p];
    float4 g_co = gco[p];
    float4 g_rgb = grgb[p];
    float qn[5];
    Geo g;
    geometry(cam, mean, sop, quat, g, qn);
    float tz = g.t[2], itz = 1.0f / tz;
    float dt[3] = {0.f, 0.f, 0.f};

    // colour: rgb = max(sum Y c + 0.5, 0)
    {
      float vx = mean.x - cam.campos[0], vy = mean.y - cam.campos[1], vz = mean.z - cam.campos[2];
      float il = 1.0f / sqrtf(vx * vx + vy * vy + vz * vz);
      float dx = vx * il, dy = vy * il, dz = vz * il;
      float Y[16];
      sh_basis<DEG>(dx, dy, dz, Y);
      float gc[3] = {g_rgb.x, g_rgb.y, g_rgb.z};
      #pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.5f;
        #pragma unroll
        for (int k = 0; k < NC; ++k) acc += Y[k] * c[3 * k + ch];
        if (acc < 0.f) gc[ch] = 0.f;
      }
      float wsum[16];
      #pragma unroll
      for (int k = 0; k < NC; ++k) {
        dsh[3 * k] += Y[k] * gc[0];
        dsh[3 * k + 1] += Y[k] * gc[1];
        dsh[3 * k + 2] += Y[k] * gc[2];
        wsum[k] = c[3 * k] * gc[0] + c[3 * k + 1] * gc[1] + c[3 * k + 2] * gc[2];
      }
      if (DEG > 0) {
        float gx, gy, gz;
        sh_grad<DEG>(dx, dy, dz, wsum, gx, gy, gz);
        float dot = gx * dx + gy * dy + gz * dz;
        dmean[0] += (gx - dot * dx) * il;
        dmean[1] += (gy - dot * dy) * il;
        dmean[2] += (gz - dot * dz) * il;
      }
    }
    // opacity
    {
      float op = 1.0f / (1.0f + expf(-sop.w));
      dlogit += g_co.w * op * (1.f - op);
    }
    // mean2D
    dt[0] += g_xy.x * cam.fx * itz;
    dt[1] += g_xy.y * cam.fy * itz;
    dt[2] += -(g_xy.x * cam.fx * g.t[0] + g_xy.y * cam.fy * g.t[1]) * itz * itz;
    // conic -> dilated 2D covariance (a, b, c)
    float a = g.a, b = g.b, cc = g.c, det = g.det;
    float id2 = 1.0f / (det * det);
    float gA = g_co.x, gB = g_co.y, gC = g_co.z;
    float da = (-cc * cc * gA + b * cc * gB - b * b * gC) * id2;
    float db = (2.f * b * cc * gA - (det + 2.f * b * b) * gB + 2.f * a * b * gC) * id2;
    float dc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
    // Gs = [[da, db/2], [db/2, dc]]; dSig = T2^T Gs T2; dT2 = 2 Gs T2 Sig
    const float* T = g.T2;
    float hb = 0.5f * db;
    float GT0[3], GT1[3];  // rows of Gs T2
    #pragma unroll
    for (int j = 0; j < 3; ++j) {
      GT0[j] = da * T[j] + hb * T[3 + j];
      GT1[j] = hb * T[j] + dc * T[3 + j];
    }
    float dSig[9];
    #pragma unroll
    for (int i2 = 0; i2 < 3; ++i2)
      #pragma unroll
      for (int j = 0; j < 3; ++j) dSig[3 * i2 + j] = T[i2] * GT0[j] + T[3 + i2] * GT1[j];
    const float* S6 = g.Sig;
    float Sg[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
    float dT2[6];
    #pragma unroll
    for (int j = 0; j < 3; ++j) {
      dT2[j] = 2.f * (GT0[0] * Sg[j] + GT0[1] * Sg[3 + j] + GT0[2] * Sg[6 + j]);
      dT2[3 + j] = 2.f * (GT1[0] * Sg[j] + GT1[1] * Sg[3 + j] + GT1[2] * Sg[6 + j]);
    }
    // T2 = J W: dJ = dT2 W^T (J00, J02 from row 0; J11, J12 from row 1)
    const float* V = cam.viewmat;
    float dJ00 = dT2[0] * V[0] + dT2[1] * V[1] + dT2[2] * V[2];
    float dJ02 = dT2[0] * V[8] + dT2[1] * V[9] + dT2[2] * V[10];
    float dJ11 = dT2[3] * V[4] + dT2[4] * V[5] + dT2[5] * V[6];
    float dJ12 = dT2[3] * V[8] + dT2[4] * V[9] + dT2[5] * V[10];
    dt[2] += -(dJ00 * cam.fx + dJ11 * cam.fy) * itz * itz;
    if (g.clx) {
      dt[2] += dJ02 * cam.fx * g.xzc * itz * itz;
    } else {
      dt[0] += -dJ02 * cam.fx * itz * itz;
      dt[2] += 2.f * dJ02 * cam.fx * g.t[0] * itz * itz * itz;
    }
    if (g.cly) {
      dt[2] += dJ12 * cam.fy * g.yzc * itz * itz;
    } else {
      dt[1] += -dJ12 * cam.fy * itz * itz;
      dt[2] += 2.f * dJ12 * cam.fy * g.t[1] * itz * itz * itz;
    }
    // t = W mu + t0
    #pragma unroll
    for (int k = 0; k < 3; ++k) dmean[k] += V[k] * dt[0] + V[4 + k] * dt[1] + V[8 + k] * dt[2];
    // Sigma = M M^T, M = Rq diag(s): dM = 2 dSig M
    float M[9];
    #pragma unroll
    for (int i2 = 0; i2 < 3; ++i2)
      #pragma unroll
      for (int j = 0; j < 3; ++j) M[3 * i2 + j] = g.Rq[3 * i2 + j] * g.s[j];
    float dR[9];
    #pragma unroll
    for (int i2 = 0; i2 < 3; ++i2)
      #pragma unroll
      for (int j = 0; j < 3; ++j) {
        float dM = 2.f * (dSig[3 * i2] * M[j] + dSig[3 * i2 + 1] * M[3 + j] + dSig[3 * i2 + 2] * M[6 + j]);
        dls[j] += dM * g.Rq[3 * i2 + j] * g.s[j];
        dR[3 * i2 + j] = dM * g.s[j];
      }
    // rotation of the normalised quaternion
    float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    float gw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    float gx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                      w * dR[7] - 2.f * x * dR[8]);
    float gy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                      z * dR[7] - 2.f * y * dR[8]);
    float gz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                      x * dR[6] + y * dR[7]);
    float dot = gw * w + gx * x + gy * y + gz * z;
    float inv = qn[4];
    dq[0] += (gw - dot * w) * inv;
    dq[1] += (gx - dot * x) * inv;
    dq[2] += (gy - dot * y) * inv;
    dq[3] += (gz - dot * z) * inv;
  }
}

template <int DEG>
__global__ void __launch_bounds__(128) k_project_bwd(const float4* __restrict__ params, int64_t N,
                                                     UnitTable U, const gs_camera* __restrict__ cams,
                                                     const int* __restrict__ radius,
                                                     const float2* __restrict__ gxy,
                                                     const float4* __restrict__ gco,
                                                     const float4* __restrict__ grgb,
                                                     float4* __restrict__ grads) {
  constexpr int NP = ShCount<DEG>::NP;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float4 mean = __ldg(params + i);
  float4 sop = __ldg(params + N + i);
  float4 quat = __ldg(params + 2 * N + i);
  float c[4 * NP];
  load_sh<DEG>(params, N, i, c);
  float dmean[3], dls[3], dq[4], dlogit, dsh[4 * NP];
  project_grads<DEG>(i, mean, sop, quat, c, U, cams, radius, gxy, gco, grgb, dmean, dls, dq, dlogit, dsh);
  grads[i] = make_float4(dmean[0], dmean[1], dmean[2], 0.f);
  grads[N + i] = make_float4(dls[0], dls[1], dls[2], dlogit);
  grads[2 * N + i] = make_float4(dq[0], dq[1], dq[2], dq[3]);
  #pragma unroll
  for (int k = 0; k < NP; ++k)
    grads[(3 + k) * N + i] = make_float4(dsh[4 * k], dsh[4 * k + 1], dsh[4 * k + 2], dsh[4 * k + 3]);
}

struct AdamLR {
  float4 init[16];
  float4 fin[16];
};

__device__ __forceinline__ bool finite4(float4 a) {
  return isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w);
}

__global__ void __launch_bounds__(256) k_adam(float4* __restrict__ p, float4* __restrict__ g,
                                              float4* __restrict__ m, float4* __restrict__ v, int64_t N,
                                              int n_planes, AdamLR lr, int lr_steps, float b1, float b2,
                                              float eps, const int32_t* __restrict__ d_step, int zero,
                                              int* __restrict__ status) {
  __shared__ float4 s_lr[16];
  int t = *d_step + 1;
  if (threadIdx.x < n_planes) {
    float frac = lr_steps > 0 ? (float)min(t, lr_steps) / (float)lr_steps : 0.f;
    float4 a = lr.init[threadIdx.x], b = lr.fin[threadIdx.x];
    auto sched = [&](float x0, float x1) { return (x0 == x1 || x0 <= 0.f) ? x0 : x0 * powf(x1 / x0, frac); };
    s_lr[threadIdx.x] = make_float4(sched(a.x, b.x), sched(a.y, b.y), sched(a.z, b.z), sched(a.w, b.w));
  }
  __syncthreads();
  float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
  float ibc1 = 1.f / bc1, ibc2 = 1.f / bc2;
  int64_t total = (int64_t)n_planes * N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int plane = (int)(k / N);
    float4 L = s_lr[plane];
    float4 P = p[k], G = g[k], Mv = m[k], Vv = v[k];
    if (zero) g[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!finite4(G)) {  // a non-finite gradient: reported, and these four values keep their state
      set_status(status, GS_ERR_NONFINITE);
      continue;
    }
    float* pp = &P.x; float* gg = &G.x; float* mm = &Mv.x; float* vv = &Vv.x; const float* ll = &L.x;
    #pragma unroll
    for (int c = 0; c < 4; ++c) {
      mm[c] = b1 * mm[c] + (1.f - b1) * gg[c];
      vv[c] = b2 * vv[c] + (1.f - b2) * gg[c] * gg[c];
      pp[c] -= ll[c] * (mm[c] * ibc1) / (sqrtf(vv[c] * ibc2) + eps);
    }
    p[k] = P; m[k] = Mv; v[k] = Vv;
  }
}

// Adam update of one float4 of parameters (textbook form, bias-corrected).
__device__ __forceinline__ void adam4(float4& P, float4 G, float4& M, float4& V, float4 L, float b1, float b2,
                                      float ibc1, float ibc2, float eps) {
  float* pp = &P.x; const float* gg = &G.x; float* mm = &M.x; float* vv = &V.x; const float* ll = &L.x;
  #pragma unroll
  for (int c = 0; c < 4; ++c) {
    mm[c] = b1 * mm[c] + (1.f - b1) * gg[c];
    vv[c] = b2 * vv[c] + (1.f - b2) * gg[c] * gg[c];
    pp[c] -= ll[c] * (mm[c] * ibc1) / (sqrtf(vv[c] * ibc2) + eps);
  }
}

// Projection backward fused with Adam: the parameter gradient of Gaussian i
// is formed in registers and applied at once, so it never goes to memory
// (optionally it is also written to `grads`).
template <int DEG>
__global__ void __launch_bounds__(128) k_project_bwd_adam(float4* __restrict__ params, int64_t N, UnitTable U,
                                                          const gs_camera* __restrict__ cams,
                                                          const int* __restrict__ radius,
                                                          const float2* __restrict__ gxy,
                                                          const float4* __restrict__ gco,
                                                          const float4* __restrict__ grgb, float4* __restrict__ m,
                                                          float4* __restrict__ v, AdamLR lr, int lr_steps, float b1,
                                                          float b2, float eps, const int32_t* __restrict__ d_step,
                                                          float4* __restrict__ grads, int sparse,
                                                          int* __restrict__ status) {
  constexpr int NP = ShCount<DEG>::NP;
  constexpr int NPL = 3 + NP;
  __shared__ float4 s_lr[16];
  int t = *d_step + 1;
  if (threadIdx.x < NPL) {
    float frac = lr_steps > 0 ? (float)min(t, lr_steps) / (float)lr_steps : 0.f;
    float4 a = lr.init[threadIdx.x], b = lr.fin[threadIdx.x];
    auto sched = [&](float x0, float x1) { return (x0 == x1 || x0 <= 0.f) ? x0 : x0 * powf(x1 / x0, frac); };
    s_lr[threadIdx.x] = make_float4(sched(a.x, b.x), sched(a.y, b.y), sched(a.z, b.z), sched(a.w, b.w));
  }
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float ibc1 = 1.f / (1.f - powf(b1, (float)t)), ibc2 = 1.f / (1.f - powf(b2, (float)t));
  float4 mean = params[i];
  float4 sop = params[N + i];
  float4 quat = params[2 * N + i];
  float c[4 * NP];
  #pragma unroll
  for (int k = 0; k < NP; ++k) {
    float4 q = params[(3 + k) * N + i];
    c[4 * k] = q.x; c[4 * k + 1] = q.y; c[4 * k + 2] = q.z; c[4 * k + 3] = q.w;
  }
  float dmean[3], dls[3], dq[4], dlogit, dsh[4 * NP];
  project_grads<DEG>(i, mean, sop, quat, c, U, cams, radius, gxy, gco, grgb, dmean, dls, dq, dlogit, dsh);
  float4 G[3] = {make_float4(dmean[0], dmean[1], dmean[2], 0.f), make_float4(dls[0], dls[1], dls[2], dlogit),
                 make_float4(dq[0], dq[1], dq[2], dq[3])};
  // a non-finite gradient is reported and leaves this Gaussian's parameters and moments as they are
  bool ok = finite4(G[0]) && finite4(G[1]) && finite4(G[2]);
  bool any = false;
  #pragma unroll
  for (int k = 0; k < 4 * NP; ++k) { ok = ok && isfinite(dsh[k]); any = any || dsh[k] != 0.f; }
  if (!ok) set_status(status, GS_ERR_NONFINITE);
  #pragma unroll
  for (int k = 0; k < 3; ++k) any = any || G[k].x != 0.f || G[k].y != 0.f || G[k].z != 0.f || G[k].w != 0.f;
  if (sparse && !any) ok = false;  // sparse: a Gaussian without gradient keeps its state
  float4 Pv[3] = {mean, sop, quat};
  #pragma unroll
  for (int k = 0; k < 3; ++k) {
    int64_t o = k * N + i;
    float4 M = m[o], V = v[o];
    adam4(Pv[k], G[k], M, V, s_lr[k], b1, b2, ibc1, ibc2, eps);
    if (ok) { params[o] = Pv[k]; m[o] = M; v[o] = V; }
    if (grads) grads[o] = G[k];
  }
  #pragma unroll
  for (int k = 0; k < NP; ++k) {
    int64_t o = (3 + k) * N + i;
    float4 P = make_float4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
    float4 Gk = make_float4(dsh[4 * k], dsh[4 * k + 1], dsh[4 * k + 2], dsh[4 * k + 3]);
    float4 M = m[o], V = v[o];
    adam4(P, Gk, M, V, s_lr[3 + k], b1, b2, ibc1, ibc2, eps);
    if (ok) { params[o] = P; m[o] = M; v[o] = V; }
    if (grads) grads[o] = Gk;
  }
}

// Async 16-byte global -> shared copies (cp.async, L2 only); each thread
// copies and later reads only its own slots, so a thread-local wait suffices.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NG>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NG) : "memory"); }

// The next step's projection, fused into the projection backward + Adam
// (cams NULL: none): camera per unit, image size and the record arrays.
struct NextProj {
  const gs_camera* cams;
  int W, H;
  float4* xy;
  float4* conic_op;
  float4* rgb;
  float* depth;
  int* radius;
  uint32_t* tiles;
};

constexpr int PBA_T = 64;  // Gaussians per block of the staged kernel
constexpr int PBA_R = 6;   // moment planes (m and v) in flight per thread (7 or more: 210 registers)

// Projection backward fused with Adam for Gaussians that belong to exactly
// one unit (one view of one partition).  On entry every thread starts async
// copies of its Gaussian's parameter planes (one commit group) and of the
// first PBA_R planes of its Adam moments, in the order the updates use them
// (SH planes, then mean, scale/opacity, rotation), into its own
// shared-memory slots; each update then starts the copy of the moments
// PBA_R planes ahead into the slot it has just consumed.  The geometry
// gradient runs once the parameters have landed.  The SH planes are read
// twice from shared memory (colour and clamp first, then each plane's
// gradient and update), so neither the 48 coefficients nor their gradients
// are held in registers.
template <int DEG>
__global__ void __launch_bounds__(PBA_T) k_project_bwd_adam1(float4* __restrict__ params, int64_t N, UnitTable U,
                                                           const gs_camera* __restrict__ cams,
                                                           const int* radius,  // overwritten by nx (own record)
                                                           const float2* __restrict__ gxy,
                                                           const float4* __restrict__ gco,
                                                           const float4* __restrict__ grgb, float4* __restrict__ m,
                                                           float4* __restrict__ v, AdamLR lr, int lr_steps, float b1,
                                                           float b2, float eps, const int32_t* __restrict__ d_step,
                                                           float4* __restrict__ grads, int sparse,
                                                           int* __restrict__ status, NextProj nx) {
  constexpr int NC = ShCount<DEG>::NC;
  constexpr int NP = ShCount<DEG>::NP;
  constexpr int NPL = 3 + NP;
  __shared__ float4 s_lr[16];
  int t = *d_step + 1;
  if (threadIdx.x < NPL) {
    float frac = lr_steps > 0 ? (float)min(t, lr_steps) / (float)lr_steps : 0.f;
    float4 a = lr.init[threadIdx.x], b = lr.fin[threadIdx.x];
    auto sched = [&](float x0, float x1) { return (x0 == x1 || x0 <= 0.f) ? x0 : x0 * powf(x1 / x0, frac); };
    s_lr[threadIdx.x] = make_float4(sched(a.x, b.x), sched(a.y, b.y), sched(a.z, b.z), sched(a.w, b.w));
  }
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  // the unit containing i (units are disjoint here)
  int uu = -1;
  int64_t pidx = 0;
  for (int u = 0; u < U.n; ++u) {
    int64_t l = i - U.gauss_begin[u];
    if (l >= 0 && l < U.proj_base[u + 1] - U.proj_base[u]) { uu = u; pidx = U.proj_base[u] + l; break; }
  }
  bool vis = uu >= 0 && __ldg(radius + pidx) > 0;
  // sparse: a Gaussian with no screen-space gradient in this step keeps its parameters and moments (no
  // load, no store), as a sparse Adam updates only the Gaussians a view touches; with the next step's
  // projection fused in it joins the other lanes at that projection (one call per warp)
  bool skip = false;
  if (sparse) {
    bool any = false;
    if (vis) {
      float2 a = gxy[pidx];
      float4 b = gco[pidx], c = grgb[pidx];
      any = a.x != 0.f || a.y != 0.f || b.x != 0.f || b.y != 0.f || b.z != 0.f || b.w != 0.f || c.x != 0.f ||
            c.y != 0.f || c.z != 0.f;
    }
    if (!any) {
      if (grads) {
        #pragma unroll
        for (int k = 0; k < NPL; ++k) grads[k * N + i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (!nx.cams) return;
      skip = true;
    }
  }
  // the parameters the next step's projection takes: as stored after the update, or unchanged
  float4 pm, ps, pq;
  const float4* shp;
  int64_t shs;
  extern __shared__ float4 s_stage[];  // [NPL][PBA_T] parameters, then [PBA_R][2][PBA_T] m, v ring
  if (!skip) {
    const int tl = threadIdx.x;
    float4* sP = s_stage;
    float4* sR = s_stage + NPL * PBA_T;
    // update sequence q = 0 .. NPL - 1 takes plane (q + 3) % NPL: the SH planes, then 0, 1, 2
    auto mv_copy = [&](int q) {
      if (q < NPL) {
        int k = (q + 3) % NPL;
        float4* slot = sR + (q % PBA_R) * 2 * PBA_T;
        cp_async16(slot + tl, m + k * N + i);
        cp_async16(slot + PBA_T + tl, v + k * N + i);
      }
      cp_async_commit();  // one group per sequence step (empty past the end) keeps the counting uniform
    };
    #pragma unroll
    for (int k = 0; k < NPL; ++k) cp_async16(sP + k * PBA_T + tl, params + k * N + i);
    cp_async_commit();
    #pragma unroll
    for (int q = 0; q < PBA_R; ++q) mv_copy(q);
    float ibc1 = 1.f / (1.f - powf(b1, (float)t)), ibc2 = 1.f / (1.f - powf(b2, (float)t));
    cp_async_wait<PBA_R>();  // this thread's parameter planes have landed
    float4 mean = sP[tl], sop = sP[PBA_T + tl], quat = sP[2 * PBA_T + tl];
    float dmean[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f}, dlogit = 0.f;
    float Y[16], gc[3] = {0.f, 0.f, 0.f}, il = 0.f, dir[3] = {0.f, 0.f, 0.f};
    bool ok = true;  // false: a non-finite gradient, reported; this Gaussian's state is then left as it is
    if (vis) {
      const gs_camera& cam = cams[uu];
      float2 g_xy = gxy[pidx];
      float4 g_co = gco[pidx];
      float4 g_rgb = grgb[pidx];
      ok = isfinite(g_xy.x) && isfinite(g_xy.y) && finite4(g_co) && finite4(g_rgb);
      // pass A: colour before the clamp
      float vx = mean.x - cam.campos[0], vy = mean.y - cam.campos[1], vz = mean.z - cam.campos[2];
      il = 1.0f / sqrtf(vx * vx + vy * vy + vz * vz);
      dir[0] = vx * il; dir[1] = vy * il; dir[2] = vz * il;
      sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
      float col[3] = {0.5f, 0.5f, 0.5f};
      #pragma unroll
      for (int k = 0; k < NP; ++k) {
        float4 q = sP[(3 + k) * PBA_T + tl];
        const float* qq = &q.x;
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          int f = 4 * k + e;
          if (f < 3 * NC) col[f % 3] += Y[f / 3] * qq[e];
        }
      }
      gc[0] = col[0] < 0.f ? 0.f : g_rgb.x;
      gc[1] = col[1] < 0.f ? 0.f : g_rgb.y;
      gc[2] = col[2] < 0.f ? 0.f : g_rgb.z;
      // everything but the SH direction term (as in project_grads)
      float qn[5];
      Geo g;
      geometry(cam, mean, sop, quat, g, qn);
      float itz = 1.0f / g.t[2];
      float dt[3] = {0.f, 0.f, 0.f};
      {
        float op = 1.0f / (1.0f + expf(-sop.w));
        dlogit = g_co.w * op * (1.f - op);
      }
      dt[0] += g_xy.x * cam.fx * itz;
      dt[1] += g_xy.y * cam.fy * itz;
      dt[2] += -(g_xy.x * cam.fx * g.t[0] + g_xy.y * cam.fy * g.t[1]) * itz * itz;
      float a = g.a, b = g.b, cc = g.c, det = g.det;
      float id2 = 1.0f / (det * det);
      float gA = g_co.x, gB = g_co.y, gC = g_co.z;
      float da = (-cc * cc * gA + b * cc * gB - b * b * gC) * id2;
      float db = (2.f * b * cc * gA - (det + 2.f * b * b) * gB + 2.f * a * b * gC) * id2;
      float dc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
      const float* T = g.T2;
      float hb = 0.5f * db;
      float GT0[3], GT1[3];
      #pragma unroll
      for (int j = 0; j < 3; ++j) {
        GT0[j] = da * T[j] + hb * T[3 + j];
        GT1[j] = hb * T[j] + dc * T[3 + j];
      }
      float dSig[9];
      #pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
        #pragma unroll
        for (int j = 0; j < 3; ++j) dSig[3 * i2 + j] = T[i2] * GT0[j] + T[3 + i2] * GT1[j];
      const float* S6 = g.Sig;
      float Sg[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
      float dT2[6];
      #pragma unroll
      for (int j = 0; j < 3; ++j) {
        dT2[j] = 2.f * (GT0[0] * Sg[j] + GT0[1] * Sg[3 + j] + GT0[2] * Sg[6 + j]);
        dT2[3 + j] = 2.f * (GT1[0] * Sg[j] + GT1[1] * Sg[3 + j] + GT1[2] * Sg[6 + j]);
      }
      const float* V = cam.viewmat;
      float dJ00 = dT2[0] * V[0] + dT2[1] * V[1] + dT2[2] * V[2];
      float dJ02 = dT2[0] * V[8] + dT2[1] * V[9] + dT2[2] * V[10];
      float dJ11 = dT2[3] * V[4] + dT2[4] * V[5] + dT2[5] * V[6];
      float dJ12 = dT2[3] * V[8] + dT2[4] * V[9] + dT2[5] * V[10];
      dt[2] += -(dJ00 * cam.fx + dJ11 * cam.fy) * itz * itz;
      if (g.clx) {
        dt[2] += dJ02 * cam.fx * g.xzc * itz * itz;
      } else {
        dt[0] += -dJ02 * cam.fx * itz * itz;
        dt[2] += 2.f * dJ02 * cam.fx * g.t[0] * itz * itz * itz;
      }
      if (g.cly) {
        dt[2] += dJ12 * cam.fy * g.yzc * itz * itz;
      } else {
        dt[1] += -dJ12 * cam.fy * itz * itz;
        dt[2] += 2.f * dJ12 * cam.fy * g.t[1] * itz * itz * itz;
      }
      #pragma unroll
      for (int k = 0; k < 3; ++k) dmean[k] += V[k] * dt[0] + V[4 + k] * dt[1] + V[8 + k] * dt[2];
      float M[9];
      #pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
        #pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i2 + j] = g.Rq[3 * i2 + j] * g.s[j];
      float dR[9];
      #pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
        #pragma unroll
        for (int j = 0; j < 3; ++j) {
          float dM = 2.f * (dSig[3 * i2] * M[j] + dSig[3 * i2 + 1] * M[3 + j] + dSig[3 * i2 + 2] * M[6 + j]);
          dls[j] += dM * g.Rq[3 * i2 + j] * g.s[j];
          dR[3 * i2 + j] = dM * g.s[j];
        }
      float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
      float gw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
      float gx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                        w * dR[7] - 2.f * x * dR[8]);
      float gy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                        z * dR[7] - 2.f * y * dR[8]);
      float gz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                        x * dR[6] + y * dR[7]);
      float dot = gw * w + gx * x + gy * y + gz * z;
      float inv = qn[4];
      dq[0] = (gw - dot * w) * inv;
      dq[1] = (gx - dot * x) * inv;
      dq[2] = (gy - dot * y) * inv;
      dq[3] = (gz - dot * z) * inv;
      // with finite screen-space gradients and parameters, every gradient below is finite
      ok = ok && finite4(make_float4(dmean[0], dmean[1], dmean[2], dlogit)) &&
           finite4(make_float4(dls[0], dls[1], dls[2], 0.f)) && finite4(make_float4(dq[0], dq[1], dq[2], dq[3]));
      #pragma unroll
      for (int k = 0; k < NP; ++k) ok = ok && finite4(sP[(3 + k) * PBA_T + tl]);
      if (!ok) set_status(status, GS_ERR_NONFINITE);
    } else {
      #pragma unroll
      for (int k = 0; k < 16; ++k) Y[k] = 0.f;
    }
    // pass B: per SH plane, its gradient, the direction term and the Adam update
    float wsum[16];
    #pragma unroll
    for (int k = 0; k < 16; ++k) wsum[k] = 0.f;
    #pragma unroll
    for (int k = 0; k < NP; ++k) {
      int64_t o = (3 + k) * N + i;
      float4 P = sP[(3 + k) * PBA_T + tl];
      cp_async_wait<PBA_R - 1>();  // the moments of sequence step k
      const float4* slot = sR + (k % PBA_R) * 2 * PBA_T;
      float* pp = &P.x;
      float G[4];
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        int f = 4 * k + e;
        G[e] = 0.f;
        if (f < 3 * NC) {
          G[e] = Y[f / 3] * gc[f % 3];
          wsum[f / 3] += pp[e] * gc[f % 3];
        }
      }
      float4 Gk = make_float4(G[0], G[1], G[2], G[3]);
      float4 Mv = slot[tl], Vv = slot[PBA_T + tl];
      adam4(P, Gk, Mv, Vv, s_lr[3 + k], b1, b2, ibc1, ibc2, eps);
      if (ok) {
        params[o] = P; m[o] = Mv; v[o] = Vv;
        if (nx.cams) sP[(3 + k) * PBA_T + tl] = P;  // the updated plane, for the next step's colour
      }
      if (grads) grads[o] = Gk;
      mv_copy(k + PBA_R);  // the slot's values are consumed: refill it PBA_R steps ahead
    }
    if (vis && DEG > 0) {
      float sx, sy, sz;
      sh_grad<DEG>(dir[0], dir[1], dir[2], wsum, sx, sy, sz);
      float d = sx * dir[0] + sy * dir[1] + sz * dir[2];
      dmean[0] += (sx - d * dir[0]) * il;
      dmean[1] += (sy - d * dir[1]) * il;
      dmean[2] += (sz - d * dir[2]) * il;
    }
    float4 Gp[3] = {make_float4(dmean[0], dmean[1], dmean[2], 0.f), make_float4(dls[0], dls[1], dls[2], dlogit),
                    make_float4(dq[0], dq[1], dq[2], dq[3])};
    float4 Pv[3] = {mean, sop, quat};
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
      int64_t o = k * N + i;
      cp_async_wait<PBA_R - 1>();  // the moments of sequence step NP + k
      const float4* slot = sR + ((NP + k) % PBA_R) * 2 * PBA_T;
      float4 Mv = slot[tl], Vv = slot[PBA_T + tl];
      adam4(Pv[k], Gp[k], Mv, Vv, s_lr[k], b1, b2, ibc1, ibc2, eps);
      if (ok) { params[o] = Pv[k]; m[o] = Mv; v[o] = Vv; }
      if (grads) grads[o] = Gp[k];
      mv_copy(NP + k + PBA_R);
    }
    pm = ok ? Pv[0] : mean; ps = ok ? Pv[1] : sop; pq = ok ? Pv[2] : quat;
    shp = sP + 3 * PBA_T + tl;
    shs = PBA_T;
  } else {
    pm = __ldg(params + i); ps = __ldg(params + N + i); pq = __ldg(params + 2 * N + i);
    shp = params + 3 * N + i;
    shs = N;
  }
  // a1 of the next step, fused: the Gaussian as stored projected for the next camera of its unit
  if (nx.cams && uu >= 0)
    project_record<DEG>(nx.cams[uu], pm, ps, pq, nx.W, nx.H, true, shp, shs, nx.xy + pidx, nx.conic_op + pidx,
                        nx.rgb + pidx, nx.depth + pidx, nx.radius + pidx, nx.tiles + pidx, status);
}

__global__ void k_step_advance(int32_t* s) { *s += 1; }

}  // namespace

// ---------------------------------------------------------------- host helpers
int gs_check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "libgs: CUDA error %s\n", cudaGetErrorString(e));
    return GS_ERR_CUDA;
  }
  return GS_OK;
}

int gs_fill_units(const gs_units* u, UnitTable& t, int64_t* total) {
  if (!u || u->n_units < 1 || u->n_units > GS_MAX_UNITS || !u->gauss_begin || !u->gauss_count)
    return GS_ERR_INVALID;
  t.n = u->n_units;
  int64_t acc = 0;
  for (int k = 0; k < t.n; ++k) {
    if (u->gauss_begin[k] < 0 || u->gauss_count[k] < 0) return GS_ERR_INVALID;
    t.proj_base[k] = acc;
    t.gauss_begin[k] = u->gauss_begin[k];
    acc += u->gauss_count[k];
  }
  t.proj_base[t.n] = acc;
  if (acc >= (int64_t)UINT32_MAX) return GS_ERR_INVALID;  // record ids are 32-bit
  if (total) *total = acc;
  return GS_OK;
}

int gs_fill_owned(const gs_owned* o, OwnedTable& t) {
  memset(&t, 0, sizeof(t));
  if (!o || o->n_parts == 0) return GS_OK;
  if (o->n_parts < 0 || o->n_parts > GS_MAX_PARTS || !o->part_offsets || !o->boxes || !o->closed_hi)
    return GS_ERR_INVALID;
  t.n = o->n_parts;
  for (int k = 0; k <= t.n; ++k) t.part_off[k] = o->part_offsets[k];
  for (int k = 0; k < t.n; ++k) {
    for (int a = 0; a < 6; ++a) t.box[k][a] = o->boxes[6 * k + a];
    t.closed_hi[k] = o->closed_hi[k];
  }
  return GS_OK;
}

static bool units_in_range(const UnitTable& t, int64_t n_gauss) {
  for (int k = 0; k < t.n; ++k)
    if (t.gauss_begin[k] + (t.proj_base[k + 1] - t.proj_base[k]) > n_gauss) return false;
  return true;
}

GS_API int gs_param_planes(int sh_degree) { return param_planes(sh_degree); }

GS_API int gs_status_read(int* d_status, int clear, gs_stream_t stream) {
  GS_RANGE("gs_status_read");
  if (!d_status) return GS_ERR_INVALID;
  int h = 0;
  if (cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return GS_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GS_ERR_CUDA;
  if (clear && cudaMemsetAsync(d_status, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess) return GS_ERR_CUDA;
  return h;
}

GS_API int gs_preprocess(const float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                         const gs_camera* cams, int width, int height, const gs_owned* owned,
                         const gs_proj* proj, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_preprocess");
  UnitTable U;
  OwnedTable O;
  int64_t P = 0;
  if ((!params && n_gauss > 0) || !cams || !proj || n_gauss < 0 || width <= 0 || height <= 0 ||
      param_planes(sh_degree) < 0)
    return GS_ERR_INVALID;
  if (!proj->xy || !proj->conic_op || !proj->rgb || !proj->depth || !proj->radius || !proj->tiles)
    return GS_ERR_INVALID;
  if (gs_fill_units(units, U, &P) != GS_OK || !units_in_range(U, n_gauss)) return GS_ERR_INVALID;
  if (gs_fill_owned(owned, O) != GS_OK) return GS_ERR_INVALID;
  if (O.n > 0 && O.part_off[O.n] != n_gauss) return GS_ERR_INVALID;
  if (P == 0) return GS_OK;
  dim3 block(256), grid((unsigned)((P + 255) / 256));
  cudaStream_t s = (cudaStream_t)stream;
  const float4* p4 = (const float4*)params;
#define GS_PRE(D)                                                                                   \
  k_preprocess<D><<<grid, block, 0, s>>>(p4, n_gauss, U, O, cams, width, height, (float4*)proj->xy, \
                                         (float4*)proj->conic_op, (float4*)proj->rgb, proj->depth,   \
                                         proj->radius, proj->tiles, d_status)
  switch (sh_degree) {
    case 0: GS_PRE(0); break;
    case 1: GS_PRE(1); break;
    case 2: GS_PRE(2); break;
    default: GS_PRE(3); break;
  }
#undef GS_PRE
  return gs_check_launch();
}

GS_API int gs_project_bwd(const float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                          const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d, float* grads,
                          gs_stream_t stream) {
  GS_RANGE("gs_project_bwd");
  UnitTable U;
  int64_t P = 0;
  if (((!params || !grads) && n_gauss > 0) || !cams || !proj || !g2d || n_gauss < 0 ||
      param_planes(sh_degree) < 0)
    return GS_ERR_INVALID;
  if (!proj->radius || !g2d->dxy || !g2d->dconic_op || !g2d->drgb) return GS_ERR_INVALID;
  if (gs_fill_units(units, U, &P) != GS_OK || !units_in_range(U, n_gauss)) return GS_ERR_INVALID;
  if (n_gauss == 0) return GS_OK;
  dim3 block(128), grid((unsigned)((n_gauss + 127) / 128));
  cudaStream_t s = (cudaStream_t)stream;
#define GS_PB(D)                                                                                           \
  k_project_bwd<D><<<grid, block, 0, s>>>((const float4*)params, n_gauss, U, cams, proj->radius,          \
                                          (const float2*)g2d->dxy, (const float4*)g2d->dconic_op,         \
                                          (const float4*)g2d->drgb, (float4*)grads)
  switch (sh_degree) {
    case 0: GS_PB(0); break;
    case 1: GS_PB(1); break;
    case 2: GS_PB(2); break;
    default: GS_PB(3); break;
  }
#undef GS_PB
  return gs_check_launch();
}

GS_API int gs_adam_step(float* params, float* grads, float* m, float* v, int64_t n_gauss, int n_planes,
                        const float* lr_init, const float* lr_final, int32_t lr_steps, float beta1, float beta2,
                        float eps, const int32_t* d_step, int zero_grad, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_adam_step");
  if (!params || !grads || !m || !v || !lr_init || !d_step || n_gauss < 0 || n_planes < 1 || n_planes > 16)
    return GS_ERR_INVALID;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f)) return GS_ERR_INVALID;
  AdamLR lr;
  memset(&lr, 0, sizeof(lr));
  for (int k = 0; k < n_planes; ++k) {
    lr.init[k] = make_float4(lr_init[4 * k], lr_init[4 * k + 1], lr_init[4 * k + 2], lr_init[4 * k + 3]);
    const float* f = lr_final ? lr_final : lr_init;
    lr.fin[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
  }
  if (n_gauss == 0) return GS_OK;
  int64_t total = (int64_t)n_planes * n_gauss;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (total + 255) / 256;
  int64_t cap = (int64_t)sms * 8;
  unsigned grid = (unsigned)(want < cap ? want : cap);
  k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>((float4*)params, (float4*)grads, (float4*)m, (float4*)v, n_gauss,
                                                 n_planes, lr, lr_steps, beta1, beta2, eps, d_step, zero_grad,
                                                 d_status);
  return gs_check_launch();
}

GS_API int gs_step_advance(int32_t* d_step, gs_stream_t stream) {
  GS_RANGE("gs_step_advance");
  if (!d_step) return GS_ERR_INVALID;
  k_step_advance<<<1, 1, 0, (cudaStream_t)stream>>>(d_step);
  return gs_check_launch();
}

static int project_bwd_adam_impl(float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                                 const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d, float* m,
                                 float* v, const float* lr_init, const float* lr_final, int32_t lr_steps, float beta1,
                                 float beta2, float eps, const int32_t* d_step, float* grads, int sparse,
                                 int* d_status, gs_stream_t stream, const gs_camera* next_cams, int width,
                                 int height) {
  UnitTable U;
  int64_t P = 0;
  int npl = param_planes(sh_degree);
  if (((!params || !m || !v) && n_gauss > 0) || !cams || !proj || !g2d || n_gauss < 0 || npl < 0 || !lr_init ||
      !d_step)
    return GS_ERR_INVALID;
  if (!proj->radius || !g2d->dxy || !g2d->dconic_op || !g2d->drgb) return GS_ERR_INVALID;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f)) return GS_ERR_INVALID;
  if (gs_fill_units(units, U, &P) != GS_OK || !units_in_range(U, n_gauss)) return GS_ERR_INVALID;
  AdamLR lr;
  memset(&lr, 0, sizeof(lr));
  for (int k = 0; k < npl; ++k) {
    const float* f = lr_final ? lr_final : lr_init;
    lr.init[k] = make_float4(lr_init[4 * k], lr_init[4 * k + 1], lr_init[4 * k + 2], lr_init[4 * k + 3]);
    lr.fin[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
  }
  // every Gaussian in at most one unit: the streaming kernel applies
  bool disjoint = true;
  for (int a = 0; a < U.n && disjoint; ++a)
    for (int b = a + 1; b < U.n && disjoint; ++b) {
      int64_t a0 = U.gauss_begin[a], a1 = a0 + (U.proj_base[a + 1] - U.proj_base[a]);
      int64_t b0 = U.gauss_begin[b], b1 = b0 + (U.proj_base[b + 1] - U.proj_base[b]);
      if (a0 < b1 && b0 < a1) disjoint = false;
    }
  NextProj nx{};
  if (next_cams) {
    if (!disjoint || width <= 0 || height <= 0 || !proj->xy || !proj->conic_op || !proj->rgb || !proj->depth ||
        !proj->tiles)
      return GS_ERR_INVALID;
    nx = NextProj{next_cams, width, height, (float4*)proj->xy, (float4*)proj->conic_op, (float4*)proj->rgb,
                  proj->depth, proj->radius, proj->tiles};
  }
  if (n_gauss == 0) return GS_OK;
  dim3 block(128), grid((unsigned)((n_gauss + 127) / 128));
  cudaStream_t s = (cudaStream_t)stream;
  if (disjoint) {
    dim3 grid1((unsigned)((n_gauss + PBA_T - 1) / PBA_T));
    size_t smem1 = sizeof(float4) * ((size_t)npl + 2 * PBA_R) * PBA_T;  // 23,552 B at degree 3
#define GS_PBA1(D)                                                                                                \
  k_project_bwd_adam1<D><<<grid1, PBA_T, smem1, s>>>((float4*)params, n_gauss, U, cams, proj->radius,            \
                                                (const float2*)g2d->dxy, (const float4*)g2d->dconic_op,          \
                                                (const float4*)g2d->drgb, (float4*)m, (float4*)v, lr, lr_steps,   \
                                                beta1, beta2, eps, d_step, (float4*)grads, sparse, d_status, nx)
    switch (sh_degree) {
      case 0: GS_PBA1(0); break;
      case 1: GS_PBA1(1); break;
      case 2: GS_PBA1(2); break;
      default: GS_PBA1(3); break;
    }
#undef GS_PBA1
    return gs_check_launch();
  }
#define GS_PBA(D)                                                                                                \
  k_project_bwd_adam<D><<<grid, block, 0, s>>>((float4*)params, n_gauss, U, cams, proj->radius,                 \
                                               (const float2*)g2d->dxy, (const float4*)g2d->dconic_op,          \
                                               (const float4*)g2d->drgb, (float4*)m, (float4*)v, lr, lr_steps,   \
                                               beta1, beta2, eps, d_step, (float4*)grads, sparse, d_status)
  switch (sh_degree) {
    case 0: GS_PBA(0); break;
    case 1: GS_PBA(1); break;
    case 2: GS_PBA(2); break;
    default: GS_PBA(3); break;
  }
#undef GS_PBA
  return gs_check_launch();
}

GS_API int gs_project_bwd_adam(float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                               const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d, float* m, float* v,
                               const float* lr_init, const float* lr_final, int32_t lr_steps, float beta1,
                               float beta2, float eps, const int32_t* d_step, float* grads, int sparse,
                               int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_project_bwd_adam");
  return project_bwd_adam_impl(params, n_gauss, sh_degree, units, cams, proj, g2d, m, v, lr_init, lr_final, lr_steps,
                               beta1, beta2, eps, d_step, grads, sparse, d_status, stream, nullptr, 0, 0);
}

GS_API int gs_project_bwd_adam_next(float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                                    const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d, float* m,
                                    float* v, const float* lr_init, const float* lr_final, int32_t lr_steps,
                                    float beta1, float beta2, float eps, const int32_t* d_step, float* grads,
                                    int sparse, const gs_camera* next_cams, int width, int height, int* d_status,
                                    gs_stream_t stream) {
  GS_RANGE("gs_project_bwd_adam_next");
  if (!next_cams) return GS_ERR_INVALID;
  return project_bwd_adam_impl(params, n_gauss, sh_degree, units, cams, proj, g2d, m, v, lr_init, lr_final, lr_steps,
                               beta1, beta2, eps, d_step, grads, sparse, d_status, stream, next_cams, width, height);
}
