// a9 (second half): the learned initialiser.  A 3-layer MLP maps each
// isosurface point's kNN geometry to its initial log-scale (relative to the
// mean 3-NN distance), rotation and opacity.
//
// Network: X[112] -> relu(X W1 + b1)[64] -> relu(. W2 + b2)[64] -> . W3 + b3 [8].
// Features (built in shared memory, never stored): the 16 neighbour offsets
// divided by the mean neighbour distance (48), the 16 neighbour normals (48),
// the point's own normal (3), zero padding to 112.  GEMM operands are bf16
// (round to nearest even), products accumulate in fp32 on the tensor cores
// (mma.sync m16n8k16 / m16n8k8); activations are rounded to bf16 where they
// become the next GEMM's operand, and back-propagated signals likewise.
//
// One CTA of 4 warps handles batches of 64 points, 16 per warp.  Layer
// outputs stay in registers: the accumulator layout of two adjacent n8 tiles
// is the A-operand layout of one k16 step, so layers chain without shared
// memory.  Weight gradients are tensor-core GEMMs over the 64-point batch
// from bf16 tiles in shared memory, accumulated per CTA in fp32 shared memory
// and added to the global gradient once per CTA.
//
// This stage is HBM-bound (about 300 bytes of gathered neighbour data per
// point against 23 kFLOP), so mma.sync at this size already saturates the
// memory system; see the design notes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

constexpr int KIN = 112, HID = 64, KOUT = 8, KNN = 16;
constexpr int W1_OFF = 0, B1_OFF = W1_OFF + KIN * HID, W2_OFF = B1_OFF + HID, B2_OFF = W2_OFF + HID * HID;
constexpr int W3_OFF = B2_OFF + HID, B3_OFF = W3_OFF + HID * KOUT, NPARAM = B3_OFF + KOUT;  // 11912
constexpr int BATCH = 64;
constexpr int THREADS = 128;
constexpr int LDX = 120;  // bf16 row stride of the feature tile and of W1^T
constexpr int LDH = 72;   // bf16 row stride of 64-wide tiles

static_assert(NPARAM == 11912, "parameter layout");

// shared-memory layout (bytes)
struct Smem {
  static constexpr int W1t = 0;                          // [64][LDX] bf16  W1^T
  static constexpr int W2t = W1t + HID * LDX * 2;        // [64][LDH] bf16  W2^T
  static constexpr int W2 = W2t + HID * LDH * 2;         // [64][LDH] bf16  W2 (in-major)
  static constexpr int W3t = W2 + HID * LDH * 2;         // [8][LDH]  bf16  W3^T
  static constexpr int W3 = W3t + KOUT * LDH * 2;        // [64][8]   bf16  W3 (in-major)
  static constexpr int Bias = W3 + HID * KOUT * 2;       // fp32 b1[64] b2[64] b3[8]
  static constexpr int X = Bias + (2 * HID + KOUT) * 4;  // [64][LDX] bf16 features
  static constexpr int Dbar = X + BATCH * LDX * 2;       // fp32 [64]
  static constexpr int FWD_END = Dbar + BATCH * 4;
  static constexpr int H1 = FWD_END;                     // [64][LDH] bf16
  static constexpr int H2 = H1 + BATCH * LDH * 2;
  static constexpr int dH1 = H2 + BATCH * LDH * 2;
  static constexpr int dH2 = dH1 + BATCH * LDH * 2;
  static constexpr int dY = dH2 + BATCH * LDH * 2;       // [64][8] bf16
  static constexpr int dW = dY + BATCH * KOUT * 2;       // fp32 [NPARAM]
  static constexpr int TRAIN_END = dW + NPARAM * 4;
};

__device__ __forceinline__ uint16_t bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack(float lo, float hi) {
  return (uint32_t)bf(lo) | ((uint32_t)bf(hi) << 16);
}
__device__ __forceinline__ float unbf(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }
__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pair(const uint16_t* lo, const uint16_t* hi) {
  return (uint32_t)(*lo) | ((uint32_t)(*hi) << 16);
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma1688(float* d, uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

// Stage the fp32 master weights as bf16 (transposed copies where the
// B operand needs them) and the biases as fp32.
__device__ void stage_weights(const float* __restrict__ w, char* sm, bool train) {
  uint16_t* W1t = (uint16_t*)(sm + Smem::W1t);
  uint16_t* W2t = (uint16_t*)(sm + Smem::W2t);
  uint16_t* W2 = (uint16_t*)(sm + Smem::W2);
  uint16_t* W3t = (uint16_t*)(sm + Smem::W3t);
  uint16_t* W3 = (uint16_t*)(sm + Smem::W3);
  float* bias = (float*)(sm + Smem::Bias);
  for (int q = threadIdx.x; q < KIN * HID; q += blockDim.x) {
    int k = q / HID, o = q % HID;
    W1t[o * LDX + k] = bf(w[W1_OFF + q]);
  }
  for (int q = threadIdx.x; q < HID * HID; q += blockDim.x) {
    int k = q / HID, o = q % HID;
    uint16_t v = bf(w[W2_OFF + q]);
    W2t[o * LDH + k] = v;
    if (train) W2[k * LDH + o] = v;
  }
  for (int q = threadIdx.x; q < HID * KOUT; q += blockDim.x) {
    int k = q / KOUT, o = q % KOUT;
    uint16_t v = bf(w[W3_OFF + q]);
    W3t[o * LDH + k] = v;
    if (train) W3[k * KOUT + o] = v;
  }
  for (int q = threadIdx.x; q < 2 * HID + KOUT; q += blockDim.x) {
    int src = q < HID ? B1_OFF + q : (q < 2 * HID ? B2_OFF + q - HID : B3_OFF + q - 2 * HID);
    bias[q] = w[src];
  }
}

// Features of the batch's points into the bf16 tile X[64][LDX].
__device__ void build_features(const float* __restrict__ pts, const float* __restrict__ nrm,
                               const int* __restrict__ knn_idx, const float* __restrict__ knn_dist, int64_t n,
                               int64_t base, char* sm) {
  uint16_t* X = (uint16_t*)(sm + Smem::X);
  float* dbar = (float*)(sm + Smem::Dbar);
  for (int p = threadIdx.x; p < BATCH; p += blockDim.x) {
    int64_t i = base + p;
    float s = 0.f;
    if (i < n)
      for (int a = 0; a < KNN; ++a) s += knn_dist[i * KNN + a];
    float d = s / (float)KNN;
    dbar[p] = d > 1e-12f ? d : 1e-12f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < BATCH * KNN; q += blockDim.x) {
    int p = q / KNN, a = q % KNN;
    int64_t i = base + p;
    float o[3] = {0.f, 0.f, 0.f}, nn[3] = {0.f, 0.f, 0.f};
    if (i < n) {
      int j = knn_idx[i * KNN + a];
      if (j >= 0) {
        float inv = dbar[p];
        for (int c = 0; c < 3; ++c) {
          o[c] = (pts[3 * (int64_t)j + c] - pts[3 * i + c]) / inv;
          nn[c] = nrm[3 * (int64_t)j + c];
        }
      }
    }
    for (int c = 0; c < 3; ++c) {
      X[p * LDX + 3 * a + c] = bf(o[c]);
      X[p * LDX + 48 + 3 * a + c] = bf(nn[c]);
    }
  }
  for (int q = threadIdx.x; q < BATCH * (KIN - 96); q += blockDim.x) {
    int p = q / (KIN - 96), f = 96 + q % (KIN - 96);
    int64_t i = base + p;
    float v = (f < 99 && i < n) ? nrm[3 * i + (f - 96)] : 0.f;
    X[p * LDX + f] = bf(v);
  }
  __syncthreads();
}

// Forward pass of the warp's 16 rows (m0 .. m0+15 of the batch).  h1, h2 are
// the post-ReLU fp32 activations in accumulator layout; y the outputs.
__device__ __forceinline__ void forward_rows(const char* sm, int m0, float (&h1)[8][4], float (&h2)[8][4],
                                             float (&y)[4]) {
  const uint16_t* X = (const uint16_t*)(sm + Smem::X);
  const uint16_t* W1t = (const uint16_t*)(sm + Smem::W1t);
  const uint16_t* W2t = (const uint16_t*)(sm + Smem::W2t);
  const uint16_t* W3t = (const uint16_t*)(sm + Smem::W3t);
  const float* bias = (const float*)(sm + Smem::Bias);
  int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  #pragma unroll
  for (int j = 0; j < 8; ++j) h1[j][0] = h1[j][1] = h1[j][2] = h1[j][3] = 0.f;
  #pragma unroll
  for (int s = 0; s < KIN / 16; ++s) {
    int k0 = 16 * s + 2 * t;
    uint32_t a[4] = {ld32(X + (m0 + g) * LDX + k0), ld32(X + (m0 + g + 8) * LDX + k0),
                     ld32(X + (m0 + g) * LDX + k0 + 8), ld32(X + (m0 + g + 8) * LDX + k0 + 8)};
    #pragma unroll
    for (int j = 0; j < 8; ++j)
      mma16816(h1[j], a, ld32(W1t + (8 * j + g) * LDX + k0), ld32(W1t + (8 * j + g) * LDX + k0 + 8));
  }
  #pragma unroll
  for (int j = 0; j < 8; ++j) {
    float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
    h1[j][0] = fmaxf(h1[j][0] + b0, 0.f); h1[j][1] = fmaxf(h1[j][1] + b1, 0.f);
    h1[j][2] = fmaxf(h1[j][2] + b0, 0.f); h1[j][3] = fmaxf(h1[j][3] + b1, 0.f);
  }
  #pragma unroll
  for (int j = 0; j < 8; ++j) h2[j][0] = h2[j][1] = h2[j][2] = h2[j][3] = 0.f;
  #pragma unroll
  for (int s = 0; s < HID / 16; ++s) {
    uint32_t a[4] = {pack(h1[2 * s][0], h1[2 * s][1]), pack(h1[2 * s][2], h1[2 * s][3]),
                     pack(h1[2 * s + 1][0], h1[2 * s + 1][1]), pack(h1[2 * s + 1][2], h1[2 * s + 1][3])};
    int k0 = 16 * s + 2 * t;
    #pragma unroll
    for (int j = 0; j < 8; ++j)
      mma16816(h2[j], a, ld32(W2t + (8 * j + g) * LDH + k0), ld32(W2t + (8 * j + g) * LDH + k0 + 8));
  }
  #pragma unroll
  for (int j = 0; j < 8; ++j) {
    float b0 = bias[HID + 8 * j + 2 * t], b1 = bias[HID + 8 * j + 2 * t + 1];
    h2[j][0] = fmaxf(h2[j][0] + b0, 0.f); h2[j][1] = fmaxf(h2[j][1] + b1, 0.f);
    h2[j][2] = fmaxf(h2[j][2] + b0, 0.f); h2[j][3] = fmaxf(h2[j][3] + b1, 0.f);
  }
  y[0] = y[1] = y[2] = y[3] = 0.f;
  #pragma unroll
  for (int s = 0; s < HID / 16; ++s) {
    uint32_t a[4] = {pack(h2[2 * s][0], h2[2 * s][1]), pack(h2[2 * s][2], h2[2 * s][3]),
                     pack(h2[2 * s + 1][0], h2[2 * s + 1][1]), pack(h2[2 * s + 1][2], h2[2 * s + 1][3])};
    int k0 = 16 * s + 2 * t;
    mma16816(y, a, ld32(W3t + g * LDH + k0), ld32(W3t + g * LDH + k0 + 8));
  }
  float b0 = bias[2 * HID + 2 * t], b1 = bias[2 * HID + 2 * t + 1];
  y[0] += b0; y[1] += b1; y[2] += b0; y[3] += b1;
}

// y rows (m0+g, m0+g+8), cols (2t, 2t+1) -> out[row][col]
__global__ void __launch_bounds__(THREADS) k_mlp_forward(const float* __restrict__ pts, const float* __restrict__ nrm,
                                                         const int* __restrict__ knn_idx,
                                                         const float* __restrict__ knn_dist, int64_t n,
                                                         const float* __restrict__ w, float* __restrict__ out) {
  extern __shared__ __align__(16) char sm[];
  stage_weights(w, sm, false);
  __syncthreads();
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  int64_t nb = (n + BATCH - 1) / BATCH;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    int64_t base = b * BATCH;
    build_features(pts, nrm, knn_idx, knn_dist, n, base, sm);
    float h1[8][4], h2[8][4], y[4];
    int m0 = warp * 16;
    forward_rows(sm, m0, h1, h2, y);
    int64_t r0 = base + m0 + g, r1 = r0 + 8;
    if (r0 < n) { out[r0 * KOUT + 2 * t] = y[0]; out[r0 * KOUT + 2 * t + 1] = y[1]; }
    if (r1 < n) { out[r1 * KOUT + 2 * t] = y[2]; out[r1 * KOUT + 2 * t + 1] = y[3]; }
    __syncthreads();  // the feature tile is rebuilt next iteration
  }
}

// Initial Gaussian parameters: plane 1 (log-scale, logit opacity) and plane 2
// (rotation).  Plain form: isotropic log(mean 3-NN distance), identity rotation,
// logit_default.  With the MLP: log-scale = log(d3) + y[0:3], rotation y[3:7],
// logit y[7]; any non-finite output (or a rotation of norm < 1e-6) falls back to
// the plain values for that Gaussian.
__device__ __forceinline__ void write_init(float4* __restrict__ params, int64_t N, int64_t i, float d3, const float* y,
                                           bool have_y, float logit_default) {
  float ls = logf(fmaxf(d3, 1e-7f));
  float4 sop = make_float4(ls, ls, ls, logit_default);
  float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
  if (have_y) {
    bool ok = true;
    for (int c = 0; c < KOUT; ++c) ok = ok && isfinite(y[c]);
    float qn = sqrtf(y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
    ok = ok && qn > 1e-6f;
    if (ok) {
      sop = make_float4(ls + y[0], ls + y[1], ls + y[2], y[7]);
      q = make_float4(y[3], y[4], y[5], y[6]);
    }
  }
  params[N + i] = sop;
  params[2 * N + i] = q;
}

__global__ void k_plain_init(const float* __restrict__ knn_dist, int k, int64_t n, float logit_default,
                             float4* __restrict__ params, int64_t N) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float d3 = (knn_dist[i * k] + knn_dist[i * k + 1] + knn_dist[i * k + 2]) / 3.f;
  write_init(params, N, i, d3, nullptr, false, logit_default);
}

__global__ void __launch_bounds__(THREADS) k_mlp_init(const float* __restrict__ pts, const float* __restrict__ nrm,
                                                      const int* __restrict__ knn_idx,
                                                      const float* __restrict__ knn_dist, int64_t n,
                                                      const float* __restrict__ w, float logit_default,
                                                      float4* __restrict__ params, int64_t N) {
  extern __shared__ __align__(16) char sm[];
  stage_weights(w, sm, false);
  __syncthreads();
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float* ybuf = (float*)(sm + Smem::H1);  // [64][8] fp32 staging of the outputs
  int64_t nb = (n + BATCH - 1) / BATCH;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    int64_t base = b * BATCH;
    build_features(pts, nrm, knn_idx, knn_dist, n, base, sm);
    float h1[8][4], h2[8][4], y[4];
    int m0 = warp * 16;
    forward_rows(sm, m0, h1, h2, y);
    ybuf[(m0 + g) * KOUT + 2 * t] = y[0];
    ybuf[(m0 + g) * KOUT + 2 * t + 1] = y[1];
    ybuf[(m0 + g + 8) * KOUT + 2 * t] = y[2];
    ybuf[(m0 + g + 8) * KOUT + 2 * t + 1] = y[3];
    __syncthreads();
    for (int p = threadIdx.x; p < BATCH; p += blockDim.x) {
      int64_t i = base + p;
      if (i >= n) continue;
      float d3 = (knn_dist[i * KNN] + knn_dist[i * KNN + 1] + knn_dist[i * KNN + 2]) / 3.f;
      write_init(params, N, i, d3, ybuf + p * KOUT, true, logit_default);
    }
    __syncthreads();
  }
}

// One training step's gradients: forward, loss (sum of squared errors times
// `scale`), backward; dW accumulated into `grad` (zeroed by the caller).
__global__ void __launch_bounds__(THREADS) k_mlp_train(const float* __restrict__ pts, const float* __restrict__ nrm,
                                                       const int* __restrict__ knn_idx,
                                                       const float* __restrict__ knn_dist,
                                                       const float* __restrict__ target, int64_t n,
                                                       const float* __restrict__ w, float scale,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) char sm[];
  stage_weights(w, sm, true);
  float* dW = (float*)(sm + Smem::dW);
  for (int q = threadIdx.x; q < NPARAM; q += blockDim.x) dW[q] = 0.f;
  __syncthreads();
  uint16_t* sX = (uint16_t*)(sm + Smem::X);
  uint16_t* sH1 = (uint16_t*)(sm + Smem::H1);
  uint16_t* sH2 = (uint16_t*)(sm + Smem::H2);
  uint16_t* sdH1 = (uint16_t*)(sm + Smem::dH1);
  uint16_t* sdH2 = (uint16_t*)(sm + Smem::dH2);
  uint16_t* sdY = (uint16_t*)(sm + Smem::dY);
  const uint16_t* W2 = (const uint16_t*)(sm + Smem::W2);
  const uint16_t* W3 = (const uint16_t*)(sm + Smem::W3);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float lsum = 0.f;
  int64_t nb = (n + BATCH - 1) / BATCH;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    int64_t base = b * BATCH;
    build_features(pts, nrm, knn_idx, knn_dist, n, base, sm);
    float h1[8][4], h2[8][4], y[4];
    int m0 = warp * 16;
    forward_rows(sm, m0, h1, h2, y);
    int64_t r0 = base + m0 + g, r1 = r0 + 8;
    float dy[4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      int64_t r = e < 2 ? r0 : r1;
      int col = 2 * t + (e & 1);
      float d = 0.f;
      if (r < n) {
        d = y[e] - target[r * KOUT + col];
        lsum += d * d;
      }
      dy[e] = 2.f * d * scale;
    }
    uint32_t ady0 = pack(dy[0], dy[1]), ady1 = pack(dy[2], dy[3]);
    *reinterpret_cast<uint32_t*>(sdY + (m0 + g) * KOUT + 2 * t) = ady0;
    *reinterpret_cast<uint32_t*>(sdY + (m0 + g + 8) * KOUT + 2 * t) = ady1;
    // activations as bf16 tiles for the weight gradients
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
      *reinterpret_cast<uint32_t*>(sH1 + (m0 + g) * LDH + 8 * j + 2 * t) = pack(h1[j][0], h1[j][1]);
      *reinterpret_cast<uint32_t*>(sH1 + (m0 + g + 8) * LDH + 8 * j + 2 * t) = pack(h1[j][2], h1[j][3]);
      *reinterpret_cast<uint32_t*>(sH2 + (m0 + g) * LDH + 8 * j + 2 * t) = pack(h2[j][0], h2[j][1]);
      *reinterpret_cast<uint32_t*>(sH2 + (m0 + g + 8) * LDH + 8 * j + 2 * t) = pack(h2[j][2], h2[j][3]);
    }
    // dH2 = dY W3^T, masked by the ReLU of layer 2, rounded to bf16
    float d2[8][4];
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
      d2[j][0] = d2[j][1] = d2[j][2] = d2[j][3] = 0.f;
      mma1688(d2[j], ady0, ady1, ld32(W3 + (8 * j + g) * KOUT + 2 * t));
      #pragma unroll
      for (int e = 0; e < 4; ++e) d2[j][e] = h2[j][e] > 0.f ? d2[j][e] : 0.f;
      *reinterpret_cast<uint32_t*>(sdH2 + (m0 + g) * LDH + 8 * j + 2 * t) = pack(d2[j][0], d2[j][1]);
      *reinterpret_cast<uint32_t*>(sdH2 + (m0 + g + 8) * LDH + 8 * j + 2 * t) = pack(d2[j][2], d2[j][3]);
    }
    // dH1 = dH2 W2^T, masked by the ReLU of layer 1
    float d1[8][4];
    #pragma unroll
    for (int j = 0; j < 8; ++j) d1[j][0] = d1[j][1] = d1[j][2] = d1[j][3] = 0.f;
    #pragma unroll
    for (int s = 0; s < HID / 16; ++s) {
      uint32_t a[4] = {pack(d2[2 * s][0], d2[2 * s][1]), pack(d2[2 * s][2], d2[2 * s][3]),
                       pack(d2[2 * s + 1][0], d2[2 * s + 1][1]), pack(d2[2 * s + 1][2], d2[2 * s + 1][3])};
      int k0 = 16 * s + 2 * t;
      #pragma unroll
      for (int j = 0; j < 8; ++j)
        mma16816(d1[j], a, ld32(W2 + (8 * j + g) * LDH + k0), ld32(W2 + (8 * j + g) * LDH + k0 + 8));
    }
    #pragma unroll
    for (int j = 0; j < 8; ++j) {
      #pragma unroll
      for (int e = 0; e < 4; ++e) d1[j][e] = h1[j][e] > 0.f ? d1[j][e] : 0.f;
      *reinterpret_cast<uint32_t*>(sdH1 + (m0 + g) * LDH + 8 * j + 2 * t) = pack(d1[j][0], d1[j][1]);
      *reinterpret_cast<uint32_t*>(sdH1 + (m0 + g + 8) * LDH + 8 * j + 2 * t) = pack(d1[j][2], d1[j][3]);
    }
    __syncthreads();
    // weight gradients over the 64-point batch: dW1 = X^T dH1 (7 x 8 tiles),
    // dW2 = H1^T dH2 (4 x 8), dW3 = H2^T dY (4 x 1); K = the 64 points
    for (int tile = warp; tile < 56 + 32 + 4; tile += THREADS / 32) {
      const uint16_t *A, *B;
      int lda, ldb, mi, nj, ncols, off;
      if (tile < 56) { A = sX; lda = LDX; B = sdH1; ldb = LDH; mi = tile / 8; nj = tile % 8; ncols = HID; off = W1_OFF; }
      else if (tile < 88) { int q = tile - 56; A = sH1; lda = LDH; B = sdH2; ldb = LDH; mi = q / 8; nj = q % 8; ncols = HID; off = W2_OFF; }
      else { int q = tile - 88; A = sH2; lda = LDH; B = sdY; ldb = KOUT; mi = q; nj = 0; ncols = KOUT; off = W3_OFF; }
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      int m = 16 * mi + g, ncol = 8 * nj + g;
      #pragma unroll
      for (int s = 0; s < BATCH / 16; ++s) {
        int p = 16 * s + 2 * t;  // batch rows (the K dimension)
        uint32_t a[4] = {pair(A + p * lda + m, A + (p + 1) * lda + m),
                         pair(A + p * lda + m + 8, A + (p + 1) * lda + m + 8),
                         pair(A + (p + 8) * lda + m, A + (p + 9) * lda + m),
                         pair(A + (p + 8) * lda + m + 8, A + (p + 9) * lda + m + 8)};
        uint32_t b0 = pair(B + p * ldb + ncol, B + (p + 1) * ldb + ncol);
        uint32_t b1 = pair(B + (p + 8) * ldb + ncol, B + (p + 9) * ldb + ncol);
        mma16816(acc, a, b0, b1);
      }
      int col = 8 * nj + 2 * t;
      dW[off + m * ncols + col] += acc[0];
      dW[off + m * ncols + col + 1] += acc[1];
      dW[off + (m + 8) * ncols + col] += acc[2];
      dW[off + (m + 8) * ncols + col + 1] += acc[3];
    }
    // bias gradients: sums of the rounded back-propagated signals
    for (int q = threadIdx.x; q < 2 * HID + KOUT; q += blockDim.x) {
      float s = 0.f;
      if (q < HID) { for (int p = 0; p < BATCH; ++p) s += unbf(sdH1[p * LDH + q]); dW[B1_OFF + q] += s; }
      else if (q < 2 * HID) { for (int p = 0; p < BATCH; ++p) s += unbf(sdH2[p * LDH + q - HID]); dW[B2_OFF + q - HID] += s; }
      else { for (int p = 0; p < BATCH; ++p) s += unbf(sdY[p * KOUT + q - 2 * HID]); dW[B3_OFF + q - 2 * HID] += s; }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < NPARAM; q += blockDim.x)
    if (dW[q] != 0.f) atomicAdd(&grad[q], dW[q]);
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0 && lsum != 0.f) atomicAdd(loss, lsum * scale);
}

__global__ void k_features_out(const float* __restrict__ pts, const float* __restrict__ nrm,
                               const int* __restrict__ knn_idx, const float* __restrict__ knn_dist, int64_t n,
                               uint16_t* __restrict__ X) {
  extern __shared__ __align__(16) char sm[];
  int64_t nb = (n + BATCH - 1) / BATCH;
  const uint16_t* sX = (const uint16_t*)(sm + Smem::X);
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    int64_t base = b * BATCH;
    build_features(pts, nrm, knn_idx, knn_dist, n, base, sm);
    for (int q = threadIdx.x; q < BATCH * KIN; q += blockDim.x) {
      int p = q / KIN, f = q % KIN;
      if (base + p < n) X[(base + p) * KIN + f] = sX[p * LDX + f];
    }
    __syncthreads();
  }
}

int grid_for(int64_t n, int per_sm) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t nb = (n + BATCH - 1) / BATCH;
  int64_t cap = (int64_t)sms * per_sm;
  return (int)(nb < cap ? (nb > 0 ? nb : 1) : cap);
}

template <typename K>
int set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess ? GS_OK
                                                                                                          : GS_ERR_CUDA;
}

bool knn_args_ok(const float* pts, const float* nrm, const int32_t* idx, const float* dist, int64_t n) {
  return pts && nrm && idx && dist && n >= 0;
}

}  // namespace

GS_API int gs_mlp_param_count(void) { return NPARAM; }

GS_API int gs_mlp_features(const float* points, const float* normals, const int32_t* knn_idx, const float* knn_dist,
                           int64_t n, uint16_t* features, gs_stream_t stream) {
  GS_RANGE("gs_mlp_features");
  if (!knn_args_ok(points, normals, knn_idx, knn_dist, n) || !features) return GS_ERR_INVALID;
  if (n == 0) return GS_OK;
  if (set_smem(k_features_out, Smem::FWD_END) != GS_OK) return GS_ERR_CUDA;
  k_features_out<<<grid_for(n, 4), THREADS, Smem::FWD_END, (cudaStream_t)stream>>>(points, normals, knn_idx, knn_dist,
                                                                                   n, features);
  return gs_check_launch();
}

GS_API int gs_mlp_forward(const float* points, const float* normals, const int32_t* knn_idx, const float* knn_dist,
                          int64_t n, const float* weights, float* out, gs_stream_t stream) {
  GS_RANGE("gs_mlp_forward");
  if (!knn_args_ok(points, normals, knn_idx, knn_dist, n) || !weights || !out) return GS_ERR_INVALID;
  if (n == 0) return GS_OK;
  if (set_smem(k_mlp_forward, Smem::FWD_END) != GS_OK) return GS_ERR_CUDA;
  k_mlp_forward<<<grid_for(n, 4), THREADS, Smem::FWD_END, (cudaStream_t)stream>>>(points, normals, knn_idx, knn_dist,
                                                                                  n, weights, out);
  return gs_check_launch();
}

GS_API int gs_mlp_train_step(const float* points, const float* normals, const int32_t* knn_idx,
                             const float* knn_dist, const float* targets, int64_t n, float* weights, float* grad,
                             float* m, float* v, float lr, const int32_t* d_step, float* d_loss, gs_stream_t stream) {
  GS_RANGE("gs_mlp_train_step");
  if (!knn_args_ok(points, normals, knn_idx, knn_dist, n) || !targets || !weights || !grad || !m || !v ||
      !d_step || !d_loss || n < 1 || !(lr > 0.f))
    return GS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, s) != cudaSuccess ||
      cudaMemsetAsync(d_loss, 0, sizeof(float), s) != cudaSuccess)
    return GS_ERR_CUDA;
  if (set_smem(k_mlp_train, Smem::TRAIN_END) != GS_OK) return GS_ERR_CUDA;
  float scale = 1.0f / (8.0f * (float)n);
  k_mlp_train<<<grid_for(n, 1), THREADS, Smem::TRAIN_END, s>>>(points, normals, knn_idx, knn_dist, targets, n,
                                                               weights, scale, grad, d_loss);
  int r = gs_check_launch();
  if (r != GS_OK) return r;
  float lr4[4] = {lr, lr, lr, lr};
  return gs_adam_step(weights, grad, m, v, NPARAM / 4, 1, lr4, lr4, 0, 0.9f, 0.999f, 1e-8f, d_step, 0, nullptr,
                      stream);
}

GS_API int gs_init_gaussians(const float* points, const float* normals, const int32_t* knn_idx,
                             const float* knn_dist, int knn_k, int64_t n, const float* weights, float logit_default,
                             float* params, int64_t n_gauss, gs_stream_t stream) {
  GS_RANGE("gs_init_gaussians");
  if (!points || !knn_dist || !params || n < 0 || n > n_gauss || knn_k < 3) return GS_ERR_INVALID;
  if (weights && (!normals || !knn_idx || knn_k != KNN)) return GS_ERR_INVALID;
  if (n == 0) return GS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // means = the points
  if (cudaMemcpy2DAsync(params, 4 * sizeof(float), points, 3 * sizeof(float), 3 * sizeof(float), (size_t)n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GS_ERR_CUDA;
  if (!weights) {
    k_plain_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(knn_dist, knn_k, n, logit_default, (float4*)params,
                                                             n_gauss);
  } else {
    if (set_smem(k_mlp_init, Smem::FWD_END + BATCH * KOUT * 4) != GS_OK) return GS_ERR_CUDA;
    k_mlp_init<<<grid_for(n, 4), THREADS, Smem::FWD_END + BATCH * KOUT * 4, s>>>(
        points, normals, knn_idx, knn_dist, n, weights, logit_default, (float4*)params, n_gauss);
  }
  return gs_check_launch();
}
