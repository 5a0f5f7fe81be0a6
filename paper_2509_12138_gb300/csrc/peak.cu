// Issue-rate microbenchmark: the denominator of the blend kernels' roofline.
//
// Every thread runs GS_PEAK_CHAINS independent dependency chains for `iters`
// rounds, so each SM sub-partition always has an instruction ready:
//   mode 0 (FP32): x = fma(x, a, b) -- one FP32 lane-operation per step;
//   mode 1 (MUFU): x = ex2(x) - 1.5 -- one ex2.approx on the multi-function
//                  unit plus one FP32 add per step (chains start at -j/8,
//                  below the repelling fixed point near 1.66, and converge
//                  to the attracting one, x = -1; nothing overflows).
// The grid fills every SM (8 blocks of 256 threads per SM), and each thread
// writes the sum of its chains so that no step is dead code.
#include "common.cuh"

namespace {

constexpr int PEAK_T = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int MODE>
__global__ void __launch_bounds__(PEAK_T) k_peak(float* out, int iters, float a, float b) {
  const int tid = blockIdx.x * PEAK_T + threadIdx.x;
  float x[GS_PEAK_CHAINS];
#pragma unroll
  for (int j = 0; j < GS_PEAK_CHAINS; ++j) x[j] = -0.125f * (float)j;
#pragma unroll 16
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int j = 0; j < GS_PEAK_CHAINS; ++j) {
      if (MODE == 0)
        x[j] = fmaf(x[j], a, b);
      else
        x[j] = ex2_approx(x[j]) - b;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < GS_PEAK_CHAINS; ++j) s += x[j];
  out[tid] = s;
}

}  // namespace

GS_API int gs_peak_threads(int n_sms) {
  if (n_sms <= 0) return -1;
  return n_sms * PEAK_BLOCKS_PER_SM * PEAK_T;
}

GS_API int gs_peak_issue(int mode, int n_sms, int iters, float a, float b, float* out,
                         gs_stream_t stream) {
  GS_RANGE("gs_peak_issue");
  if (!out || n_sms <= 0 || iters <= 0 || (mode != 0 && mode != 1)) return GS_ERR_INVALID;
  const dim3 grid(n_sms * PEAK_BLOCKS_PER_SM);
  cudaStream_t s = (cudaStream_t)stream;
  if (mode == 0)
    k_peak<0><<<grid, PEAK_T, 0, s>>>(out, iters, a, b);
  else
    k_peak<1><<<grid, PEAK_T, 0, s>>>(out, iters, a, b);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
