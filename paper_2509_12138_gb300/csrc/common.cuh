// Device helpers shared by the libgs kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"
#include <nvtx3/nvToolsExt.h>

#define GS_API extern "C" __attribute__((visibility("default")))

namespace gs {

constexpr int TILE = GS_TILE;
constexpr int TILE_PIX = TILE * TILE;
constexpr float DILATION = 0.3f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float ALPHA_MIN = 1.0f / 255.0f;
constexpr float T_MIN = 1e-4f;
constexpr float JCLAMP = 1.3f;
constexpr float LAMBDA_FLOOR = 0.1f;

// Unit table passed by value: proj_base has n_units + 1 entries.
struct UnitTable {
  int32_t n;
  int64_t proj_base[GS_MAX_UNITS + 1];
  int64_t gauss_begin[GS_MAX_UNITS];
};

struct OwnedTable {
  int32_t n;  // 0 = no filter
  int64_t part_off[GS_MAX_PARTS + 1];
  float box[GS_MAX_PARTS][6];
  int32_t closed_hi[GS_MAX_PARTS];
};

// unit containing projected index p (proj_base sorted ascending)
__device__ __forceinline__ int unit_of(const UnitTable& U, int64_t p) {
  int lo = 0, hi = U.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (U.proj_base[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int part_of(const OwnedTable& O, int64_t i) {
  int lo = 0, hi = O.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (O.part_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int floordiv16(int a) { return a >> 4; }  // arithmetic shift = floor
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ---- float pairs (unevaluated sums hi + lo): error-free transformations
// Knuth's TwoSum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker's TwoProduct with a fused multiply-add: p + e = a b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// floor of the pair u = hi + lo (|lo| <= half an ulp of hi): one below
// floor(hi) when hi is an integer and lo is negative.
__device__ __forceinline__ int floor_pair(float hi, float lo) {
  float f = floorf(hi);
  return (int)f - ((f == hi && lo < 0.f) ? 1 : 0);
}

// Tile rectangle [x0, x1) x [y0, y1) of a splat at m = (u, v) with radius r,
// the pixel position given as float pairs (m.x + m.z, m.y + m.w).
// floor((u - r)/16) = floor((floor(u) - r)/16) for integer r, so the integer
// form is exact and matches any exact evaluation of the formula.
__device__ __forceinline__ void tile_rect(float4 m, int r, int TX, int TY, int& x0, int& y0, int& x1, int& y1) {
  int fu = floor_pair(m.x, m.z), fv = floor_pair(m.y, m.w);
  x0 = clampi(floordiv16(fu - r), 0, TX);
  y0 = clampi(floordiv16(fv - r), 0, TY);
  x1 = clampi(floordiv16(fu + r + TILE - 1), 0, TX);
  y1 = clampi(floordiv16(fv + r + TILE - 1), 0, TY);
}

// Offset of a record's pixel position from the origin o (an integer pixel
// coordinate) along one axis: (hi - o) + lo.  The blend kernels evaluate every
// (pixel, record) pair as this offset minus the pixel's own offset from the
// same origin (the tile's corner), so the power is computed from a small,
// accurate difference rather than from coordinates of ~10^3 pixels, and all
// kernels (forward, backward, any pixel-block shape) get bit-identical values.
__device__ __forceinline__ float rel_pos(float hi, float lo, float o) {
  return __fadd_rn(__fsub_rn(hi, o), lo);
}

// power = -(A dx^2 + C dy^2)/2 - B dx dy, written with explicit fmas so that
// the forward and backward kernels evaluate bit-identical values.
__device__ __forceinline__ float splat_power(float A, float B, float C, float dx, float dy) {
  float q = __fmul_rn(A, __fmul_rn(dx, dx));
  q = __fmaf_rn(C, __fmul_rn(dy, dy), q);
  float r = __fmul_rn(B, __fmul_rn(dx, dy));
  return __fmaf_rn(-0.5f, q, -r);
}

// Power below which alpha = o e^power < 1/255 for certain (with margin):
// -(ln(255 o) + 1e-3) * 1.001 - 1e-3.  Lets the blend skip the exponential.
__device__ __forceinline__ float power_floor(float o) {
  float tau = logf(255.f * o) + 1e-3f;
  return -tau * 1.001f - 1e-3f;
}

// Bounding box (xmin, xmax, ymin, ymax) of {d : o exp(-d^T Q d / 2) >= 1/255},
// i.e. d^T Q d <= 2 ln(255 o), half-widths sqrt(2 ln(255 o) Sigma_xx) with
// Sigma = Q^-1; inflated so float rounding can never cull a passing pixel.
// An empty box (xmin > xmax) when o < 1/255.  Also returns power_floor(o).
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

// 16-bit mask of the 4x4-pixel blocks (bit 4 by + bx) of tile (tx, ty) whose
// pixel centres the box reaches.  Block bx covers pixel centres
// [16 tx + 4 bx, 16 tx + 4 bx + 3]; it is reached iff b.x <= its right end and
// b.y >= its left end, which holds for a contiguous run of bx (and of by).
__device__ __forceinline__ uint32_t axis_bits(float lo, float hi, int origin) {
  uint32_t m = 0;
  #pragma unroll
  for (int k = 0; k < 4; ++k) {
    float a = (float)(origin + 4 * k);
    if (!(hi < a || lo > a + 3.f)) m |= 1u << k;
  }
  return m;
}
__device__ __forceinline__ uint32_t block_mask(float4 b, int tx, int ty) {
  if (!(b.x <= b.y)) return 0u;
  uint32_t cx = axis_bits(b.x, b.y, tx * TILE), ry = axis_bits(b.z, b.w, ty * TILE);
  // row by of the mask gets the column bits when ry has bit by
  uint32_t spread = (ry & 1u) | ((ry & 2u) << 3) | ((ry & 4u) << 6) | ((ry & 8u) << 9);
  return cx * spread;
}

__device__ __forceinline__ void set_status(int* st, int bits) {
  if (st) atomicOr(st, bits);
}

__host__ __device__ __forceinline__ int param_planes(int deg) {
  return (deg < 0 || deg > 3) ? -1 : 3 + (3 * (deg + 1) * (deg + 1) + 3) / 4;
}

}  // namespace gs

// NVTX range around a host entry point (header-only NVTX3: a no-op unless a
// profiler is attached), so that every gs_* call shows on a timeline.
struct GsRange {
  explicit GsRange(const char* name) { nvtxRangePushA(name); }
  ~GsRange() { nvtxRangePop(); }
  GsRange(const GsRange&) = delete;
  GsRange& operator=(const GsRange&) = delete;
};
#define GS_RANGE(name) GsRange gs_range_guard_(name)

// host-side helpers
int gs_fill_units(const gs_units* u, gs::UnitTable& t, int64_t* total);
int gs_fill_owned(const gs_owned* o, gs::OwnedTable& t);
int gs_check_launch();
size_t gs_scan_ws_bytes(int64_t n);
int gs_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws, uint32_t* d_total, cudaStream_t s);
