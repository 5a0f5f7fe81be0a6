// a9 (first half): exact k nearest neighbours of the isosurface points on a
// uniform grid.  Their distances give the plain initial scale (mean 3-NN
// distance) and, with k = 16, the geometry features of the learned initialiser.
//
// Build: count points per cell, exclusive scan, scatter the points (as float4
// with the index in .w) into cell order.  Query: one thread per point keeps
// the k best (squared distance, index) pairs in registers and visits cubic
// shells of cells of growing radius R until the k-th best distance is no
// larger than the distance from the point to the outside of the searched cube.
// Ties in distance are broken by the smaller index, so the result is unique.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

__host__ __device__ inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Grid {
  float lo[3];
  float h, inv_h;
  int dim[3];
};

struct KnnWs {
  size_t count, start, cursor, scan, sorted, total_cnt, total;
};
KnnWs knn_ws(int64_t n, int64_t cells) {
  KnnWs L;
  size_t o = 0;
  L.count = o; o += a256(sizeof(uint32_t) * (size_t)cells);
  L.start = o; o += a256(sizeof(uint32_t) * (size_t)(cells + 1));
  L.cursor = o; o += a256(sizeof(uint32_t) * (size_t)cells);
  L.scan = o; o += a256(gs_scan_ws_bytes(cells));
  L.sorted = o; o += a256(sizeof(float4) * (size_t)(n > 0 ? n : 1));
  L.total_cnt = o; o += a256(sizeof(uint32_t));
  L.total = o;
  return L;
}

__device__ __forceinline__ int cell_coord(float x, float lo, float inv_h, int dim) {
  int c = (int)floorf((x - lo) * inv_h);
  return min(max(c, 0), dim - 1);
}

__global__ void k_cell_count(const float* __restrict__ pts, int64_t n, Grid g, uint32_t* __restrict__ count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx = cell_coord(pts[3 * i], g.lo[0], g.inv_h, g.dim[0]);
  int cy = cell_coord(pts[3 * i + 1], g.lo[1], g.inv_h, g.dim[1]);
  int cz = cell_coord(pts[3 * i + 2], g.lo[2], g.inv_h, g.dim[2]);
  atomicAdd(&count[((int64_t)cz * g.dim[1] + cy) * g.dim[0] + cx], 1u);
}

__global__ void k_cell_scatter(const float* __restrict__ pts, int64_t n, Grid g, const uint32_t* __restrict__ start,
                               uint32_t* __restrict__ cursor, float4* __restrict__ sorted) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
  int cx = cell_coord(x, g.lo[0], g.inv_h, g.dim[0]);
  int cy = cell_coord(y, g.lo[1], g.inv_h, g.dim[1]);
  int cz = cell_coord(z, g.lo[2], g.inv_h, g.dim[2]);
  int64_t c = ((int64_t)cz * g.dim[1] + cy) * g.dim[0] + cx;
  uint32_t pos = start[c] + atomicAdd(&cursor[c], 1u);
  sorted[pos] = make_float4(x, y, z, __int_as_float((int)i));
}

template <int K>
__device__ __forceinline__ void offer(float d, int j, float* bd, int* bi) {
  if (d > bd[K - 1] || (d == bd[K - 1] && j > bi[K - 1])) return;
  float cd = d;
  int ci = j;
  #pragma unroll
  for (int q = 0; q < K; ++q) {
    bool less = cd < bd[q] || (cd == bd[q] && ci < bi[q]);
    if (less) {
      float td = bd[q]; bd[q] = cd; cd = td;
      int ti = bi[q]; bi[q] = ci; ci = ti;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(128) k_knn_query(const float* __restrict__ pts, int64_t n, Grid g,
                                                   const uint32_t* __restrict__ start,
                                                   const float4* __restrict__ sorted, int* __restrict__ out_idx,
                                                   float* __restrict__ out_dist) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
  int c[3] = {cell_coord(px, g.lo[0], g.inv_h, g.dim[0]), cell_coord(py, g.lo[1], g.inv_h, g.dim[1]),
              cell_coord(pz, g.lo[2], g.inv_h, g.dim[2])};
  float bd[K];
  int bi[K];
  #pragma unroll
  for (int q = 0; q < K; ++q) { bd[q] = INFINITY; bi[q] = 0x7fffffff; }
  int maxdim = max(g.dim[0], max(g.dim[1], g.dim[2]));
  float p[3] = {px, py, pz};
  for (int R = 0; R <= maxdim; ++R) {
    for (int dz = -R; dz <= R; ++dz) {
      int z = c[2] + dz;
      if (z < 0 || z >= g.dim[2]) continue;
      for (int dy = -R; dy <= R; ++dy) {
        int y = c[1] + dy;
        if (y < 0 || y >= g.dim[1]) continue;
        bool face = (dz == -R || dz == R || dy == -R || dy == R);
        for (int dx = -R; dx <= R; dx += (face ? 1 : 2 * R)) {
          int x = c[0] + dx;
          if (x >= 0 && x < g.dim[0]) {
            int64_t cell = ((int64_t)z * g.dim[1] + y) * g.dim[0] + x;
            uint32_t s = start[cell], e = start[cell + 1];
            for (uint32_t q = s; q < e; ++q) {
              float4 o = sorted[q];
              int j = __float_as_int(o.w);
              if (j == (int)i) continue;
              float ex = o.x - px, ey = o.y - py, ez = o.z - pz;
              offer<K>(ex * ex + ey * ey + ez * ez, j, bd, bi);
            }
          }
          if (R == 0) break;
        }
      }
    }
    // distance from p to the outside of the searched cube of cells
    float guard = INFINITY;
    bool whole = true;
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
      int lo = c[a] - R, hi = c[a] + R;
      if (lo > 0) guard = fminf(guard, p[a] - (g.lo[a] + lo * g.h));
      if (hi < g.dim[a] - 1) guard = fminf(guard, (g.lo[a] + (hi + 1) * g.h) - p[a]);
      whole = whole && lo <= 0 && hi >= g.dim[a] - 1;
    }
    if (whole) break;
    // the k-th best must be strictly inside: a point outside the cube is at least `guard` away
    if (bd[K - 1] < guard * guard * 0.999f) break;
  }
  #pragma unroll
  for (int q = 0; q < K; ++q) {
    bool ok = bd[q] < INFINITY;
    out_idx[i * K + q] = ok ? bi[q] : -1;
    out_dist[i * K + q] = ok ? sqrtf(bd[q]) : INFINITY;
  }
}

}  // namespace

GS_API size_t gs_knn_workspace_size(int64_t n, const int32_t* grid_dims) {
  if (n < 0 || !grid_dims || grid_dims[0] < 1 || grid_dims[1] < 1 || grid_dims[2] < 1) return 0;
  int64_t cells = (int64_t)grid_dims[0] * grid_dims[1] * grid_dims[2];
  return knn_ws(n, cells).total;
}

GS_API int gs_knn(const float* points, int64_t n, int k, const float* grid_lo, float cell_size,
                  const int32_t* grid_dims, void* workspace, size_t workspace_bytes, int32_t* idx, float* dist,
                  gs_stream_t stream) {
  GS_RANGE("gs_knn");
  if (!points || !idx || !dist || !grid_lo || !grid_dims || !workspace || n < 0 || !(cell_size > 0.f) ||
      !(k == 3 || k == 8 || k == 16))
    return GS_ERR_INVALID;
  Grid g;
  for (int a = 0; a < 3; ++a) {
    if (grid_dims[a] < 1) return GS_ERR_INVALID;
    g.lo[a] = grid_lo[a];
    g.dim[a] = grid_dims[a];
  }
  g.h = cell_size;
  g.inv_h = 1.0f / cell_size;
  int64_t cells = (int64_t)g.dim[0] * g.dim[1] * g.dim[2];
  if (cells >= (int64_t)UINT32_MAX) return GS_ERR_INVALID;
  KnnWs L = knn_ws(n, cells);
  if (workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) return GS_ERR_INVALID;
  if (n == 0) return GS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  uint32_t* count = (uint32_t*)(ws + L.count);
  uint32_t* start = (uint32_t*)(ws + L.start);
  uint32_t* cursor = (uint32_t*)(ws + L.cursor);
  float4* sorted = (float4*)(ws + L.sorted);
  if (cudaMemsetAsync(count, 0, sizeof(uint32_t) * cells, s) != cudaSuccess ||
      cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * cells, s) != cudaSuccess)
    return GS_ERR_CUDA;
  unsigned nb = (unsigned)((n + 255) / 256);
  k_cell_count<<<nb, 256, 0, s>>>(points, n, g, count);
  // start[c] = exclusive prefix; start[cells] = n
  int r = gs_scan_u32(count, start, cells, ws + L.scan, start + cells, s);
  if (r != GS_OK) return r;
  k_cell_scatter<<<nb, 256, 0, s>>>(points, n, g, start, cursor, sorted);
  unsigned qb = (unsigned)((n + 127) / 128);
#define GS_KQ(K) k_knn_query<K><<<qb, 128, 0, s>>>(points, n, g, start, sorted, idx, dist)
  switch (k) {
    case 3: GS_KQ(3); break;
    case 8: GS_KQ(8); break;
    default: GS_KQ(16); break;
  }
#undef GS_KQ
  return gs_check_launch();
}
