// gs_train_batch: one optimiser step of every (partition, view) unit, a1-a6,
// enqueued on one stream with no host work that depends on the step.
//
// The paper trains each data partition independently (Sec. II, "Data
// Partitioning", "Parallel Training"); here all partitions and a batch of
// views per partition are the units of one launch chain.  The views of step t
// are chosen on the device from the step counter t = *d_step, so a CUDA graph
// that captures one call replays every later step unchanged: a gather kernel
// copies each unit's camera, ground-truth image and mask from the training
// set's pools into the step buffers, then the projection, sort, blend, loss,
// blend backward and fused projection backward + Adam run over all units, and
// the counter advances.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "common.cuh"

using namespace gs;

namespace {

// View of unit u = (partition k, slot j) at step t: train_views[(t vps + j + k) mod n_train]
// (consecutive steps walk the training views; partitions are staggered by one view).
__device__ __forceinline__ int unit_view(int64_t t, int u, int vps, const int32_t* __restrict__ train_views,
                                         int n_train) {
  int k = u / vps, j = u % vps;
  return train_views[(int)((t * vps + j + k) % n_train)];
}

// One block column per unit (blockIdx.y): copies the unit's camera, its
// partition's ground truth and mask of the chosen view.  vec: 16-byte copies
// (pointers 16-byte aligned, sizes multiples of 16 bytes), else element copies.
__global__ void __launch_bounds__(256) k_gather_views(const gs_camera* __restrict__ cam_pool,
                                                      const float* __restrict__ gt_pool,
                                                      const uint8_t* __restrict__ mask_pool,
                                                      const int32_t* __restrict__ train_views, int n_train,
                                                      int n_views, int vps, const int32_t* __restrict__ d_step,
                                                      int64_t plane, int vec, gs_camera* __restrict__ cams_step,
                                                      float* __restrict__ gt_step, uint8_t* __restrict__ mask_step) {
  int u = blockIdx.y;
  int v = unit_view((int64_t)*d_step, u, vps, train_views, n_train);
  int k = u / vps;
  if (blockIdx.x == 0 && threadIdx.x == 0) cams_step[u] = cam_pool[v];
  const int64_t src_img = (int64_t)k * n_views + v;
  const float* gs_src = gt_pool + src_img * 3 * plane;
  float* gs_dst = gt_step + (int64_t)u * 3 * plane;
  const uint8_t* ms_src = mask_pool + src_img * plane;
  uint8_t* ms_dst = mask_step + (int64_t)u * plane;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const int64_t ng = 3 * plane / 4, nm = plane / 16;
    for (int64_t e = first; e < ng; e += stride)
      reinterpret_cast<float4*>(gs_dst)[e] = __ldg(reinterpret_cast<const float4*>(gs_src) + e);
    for (int64_t e = first; e < nm; e += stride)
      reinterpret_cast<uint4*>(ms_dst)[e] = __ldg(reinterpret_cast<const uint4*>(ms_src) + e);
  } else {
    for (int64_t e = first; e < 3 * plane; e += stride) gs_dst[e] = gs_src[e];
    for (int64_t e = first; e < plane; e += stride) ms_dst[e] = ms_src[e];
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

GS_API int gs_gather_views(const gs_train_batch_desc* d, const int32_t* d_step, gs_stream_t stream) {
  GS_RANGE("gs_gather_views");
  if (!d || !d->units || !d_step || !d->cam_pool || !d->gt_pool || !d->mask_pool || !d->train_views ||
      !d->cams_step || !d->gt_step || !d->mask_step || d->views_per_step < 1 || d->n_train < 1 || d->n_views < 1 ||
      d->width <= 0 || d->height <= 0)
    return GS_ERR_INVALID;
  int U = d->units->n_units;
  if (U < 1 || U > GS_MAX_UNITS || U % d->views_per_step != 0) return GS_ERR_INVALID;
  int64_t plane = (int64_t)d->width * d->height;
  int vec = aligned16(d->gt_pool) && aligned16(d->gt_step) && aligned16(d->mask_pool) && aligned16(d->mask_step) &&
            (3 * plane) % 4 == 0 && plane % 16 == 0;
  int64_t per_unit = (3 * plane / 4 + 255) / 256;
  unsigned gx = (unsigned)(per_unit < 64 ? (per_unit > 0 ? per_unit : 1) : 64);
  k_gather_views<<<dim3(gx, (unsigned)U), 256, 0, (cudaStream_t)stream>>>(
      d->cam_pool, d->gt_pool, d->mask_pool, d->train_views, d->n_train, d->n_views, d->views_per_step, d_step, plane,
      vec, d->cams_step, d->gt_step, d->mask_step);
  return gs_check_launch();
}

GS_API int gs_train_batch(const gs_train_batch_desc* d, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_train_batch");
  if (!d || !d->params || !d->adam_m || !d->adam_v || !d->proj || !d->g2d || !d->d_step || !d->lr_init ||
      !d->sorted_vals || !d->ranges || !d->d_num_instances || !d->img || !d->final_T || !d->n_contrib ||
      !d->d_loss || !d->dL_dimg)
    return GS_ERR_INVALID;
  int U = d->units ? d->units->n_units : 0;
  int r;
  if ((r = gs_gather_views(d, d->d_step, stream)) != GS_OK) return r;
  if ((r = gs_preprocess(d->params, d->n_gauss, d->sh_degree, d->units, d->cams_step, d->width, d->height, nullptr,
                         d->proj, d_status, stream)) != GS_OK)
    return r;
  if ((r = gs_bin_sort(d->proj, d->units, d->width, d->height, d->max_instances, d->sort_ws, d->sort_ws_bytes,
                       d->sorted_vals, d->ranges, d->d_num_instances, d->sched, d_status, stream)) != GS_OK)
    return r;
  if ((r = gs_render_fwd(d->proj, d->sorted_vals, d->ranges, U, d->width, d->height, d->bg, d->img, d->final_T,
                         d->n_contrib, d->variant, d->sched, stream)) != GS_OK)
    return r;
  if ((r = gs_loss(d->img, d->gt_step, d->mask_step, U, d->width, d->height, d->lambda_ssim, d->loss_ws,
                   d->loss_ws_bytes, d->d_loss, d->dL_dimg, stream)) != GS_OK)
    return r;
  const bool pen = d->lambda_bg > 0.f;
  if (pen && (r = gs_bg_penalty(d->final_T, d->mask_step, U, d->width, d->height, d->lambda_bg, d->bg_ws,
                                d->bg_ws_bytes, d->d_loss, d->dL_dT, stream)) != GS_OK)
    return r;
  int64_t P = 0;
  for (int u = 0; u < U; ++u) P += d->units->gauss_count[u];
  if ((r = gs_blend_bwd(d->proj, d->sorted_vals, d->ranges, U, d->width, d->height, d->bg, d->img, d->final_T,
                        d->n_contrib, d->dL_dimg, pen ? d->dL_dT : nullptr, d->g2d, P, d->variant, d->sched,
                        stream)) != GS_OK)
    return r;
  if ((r = gs_project_bwd_adam(d->params, d->n_gauss, d->sh_degree, d->units, d->cams_step, d->proj, d->g2d,
                               d->adam_m, d->adam_v, d->lr_init, d->lr_final, d->lr_steps, d->beta1, d->beta2, d->eps,
                               d->d_step, d->grads, d->sparse_adam, d_status, stream)) != GS_OK)
    return r;
  return gs_step_advance(d->d_step, stream);
}
