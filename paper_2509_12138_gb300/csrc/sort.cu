// a2: the per-tile lists in (depth, record index) order and their ranges.
// gs_bin_sort (depth-first design): the visible records sorted by depth once,
// their tile instances emitted in that order as 32-bit (mask | unit | tile)
// keys and sorted stably on the unit | tile bits.  gs_bin_sort_global: one
// stable LSD radix sort of 64-bit (unit | tile | depth) instance keys.
//
// Radix passes (one pass per 8- or 9-bit digit, three kernels per pass, all
// sized from the capacity so the chain is CUDA-graph capturable):
//   hist    : each 4096-key block builds a 256-bin digit histogram (per-warp
//             shared-memory bins) and adds it to the pass totals;
//   scan    : one CTA per digit scans that digit's per-block counts in block
//             order and adds the digit's global base; a pass whose keys all
//             share one digit is detected here and skipped (no data moves);
//   scatter : each block ranks its keys stably (warp match + per-warp digit
//             counts, in key order) and writes them to the other buffer.
// Which buffer holds the current keys is tracked on the device (cur[pass]),
// so skipped passes need no host decision.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"

using namespace gs;

// words of the bucketed sort's long-list scratch (sort_seg.cu), held in the value buffers
void gs_seg_ws_words(int64_t cap, size_t* words_s, size_t* words_l);

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_BLOCK = SCAN_T * SCAN_ITEMS;  // 2048 records per scan block
constexpr int RS_T = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_T * RS_ITEMS;  // 4096 keys per sort block
constexpr int RS_BINS_MAX = 512;  // digits of up to 9 bits
constexpr int MAX_PASSES = 8;
constexpr int SCATTER_DYN_SMEM = RS_TILE * (int)(sizeof(uint64_t) + sizeof(uint32_t));  // 48 KB

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
  size_t offsets, bsums, keys0, keys1, vals0, vals1, hist, totals, cur, misc, order, jscan, total;
};

// per-(unit, tile) scan scratch is sized for the largest tile grid (4K, 256 units)
constexpr int64_t MAX_SCHED_TILES = (int64_t)GS_MAX_UNITS * 240 * 135;

WsLayout ws_layout(int64_t P, int64_t C) {
  WsLayout L;
  size_t o = 0;
  int64_t nsb = (P + SCAN_BLOCK - 1) / SCAN_BLOCK;
  // the depth-first design sorts up to P records before it bins up to C instances
  const int64_t K = C > P ? C : P;
  int64_t nrb = (K + RS_TILE - 1) / RS_TILE;
  L.offsets = o; o += align256(sizeof(uint32_t) * (size_t)(P > 0 ? P : 1));
  L.bsums = o; o += align256(sizeof(uint32_t) * (size_t)(nsb + 1));
  L.keys0 = o; o += align256(sizeof(uint64_t) * (size_t)(K > 0 ? K : 1));
  L.keys1 = o; o += align256(sizeof(uint64_t) * (size_t)(K > 0 ? K : 1));
  size_t ws_s = 0, ws_l = 0;
  gs_seg_ws_words(C, &ws_s, &ws_l);
  const size_t cw = (size_t)(C > 0 ? C : 1);
  L.vals0 = o; o += align256(sizeof(uint32_t) * (cw > ws_s ? cw : ws_s));
  L.vals1 = o; o += align256(sizeof(uint32_t) * (cw > ws_l ? cw : ws_l));
  L.hist = o; o += align256(sizeof(uint32_t) * RS_BINS_MAX * (size_t)(nrb > 0 ? nrb : 1));
  L.totals = o; o += align256(sizeof(uint32_t) * RS_BINS_MAX * MAX_PASSES);
  L.cur = o; o += align256(sizeof(int32_t) * 2 * (MAX_PASSES + 1));
  L.misc = o; o += align256(sizeof(uint32_t) * 4);
  L.order = o; o += align256(sizeof(uint32_t) * 66);
  L.jscan = o; o += align256(sizeof(uint32_t) * (size_t)((MAX_SCHED_TILES + SCAN_BLOCK - 1) / SCAN_BLOCK + 1));
  L.total = o;
  return L;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  int lane = threadIdx.x & 31;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// exclusive scan of one value per thread over a 256-thread block; returns
// the block total through *total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
    uint32_t xi = warp_incl_scan(x);
    if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = xi - x;
    if (lane == (int)(blockDim.x >> 5) - 1) s_warp[32] = xi;
  }
  __syncthreads();
  uint32_t r = inc - v + s_warp[w];
  if (total) *total = s_warp[32];
  __syncthreads();
  return r;
}

// ---- exclusive scan of tiles_touched -> instance offsets
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t* __restrict__ in, int64_t P,
                                                        uint32_t* __restrict__ bsums) {
  __shared__ uint32_t s_warp[33];
  int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  uint32_t s = 0;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SCAN_T + threadIdx.x;
    if (k < P) s += in[k];
  }
  uint32_t tot;
  block_excl_scan(s, s_warp, &tot);
  if (threadIdx.x == 0) bsums[blockIdx.x] = tot;
}

// bmins (may be NULL): per-block minima reduced on the way into *dmin
__global__ void __launch_bounds__(1024) k_scan_bsums(uint32_t* bsums, int64_t nb, const uint32_t* bmins,
                                                     uint32_t* dmin) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_carry;
  __shared__ uint32_t s_min;
  if (threadIdx.x == 0) { s_carry = 0; s_min = 0xffffffffu; }
  __syncthreads();
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t k = base + threadIdx.x;
    if (bmins) {
      uint32_t mn = __reduce_min_sync(0xffffffffu, k < nb ? bmins[k] : 0xffffffffu);
      if ((threadIdx.x & 31) == 0) atomicMin(&s_min, mn);
    }
    uint32_t v = k < nb ? bsums[k] : 0u;
    uint32_t tot;
    uint32_t ex = block_excl_scan(v, s_warp, &tot);
    uint32_t carry = s_carry;
    if (k < nb) bsums[k] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bsums[nb] = s_carry;
    if (bmins) *dmin = s_min;
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_down(const uint32_t* __restrict__ in, int64_t P,
                                                      const uint32_t* __restrict__ bsums, int64_t nb,
                                                      uint32_t* __restrict__ out, int64_t cap,
                                                      uint32_t* d_count, int* status) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_items[SCAN_BLOCK];
  int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  // blocked arrangement: thread t owns items [t*ITEMS, (t+1)*ITEMS) of the block
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SCAN_T + threadIdx.x;
    s_items[j * SCAN_T + threadIdx.x] = k < P ? in[k] : 0u;
  }
  __syncthreads();
  uint32_t loc[SCAN_ITEMS];
  uint32_t s = 0;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    loc[j] = s;
    s += s_items[threadIdx.x * SCAN_ITEMS + j];
  }
  uint32_t ex = block_excl_scan(s, s_warp, nullptr) + bsums[blockIdx.x];
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) s_items[threadIdx.x * SCAN_ITEMS + j] = loc[j] + ex;
  __syncthreads();
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SCAN_T + threadIdx.x;
    if (k < P) out[k] = s_items[j * SCAN_T + threadIdx.x];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t total = bsums[nb];
    if ((int64_t)total > cap) {
      set_status(status, GS_ERR_CAPACITY);
      total = (uint32_t)cap;
    }
    *d_count = total;
  }
}

// ---- duplication: one key per (record, covered tile)
// With key_masks set, the 16-bit block mask of each (record, tile) instance
// rides in key bits 48..63, above every bit the radix passes sort on, so the
// sort carries it to the instance's sorted position at no extra traffic.
__global__ void __launch_bounds__(256) k_duplicate(UnitTable U, const float4* __restrict__ xy,
                                                   const float4* __restrict__ conic_op,
                                                   const float* __restrict__ depth,
                                                   const int* __restrict__ radius,
                                                   const uint32_t* __restrict__ tiles,
                                                   const uint32_t* __restrict__ offsets, int W, int H,
                                                   int tile_bits, int64_t cap, int key_masks,
                                                   uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t P = U.proj_base[U.n];
  if (p >= P) return;
  uint32_t nt = tiles[p];
  if (nt == 0) return;
  int u = unit_of(U, p);
  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  float4 m = xy[p];
  int x0, y0, x1, y1;
  tile_rect(m, radius[p], TX, TY, x0, y0, x1, y1);
  uint64_t dbits = (uint64_t)__float_as_uint(depth[p]);
  uint64_t hi = (uint64_t)u << (tile_bits + 32);
  float4 box = make_float4(1.f, -1.f, 1.f, -1.f);
  if (key_masks) {
    float pm;
    box = alpha_box(make_float2(m.x, m.y), conic_op[p], pm);
  }
  int64_t o = offsets[p];
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx) {
      if (o < cap) {
        uint64_t mk = key_masks ? (uint64_t)block_mask(box, tx, ty) << 48 : 0ull;
        keys[o] = mk | hi | ((uint64_t)(ty * TX + tx) << 32) | dbits;
        vals[o] = (uint32_t)p;
      }
      ++o;
    }
}

// ---- radix pass kernels
template <int BITS, typename KT>
__global__ void __launch_bounds__(RS_T) k_radix_hist(const KT* __restrict__ k0, const KT* __restrict__ k1,
                                                     const int32_t* __restrict__ cur, int pass,
                                                     const uint32_t* __restrict__ d_count, int shift,
                                                     uint32_t* __restrict__ hist, int64_t stride,
                                                     uint32_t* __restrict__ totals) {
  constexpr int BINS = 1 << BITS;
  __shared__ uint32_t s_h[RS_T / 32][BINS];
  int64_t I = *d_count;
  const KT* keys = cur[pass] ? k1 : k0;
  int w = threadIdx.x >> 5;
  // the grid holds as many blocks as stay resident; they take the 4096-key tiles in turn
  for (int64_t t = blockIdx.x; t * RS_TILE < I; t += gridDim.x) {
    int64_t base = t * RS_TILE;
    for (int k = threadIdx.x; k < (RS_T / 32) * BINS; k += RS_T) (&s_h[0][0])[k] = 0u;
    // every load of the tile's keys in flight at once, then the counting
    uint32_t dg[RS_ITEMS];
    #pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      int64_t k = base + (int64_t)j * RS_T + threadIdx.x;
      dg[j] = k < I ? ((uint32_t)(keys[k] >> shift) & (BINS - 1u)) : 0xffffffffu;
    }
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j)
      if (dg[j] != 0xffffffffu) atomicAdd(&s_h[w][dg[j]], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < BINS; d += RS_T) {
      uint32_t c = 0;
      #pragma unroll
      for (int q = 0; q < RS_T / 32; ++q) c += s_h[q][d];
      hist[(int64_t)d * stride + t] = c;
      if (c) atomicAdd(&totals[pass * RS_BINS_MAX + d], c);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t* __restrict__ hist, int64_t stride,
                                                     const uint32_t* __restrict__ totals, int pass, int bins,
                                                     const uint32_t* __restrict__ d_count,
                                                     int32_t* __restrict__ cur) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_carry;
  __shared__ int s_skip;
  __shared__ uint32_t s_base;
  int64_t I = *d_count;
  int d = blockIdx.x;
  const uint32_t* tot = totals + pass * RS_BINS_MAX;
  if (threadIdx.x == 0) { s_skip = 0; s_base = 0; s_carry = 0; }
  __syncthreads();
  if ((int)threadIdx.x < bins) {
    uint32_t t = tot[threadIdx.x];
    if ((int64_t)t == I) s_skip = 1;  // every key has this digit (or I == 0)
    if ((int)threadIdx.x < d) atomicAdd(&s_base, t);
  }
  if (I == 0 && threadIdx.x == 0) s_skip = 1;
  __syncthreads();
  if (d == 0 && threadIdx.x == 0) cur[pass + 1] = s_skip ? cur[pass] : 1 - cur[pass];
  if (s_skip) return;
  int64_t nb = (I + RS_TILE - 1) / RS_TILE;
  uint32_t* row = hist + (int64_t)d * stride;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    int64_t b = b0 + threadIdx.x;
    uint32_t v = b < nb ? row[b] : 0u;
    uint32_t t;
    uint32_t ex = block_excl_scan(v, s_warp, &t);
    uint32_t carry = s_carry;
    if (b < nb) row[b] = ex + carry + s_base;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + t;
    __syncthreads();
  }
}

// Stable scatter of one 4096-key block.  Warp w owns the block's keys
// [512 w, 512 (w + 1)) (16 rounds of 32 consecutive keys), so ranking each
// warp's keys in round order with warp-private digit counters (warp match,
// no block barrier) ranks the block's keys in key order once the per-warp
// counts are scanned across warps.  Keys are then placed in a block-local
// digit-sorted buffer in shared memory and written out so that each digit's
// run goes to consecutive global positions (coalesced stores).
template <int BITS, typename KT, bool FINAL = false>
__global__ void __launch_bounds__(RS_T, sizeof(KT) == 4 ? 3 : 2) k_radix_scatter(KT* __restrict__ k0, KT* __restrict__ k1,
                                                        uint32_t* __restrict__ v0, uint32_t* __restrict__ v1,
                                                        const int32_t* __restrict__ cur, int pass,
                                                        const uint32_t* __restrict__ d_count, int shift,
                                                        const uint32_t* __restrict__ hist, int64_t stride,
                                                        uint32_t* __restrict__ vfinal, uint16_t* __restrict__ mfinal) {
  // FINAL: the values go to vfinal instead of the other value buffer (the last pass of a sort writes the
  // caller's output directly), and bits 16-31 of each key (the block mask) to mfinal unless it is NULL
  constexpr int BINS = 1 << BITS;
  constexpr int NW = RS_T / 32;
  constexpr int DPT = BINS / RS_T;      // digits per thread in the per-digit steps
  constexpr int WKEYS = RS_TILE / NW;   // keys per warp
  __shared__ uint32_t s_off[BINS];      // global start of this block's run of each digit
  __shared__ uint32_t s_lstart[BINS];   // block-local start of each digit
  __shared__ uint32_t s_wc[NW][BINS];   // per-warp digit counts, then each warp's offset within the digit
  __shared__ uint32_t s_warp[33];
  extern __shared__ __align__(16) unsigned char s_dyn[];  // RS_TILE keys, then RS_TILE values
  KT* s_keys = reinterpret_cast<KT*>(s_dyn);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_dyn + sizeof(KT) * RS_TILE);
  int64_t I = *d_count;
  int c = cur[pass];
  if (cur[pass + 1] == c) return;  // skipped pass
  const KT* kin = c ? k1 : k0;
  const uint32_t* vin = c ? v1 : v0;
  KT* kout = c ? k0 : k1;
  uint32_t* vout = FINAL ? vfinal : (c ? v0 : v1);
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // the grid holds as many blocks as stay resident; they take the 4096-key tiles in turn
  for (int64_t t = blockIdx.x; t * RS_TILE < I; t += gridDim.x) {
    int64_t base = t * RS_TILE;
    #pragma unroll
    for (int e = 0; e < DPT; ++e) {
      int dd = tid + e * RS_T;
      s_off[dd] = hist[(int64_t)dd * stride + t];
      #pragma unroll
      for (int q = 0; q < NW; ++q) s_wc[q][dd] = 0u;
    }
    uint32_t lt = (1u << lane) - 1u;
    KT key[RS_ITEMS];
    uint32_t val[RS_ITEMS];
    uint32_t rnk[RS_ITEMS / 2];  // ranks within the digit among this warp's keys, two 16-bit ranks a word
    int64_t wk = base + (int64_t)w * WKEYS + lane;  // this lane's key of round 0
    int64_t rem64 = I - wk;
    int rem = rem64 > RS_TILE ? RS_TILE : (int)rem64;  // round j holds a key iff 32 j < rem
    const KT* kp = kin + wk;
    const uint32_t* vp = vin + wk;
    #pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      bool valid = j * 32 < rem;
      key[j] = valid ? kp[j * 32] : (KT)0;
      val[j] = valid ? vp[j * 32] : 0u;
    }
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      bool valid = j * 32 < rem;
      uint32_t d = valid ? ((uint32_t)(key[j] >> shift) & (BINS - 1u)) : (uint32_t)BINS;
      uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = valid ? s_wc[w][d] : 0u;
      uint32_t r = before + __popc(peers & lt);  // < WKEYS: fits 16 bits
      if (j & 1) rnk[j >> 1] |= r << 16; else rnk[j >> 1] = r;
      __syncwarp();
      if (valid && (peers & lt) == 0u) s_wc[w][d] = before + __popc(peers);  // lowest lane of the group
      __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive scan of the warp counts (warp order = key order); thread tid
    // owns digits tid * DPT .. tid * DPT + DPT - 1, then a block scan gives digit starts
    {
      uint32_t cnts[DPT];
      uint32_t cnt = 0;
      #pragma unroll
      for (int e = 0; e < DPT; ++e) {
        int dd = tid * DPT + e;
        uint32_t acc = 0;
        #pragma unroll
        for (int q = 0; q < NW; ++q) {
          uint32_t cq = s_wc[q][dd];
          s_wc[q][dd] = acc;
          acc += cq;
        }
        cnts[e] = acc;
        cnt += acc;
      }
      uint32_t inc = cnt;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t nb = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += nb;
      }
      if (lane == 31) s_warp[w] = inc;
      __syncthreads();
      if (w == 0) {
        uint32_t x = lane < NW ? s_warp[lane] : 0u, xi = x;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t nb = __shfl_up_sync(0xffffffffu, xi, o);
          if (lane >= o) xi += nb;
        }
        if (lane < NW) s_warp[lane] = xi - x;
      }
      __syncthreads();
      uint32_t st = inc - cnt + s_warp[w];
      #pragma unroll
      for (int e = 0; e < DPT; ++e) { s_lstart[tid * DPT + e] = st; st += cnts[e]; }
    }
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
      if (j * 32 >= rem) continue;
      uint32_t d = (uint32_t)(key[j] >> shift) & (BINS - 1u);
      uint32_t r = (j & 1) ? (rnk[j >> 1] >> 16) : (rnk[j >> 1] & 0xffffu);
      uint32_t pos = s_lstart[d] + s_wc[w][d] + r;
      s_keys[pos] = key[j];
      s_vals[pos] = val[j];
    }
    __syncthreads();
    int n_here = (int)min((int64_t)RS_TILE, I - base);
    for (int i = tid; i < n_here; i += RS_T) {
      KT kk = s_keys[i];
      uint32_t d = (uint32_t)(kk >> shift) & (BINS - 1u);
      uint32_t gp = s_off[d] + (uint32_t)i - s_lstart[d];
      kout[gp] = kk;
      vout[gp] = s_vals[i];
      if (FINAL && mfinal) mfinal[gp] = (uint16_t)((uint64_t)kk >> 16);
    }
    __syncthreads();  // the tile's shared-memory staging is read out before the next tile reuses it
  }
}

__global__ void __launch_bounds__(256) k_ranges(const uint64_t* __restrict__ k0, const uint64_t* __restrict__ k1,
                                                const uint32_t* __restrict__ v0, const uint32_t* __restrict__ v1,
                                                const int32_t* __restrict__ cur, int final_pass,
                                                const uint32_t* __restrict__ d_count, int tile_bits,
                                                int n_tiles, int TX, uint32_t* __restrict__ ranges,
                                                uint32_t* __restrict__ out_vals, const float4* __restrict__ xy,
                                                const float4* __restrict__ conic_op, uint16_t* __restrict__ masks,
                                                int key_masks) {
  int64_t I = *d_count;
  int c = cur[final_pass];
  const uint64_t* keys = c ? k1 : k0;
  const uint32_t* vals = c ? v1 : v0;
  // unit | tile bits (key bits 32..47 when the block masks ride in bits 48..63)
  uint32_t utm = key_masks ? 0xffffu : 0xffffffffu;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < I; k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t kk = keys[k];
    uint32_t ut = (uint32_t)(kk >> 32) & utm;
    uint32_t p = vals[k];
    out_vals[k] = p;
    uint32_t mask = (1u << tile_bits) - 1u;
    uint32_t tile = ut & mask;
    int64_t flat = (int64_t)(ut >> tile_bits) * n_tiles + tile;
    if (k == 0 || ((uint32_t)(keys[k - 1] >> 32) & utm) != ut) ranges[2 * flat] = (uint32_t)k;
    if (k == I - 1 || ((uint32_t)(keys[k + 1] >> 32) & utm) != ut) ranges[2 * flat + 1] = (uint32_t)(k + 1);
    if (masks && key_masks) {
      masks[k] = (uint16_t)(kk >> 48);
    } else if (masks) {
      // which 4x4 pixel blocks of its tile the record's alpha >= 1/255 box reaches
      float pm;
      float4 m = xy[p];
      float4 b = alpha_box(make_float2(m.x, m.y), conic_op[p], pm);
      masks[k] = (uint16_t)block_mask(b, (int)(tile % (uint32_t)TX), (int)(tile / (uint32_t)TX));
    }
  }
}

// ---- depth-first design: sort the visible records by depth once, then bin their instances by
// (unit, tile) with a stable sort on 32-bit keys (block mask << 16 | unit | tile).  Stability makes
// each list come out in (depth, record index) order, the order of the global key sort.

// visible records (tiles > 0) per 2048-record scan block, and the smallest depth key among them
// (bmins: float32 depth bits, which order as unsigned integers for positive depths; all ones for a block
// without visible records).  k_scan_bsums reduces the block minima: one global atomic per block on a
// single address took ~30 us at 10M records.
__global__ void __launch_bounds__(SCAN_T) k_vis_reduce(const uint32_t* __restrict__ tiles,
                                                       const float* __restrict__ depth, int64_t P,
                                                       uint32_t* __restrict__ bsums, uint32_t* __restrict__ bmins) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_min;
  if (threadIdx.x == 0) s_min = 0xffffffffu;
  int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  uint32_t s = 0, mn = 0xffffffffu;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SCAN_T + threadIdx.x;
    if (k < P) {
      // both loads issued before either is tested (a depth load behind the visibility test doubled the
      // kernel's time)
      uint32_t tk = tiles[k], dk = __float_as_uint(depth[k]);
      if (tk > 0u) {
        ++s;
        mn = min(mn, dk);
      }
    }
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  __syncthreads();  // s_min initialised
  if ((threadIdx.x & 31) == 0) atomicMin(&s_min, mn);
  uint32_t tot;
  block_excl_scan(s, s_warp, &tot);  // (its barriers also order the shared minimum)
  if (threadIdx.x == 0) {
    bsums[blockIdx.x] = tot;
    bmins[blockIdx.x] = s_min;
  }
}

// compaction in record order: (depth bits - *dmin, record index) of every visible record; *d_vis = their
// number.  Keys relative to the nearest visible depth keep the order and leave the top byte zero when the
// view's depths stay within a factor of ~4 (then the device skips the top radix pass).
// Round j of a block covers its records [256 j, 256 j + 256) (coalesced loads); a record's slot is the
// block's base, the visible records of earlier (round, warp) pairs and those of lower lanes.
__global__ void __launch_bounds__(SCAN_T) k_vis_compact(const uint32_t* __restrict__ tiles,
                                                        const float* __restrict__ depth, int64_t P,
                                                        const uint32_t* __restrict__ bsums, int64_t nb,
                                                        const uint32_t* __restrict__ dmin,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        uint32_t* __restrict__ d_vis) {
  constexpr int NW = SCAN_T / 32;
  static_assert(SCAN_ITEMS * NW == 64, "one warp scans the (round, warp) counts two per lane");
  __shared__ uint32_t s_cnt[SCAN_ITEMS * NW];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  uint32_t bal[SCAN_ITEMS];
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SCAN_T + threadIdx.x;
    bal[j] = __ballot_sync(0xffffffffu, k < P && tiles[k] > 0u);
    if (lane == 0) s_cnt[j * NW + w] = __popc(bal[j]);
  }
  __syncthreads();
  if (w == 0) {  // exclusive scan of the 64 (round, warp) counts, two per lane
    uint32_t a = s_cnt[2 * lane], b = s_cnt[2 * lane + 1];
    uint32_t inc = warp_incl_scan(a + b);
    s_cnt[2 * lane] = inc - a - b;
    s_cnt[2 * lane + 1] = inc - b;
  }
  __syncthreads();
  uint32_t c0 = bsums[blockIdx.x];
  const uint32_t d0 = *dmin;
  uint32_t lt = (1u << lane) - 1u;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j)
    if (bal[j] >> lane & 1u) {
      int64_t k = base + (int64_t)j * SCAN_T + threadIdx.x;
      uint32_t c = c0 + s_cnt[j * NW + w] + __popc(bal[j] & lt);
      keys[c] = __float_as_uint(depth[k]) - d0;
      vals[c] = (uint32_t)k;
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_vis = bsums[nb];
}

// instance count of every 2048 records in depth order (scan blocks), for the scan of the offsets
__global__ void __launch_bounds__(SCAN_T) k_dup_reduce(const uint32_t* __restrict__ vA,
                                                       const uint32_t* __restrict__ vB,
                                                       const int32_t* __restrict__ cur, int final_pass,
                                                       const uint32_t* __restrict__ d_vis,
                                                       const uint32_t* __restrict__ tiles,
                                                       uint32_t* __restrict__ bsums) {
  __shared__ uint32_t s_warp[33];
  const uint32_t* v = cur[final_pass] ? vB : vA;
  int64_t V = *d_vis;
  int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  uint32_t s = 0;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + (int64_t)j * SCAN_T + threadIdx.x;
    if (i < V) s += tiles[v[i]];
  }
  uint32_t tot;
  block_excl_scan(s, s_warp, &tot);
  if (threadIdx.x == 0) bsums[blockIdx.x] = tot;
}

// one 32-bit key per (record, covered tile), records taken in depth order.  Block b takes sorted records
// [2048 b, 2048 b + 2048), thread t the 8 consecutive ones from 2048 b + 8 t; their instances are numbered
// from the block's scanned base in record order.  The block stages its instances in shared memory in
// windows of EMIT_WIN and writes each window out with coalesced stores (a thread only visits the
// instances of its records that fall in the window, so a window costs O(its instances + 8) per thread).
// Block 0 also writes the instance count (clamped to the capacity, GS_ERR_CAPACITY beyond it).
constexpr int EMIT_WIN = 4096;
__global__ void __launch_bounds__(SCAN_T, 3) k_dup_emit(UnitTable U, const float4* __restrict__ xy,
                                                     const float4* __restrict__ conic_op,
                                                     const int* __restrict__ radius, const uint32_t* __restrict__ vA,
                                                     const uint32_t* __restrict__ vB, const int32_t* __restrict__ cur,
                                                     int final_pass, const uint32_t* __restrict__ d_vis,
                                                     const uint32_t* __restrict__ bsums, int64_t nb, int W, int H,
                                                     int tile_bits, int64_t cap, int key_masks,
                                                     uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                     uint32_t* __restrict__ d_count, int* __restrict__ status) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_p[SCAN_BLOCK];
  __shared__ uint32_t s_key[EMIT_WIN];
  __shared__ uint32_t s_val[EMIT_WIN];
  const uint32_t* v = cur[final_pass] ? vB : vA;
  int64_t V = *d_vis;
  int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + (int64_t)j * SCAN_T + threadIdx.x;
    s_p[j * SCAN_T + threadIdx.x] = i < V ? v[i] : 0xffffffffu;
  }
  __syncthreads();
  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  int rx0[SCAN_ITEMS], ry0[SCAN_ITEMS], rw[SCAN_ITEMS], rh[SCAN_ITEMS];
  float4 box[SCAN_ITEMS];
  uint32_t n = 0;
  #pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    uint32_t p = s_p[threadIdx.x * SCAN_ITEMS + j];
    rx0[j] = ry0[j] = rw[j] = rh[j] = 0;
    box[j] = make_float4(1.f, -1.f, 1.f, -1.f);
    if (p != 0xffffffffu) {
      float4 m = xy[p];
      int x0, y0, x1, y1;
      tile_rect(m, radius[p], TX, TY, x0, y0, x1, y1);
      rx0[j] = x0; ry0[j] = y0; rw[j] = x1 - x0; rh[j] = y1 - y0;
      n += (uint32_t)((x1 - x0) * (y1 - y0));
      if (key_masks) {
        float pm;
        box[j] = alpha_box(make_float2(m.x, m.y), conic_op[p], pm);
      }
    }
  }
  uint32_t tot;
  uint32_t lo = block_excl_scan(n, s_warp, &tot);  // this thread's first instance within the block
  int64_t ob = (int64_t)bsums[blockIdx.x];           // the block's first instance
  for (uint32_t win = 0; win < tot; win += EMIT_WIN) {
    uint32_t a = lo;
    #pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      uint32_t c = (uint32_t)(rw[j] * rh[j]);
      uint32_t k0 = a > win ? a : win;
      uint32_t k1 = a + c < win + EMIT_WIN ? a + c : win + EMIT_WIN;
      if (k0 < k1) {
        uint32_t p = s_p[threadIdx.x * SCAN_ITEMS + j];
        uint32_t hi = (uint32_t)unit_of(U, p) << tile_bits;
        uint32_t t = k0 - a;
        int ty = ry0[j] + (int)(t / (uint32_t)rw[j]), tx = rx0[j] + (int)(t % (uint32_t)rw[j]);
        for (uint32_t k = k0; k < k1; ++k) {
          uint32_t mk = key_masks ? block_mask(box[j], tx, ty) << 16 : 0u;
          s_key[k - win] = mk | hi | (uint32_t)(ty * TX + tx);
          s_val[k - win] = p;
          if (++tx == rx0[j] + rw[j]) { tx = rx0[j]; ++ty; }
        }
      }
      a += c;
    }
    __syncthreads();
    uint32_t wn = tot - win < (uint32_t)EMIT_WIN ? tot - win : (uint32_t)EMIT_WIN;
    for (uint32_t i = threadIdx.x; i < wn; i += SCAN_T) {
      int64_t g = ob + win + i;
      if (g < cap) {
        keys[g] = s_key[i];
        vals[g] = s_val[i];
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t total = bsums[nb];
    if ((int64_t)total > cap) {
      set_status(status, GS_ERR_CAPACITY);
      total = (uint32_t)cap;
    }
    *d_count = total;
  }
}

// list ranges from the sorted 32-bit instance keys, and the record ids and block masks when the last
// instance pass was skipped (otherwise that pass wrote them)
__global__ void __launch_bounds__(256) k_ranges32(const uint32_t* __restrict__ kA, const uint32_t* __restrict__ kB,
                                                  const uint32_t* __restrict__ vA, const uint32_t* __restrict__ vB,
                                                  const int32_t* __restrict__ cur, int final_pass,
                                                  const uint32_t* __restrict__ d_count, int tile_bits, int n_tiles,
                                                  uint32_t* __restrict__ ranges, uint32_t* __restrict__ out_vals,
                                                  uint16_t* __restrict__ masks) {
  int64_t I = *d_count;
  int c = cur[final_pass];
  const bool copy = final_pass < 1 || cur[final_pass - 1] == c;  // the last pass was skipped
  const uint32_t* keys = c ? kB : kA;
  const uint32_t* vals = c ? vB : vA;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < I; k += (int64_t)gridDim.x * blockDim.x) {
    uint32_t kk = keys[k];
    uint32_t ut = kk & 0xffffu;
    int64_t flat = (int64_t)(ut >> tile_bits) * n_tiles + (ut & ((1u << tile_bits) - 1u));
    if (k == 0 || (keys[k - 1] & 0xffffu) != ut) ranges[2 * flat] = (uint32_t)k;
    if (k == I - 1 || (keys[k + 1] & 0xffffu) != ut) ranges[2 * flat + 1] = (uint32_t)(k + 1);
    if (copy) {
      out_vals[k] = vals[k];
      if (masks) masks[k] = (uint16_t)(kk >> 16);
    }
  }
}

// number of chunks of each list, in tile order
__global__ void k_chunk_count(const uint2* __restrict__ ranges, const uint32_t* __restrict__ order, int NT, int K,
                              uint32_t* __restrict__ counts) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= NT) return;
  uint2 r = ranges[order[o]];
  counts[o] = (r.y - r.x + (uint32_t)K - 1u) / (uint32_t)K;
}

// (order position, chunk) of every chunk job
__global__ void k_chunk_jobs(const uint32_t* __restrict__ job_base, int NT, int64_t max_jobs,
                             uint32_t* __restrict__ jobs) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= NT) return;
  uint32_t b = job_base[o], e = job_base[o + 1];
  for (uint32_t j = b; j < e && (int64_t)j < max_jobs; ++j) {
    jobs[2 * (int64_t)j] = (uint32_t)o;
    jobs[2 * (int64_t)j + 1] = j - b;
  }
}

// As many blocks of `threads` as stay resident on the device, at most `units`: the grid of a kernel
// whose blocks take equal units of work in turn (a grid sized for the capacity would mostly hold
// blocks that find nothing to do).
template <typename K>
unsigned resident_blocks(K kernel, int threads, size_t dyn_smem, int64_t units) {
  int dev = 0, sms = 0, per = 0;
  if (units < 1) return 1u;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, dyn_smem) != cudaSuccess || sms < 1 || per < 1)
    return (unsigned)units;
  int64_t g = (int64_t)sms * per;
  return (unsigned)(g < units ? g : units);
}

int bits_for(int64_t n) {
  int b = 0;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}

}  // namespace

// Exclusive scan of n uint32 values (helper for other stages): out[i] = sum in[0..i);
// *d_total receives the sum.  ws must hold gs_scan_ws_bytes(n) bytes.
size_t gs_scan_ws_bytes(int64_t n) { return sizeof(uint32_t) * (size_t)((n + SCAN_BLOCK - 1) / SCAN_BLOCK + 1); }

int gs_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws, uint32_t* d_total, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  int64_t nsb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  uint32_t* bsums = (uint32_t*)ws;
  k_scan_reduce<<<(unsigned)nsb, SCAN_T, 0, s>>>(in, n, bsums);
  k_scan_bsums<<<1, 1024, 0, s>>>(bsums, nsb, nullptr, nullptr);
  k_scan_down<<<(unsigned)nsb, SCAN_T, 0, s>>>(in, n, bsums, nsb, out, INT64_MAX, d_total, nullptr);
  return gs_check_launch();
}

GS_API size_t gs_bin_sort_workspace_size(int64_t n_proj, int64_t max_instances) {
  if (n_proj < 0 || max_instances < 0) return 0;
  return ws_layout(n_proj, max_instances).total;
}

// The sort chain, shared by gs_bin_sort and the fixed-scratch variant.
int gs_tile_order_impl(const uint32_t* ranges, int n, uint32_t* ws, uint32_t* order, cudaStream_t s);

// Tile order (unless the sort already made it), then the chunk jobs in that order.
int gs_schedule_jobs(const uint32_t* ranges, int NT, char* order_ws, char* scan_ws, const gs_schedule* sched,
                     cudaStream_t s, bool order_done = false) {
  int r = order_done ? GS_OK : gs_tile_order_impl(ranges, NT, (uint32_t*)order_ws, sched->tile_order, s);
  if (r != GS_OK) return r;
  unsigned nb = (unsigned)((NT + 255) / 256);
  k_chunk_count<<<nb, 256, 0, s>>>((const uint2*)ranges, sched->tile_order, NT, sched->chunk, sched->job_base);
  r = gs_scan_u32(sched->job_base, sched->job_base, NT, scan_ws, sched->job_base + NT, s);
  if (r != GS_OK) return r;
  k_chunk_jobs<<<nb, 256, 0, s>>>(sched->job_base, NT, sched->max_jobs, sched->jobs);
  return gs_check_launch();
}

int gs_schedule_check(const gs_schedule* sched, int n_units, int n_tiles, int64_t max_instances) {
  if (!sched) return GS_OK;
  if (!sched->tile_order || !sched->block_masks || !sched->job_base || !sched->jobs || !sched->checkpoints ||
      !sched->chunk_last || !sched->stop_queue ||
      sched->chunk < 32 || (sched->chunk & 31))
    return GS_ERR_INVALID;
  int64_t NT = (int64_t)n_units * n_tiles;
  if (NT > MAX_SCHED_TILES) return GS_ERR_INVALID;
  if (sched->max_jobs < NT + max_instances / sched->chunk + 1) return GS_ERR_INVALID;
  if (sched->max_checkpoints < max_instances / sched->chunk + 1) return GS_ERR_INVALID;
  return GS_OK;
}

int gs_seg_sort(const UnitTable& U, int64_t P, const gs_proj* proj, int width, int height, int64_t cap,
                uint64_t* keysA, uint64_t* keysB, uint32_t* wsS, uint32_t* wsL, uint32_t* bsums, uint32_t* ctr,
                uint32_t* sorted_vals, uint32_t* ranges, uint16_t* masks, cudaStream_t s);

// The depth-first design (method 2): compact the visible records in record order, sort them by their
// 32-bit depth keys taken relative to the nearest visible depth (stable 8-bit passes; a pass whose digit
// all keys share is skipped on the device: the top one whenever the view's depths stay within a factor
// of ~4 of each other, so that every relative key is below 2^24), scan their
// instance counts in that order, emit one 32-bit (mask | unit | tile) key per instance, sort those
// stably on the unit | tile bits (ut_bits <= 16: one or two 8-bit passes) and read off the lists.
// Buffers: the record pairs ping-pong between keys0 (keys at word 0, ids at word P) and keys1; the
// instance pairs between (vals0, vals1) and (keys0, keys1) reinterpreted as 32-bit words.
static int depth_first_sort(const UnitTable& U, int64_t P, const gs_proj* proj, int width, int height, int64_t cap,
                     int tile_bits, int ut_bits, int64_t nsb, int64_t stride, uint32_t* bsums,
                     uint64_t* k0, uint64_t* k1, uint32_t* v0, uint32_t* v1, uint32_t* hist, uint32_t* totals,
                     int32_t* cur, uint32_t* d_vis, uint32_t* bmin_ws, uint32_t* sorted_vals, uint32_t* ranges,
                     uint32_t* d_num_instances, uint16_t* block_masks, int* d_status, cudaStream_t s) {
  constexpr size_t DYN32 = RS_TILE * (sizeof(uint32_t) + sizeof(uint32_t));
  int n_tiles = ((width + TILE - 1) / TILE) * ((height + TILE - 1) / TILE);
  uint32_t* dkA = (uint32_t*)k0;
  uint32_t* dvA = dkA + P;
  uint32_t* dkB = (uint32_t*)k1;
  uint32_t* dvB = dkB + P;
  if (cudaFuncSetAttribute(k_radix_scatter<8, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DYN32) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_radix_scatter<8, uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)DYN32) != cudaSuccess)
    return GS_ERR_CUDA;
  unsigned gh = resident_blocks(k_radix_hist<8, uint32_t>, RS_T, 0, stride);
  unsigned gsc = resident_blocks(k_radix_scatter<8, uint32_t>, RS_T, DYN32, stride);
  unsigned gscf = resident_blocks(k_radix_scatter<8, uint32_t, true>, RS_T, DYN32, stride);
  uint32_t* d_min = d_vis + 1;
  uint32_t* bmins = bmin_ws;  // nsb entries
  k_vis_reduce<<<(unsigned)nsb, SCAN_T, 0, s>>>(proj->tiles, proj->depth, P, bsums, bmins);
  k_scan_bsums<<<1, 1024, 0, s>>>(bsums, nsb, bmins, d_min);
  k_vis_compact<<<(unsigned)nsb, SCAN_T, 0, s>>>(proj->tiles, proj->depth, P, bsums, nsb, d_min, dkA, dvA, d_vis);
  // (three 9-bit passes and a skipped top pass measured slower: a 9-bit scatter pass took 76 us against
  // 48 us for an 8-bit one at 10M records)
  constexpr int DEPTH_PASSES = 4;
  for (int pass = 0; pass < DEPTH_PASSES; ++pass) {
    k_radix_hist<8, uint32_t><<<gh, RS_T, 0, s>>>(dkA, dkB, cur, pass, d_vis, 8 * pass, hist, stride, totals);
    k_radix_scan<<<256, 1024, 0, s>>>(hist, stride, totals, pass, 256, d_vis, cur);
    k_radix_scatter<8, uint32_t><<<gsc, RS_T, DYN32, s>>>(dkA, dkB, dvA, dvB, cur, pass, d_vis, 8 * pass, hist,
                                                          stride, nullptr, nullptr);
  }
  k_dup_reduce<<<(unsigned)nsb, SCAN_T, 0, s>>>(dvA, dvB, cur, DEPTH_PASSES, d_vis, proj->tiles, bsums);
  k_scan_bsums<<<1, 1024, 0, s>>>(bsums, nsb, nullptr, nullptr);
  int key_masks = block_masks ? 1 : 0;
  uint32_t* ikA = v0;
  uint32_t* ivA = v1;
  uint32_t* ikB = (uint32_t*)k0;
  uint32_t* ivB = (uint32_t*)k1;
  k_dup_emit<<<(unsigned)nsb, SCAN_T, 0, s>>>(U, (const float4*)proj->xy, (const float4*)proj->conic_op,
                                              proj->radius, dvA, dvB, cur, DEPTH_PASSES, d_vis, bsums, nsb, width,
                                              height, tile_bits, cap, key_masks, ikA, ivA, d_num_instances,
                                              d_status);
  if (cap == 0) return gs_check_launch();
  // the instance passes keep their own buffer parity and digit totals
  int32_t* cur_t = cur + MAX_PASSES + 1;
  uint32_t* totals_t = totals + DEPTH_PASSES * RS_BINS_MAX;
  int tpasses = (ut_bits + 7) / 8;
  for (int pass = 0; pass < tpasses; ++pass) {
    k_radix_hist<8, uint32_t><<<gh, RS_T, 0, s>>>(ikA, ikB, cur_t, pass, d_num_instances, 8 * pass, hist, stride,
                                                  totals_t);
    k_radix_scan<<<256, 1024, 0, s>>>(hist, stride, totals_t, pass, 256, d_num_instances, cur_t);
    // the last pass writes the record ids and block masks to the outputs (k_ranges32 copies them only
    // when the device skips that pass)
    if (pass == tpasses - 1)
      k_radix_scatter<8, uint32_t, true><<<gscf, RS_T, DYN32, s>>>(ikA, ikB, ivA, ivB, cur_t, pass, d_num_instances,
                                                                   8 * pass, hist, stride, sorted_vals, block_masks);
    else
      k_radix_scatter<8, uint32_t><<<gsc, RS_T, DYN32, s>>>(ikA, ikB, ivA, ivB, cur_t, pass, d_num_instances, 8 * pass,
                                                            hist, stride, nullptr, nullptr);
  }
  k_ranges32<<<resident_blocks(k_ranges32, 256, 0, (cap + 255) / 256), 256, 0, s>>>(
      ikA, ikB, ivA, ivB, cur_t, tpasses, d_num_instances, tile_bits, n_tiles, ranges, sorted_vals, block_masks);
  return gs_check_launch();
}

// method 0: the global LSD radix sort of (unit | tile | depth) keys; 1: the bucketed sort (sort_seg.cu);
// 2: the depth-first design (falls back to 0 when unit | tile needs more than 16 bits).  All give the
// same lists, ranges and masks.
int gs_bin_sort_impl(const gs_proj* proj, const gs_units* units, int width, int height, int64_t max_instances,
                     void* workspace, size_t workspace_bytes, uint32_t* sorted_vals, uint32_t* ranges,
                     uint32_t* d_num_instances, const gs_schedule* sched, int* d_status, cudaStream_t s,
                     int method) {
  uint16_t* block_masks = sched ? sched->block_masks : nullptr;
  UnitTable U;
  int64_t P = 0;
  if (!proj || !proj->xy || !proj->depth || !proj->radius || !proj->tiles || width <= 0 || height <= 0 ||
      (block_masks && !proj->conic_op) ||
      !workspace || !sorted_vals || !ranges || !d_num_instances || max_instances < 0 ||
      max_instances >= (int64_t)UINT32_MAX)
    return GS_ERR_INVALID;
  if (gs_fill_units(units, U, &P) != GS_OK) return GS_ERR_INVALID;
  WsLayout L = ws_layout(P, max_instances);
  if (workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) return GS_ERR_INVALID;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  int n_tiles = TX * TY;
  if (gs_schedule_check(sched, U.n, n_tiles, max_instances) != GS_OK) return GS_ERR_INVALID;
  int tile_bits = bits_for(n_tiles);
  int unit_bits = bits_for(U.n);
  if (tile_bits + unit_bits > 32) return GS_ERR_INVALID;
  int key_bits = 32 + tile_bits + unit_bits;
  if (method == 2 && tile_bits + unit_bits > 16) method = 0;  // unit | tile beside the mask in 32 bits
  // 9-bit digits when they save a pass (45-bit keys at 1080p: 5 passes instead of 6)
  int digit = ((key_bits + 8) / 9 < (key_bits + 7) / 8) ? 9 : 8;
  int passes = (key_bits + digit - 1) / digit;
  char* ws = (char*)workspace;
  uint32_t* offsets = (uint32_t*)(ws + L.offsets);
  uint32_t* bsums = (uint32_t*)(ws + L.bsums);
  uint64_t* k0 = (uint64_t*)(ws + L.keys0);
  uint64_t* k1 = (uint64_t*)(ws + L.keys1);
  uint32_t* v0 = (uint32_t*)(ws + L.vals0);
  uint32_t* v1 = (uint32_t*)(ws + L.vals1);
  uint32_t* hist = (uint32_t*)(ws + L.hist);
  uint32_t* totals = (uint32_t*)(ws + L.totals);
  int32_t* cur = (int32_t*)(ws + L.cur);
  int64_t stride = ((max_instances > P ? max_instances : P) + RS_TILE - 1) / RS_TILE;
  if (stride < 1) stride = 1;

  if (cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_tiles * U.n, s) != cudaSuccess ||
      cudaMemsetAsync(totals, 0, sizeof(uint32_t) * RS_BINS_MAX * MAX_PASSES, s) != cudaSuccess ||
      cudaMemsetAsync(cur, 0, sizeof(int32_t) * 2 * (MAX_PASSES + 1), s) != cudaSuccess ||
      cudaMemsetAsync(d_num_instances, 0, sizeof(uint32_t), s) != cudaSuccess)
    return GS_ERR_CUDA;
  if (P == 0) {
    if (sched) return gs_schedule_jobs(ranges, n_tiles * U.n, ws + L.order, ws + L.jscan, sched, s);
    return gs_check_launch();
  }
  int64_t nsb = (P + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (method == 2) {
    int r = depth_first_sort(U, P, proj, width, height, max_instances, tile_bits, tile_bits + unit_bits, nsb, stride,
                             bsums, k0, k1, v0, v1, hist, totals, cur, (uint32_t*)(ws + L.misc), offsets,
                             sorted_vals, ranges, d_num_instances, block_masks, d_status, s);
    if (r != GS_OK) return r;
    if (sched) return gs_schedule_jobs(ranges, n_tiles * U.n, ws + L.order, ws + L.jscan, sched, s);
    return gs_check_launch();
  }
  k_scan_reduce<<<(unsigned)nsb, SCAN_T, 0, s>>>(proj->tiles, P, bsums);
  k_scan_bsums<<<1, 1024, 0, s>>>(bsums, nsb, nullptr, nullptr);
  k_scan_down<<<(unsigned)nsb, SCAN_T, 0, s>>>(proj->tiles, P, bsums, nsb, offsets, max_instances,
                                               d_num_instances, d_status);
  if (method == 1) {
    if ((int64_t)n_tiles * U.n > MAX_SCHED_TILES) return GS_ERR_INVALID;
    int r = gs_seg_sort(U, P, proj, width, height, max_instances, k0, k1, v0, v1, (uint32_t*)(ws + L.jscan),
                        (uint32_t*)cur, sorted_vals, ranges, block_masks, s);
    if (r != GS_OK) return r;
    if (sched) return gs_schedule_jobs(ranges, n_tiles * U.n, ws + L.order, ws + L.jscan, sched, s);
    return gs_check_launch();
  }
  // block masks ride in the keys when unit | tile | depth leave bits 48..63 free
  int key_masks = (block_masks && key_bits <= 48) ? 1 : 0;
  k_duplicate<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(U, (const float4*)proj->xy, (const float4*)proj->conic_op,
                                                          proj->depth, proj->radius, proj->tiles, offsets, width,
                                                          height, tile_bits, max_instances, key_masks, k0, v0);
  if (max_instances > 0) {
    if (cudaFuncSetAttribute(k_radix_scatter<8, uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, SCATTER_DYN_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_radix_scatter<9, uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, SCATTER_DYN_SMEM) !=
            cudaSuccess)
      return GS_ERR_CUDA;
    unsigned gh = digit == 9 ? resident_blocks(k_radix_hist<9, uint64_t>, RS_T, 0, stride)
                             : resident_blocks(k_radix_hist<8, uint64_t>, RS_T, 0, stride);
    unsigned gs = digit == 9 ? resident_blocks(k_radix_scatter<9, uint64_t>, RS_T, SCATTER_DYN_SMEM, stride)
                             : resident_blocks(k_radix_scatter<8, uint64_t>, RS_T, SCATTER_DYN_SMEM, stride);
    for (int pass = 0; pass < passes; ++pass) {
      int shift = digit * pass;
      if (digit == 9) {
        k_radix_hist<9, uint64_t><<<gh, RS_T, 0, s>>>(k0, k1, cur, pass, d_num_instances, shift, hist, stride, totals);
        k_radix_scan<<<512, 1024, 0, s>>>(hist, stride, totals, pass, 512, d_num_instances, cur);
        k_radix_scatter<9, uint64_t><<<gs, RS_T, SCATTER_DYN_SMEM, s>>>(k0, k1, v0, v1, cur, pass, d_num_instances, shift,
                                                               hist, stride, nullptr, nullptr);
      } else {
        k_radix_hist<8, uint64_t><<<gh, RS_T, 0, s>>>(k0, k1, cur, pass, d_num_instances, shift, hist, stride, totals);
        k_radix_scan<<<256, 1024, 0, s>>>(hist, stride, totals, pass, 256, d_num_instances, cur);
        k_radix_scatter<8, uint64_t><<<gs, RS_T, SCATTER_DYN_SMEM, s>>>(k0, k1, v0, v1, cur, pass, d_num_instances, shift,
                                                               hist, stride, nullptr, nullptr);
      }
    }
    k_ranges<<<resident_blocks(k_ranges, 256, 0, (max_instances + 255) / 256), 256, 0, s>>>(
        k0, k1, v0, v1, cur, passes, d_num_instances, tile_bits, n_tiles, TX, ranges, sorted_vals,
        (const float4*)proj->xy, (const float4*)proj->conic_op, block_masks, key_masks);
  }
  if (sched) return gs_schedule_jobs(ranges, n_tiles * U.n, ws + L.order, ws + L.jscan, sched, s);
  return gs_check_launch();
}

GS_API int gs_bin_sort(const gs_proj* proj, const gs_units* units, int width, int height, int64_t max_instances,
                       void* workspace, size_t workspace_bytes, uint32_t* sorted_vals, uint32_t* ranges,
                       uint32_t* d_num_instances, const gs_schedule* sched, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_bin_sort");
  return gs_bin_sort_impl(proj, units, width, height, max_instances, workspace, workspace_bytes, sorted_vals,
                          ranges, d_num_instances, sched, d_status, (cudaStream_t)stream, 2);
}

GS_API int gs_bin_sort_global(const gs_proj* proj, const gs_units* units, int width, int height,
                              int64_t max_instances, void* workspace, size_t workspace_bytes, uint32_t* sorted_vals,
                              uint32_t* ranges, uint32_t* d_num_instances, const gs_schedule* sched, int* d_status,
                              gs_stream_t stream) {
  GS_RANGE("gs_bin_sort_global");
  return gs_bin_sort_impl(proj, units, width, height, max_instances, workspace, workspace_bytes, sorted_vals,
                          ranges, d_num_instances, sched, d_status, (cudaStream_t)stream, 0);
}

GS_API int gs_bin_sort_bucketed(const gs_proj* proj, const gs_units* units, int width, int height,
                                int64_t max_instances, void* workspace, size_t workspace_bytes,
                                uint32_t* sorted_vals, uint32_t* ranges, uint32_t* d_num_instances,
                                const gs_schedule* sched, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_bin_sort_bucketed");
  return gs_bin_sort_impl(proj, units, width, height, max_instances, workspace, workspace_bytes, sorted_vals,
                          ranges, d_num_instances, sched, d_status, (cudaStream_t)stream, 1);
}

GS_API int gs_schedule_sizes(int n_units, int width, int height, int64_t max_instances, int chunk, int64_t* max_jobs,
                             int64_t* max_checkpoints) {
  if (n_units < 1 || width <= 0 || height <= 0 || max_instances < 0 || chunk < 32 || (chunk & 31) || !max_jobs ||
      !max_checkpoints)
    return GS_ERR_INVALID;
  int64_t nt = (int64_t)n_units * ((width + TILE - 1) / TILE) * ((height + TILE - 1) / TILE);
  *max_jobs = nt + max_instances / chunk + 1;
  *max_checkpoints = max_instances / chunk + 1;
  return GS_OK;
}

int gs_render_fwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                       int width, int height, const float* bg, float* img, float* final_T, uint32_t* n_contrib,
                       int variant, const gs_schedule* sched, cudaStream_t s);

GS_API int gs_merge_render(const float* params, int64_t n_gauss, int sh_degree, const gs_owned* owned,
                           const gs_camera* cam, int width, int height, const float* bg, const gs_proj* proj,
                           int64_t max_instances, void* workspace, size_t workspace_bytes, uint32_t* sorted_vals,
                           uint32_t* ranges, uint32_t* d_num_instances, float* img, float* final_T,
                           uint32_t* n_contrib, const gs_schedule* sched, int* d_status, gs_stream_t stream) {
  GS_RANGE("gs_merge_render");
  if (!owned || owned->n_parts < 1) return GS_ERR_INVALID;
  int64_t begin = 0, count = n_gauss;
  gs_units one = {1, &begin, &count};
  int r = gs_preprocess(params, n_gauss, sh_degree, &one, cam, width, height, owned, proj, d_status, stream);
  if (r != GS_OK) return r;
  r = gs_bin_sort_impl(proj, &one, width, height, max_instances, workspace, workspace_bytes, sorted_vals, ranges,
                       d_num_instances, sched, d_status, (cudaStream_t)stream, 2);
  if (r != GS_OK) return r;
  return gs_render_fwd_impl(proj, sorted_vals, ranges, 1, width, height, bg, img, final_T, n_contrib, 0, sched,
                            (cudaStream_t)stream);
}
