// a2, bucketed form: the tile instances are gathered per (unit, tile) list
// and every list is sorted on its own.
//
//   count   : every visible record adds one to the count of each (unit, tile)
//             it covers (warp-aggregated atomics: records in Z-order share
//             most of their tiles with their neighbours);
//   scan    : exclusive scan of the counts gives each list's [start, end),
//             the tile ranges;
//   scatter : every record writes (float bits of its depth, record index) to
//             a slot of each list it covers, slots taken by warp-aggregated
//             atomics, so the order inside a list is arbitrary;
//   sort    : one CTA per list, heaviest lists first, sorts the list by
//             depth with stable LSD radix passes of 8-bit digits over the
//             list's own depth range (in shared memory for lists of up to
//             SG_SMEM keys, through L2-resident scratch otherwise), then
//             orders each run of equal depths by record index.  A run longer
//             than SG_RUN sends the list through radix passes over (depth,
//             record index) instead.  Either way the list ends in the order
//             of a stable depth sort of its records in index order, the
//             order the global radix sort produces; the block masks of the
//             sorted instances are written with it.
// Every launch is sized without a host round trip (CUDA-graph capturable).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

constexpr int SG_T = 256;                  // threads of a list-sorting CTA
constexpr int SG_W = SG_T / 32;
constexpr int SG_R = 8;                    // rounds of 32 keys per warp and tile
constexpr int SG_TILE = SG_T * SG_R;       // 2048 keys per tile of a pass
constexpr int SG_SMEM = 4096;              // lists of up to this many keys sort in shared memory
constexpr int SG_RUN = 64;                 // longest run of equal depths ordered in place
constexpr int SC_T = 256, SC_ITEMS = 8, SC_BLOCK = SC_T * SC_ITEMS;  // segment scan

struct SegShared {
  uint64_t buf[2][SG_SMEM];
  uint16_t mbuf[2][SG_SMEM];  // the keys' block masks
  uint32_t cnt[SG_W][256];
  uint32_t base[256];
  uint32_t tot[256];
  uint32_t red[4][SG_W];
  uint32_t warp[SG_W + 1];
  uint32_t seg;
  int flag;
};

__device__ __forceinline__ uint32_t warp_incl(uint32_t v) {
  int lane = threadIdx.x & 31;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// exclusive scan of one value per thread of a 256-thread block; *total = the sum
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = warp_incl(v);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < SG_W ? s_warp[lane] : 0u;
    uint32_t xi = warp_incl(x);
    if (lane < SG_W) s_warp[lane] = xi - x;
    if (lane == SG_W - 1) s_warp[SG_W] = xi;
  }
  __syncthreads();
  uint32_t r = inc - v + s_warp[w];
  if (total) *total = s_warp[SG_W];
  __syncthreads();
  return r;
}

// The (unit, tile) list of the k-th tile (row-major) of a record's rectangle.
struct RecTiles {
  uint32_t nt;
  int x0, y0, wdt;
  int64_t ubase;
};
__device__ __forceinline__ RecTiles rec_tiles(const UnitTable& U, const float4* __restrict__ xy,
                                              const int* __restrict__ radius, const uint32_t* __restrict__ tiles,
                                              int64_t p, int64_t P, int TX, int TY, int n_tiles) {
  RecTiles r{0u, 0, 0, 1, 0};
  if (p < P) {
    r.nt = tiles[p];
    if (r.nt) {
      int x1, y1;
      tile_rect(xy[p], radius[p], TX, TY, r.x0, r.y0, x1, y1);
      r.wdt = x1 - r.x0;
      r.ubase = (int64_t)unit_of(U, p) * n_tiles;
    }
  }
  return r;
}
__device__ __forceinline__ long long rec_list(const RecTiles& r, uint32_t k, int TX) {
  if (k >= r.nt) return -1;
  return r.ubase + (int64_t)(r.y0 + (int)(k / (uint32_t)r.wdt)) * TX + (r.x0 + (int)(k % (uint32_t)r.wdt));
}

__global__ void __launch_bounds__(256) k_seg_count(UnitTable U, const float4* __restrict__ xy,
                                                   const int* __restrict__ radius, const uint32_t* __restrict__ tiles,
                                                   int TX, int TY, int n_tiles, uint32_t* __restrict__ ranges) {
  const int64_t P = U.proj_base[U.n];
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  RecTiles r = rec_tiles(U, xy, radius, tiles, p, P, TX, TY, n_tiles);
  const uint32_t kmax = __reduce_max_sync(0xffffffffu, r.nt);
  for (uint32_t k = 0; k < kmax; ++k) {
    long long f = rec_list(r, k, TX);
    unsigned peers = __match_any_sync(0xffffffffu, f);
    if (f >= 0 && lane == __ffs(peers) - 1) atomicAdd(&ranges[2 * f + 1], (uint32_t)__popc(peers));
  }
}

__global__ void __launch_bounds__(256) k_seg_scatter(UnitTable U, const float4* __restrict__ xy,
                                                     const float4* __restrict__ conic_op,
                                                     const int* __restrict__ radius,
                                                     const uint32_t* __restrict__ tiles,
                                                     const float* __restrict__ depth, int TX, int TY, int n_tiles,
                                                     int64_t cap, uint32_t* __restrict__ ranges,
                                                     uint64_t* __restrict__ keys, uint16_t* __restrict__ kmasks) {
  const int64_t P = U.proj_base[U.n];
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  RecTiles r = rec_tiles(U, xy, radius, tiles, p, P, TX, TY, n_tiles);
  const uint64_t key = r.nt ? ((uint64_t)__float_as_uint(depth[p]) << 32) | (uint64_t)(uint32_t)p : 0ull;
  // the record's alpha >= 1/255 box: which 4x4 pixel blocks of each covered tile it reaches
  float4 box = make_float4(1.f, -1.f, 1.f, -1.f);
  if (kmasks && r.nt) {
    float pm;
    float4 m = xy[p];
    box = alpha_box(make_float2(m.x, m.y), conic_op[p], pm);
  }
  const uint32_t kmax = __reduce_max_sync(0xffffffffu, r.nt);
  for (uint32_t k = 0; k < kmax; ++k) {
    long long f = rec_list(r, k, TX);
    unsigned peers = __match_any_sync(0xffffffffu, f);
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (f >= 0 && lane == leader) base = atomicAdd(&ranges[2 * f + 1], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (f >= 0) {
      uint32_t pos = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
      if ((int64_t)pos < cap) {
        keys[pos] = key;
        if (kmasks) {
          const uint32_t t = (uint32_t)(f - r.ubase);
          kmasks[pos] = (uint16_t)block_mask(box, (int)(t % (uint32_t)TX), (int)(t / (uint32_t)TX));
        }
      }
    }
  }
}

// ---- exclusive scan of the list counts (odd words of ranges): start into
// both words of each list (the second is the scatter's cursor)
__global__ void __launch_bounds__(SC_T) k_seg_scan_reduce(const uint32_t* __restrict__ ranges, int64_t n,
                                                          uint32_t* __restrict__ bsums) {
  __shared__ uint32_t s_warp[SG_W + 1];
  int64_t base = (int64_t)blockIdx.x * SC_BLOCK;
  uint32_t s = 0;
  #pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SC_T + threadIdx.x;
    if (k < n) s += ranges[2 * k + 1];
  }
  uint32_t tot;
  scan256(s, s_warp, &tot);
  if (threadIdx.x == 0) bsums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_seg_scan_bsums(uint32_t* bsums, int64_t nb) {
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int64_t k = 0; k < nb; ++k) {
      uint32_t v = bsums[k];
      bsums[k] = acc;
      acc += v;
    }
    s_carry = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) bsums[nb] = s_carry;
}

__global__ void __launch_bounds__(SC_T) k_seg_scan_down(uint32_t* __restrict__ ranges, int64_t n,
                                                        const uint32_t* __restrict__ bsums) {
  __shared__ uint32_t s_warp[SG_W + 1];
  __shared__ uint32_t s_items[SC_BLOCK];
  int64_t base = (int64_t)blockIdx.x * SC_BLOCK;
  #pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SC_T + threadIdx.x;
    s_items[j * SC_T + threadIdx.x] = k < n ? ranges[2 * k + 1] : 0u;
  }
  __syncthreads();
  uint32_t loc[SC_ITEMS];
  uint32_t s = 0;
  #pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    loc[j] = s;
    s += s_items[threadIdx.x * SC_ITEMS + j];
  }
  uint32_t ex = scan256(s, s_warp, nullptr) + bsums[blockIdx.x];
  #pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) s_items[threadIdx.x * SC_ITEMS + j] = loc[j] + ex;
  __syncthreads();
  #pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    int64_t k = base + (int64_t)j * SC_T + threadIdx.x;
    if (k < n) {  // an empty list keeps [0, 0)
      uint32_t st = ranges[2 * k + 1] ? s_items[j * SC_T + threadIdx.x] : 0u;
      ranges[2 * k] = st;
      ranges[2 * k + 1] = st;
    }
  }
}

// One stable LSD pass of a list: 8-bit digit `digit(key)` of each key of src
// [0, L) ordered into dst.  Keys are taken in tiles of SG_TILE; in a tile, warp
// w ranks its 8 rounds of 32 consecutive keys with warp-private digit counts
// (round order, lane order), and the (digit, warp) offsets are scanned across
// the CTA; the list's digit bases advance tile by tile.
template <class DigitF>
__device__ void seg_pass(const uint64_t* src, uint64_t* dst, const uint16_t* srcm, uint16_t* dstm, int L,
                         DigitF digit, SegShared& S) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  S.tot[tid] = 0;
  __syncthreads();
  for (int k = tid; k < L; k += SG_T) atomicAdd(&S.tot[digit(src[k])], 1u);
  __syncthreads();
  S.base[tid] = scan256(S.tot[tid], S.warp, nullptr);
  __syncthreads();
  for (int t0 = 0; t0 < L; t0 += SG_TILE) {
    for (int d = lane; d < 256; d += 32) S.cnt[w][d] = 0u;
    __syncwarp();
    uint64_t kv[SG_R];
    uint32_t dg[SG_R], rk[SG_R];
    uint16_t mk[SG_R];
    #pragma unroll
    for (int r = 0; r < SG_R; ++r) {
      int k = t0 + w * (32 * SG_R) + r * 32 + lane;
      bool valid = k < L;
      kv[r] = valid ? src[k] : 0ull;
      mk[r] = valid ? srcm[k] : (uint16_t)0;
      uint32_t d = valid ? digit(kv[r]) : 256u;
      dg[r] = d;
      unsigned peers = __match_any_sync(FULL, d);
      uint32_t old = valid ? S.cnt[w][d] : 0u;
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) S.cnt[w][d] = old + (uint32_t)__popc(peers);
      __syncwarp();
      rk[r] = old + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    uint32_t run = 0;  // thread tid: digit tid over the warps, in warp order
    #pragma unroll
    for (int ww = 0; ww < SG_W; ++ww) {
      uint32_t c = S.cnt[ww][tid];
      S.cnt[ww][tid] = run;
      run += c;
    }
    __syncthreads();
    #pragma unroll
    for (int r = 0; r < SG_R; ++r) {
      int k = t0 + w * (32 * SG_R) + r * 32 + lane;
      if (k < L) {
        const uint32_t q = S.base[dg[r]] + S.cnt[w][dg[r]] + rk[r];
        dst[q] = kv[r];
        dstm[q] = mk[r];
      }
    }
    __syncthreads();
    S.base[tid] += run;
    __syncthreads();
  }
}

__device__ __forceinline__ int bits_of(uint32_t range) { return range ? 32 - __clz(range) : 0; }

// ---- short lists (1 .. SG_SMEM keys): one CTA per list, in shared memory.
// CTAs take the short lists (compacted by the classify kernel) from a ticket
// counter: sort the keys with their block masks, then write the record ids
// and (with_masks) the masks in list order.
__global__ void __launch_bounds__(SG_T) k_seg_short(const uint32_t* __restrict__ ranges,
                                                    const uint32_t* __restrict__ short_list,
                                                    const uint32_t* __restrict__ n_short,
                                                    const uint64_t* __restrict__ keys,
                                                    const uint16_t* __restrict__ kmasks,
                                                    uint32_t* __restrict__ out_vals, uint16_t* __restrict__ masks,
                                                    uint32_t* __restrict__ ticket) {
  extern __shared__ __align__(16) char s_raw[];
  SegShared& S = *reinterpret_cast<SegShared*>(s_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t NS = *n_short;
  for (;;) {
    if (tid == 0) S.seg = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t o = S.seg;
    __syncthreads();
    if (o >= NS) break;
    const uint32_t f = short_list[o];
    const uint32_t a = ranges[2 * f], b = ranges[2 * f + 1];
    const int L = (int)(b - a);
    uint64_t* src = S.buf[0];
    uint64_t* dst = S.buf[1];
    uint16_t* srcm = S.mbuf[0];
    uint16_t* dstm = S.mbuf[1];
    // the list's depth and record-index ranges
    uint32_t dmin = 0xffffffffu, dmax = 0u, pmin = 0xffffffffu, pmax = 0u;
    for (int k = tid; k < L; k += SG_T) {
      uint64_t key = keys[a + k];
      src[k] = key;
      srcm[k] = kmasks ? kmasks[a + k] : (uint16_t)0;
      uint32_t d = (uint32_t)(key >> 32), p = (uint32_t)key;
      dmin = min(dmin, d); dmax = max(dmax, d); pmin = min(pmin, p); pmax = max(pmax, p);
    }
    dmin = __reduce_min_sync(0xffffffffu, dmin); dmax = __reduce_max_sync(0xffffffffu, dmax);
    pmin = __reduce_min_sync(0xffffffffu, pmin); pmax = __reduce_max_sync(0xffffffffu, pmax);
    if (lane == 0) { S.red[0][w] = dmin; S.red[1][w] = dmax; S.red[2][w] = pmin; S.red[3][w] = pmax; }
    if (tid == 0) S.flag = 0;
    __syncthreads();
    dmin = S.red[0][0]; dmax = S.red[1][0]; pmin = S.red[2][0]; pmax = S.red[3][0];
    #pragma unroll
    for (int ww = 1; ww < SG_W; ++ww) {
      dmin = min(dmin, S.red[0][ww]); dmax = max(dmax, S.red[1][ww]);
      pmin = min(pmin, S.red[2][ww]); pmax = max(pmax, S.red[3][ww]);
    }
    __syncthreads();
    // stable passes over the depth bits that vary in this list
    const int db = bits_of(dmax - dmin);
    for (int sh = 0; sh < db; sh += 8) {
      seg_pass(src, dst, srcm, dstm, L, [=](uint64_t key) { return (((uint32_t)(key >> 32) - dmin) >> sh) & 255u; },
               S);
      uint64_t* t = src; src = dst; dst = t;
      uint16_t* tm = srcm; srcm = dstm; dstm = tm;
    }
    // runs of equal depth: ordered by record index in place, or (a run longer than SG_RUN) the whole
    // list through passes over (depth, record index)
    for (int k = tid; k < L; k += SG_T) {
      uint32_t d = (uint32_t)(src[k] >> 32);
      bool start = (k == 0 || (uint32_t)(src[k - 1] >> 32) != d) && k + 1 < L && (uint32_t)(src[k + 1] >> 32) == d;
      if (!start) continue;
      int e = k + 1;
      while (e < L && (uint32_t)(src[e] >> 32) == d && e - k <= SG_RUN) ++e;
      if (e - k > SG_RUN) { S.flag = 1; continue; }
      for (int i = k + 1; i < e; ++i) {  // insertion sort of the run by record index
        uint64_t x = src[i];
        uint16_t xm = srcm[i];
        int j = i - 1;
        while (j >= k && (uint32_t)src[j] > (uint32_t)x) { src[j + 1] = src[j]; srcm[j + 1] = srcm[j]; --j; }
        src[j + 1] = x;
        srcm[j + 1] = xm;
      }
    }
    __syncthreads();
    if (S.flag) {
      const int pb = bits_of(pmax - pmin);
      for (int sh = 0; sh < db + pb; sh += 8) {
        seg_pass(src, dst, srcm, dstm, L, [=](uint64_t key) {
          uint64_t rk = ((uint64_t)((uint32_t)(key >> 32) - dmin) << pb) | (uint64_t)((uint32_t)key - pmin);
          return (uint32_t)(rk >> sh) & 255u;
        }, S);
        uint64_t* t = src; src = dst; dst = t;
        uint16_t* tm = srcm; srcm = dstm; dstm = tm;
      }
    }
    for (int k = tid; k < L; k += SG_T) {
      out_vals[a + k] = (uint32_t)src[k];
      if (masks) masks[a + k] = srcm[k];
    }
    __syncthreads();
  }
}

// ---- long lists (more than SG_SMEM keys): every list is cut into jobs of
// LG_KEYS consecutive keys, and every job takes part in each pass, so a long
// list is sorted by as many CTAs as it has jobs.  Per pass (9-bit digits of the
// keys' depth offsets from their list's minimum):
//   hist    : each job counts its digits (H[job][digit]);
//   scan    : one CTA per list, one thread per digit, walks the list's jobs:
//             each job's prefix within its list (P[job][digit]) and the list's
//             digit totals (T[list][digit]);
//   scatter : each job ranks its keys stably (warp match + per-warp counts),
//             orders them by digit in shared memory and writes each digit's
//             run (with the keys' block masks) to the other buffers at list
//             start + the list's count of smaller digits + the job's prefix.
// A list takes ceil(depth bits / 9) passes (its depth bits: those of its
// largest depth offset); its last pass also writes the record ids and block
// masks.  A final kernel then orders each run of equal depths by record index.
constexpr int LG_T = 256;
constexpr int LG_ITEMS = 16;
constexpr int LG_KEYS = LG_T * LG_ITEMS;  // 4096 keys per job
constexpr int LG_BITS = 9;
constexpr int LG_BINS = 1 << LG_BITS;
constexpr int LG_PASSES = (32 + LG_BITS - 1) / LG_BITS;

struct LongTables {
  uint32_t* list;   // [nl_max] list id of each long-list slot
  uint32_t* base;   // [nl_max + 1] jobs of each slot, scanned in place into its first job; total at the end
  uint32_t* dmin;   // [nl_max] smallest depth bits of the slot's list
  uint32_t* dmax;   // [nl_max] largest
  uint2* jobs;      // [j_max] (slot, job within the list)
  uint4* desc;      // [j_max] (first key, end key, list start, list's smallest depth bits) of each job
  uint4* desc2;     // [j_max] (slot, the list's pass count, list end, 0)
  uint32_t* T;      // [nl_max][LG_BINS] the slot's digit totals of the current pass
  uint32_t* H;      // [j_max][LG_BINS] digit counts of each job
  uint32_t* P;      // [j_max][LG_BINS] the job's prefix within its list
  int64_t j_max;
  int64_t nl_max;
  uint32_t* npass;  // the largest pass count of any long list
};

struct SegSizes {
  int64_t nl_max, j_max;
  size_t tables_s, tables_l;  // words of the long-list tables in each scratch region
  size_t words_s, words_l;    // the regions: tables, then a 256-byte aligned [cap] uint16 mask buffer
};

SegSizes seg_sizes(int64_t cap) {
  SegSizes z;
  // long lists hold more than SG_SMEM keys; a list of L keys has ceil(L / LG_KEYS) <= L / LG_KEYS + 1 jobs
  const bool longs = cap > SG_SMEM;
  z.nl_max = longs ? cap / (SG_SMEM + 1) + 1 : 0;
  z.j_max = longs ? cap / LG_KEYS + z.nl_max + 1 : 0;
  z.tables_s = (2 * (size_t)LG_BINS * (size_t)z.j_max + 63) & ~(size_t)63;  // H, P
  const size_t desc_at = ((size_t)(4 * z.nl_max + 2) + 2 * (size_t)z.j_max + (size_t)LG_BINS * (size_t)z.nl_max + 3) &
                        ~(size_t)3;
  z.tables_l = longs ? (desc_at + 8 * (size_t)z.j_max + 63) & ~(size_t)63 : 0;
  const size_t mw = ((size_t)cap + 1) / 2;
  z.words_s = z.tables_s + mw;
  z.words_l = z.tables_l + mw;
  return z;
}

LongTables long_tables(const SegSizes& z, uint32_t* wsS, uint32_t* wsL, uint32_t* npass) {
  LongTables T;
  T.nl_max = z.nl_max;
  T.j_max = z.j_max;
  T.list = wsL;
  T.base = T.list + z.nl_max;
  T.dmin = T.base + z.nl_max + 1;
  T.dmax = T.dmin + z.nl_max;
  T.jobs = reinterpret_cast<uint2*>(T.dmax + z.nl_max + 1);  // 4 nl_max + 2 words: 8-byte aligned
  T.T = reinterpret_cast<uint32_t*>(T.jobs + z.j_max);
  const size_t desc_at = ((size_t)(4 * z.nl_max + 2) + 2 * (size_t)z.j_max + (size_t)LG_BINS * (size_t)z.nl_max + 3) &
                         ~(size_t)3;
  T.desc = reinterpret_cast<uint4*>(wsL + desc_at);  // 16-byte aligned (wsL is 256-byte aligned)
  T.desc2 = T.desc + z.j_max;
  T.H = wsS;
  T.P = wsS + (size_t)LG_BINS * (size_t)z.j_max;
  T.npass = npass;
  return T;
}

__device__ __forceinline__ int lg_passes(uint32_t dmin, uint32_t dmax) {
  return (bits_of(dmax - dmin) + LG_BITS - 1) / LG_BITS;
}

// Clamps every list at the instance capacity (the instances past it were not
// stored) and gives each non-empty list a slot: short lists in short_list,
// long ones in the long tables.
__global__ void __launch_bounds__(256) k_seg_classify(uint32_t* __restrict__ ranges, int64_t NT, int64_t cap,
                                                      uint32_t* __restrict__ ctr, uint32_t* __restrict__ short_list,
                                                      LongTables T) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= NT) return;
  uint32_t a = ranges[2 * f], b = ranges[2 * f + 1];
  if ((int64_t)b > cap) {
    a = (uint32_t)min((int64_t)a, cap);
    b = (uint32_t)cap;
    ranges[2 * f] = a;
    ranges[2 * f + 1] = b;
  }
  if (b == a) return;
  if (b - a > (uint32_t)SG_SMEM) {
    uint32_t slot = atomicAdd(&ctr[1], 1u);
    T.list[slot] = (uint32_t)f;
    T.base[slot] = (b - a + LG_KEYS - 1) / LG_KEYS;
    T.dmin[slot] = 0xffffffffu;
    T.dmax[slot] = 0u;
  } else {
    short_list[atomicAdd(&ctr[2], 1u)] = (uint32_t)f;
  }
}

// (slot, job) of every job of every long list
__global__ void __launch_bounds__(256) k_lg_jobs(const uint32_t* __restrict__ ranges,
                                                 const uint32_t* __restrict__ n_long, LongTables T) {
  const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= *n_long) return;
  const uint32_t f = T.list[slot];
  const uint32_t nj = (ranges[2 * f + 1] - ranges[2 * f] + LG_KEYS - 1) / LG_KEYS;
  const uint32_t b = T.base[slot];
  for (uint32_t j = 0; j < nj; ++j) T.jobs[b + j] = make_uint2(slot, j);
}

struct LgJob {
  uint32_t slot, j, f, s, e, k0, k1;
};
__device__ __forceinline__ LgJob lg_job(uint32_t job, const uint32_t* __restrict__ ranges, const LongTables& T) {
  LgJob J;
  uint2 jb = T.jobs[job];
  J.slot = jb.x; J.j = jb.y;
  J.f = T.list[J.slot];
  J.s = ranges[2 * J.f]; J.e = ranges[2 * J.f + 1];
  J.k0 = J.s + J.j * LG_KEYS;
  J.k1 = min(J.e, J.k0 + LG_KEYS);
  return J;
}

// depth range of each long list (its jobs reduce their keys and combine atomically)
__global__ void __launch_bounds__(LG_T) k_lg_range(const uint32_t* __restrict__ ranges, LongTables T,
                                                   const uint64_t* __restrict__ keys) {
  __shared__ uint32_t s_red[2][LG_T / 32];
  const uint32_t NJ = T.base[T.nl_max];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t job = blockIdx.x; job < NJ; job += gridDim.x) {
    LgJob J = lg_job(job, ranges, T);
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (uint32_t k = J.k0 + threadIdx.x; k < J.k1; k += LG_T) {
      uint32_t d = (uint32_t)(keys[k] >> 32);
      lo = min(lo, d); hi = max(hi, d);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) { s_red[0][w] = lo; s_red[1][w] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < LG_T / 32; ++q) { lo = min(lo, s_red[0][q]); hi = max(hi, s_red[1][q]); }
      atomicMin(&T.dmin[J.slot], lo);
      atomicMax(&T.dmax[J.slot], hi);
    }
    __syncthreads();
  }
}

// every job's descriptor (after the depth ranges are known) and the largest pass count
__global__ void __launch_bounds__(256) k_lg_desc(const uint32_t* __restrict__ ranges, LongTables T) {
  const uint32_t job = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t np = 0;
  if (job < T.base[T.nl_max]) {
    LgJob J = lg_job(job, ranges, T);
    const uint32_t dmin = T.dmin[J.slot];
    np = (uint32_t)lg_passes(dmin, T.dmax[J.slot]);
    T.desc[job] = make_uint4(J.k0, J.k1, J.s, dmin);
    T.desc2[job] = make_uint4(J.slot, np, J.e, 0u);
  }
  np = __reduce_max_sync(0xffffffffu, np);
  if ((threadIdx.x & 31) == 0 && np) atomicMax(T.npass, np);
}

__device__ __forceinline__ uint32_t lg_digit(uint64_t key, uint32_t dmin, int shift) {
  return (((uint32_t)(key >> 32) - dmin) >> shift) & (LG_BINS - 1u);
}

__global__ void __launch_bounds__(LG_T) k_lg_hist(int pass, LongTables T,
                                                  const uint64_t* __restrict__ A, const uint64_t* __restrict__ B) {
  __shared__ uint32_t s_h[LG_T / 32][LG_BINS];
  if ((uint32_t)pass >= *T.npass) return;
  const uint32_t NJ = T.base[T.nl_max];
  const int w = threadIdx.x >> 5, shift = LG_BITS * pass;
  const uint64_t* src = (pass & 1) ? B : A;
  for (uint32_t job = blockIdx.x; job < NJ; job += gridDim.x) {
    const uint4 D = T.desc[job];  // k0, k1, list start, dmin
    if ((uint32_t)pass >= T.desc2[job].y) continue;  // the list is sorted (uniform in the block)
    for (int k = threadIdx.x; k < (LG_T / 32) * LG_BINS; k += LG_T) (&s_h[0][0])[k] = 0u;
    uint32_t dg[LG_ITEMS];
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r) {
      uint32_t k = D.x + r * LG_T + threadIdx.x;
      dg[r] = k < D.y ? lg_digit(src[k], D.w, shift) : 0xffffffffu;
    }
    __syncthreads();
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r)
      if (dg[r] != 0xffffffffu) atomicAdd(&s_h[w][dg[r]], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < LG_BINS; d += LG_T) {
      uint32_t c = 0;
      #pragma unroll
      for (int q = 0; q < LG_T / 32; ++q) c += s_h[q][d];
      T.H[(int64_t)job * LG_BINS + d] = c;
    }
    __syncthreads();
  }
}

// One CTA per long list, thread d for digit d: over the list's jobs, each job's exclusive prefix within the
// list (P) and the list's total (T).
__global__ void __launch_bounds__(LG_BINS) k_lg_scan(int pass, const uint32_t* __restrict__ ranges,
                                                     const uint32_t* __restrict__ n_long, LongTables T) {
  if ((uint32_t)pass >= *T.npass) return;
  const uint32_t NL = *n_long;
  const int d = threadIdx.x;
  for (uint32_t slot = blockIdx.x; slot < NL; slot += gridDim.x) {
    if (pass >= lg_passes(T.dmin[slot], T.dmax[slot])) continue;
    const uint32_t f = T.list[slot];
    const uint32_t nj = (ranges[2 * f + 1] - ranges[2 * f] + LG_KEYS - 1) / LG_KEYS;
    const int64_t fj = T.base[slot];
    uint32_t acc = 0;
    for (uint32_t j = 0; j < nj; ++j) {
      const int64_t o = (fj + j) * LG_BINS + d;
      const uint32_t v = T.H[o];
      T.P[o] = acc;
      acc += v;
    }
    T.T[(int64_t)slot * LG_BINS + d] = acc;
  }
}

// Stable scatter of one job's keys.  The keys are staged in shared memory in
// job order; warp w ranks keys [512 w, 512 (w + 1)) in 16 rounds of 32 (warp
// match, warp-private digit counts), the per-warp counts are scanned across
// warps, the keys are reordered by digit in shared memory, and each digit's run
// is written to consecutive places of the other buffer (coalesced): the list's
// start + the list's count of smaller digits + the job's prefix for the digit.
// In the list's last pass the record ids and masks go to the outputs as well.
__global__ void __launch_bounds__(LG_T, 3) k_lg_scatter(int pass, LongTables T,
                                                        uint64_t* __restrict__ A, uint64_t* __restrict__ B,
                                                        uint16_t* __restrict__ mA, uint16_t* __restrict__ mB,
                                                        uint32_t* __restrict__ out_vals,
                                                        uint16_t* __restrict__ masks) {
  constexpr int NW = LG_T / 32;
  constexpr int WKEYS = LG_KEYS / NW;
  constexpr int DPT = LG_BINS / LG_T;      // digits per thread in the per-digit steps
  __shared__ uint32_t s_off[LG_BINS];      // global position of this job's first key of each digit
  __shared__ uint16_t s_lstart[LG_BINS];   // job-local start of each digit
  __shared__ uint16_t s_wc[NW][LG_BINS];   // per-warp digit counts, then the warp's offset within the digit
  __shared__ uint32_t s_warp[SG_W + 1];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);                      // [LG_KEYS]
  uint16_t* s_msk = reinterpret_cast<uint16_t*>(s_dyn + 8 * (size_t)LG_KEYS);  // [LG_KEYS]
  if ((uint32_t)pass >= *T.npass) return;
  const uint32_t NJ = T.base[T.nl_max];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, shift = LG_BITS * pass;
  const uint64_t* src = (pass & 1) ? B : A;
  uint64_t* dst = (pass & 1) ? A : B;
  const uint16_t* srcm = (pass & 1) ? mB : mA;
  uint16_t* dstm = (pass & 1) ? mA : mB;
  for (uint32_t job = blockIdx.x; job < NJ; job += gridDim.x) {
    const uint4 D = T.desc[job];    // k0, k1, list start, dmin
    const uint4 D2 = T.desc2[job];  // slot, passes, list end
    if ((uint32_t)pass >= D2.y) continue;  // uniform in the block
    const bool last = (uint32_t)pass + 1 == D2.y;
    const uint32_t dmin = D.w;
    const int n = (int)(D.y - D.x);
    // every load of the job in flight at once: its keys and masks, the list's digit totals and the job's
    // prefixes
    uint64_t kk[LG_ITEMS];
    uint32_t mm[LG_ITEMS / 2];
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r) {
      const int i = r * LG_T + tid;
      kk[r] = i < n ? src[D.x + i] : 0ull;
      const uint32_t m = (i < n && srcm) ? (uint32_t)srcm[D.x + i] : 0u;
      if (r & 1) mm[r >> 1] |= m << 16; else mm[r >> 1] = m;
    }
    uint32_t tot[DPT], pre[DPT];
    #pragma unroll
    for (int q = 0; q < DPT; ++q) {
      tot[q] = T.T[(int64_t)D2.x * LG_BINS + tid * DPT + q];
      pre[q] = T.P[(int64_t)job * LG_BINS + tid * DPT + q];
    }
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r) {
      const int i = r * LG_T + tid;
      if (i < n) {
        s_keys[i] = kk[r];
        s_msk[i] = (uint16_t)((r & 1) ? (mm[r >> 1] >> 16) : (mm[r >> 1] & 0xffffu));
      }
    }
    // the digit totals' exclusive scan over digits, plus the job's prefix
    {
      uint32_t c = 0;
      #pragma unroll
      for (int q = 0; q < DPT; ++q) c += tot[q];
      uint32_t st = scan256(c, s_warp, nullptr) + D.z;
      #pragma unroll
      for (int q = 0; q < DPT; ++q) {
        s_off[tid * DPT + q] = st + pre[q];
        st += tot[q];
        #pragma unroll
        for (int ww = 0; ww < NW; ++ww) s_wc[ww][tid * DPT + q] = 0;
      }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t rnk[LG_ITEMS / 2];
    const int wbase = w * WKEYS;
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r) {
      const int i = wbase + r * 32 + lane;
      const bool valid = i < n;
      const uint32_t d = valid ? lg_digit(s_keys[i], dmin, shift) : (uint32_t)LG_BINS;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = valid ? (uint32_t)s_wc[w][d] : 0u;
      const uint32_t rk = before + __popc(peers & lt);  // < WKEYS
      if (r & 1) rnk[r >> 1] |= rk << 16; else rnk[r >> 1] = rk;
      __syncwarp();
      if (valid && (peers & lt) == 0u) s_wc[w][d] = (uint16_t)(before + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    // per digit: the warps' offsets within the digit (warp order = key order), then the digit starts
    {
      uint32_t cnt[DPT], c = 0;
      #pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const int dd = tid * DPT + q;
        uint32_t acc = 0;
        #pragma unroll
        for (int ww = 0; ww < NW; ++ww) {
          const uint32_t x = s_wc[ww][dd];
          s_wc[ww][dd] = (uint16_t)acc;
          acc += x;
        }
        cnt[q] = acc;
        c += acc;
      }
      uint32_t st = scan256(c, s_warp, nullptr);
      #pragma unroll
      for (int q = 0; q < DPT; ++q) { s_lstart[tid * DPT + q] = (uint16_t)st; st += cnt[q]; }
    }
    __syncthreads();
    // reorder by digit in shared memory (this thread's keys of the ranking rounds, into registers first)
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r) {
      const int i = wbase + r * 32 + lane;
      kk[r] = i < n ? s_keys[i] : 0ull;
      const uint32_t m = i < n ? (uint32_t)s_msk[i] : 0u;
      if (r & 1) mm[r >> 1] |= m << 16; else mm[r >> 1] = m;
    }
    __syncthreads();
    #pragma unroll
    for (int r = 0; r < LG_ITEMS; ++r) {
      const int i = wbase + r * 32 + lane;
      if (i >= n) break;
      const uint32_t d = lg_digit(kk[r], dmin, shift);
      const uint32_t rk = (r & 1) ? (rnk[r >> 1] >> 16) : (rnk[r >> 1] & 0xffffu);
      const uint32_t q = (uint32_t)s_lstart[d] + s_wc[w][d] + rk;
      s_keys[q] = kk[r];
      s_msk[q] = (uint16_t)((r & 1) ? (mm[r >> 1] >> 16) : (mm[r >> 1] & 0xffffu));
    }
    __syncthreads();
    for (int i = tid; i < n; i += LG_T) {
      const uint64_t k = s_keys[i];
      const uint32_t d = lg_digit(k, dmin, shift);
      const uint32_t q = s_off[d] + (uint32_t)i - s_lstart[d];
      dst[q] = k;
      if (dstm) dstm[q] = s_msk[i];
      if (last) {
        out_vals[q] = (uint32_t)k;
        if (masks) masks[q] = s_msk[i];
      }
    }
    __syncthreads();
  }
}

// Runs of equal depth in the long lists: the record ids and masks of a run
// are rewritten in record-index order by the thread of the run's first key
// (the whole 64-bit keys, whose depth halves are equal, are sorted with their
// masks).  The job's keys and masks are staged in shared memory; a run that
// ends inside the job is sorted there (insertion sort up to SG_RUN keys, else
// heapsort), one that runs on past the job's end in place in global memory
// (heapsort).  A list of one depth had no pass: it is all one run.
__device__ __forceinline__ uint32_t dhi(uint64_t k) { return (uint32_t)(k >> 32); }

// heapsort of m elements given by key(i) (ascending), moved by swap(i, j)
template <class KeyAt, class Swap>
__device__ void heap_sort(uint32_t m, KeyAt key, Swap swap) {
  auto sift = [&](uint32_t root, uint32_t end) {
    for (;;) {
      uint32_t c = 2 * root + 1;
      if (c >= end) break;
      if (c + 1 < end && key(c + 1) > key(c)) ++c;
      if (key(root) >= key(c)) break;
      swap(root, c);
      root = c;
    }
  };
  for (uint32_t q = m / 2; q-- > 0;) sift(q, m);
  for (uint32_t end = m - 1; end > 0; --end) {
    swap(0, end);
    sift(0, end);
  }
}

__global__ void __launch_bounds__(LG_T) k_lg_ties(LongTables T, uint64_t* __restrict__ A, uint64_t* __restrict__ B,
                                                  uint16_t* __restrict__ mA, uint16_t* __restrict__ mB,
                                                  uint32_t* __restrict__ out_vals, uint16_t* __restrict__ masks) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);                             // keys k0 - 1 .. k1
  uint16_t* s_m = reinterpret_cast<uint16_t*>(s_dyn + 8 * (size_t)(LG_KEYS + 2));  // masks k0 .. k1 - 1
  const uint32_t NJ = T.base[T.nl_max];
  const int tid = threadIdx.x;
  const uint64_t END = ~0ull;  // depth half 0xffffffff (a NaN): never equal to a key's
  for (uint32_t job = blockIdx.x; job < NJ; job += gridDim.x) {
    const uint4 D = T.desc[job];    // k0, k1, list start, dmin
    const uint4 D2 = T.desc2[job];  // slot, passes, list end
    const bool odd = D2.y & 1;
    uint64_t* buf = odd ? B : A;
    uint16_t* mb = odd ? mB : mA;
    const int n = (int)(D.y - D.x);
    {
      uint64_t kk[LG_ITEMS];
      uint16_t mm[LG_ITEMS];
      #pragma unroll
      for (int r = 0; r < LG_ITEMS; ++r) {
        const int i = r * LG_T + tid;
        kk[r] = i < n ? buf[D.x + i] : 0ull;
        mm[r] = (i < n && mb) ? mb[D.x + i] : (uint16_t)0;
      }
      #pragma unroll
      for (int r = 0; r < LG_ITEMS; ++r) {
        const int i = r * LG_T + tid;
        if (i < n) { s_k[i + 1] = kk[r]; s_m[i] = mm[r]; }
      }
    }
    if (tid == 0) s_k[0] = D.x > D.z ? buf[D.x - 1] : END;
    if (tid == 1) s_k[n + 1] = D.y < D2.z ? buf[D.y] : END;
    __syncthreads();
    for (int i = tid; i < n; i += LG_T) {
      const uint32_t d = dhi(s_k[i + 1]);
      if (dhi(s_k[i]) == d || dhi(s_k[i + 2]) != d) continue;  // not the first key of a run
      int r = i + 2;
      while (r < n && dhi(s_k[r + 1]) == d) ++r;
      const uint32_t i0 = D.x + i;
      if (r < n || dhi(s_k[n + 1]) != d) {
        // the run [i, r) lies in this job: sort it in shared memory
        const uint32_t m = (uint32_t)(r - i);
        uint64_t* h = s_k + i + 1;
        uint16_t* hm = s_m + i;
        if (m <= (uint32_t)SG_RUN) {
          for (uint32_t q = 1; q < m; ++q) {
            const uint64_t x = h[q];
            const uint16_t xm = hm[q];
            int t = (int)q - 1;
            while (t >= 0 && h[t] > x) { h[t + 1] = h[t]; hm[t + 1] = hm[t]; --t; }
            h[t + 1] = x;
            hm[t + 1] = xm;
          }
        } else {
          heap_sort(
              m, [&](uint32_t q) { return h[q]; },
              [&](uint32_t x, uint32_t y) {
                uint64_t t = h[x]; h[x] = h[y]; h[y] = t;
                uint16_t tm = hm[x]; hm[x] = hm[y]; hm[y] = tm;
              });
        }
        for (uint32_t q = 0; q < m; ++q) {
          out_vals[i0 + q] = (uint32_t)h[q];
          if (masks) masks[i0 + q] = hm[q];
        }
      } else {
        // the run goes on past the job: sort it in place in global memory (the other threads read only
        // its depth halves)
        uint32_t e = D.y;
        while (e < D2.z && dhi(buf[e]) == d) ++e;
        const uint32_t m = e - i0;
        uint64_t* h = buf + i0;
        uint16_t* hm = mb ? mb + i0 : nullptr;
        heap_sort(
            m, [&](uint32_t q) { return h[q]; },
            [&](uint32_t x, uint32_t y) {
              uint64_t t = h[x]; h[x] = h[y]; h[y] = t;
              if (hm) { uint16_t tm = hm[x]; hm[x] = hm[y]; hm[y] = tm; }
            });
        for (uint32_t q = 0; q < m; ++q) {
          out_vals[i0 + q] = (uint32_t)h[q];
          if (masks) masks[i0 + q] = hm ? hm[q] : (uint16_t)0;
        }
      }
    }
    __syncthreads();
  }
}

template <typename K>
unsigned seg_resident(K kernel, int threads, size_t smem, int64_t units) {
  int dev = 0, sms = 0, per = 0;
  if (units < 1) return 1u;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || sms < 1 || per < 1)
    return 0u;
  int64_t g = (int64_t)sms * per;
  return (unsigned)(g < units ? g : units);
}

}  // namespace

// Words of the bucketed sort's two scratch regions for an instance capacity
// cap: the long-list tables and a [cap] uint16 mask buffer in each.
void gs_seg_ws_words(int64_t cap, size_t* words_s, size_t* words_l) {
  SegSizes z = seg_sizes(cap);
  *words_s = z.words_s;
  *words_l = z.words_l;
}

// Buckets and sorts the tile instances of the visible records (see above).
// ranges: [NT][2], zeroed by the caller; keysA, keysB: [cap] scratch (keysB
// also holds the short-list slots until the long passes); wsS, wsL: the
// scratch regions of gs_seg_ws_words; bsums: (NT / SC_BLOCK + 2) words, also
// the long-list job scan's scratch; ctr: four words.  masks NULL: no block
// masks (conic_op unused).
int gs_seg_sort(const UnitTable& U, int64_t P, const gs_proj* proj, int width, int height, int64_t cap,
                uint64_t* keysA, uint64_t* keysB, uint32_t* wsS, uint32_t* wsL, uint32_t* bsums, uint32_t* ctr,
                uint32_t* sorted_vals, uint32_t* ranges, uint16_t* masks, cudaStream_t s) {
  const int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE, n_tiles = TX * TY;
  const int64_t NT = (int64_t)U.n * n_tiles;
  if (P == 0 || cap == 0) return gs_check_launch();
  const SegSizes z = seg_sizes(cap);
  uint16_t* mA = masks ? reinterpret_cast<uint16_t*>(wsS + z.tables_s) : nullptr;
  uint16_t* mB = masks ? reinterpret_cast<uint16_t*>(wsL + z.tables_l) : nullptr;
  const unsigned gb = (unsigned)((P + 255) / 256);
  k_seg_count<<<gb, 256, 0, s>>>(U, (const float4*)proj->xy, proj->radius, proj->tiles, TX, TY, n_tiles, ranges);
  const int64_t nb = (NT + SC_BLOCK - 1) / SC_BLOCK;
  k_seg_scan_reduce<<<(unsigned)nb, SC_T, 0, s>>>(ranges, NT, bsums);
  k_seg_scan_bsums<<<1, 32, 0, s>>>(bsums, nb);
  k_seg_scan_down<<<(unsigned)nb, SC_T, 0, s>>>(ranges, NT, bsums);
  k_seg_scatter<<<gb, 256, 0, s>>>(U, (const float4*)proj->xy, (const float4*)proj->conic_op, proj->radius,
                                   proj->tiles, proj->depth, TX, TY, n_tiles, cap, ranges, keysA, mA);
  if (cudaMemsetAsync(ctr, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
  // long lists exist only when the capacity exceeds the shared-memory list length
  const bool longs = z.nl_max > 0;
  LongTables T{};
  if (longs) {
    T = long_tables(z, wsS, wsL, ctr + 3);
    if (cudaMemsetAsync(T.base, 0, sizeof(uint32_t) * (size_t)(T.nl_max + 1), s) != cudaSuccess) return GS_ERR_CUDA;
  }
  uint32_t* short_list = reinterpret_cast<uint32_t*>(keysB);  // free until the first long pass
  k_seg_classify<<<(unsigned)((NT + 255) / 256), 256, 0, s>>>(ranges, NT, cap, ctr, short_list, T);
  const size_t smem = sizeof(SegShared);
  if (cudaFuncSetAttribute(k_seg_short, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GS_ERR_CUDA;
  const unsigned g_short = seg_resident(k_seg_short, SG_T, smem, NT);
  if (!g_short) return GS_ERR_CUDA;
  k_seg_short<<<g_short, SG_T, smem, s>>>(ranges, short_list, ctr + 2, keysA, mA, sorted_vals, masks, ctr);
  if (longs) {
    int r = gs_scan_u32(T.base, T.base, T.nl_max, bsums, T.base + T.nl_max, s);
    if (r != GS_OK) return r;
    const unsigned g_nl = (unsigned)((T.nl_max + 255) / 256);
    k_lg_jobs<<<g_nl, 256, 0, s>>>(ranges, ctr + 1, T);
    const size_t sc_smem = (sizeof(uint64_t) + sizeof(uint16_t)) * LG_KEYS;
    if (cudaFuncSetAttribute(k_lg_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc_smem) != cudaSuccess)
      return GS_ERR_CUDA;
    const unsigned g_range = seg_resident(k_lg_range, LG_T, 0, T.j_max);
    const unsigned g_hist = seg_resident(k_lg_hist, LG_T, 0, T.j_max);
    const unsigned g_scat = seg_resident(k_lg_scatter, LG_T, sc_smem, T.j_max);
    const size_t ties_smem = sizeof(uint64_t) * (LG_KEYS + 2) + sizeof(uint16_t) * LG_KEYS;
    if (cudaFuncSetAttribute(k_lg_ties, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ties_smem) != cudaSuccess)
      return GS_ERR_CUDA;
    const unsigned g_fin = seg_resident(k_lg_ties, LG_T, ties_smem, T.j_max);
    const unsigned g_lscan = seg_resident(k_lg_scan, LG_BINS, 0, T.nl_max);
    if (!g_range || !g_hist || !g_scat || !g_fin || !g_lscan) return GS_ERR_CUDA;
    k_lg_range<<<g_range, LG_T, 0, s>>>(ranges, T, keysA);
    k_lg_desc<<<(unsigned)((T.j_max + 255) / 256), 256, 0, s>>>(ranges, T);
    for (int pass = 0; pass < LG_PASSES; ++pass) {
      k_lg_hist<<<g_hist, LG_T, 0, s>>>(pass, T, keysA, keysB);
      k_lg_scan<<<g_lscan, LG_BINS, 0, s>>>(pass, ranges, ctr + 1, T);
      k_lg_scatter<<<g_scat, LG_T, sc_smem, s>>>(pass, T, keysA, keysB, mA, mB, sorted_vals, masks);
    }
    k_lg_ties<<<g_fin, LG_T, ties_smem, s>>>(T, keysA, keysB, mA, mB, sorted_vals, masks);
  }
  return gs_check_launch();
}
