// a3 / a5: front-to-back alpha blending per 16x16 tile and its reverse replay.
//
// One thread per pixel; each warp owns a BW x (32/BW) pixel block of a 16x16
// tile (BW = 8, 16 or 4: the tunable variant).  With the sort's block masks
// every (tile, pixel block) is a one-warp CTA; without them one CTA covers a
// tile.  Each warp walks the tile's list
// independently of the other warps (no block barriers: warps whose block few
// splats reach do not wait for the busy ones).  A record is blended by a warp
// only if the bounding box of the ellipse where its alpha can reach 1/255
// meets the warp's block; this skips only (pixel, record) pairs that the
// per-pixel alpha test would reject anyway, so results are unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

using namespace gs;

namespace {

__device__ __forceinline__ void atomic_add2(float* p, float a, float b) {
#if __CUDA_ARCH__ >= 900
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(a, b));
#else
  atomicAdd(p, a); atomicAdd(p + 1, b);
#endif
}
__device__ __forceinline__ void atomic_add4(float* p, float a, float b, float c, float d) {
#if __CUDA_ARCH__ >= 900
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
#else
  atomicAdd(p, a); atomicAdd(p + 1, b); atomicAdd(p + 2, c); atomicAdd(p + 3, d);
#endif
}

// Deterministic mode: gradients accumulate as int64 fixed point (value x 2^40,
// rounded to nearest).  Integer addition is associative, so the sums do not
// depend on the order in which warps add their contributions.  |value| is
// clamped to 2^22 (|value| 2^40 stays below 2^62); NaN adds 0.
constexpr float FIX_SCALE = 1099511627776.0f;  // 2^40
constexpr float FIX_LIMIT = 4194304.0f;        // 2^22
__device__ __forceinline__ unsigned long long to_fixed(float v) {
  float c = (v == v) ? fminf(fmaxf(v, -FIX_LIMIT), FIX_LIMIT) : 0.f;
  return (unsigned long long)__float2ll_rn(c * FIX_SCALE);
}

// One lane's nine gradient values of record pr (dx, dy | dA, dB, dC, dopacity | dr, dg, db).
__device__ __forceinline__ void add_lane(float* dxy, float* dco, float* drgb, unsigned long long* fixed, int64_t pr,
                                         const float* v) {
  if (fixed) {
    #pragma unroll
    for (int q = 0; q < 9; ++q) atomicAdd(fixed + 9 * pr + q, to_fixed(v[q]));
  } else {
    atomic_add2(dxy + 2 * pr, v[0], v[1]);
    atomic_add4(dco + 4 * pr, v[2], v[3], v[4], v[5]);
    atomic_add4(drgb + 4 * pr, v[6], v[7], v[8], 0.f);
  }
}

// Value q (0..8, order as above) of record pr.
__device__ __forceinline__ void add_one(float* dxy, float* dco, float* drgb, unsigned long long* fixed, int64_t pr,
                                        int q, float x) {
  if (fixed) {
    atomicAdd(fixed + 9 * pr + q, to_fixed(x));
    return;
  }
  float* dst = q < 2 ? dxy + 2 * pr + q : (q < 6 ? dco + 4 * pr + (q - 2) : drgb + 4 * pr + (q - 6));
  atomicAdd(dst, x);
}

__device__ __forceinline__ bool box_misses(float4 b, float x0, float x1, float y0, float y1) {
  return b.y < x0 || b.x > x1 || b.w < y0 || b.z > y1;
}

// Per-warp staging of one round of 32 records in shared memory: lane k writes
// record k, then every hit is read back as a broadcast.
struct __align__(16) Rec {
  float4 a;  // x, y, A, B
  float4 b;  // C, opacity, power floor, record id (bits)
  float4 c;  // r, g, b, unused
};

// Block index -> (unit, tile): heaviest tiles first when an order is given.
__device__ __forceinline__ void block_tile(const uint32_t* __restrict__ order, int n_tiles, int& u, int& tile) {
  uint32_t f = order ? order[blockIdx.x] : blockIdx.x;
  u = (int)(f / (uint32_t)n_tiles);
  tile = (int)(f % (uint32_t)n_tiles);
}

// Forward.  Each warp walks its tile's list on its own, 32 records per round
// (one per lane): a lane loads a record and tests its alpha box against the
// warp's pixel block; the records that hit are taken in list order, read back
// from the warp's staging area.  The next round's loads are issued before the
// current round is blended.
template <int BW>
__global__ void __launch_bounds__(TILE_PIX) k_render_fwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ vals,
                                                         const float4* __restrict__ xy,
                                                         const float4* __restrict__ conic_op,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         int n_tiles, float bg0, float bg1, float bg2,
                                                         float* __restrict__ img, float* __restrict__ final_T,
                                                         uint32_t* __restrict__ n_contrib) {
  const unsigned FULL = 0xffffffffu;
  __shared__ Rec s_rec[TILE_PIX / 32][32];
  int u, tile;
  block_tile(order, n_tiles, u, tile);
  int tx = tile % TX, ty = tile / TX;
  constexpr int BH = 32 / BW, NWX = TILE / BW;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float wx0 = (float)(tx * TILE + (w % NWX) * BW), wy0 = (float)(ty * TILE + (w / NWX) * BH);
  float wx1 = wx0 + (float)(BW - 1), wy1 = wy0 + (float)(BH - 1);
  int px = (int)wx0 + (lane % BW), py = (int)wy0 + (lane / BW);
  bool inside = px < W && py < H;
  uint2 rg = ranges[(int64_t)u * n_tiles + tile];
  int n = (int)(rg.y - rg.x);
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  int last = 0;
  bool done = !inside;
  // pixel offsets from the tile's corner, the origin of the staged record positions (rel_pos)
  float tox = (float)(tx * TILE), toy = (float)(ty * TILE);
  float fx = (float)(px - tx * TILE), fy = (float)(py - ty * TILE);
  Rec* my = &s_rec[w][0];
  uint32_t p_n = 0;
  float4 m_n = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 co_n = make_float4(0.f, 0.f, 0.f, 0.f), c_n = co_n;
  if (lane < n) { p_n = vals[rg.x + lane]; m_n = xy[p_n]; co_n = conic_op[p_n]; c_n = rgb[p_n]; }
  for (int base = 0; base < n; base += 32) {
    if (__all_sync(FULL, done)) break;
    float4 m = m_n;
    float4 co = co_n, c = c_n;
    bool valid = base + lane < n;
    int kn = base + 32 + lane;
    if (kn < n) { p_n = vals[rg.x + kn]; m_n = xy[p_n]; co_n = conic_op[p_n]; c_n = rgb[p_n]; }
    float pmin = 0.f;
    bool hit = false;
    if (valid) {
      float4 b = alpha_box(make_float2(m.x, m.y), co, pmin);
      hit = !box_misses(b, wx0, wx1, wy0, wy1);
    }
    unsigned mask = __ballot_sync(FULL, hit);
    if (hit) {
      my[lane].a = make_float4(rel_pos(m.x, m.z, tox), rel_pos(m.y, m.w, toy), co.x, co.y);
      my[lane].b = make_float4(co.z, co.w, pmin, 0.f);
      my[lane].c = c;
    }
    __syncwarp();
    while (mask) {
      int j = __ffs(mask) - 1;
      mask &= mask - 1;
      if (done) continue;
      float4 ra = my[j].a, rb = my[j].b;
      float power = splat_power(ra.z, ra.w, rb.x, ra.x - fx, ra.y - fy);
      if (power > 0.f || power < rb.z) continue;
      float alpha = fminf(ALPHA_MAX, rb.y * __expf(power));
      if (alpha < ALPHA_MIN) continue;
      float tT = T * (1.f - alpha);
      if (tT < T_MIN) { done = true; continue; }
      float4 rc = my[j].c;
      float wgt = alpha * T;
      c0 += rc.x * wgt; c1 += rc.y * wgt; c2 += rc.z * wgt;
      T = tT;
      last = base + j + 1;
    }
    __syncwarp();
  }
  if (inside) {
    int64_t plane = (int64_t)W * H;
    int64_t pix = (int64_t)py * W + px;
    float* im = img + (int64_t)u * 3 * plane;
    im[pix] = c0 + T * bg0;
    im[plane + pix] = c1 + T * bg1;
    im[2 * plane + pix] = c2 + T * bg2;
    final_T[(int64_t)u * plane + pix] = T;
    n_contrib[(int64_t)u * plane + pix] = (uint32_t)last;
  }
}

// Sum of 8 values over the warp in 9 shuffles: each butterfly level halves the
// set of values a lane carries; afterwards lane l holds the total of value
// 4 bit4(l) + 2 bit3(l) + bit2(l).
__device__ __forceinline__ float reduce8(const float* v, int lane) {
  const unsigned FULL = 0xffffffffu;
  float a[4], b[2];
  bool h = lane & 16;
  #pragma unroll
  for (int i = 0; i < 4; ++i) {
    float send = h ? v[i] : v[i + 4], keep = h ? v[i + 4] : v[i];
    a[i] = keep + __shfl_xor_sync(FULL, send, 16);
  }
  h = lane & 8;
  #pragma unroll
  for (int i = 0; i < 2; ++i) {
    float send = h ? a[i] : a[i + 2], keep = h ? a[i + 2] : a[i];
    b[i] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  h = lane & 4;
  float send = h ? b[0] : b[1], keep = h ? b[1] : b[0];
  float c = keep + __shfl_xor_sync(FULL, send, 4);
  c += __shfl_xor_sync(FULL, c, 2);
  c += __shfl_xor_sync(FULL, c, 1);
  return c;
}

// Backward.  Each warp replays its tile's list back to front from the largest
// n_contrib among its pixels, in rounds of 32 records; hits are taken in
// reverse list order.  The 9 gradient values of a record (d xy, d conic,
// d opacity, d rgb) are summed over the warp (butterfly for 8, a plain xor
// tree for the ninth) only if some lane contributed, and the lanes holding
// the totals add them to the record's gradients with one atomic instruction.
template <int BW>
__global__ void __launch_bounds__(TILE_PIX) k_render_bwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ vals,
                                                         const float4* __restrict__ xy,
                                                         const float4* __restrict__ conic_op,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         int n_tiles, float bg0, float bg1, float bg2,
                                                         const float* __restrict__ final_T,
                                                         const uint32_t* __restrict__ n_contrib,
                                                         const float* __restrict__ dimg,
                                                         const float* __restrict__ dLdT, float* __restrict__ dxy,
                                                         float* __restrict__ dco, float* __restrict__ drgb,
                                                           unsigned long long* __restrict__ fixed) {
  const unsigned FULL = 0xffffffffu;
  __shared__ Rec s_rec[TILE_PIX / 32][32];
  int u, tile;
  block_tile(order, n_tiles, u, tile);
  int tx = tile % TX, ty = tile / TX;
  constexpr int BH = 32 / BW, NWX = TILE / BW;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float wx0 = (float)(tx * TILE + (w % NWX) * BW), wy0 = (float)(ty * TILE + (w / NWX) * BH);
  float wx1 = wx0 + (float)(BW - 1), wy1 = wy0 + (float)(BH - 1);
  int px = (int)wx0 + (lane % BW), py = (int)wy0 + (lane / BW);
  bool inside = px < W && py < H;
  uint2 rg = ranges[(int64_t)u * n_tiles + tile];
  int64_t plane = (int64_t)W * H;
  int64_t pix = (int64_t)py * W + px;
  float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  float qT = 0.f;  // dL/dT_final x T_final: a blended entry adds -qT / (1 - alpha) to dL/dalpha
  int last = 0;
  if (inside) {
    T = final_T[(int64_t)u * plane + pix];
    last = (int)n_contrib[(int64_t)u * plane + pix];
    const float* d = dimg + (int64_t)u * 3 * plane;
    g0 = d[pix]; g1 = d[plane + pix]; g2 = d[2 * plane + pix];
    if (dLdT) qT = dLdT[(int64_t)u * plane + pix] * T;
  }
  int n = min(__reduce_max_sync(FULL, last), (int)(rg.y - rg.x));
  float S0 = bg0, S1 = bg1, S2 = bg2;  // colour behind the current entry
  float tox = (float)(tx * TILE), toy = (float)(ty * TILE);
  float fx = (float)(px - tx * TILE), fy = (float)(py - ty * TILE);
  Rec* my = &s_rec[w][0];
  // lanes (l & 3) == 0 hold butterfly value q(l); value 8 (d blue) is held by all lanes
  int q = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  for (int top = n; top > 0; top -= 32) {
    int base = top - 32;
    int k = base + lane;
    bool hit = false;
    if (k >= 0) {
      uint32_t p = vals[rg.x + k];
      float4 m = xy[p];
      float4 co = conic_op[p];
      float pm;
      float4 b = alpha_box(make_float2(m.x, m.y), co, pm);
      hit = !box_misses(b, wx0, wx1, wy0, wy1);
      if (hit) {
        my[lane].a = make_float4(rel_pos(m.x, m.z, tox), rel_pos(m.y, m.w, toy), co.x, co.y);
        my[lane].b = make_float4(co.z, co.w, pm, __uint_as_float(p));
        my[lane].c = rgb[p];
      }
    }
    unsigned mask = __ballot_sync(FULL, hit);
    __syncwarp();
    while (mask) {
      int j = 31 - __clz(mask);
      mask &= ~(1u << j);
      int pos = base + j;
      float v[9];
      #pragma unroll
      for (int e = 0; e < 9; ++e) v[e] = 0.f;
      bool contrib = false;
      float4 ra = my[j].a, rb = my[j].b;
      if (pos < last) {
        float dx = ra.x - fx, dy = ra.y - fy;
        float A = ra.z, B = ra.w, Cc = rb.x, op = rb.y;
        float power = splat_power(A, B, Cc, dx, dy);
        if (power <= 0.f && power >= rb.z) {
          float G = __expf(power);
          float araw = op * G;
          bool clamped = araw > ALPHA_MAX;
          float alpha = clamped ? ALPHA_MAX : araw;
          if (alpha >= ALPHA_MIN) {
            contrib = true;
            float4 rc = my[j].c;
            T = __fdividef(T, 1.f - alpha);  // transmittance in front of this entry
            float wgt = alpha * T;
            v[6] = wgt * g0; v[7] = wgt * g1; v[8] = wgt * g2;
            float dalpha = T * ((rc.x - S0) * g0 + (rc.y - S1) * g1 + (rc.z - S2) * g2);
            if (qT != 0.f) dalpha -= __fdividef(qT, 1.f - alpha);
            S0 = alpha * rc.x + (1.f - alpha) * S0;
            S1 = alpha * rc.y + (1.f - alpha) * S1;
            S2 = alpha * rc.z + (1.f - alpha) * S2;
            if (!clamped) {
              v[5] = G * dalpha;
              float dp = araw * dalpha;
              v[2] = -0.5f * dx * dx * dp;
              v[3] = -dx * dy * dp;
              v[4] = -0.5f * dy * dy * dp;
              v[0] = -(A * dx + B * dy) * dp;
              v[1] = -(Cc * dy + B * dx) * dp;
            }
          }
        }
      }
      unsigned cm = __ballot_sync(FULL, contrib);
      if (cm) {
        int64_t pr = (int64_t)__float_as_uint(rb.w);
        if ((cm & (cm - 1)) == 0) {
          // a single contributing lane: no reduction
          if (contrib) add_lane(dxy, dco, drgb, fixed, pr, v);
        } else {
          float tot = reduce8(v, lane);
          float e8 = v[8];
          #pragma unroll
          for (int o = 16; o > 0; o >>= 1) e8 += __shfl_xor_sync(FULL, e8, o);
          if ((lane & 3) == 0) {
            add_one(dxy, dco, drgb, fixed, pr, q, tot);
          } else if (lane == 1) {
            add_one(dxy, dco, drgb, fixed, pr, 8, e8);
          }
        }
      }
    }
    __syncwarp();
  }
}

// Bits of the 4x4 pixel blocks that a warp's BW x (32/BW) pixel block overlaps.
template <int BW>
__device__ __forceinline__ uint32_t warp_block_bits(int w) {
  constexpr int BH = 32 / BW, NWX = TILE / BW;
  int ox = (w % NWX) * BW, oy = (w / NWX) * BH;
  uint32_t bits = 0;
  #pragma unroll
  for (int by = 0; by < 4; ++by)
    #pragma unroll
    for (int bx = 0; bx < 4; ++bx)
      if (4 * bx <= ox + BW - 1 && 4 * bx + 3 >= ox && 4 * by <= oy + BH - 1 && 4 * by + 3 >= oy)
        bits |= 1u << (4 * by + bx);
  return bits;
}

// Transpose of a 32 x 32 bit matrix held one row per lane: bit j of the
// result in lane p is bit p of lane j's word (five butterfly exchanges of
// 16-, 8-, 4-, 2- and 1-bit blocks).
__device__ __forceinline__ uint32_t transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
  const uint32_t MS[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
  #pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int s = 16 >> k;
    const uint32_t m = MS[k];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? (((y & ~m) >> s) | (x & ~m)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

// Lanes of a warp's pixel block (bw x 32 / bw pixels from tile-local origin
// (ox, oy), lane = row bw + column) whose pixel centre lies in a record's
// alpha >= 1/255 box (alpha_box: conservative, so every pixel outside it has
// alpha < 1/255 and would be skipped by the blend).  (rx, ry): the record's
// tile-local position; co: conic and opacity.
__device__ __forceinline__ uint32_t hit_lanes(float rx, float ry, float4 co, float ox, float oy, int bw) {
  float pm;
  const float4 b = alpha_box(make_float2(rx, ry), co, pm);
  if (!(b.x <= b.y)) return 0u;
  const int bh = 32 / bw;
  const float c0 = fmaxf(ceilf(b.x - ox), 0.f), c1 = fminf(floorf(b.y - ox), (float)(bw - 1));
  const float r0 = fmaxf(ceilf(b.z - oy), 0.f), r1 = fminf(floorf(b.w - oy), (float)(bh - 1));
  if (!(c0 <= c1) || !(r0 <= r1)) return 0u;
  const int lo = (int)c0, rl = (int)r0, rh = (int)r1;
  const uint32_t cm = ((2u << ((int)c1 - lo)) - 1u) << lo;
  uint32_t m = 0u;
  for (int r = rl; r <= rh; ++r) m |= cm << (r * bw);
  return m;
}

// Rounds with at least this many hits walk per-lane hit lists: each lane
// takes, in list order, only the hits whose alpha box reaches its pixel
// (forward walk; reverse replay).  Below them the box and the transpose cost
// more than the hits they spare (10M Gaussians at 1080p, thresholds swept
// over 1-24: 12 and 8 were fastest).
constexpr int HIT_LISTS_FWD = 12;
constexpr int HIT_LISTS_BWD = 8;

// Front-to-back walk of list entries [beg, end) (indices from the list's
// start `off`) for one warp's pixel block, compositing into (T, c, last) of
// the lanes that are not done; a lane whose transmittance would fall below
// T_MIN stops (done).  A warp reads 2 bytes (mask) and 4 bytes (record id)
// per entry, two rounds ahead, and gathers the records of its hits one round
// ahead; the blend itself is that of k_render_fwd.
// With LOCAL, it also accumulates this walk's own partial (transmittance tl and
// colour cl from tl = 1, cl = 0: the walk's contribution per unit incoming T),
// which the checkpoints' colour-behind terms are composed from.
struct LocalAcc {
  float t, c0, c1, c2;
};

template <bool LOCAL = false>
__device__ __forceinline__ void walk_fwd(const uint32_t* __restrict__ vals, const uint16_t* __restrict__ masks,
                                         const float4* __restrict__ xy, const float4* __restrict__ conic_op,
                                         const float4* __restrict__ rgb, uint32_t off, int beg, int end,
                                         uint32_t wbits, float tox, float toy, float fx, float fy, Rec* my, float& T,
                                         float& c0, float& c1, float& c2, int& last, bool& done,
                                         LocalAcc* loc = nullptr) {
  const unsigned FULL = 0xffffffffu;
  int lane = threadIdx.x & 31;
  // the warp's pixel block: tile-local origin and width
  const float ox = __shfl_sync(FULL, fx, 0), oy = __shfl_sync(FULL, fy, 0);
  const int bw = __popc(__ballot_sync(FULL, fy == oy));
  bool h1 = false;
  float4 m1 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 co1 = make_float4(0.f, 0.f, 0.f, 0.f), cc1 = co1;
  uint32_t mk2 = 0, pk2 = 0;
  if (beg + lane < end) {
    uint32_t mk = masks[off + beg + lane];
    if (mk & wbits) {
      uint32_t pk = vals[off + beg + lane];
      h1 = true; m1 = xy[pk]; co1 = conic_op[pk]; cc1 = rgb[pk];
    }
  }
  if (beg + 32 + lane < end) { mk2 = masks[off + beg + 32 + lane]; pk2 = vals[off + beg + 32 + lane]; }
  for (int base = beg; base < end; base += 32) {
    if (__all_sync(FULL, done)) break;
    bool hit = h1;
    float4 m = m1;
    float4 co = co1, c = cc1;
    h1 = (mk2 & wbits) != 0;
    if (h1) { m1 = xy[pk2]; co1 = conic_op[pk2]; cc1 = rgb[pk2]; }
    int k2 = base + 64 + lane;
    mk2 = 0;
    if (k2 < end) { mk2 = masks[off + k2]; pk2 = vals[off + k2]; }
    unsigned mask = __ballot_sync(FULL, hit);
    const float rx = rel_pos(m.x, m.z, tox), ry = rel_pos(m.y, m.w, toy);
    if (hit) {
      my[lane].a = make_float4(rx, ry, co.x, co.y);
      my[lane].b = make_float4(co.z, co.w, c.w, 0.f);
      my[lane].c = c;
    }
    __syncwarp();
    // hits two at a time: both alphas are evaluated independently (more independent instructions
    // in flight per warp), then composited in list order
    auto hit_alpha = [&](int j) -> float {  // 0 when the record cannot blend at this pixel
      float4 ra = my[j].a, rb = my[j].b;
      float power = splat_power(ra.z, ra.w, rb.x, ra.x - fx, ra.y - fy);
      if (power > 0.f || power < rb.z) return 0.f;
      return fminf(ALPHA_MAX, rb.y * __expf(power));
    };
    auto composite = [&](int j, float alpha) {
      if (done || alpha < ALPHA_MIN) return;
      float tT = T * (1.f - alpha);
      if (tT < T_MIN) { done = true; return; }
      float4 rc = my[j].c;
      float wgt = alpha * T;
      c0 += rc.x * wgt; c1 += rc.y * wgt; c2 += rc.z * wgt;
      T = tT;
      last = base + j + 1;
      if (LOCAL) {
        float lw = alpha * loc->t;
        loc->c0 += rc.x * lw; loc->c1 += rc.y * lw; loc->c2 += rc.z * lw;
        loc->t *= 1.f - alpha;
      }
    };
    if (__popc(mask) >= HIT_LISTS_FWD) {
      // per-lane hit lists: bit j of `mine` = hit j's alpha box reaches this lane's pixel
      uint32_t mine = transpose32(hit ? hit_lanes(rx, ry, co, ox, oy, bw) : 0u);
      while (mine && !done) {
        int j1 = __ffs(mine) - 1;
        mine &= mine - 1;
        bool two = mine != 0u;
        int j2 = two ? __ffs(mine) - 1 : j1;
        if (two) mine &= mine - 1;
        float a1 = hit_alpha(j1);
        float a2 = two ? hit_alpha(j2) : 0.f;
        composite(j1, a1);
        if (two) composite(j2, a2);
      }
    } else {
      while (mask) {
        int j1 = __ffs(mask) - 1;
        mask &= mask - 1;
        bool two = mask != 0u;
        int j2 = two ? __ffs(mask) - 1 : j1;
        if (two) mask &= mask - 1;
        float a1 = hit_alpha(j1);
        float a2 = two ? hit_alpha(j2) : 0.f;
        composite(j1, a1);
        if (two) composite(j2, a2);
      }
    }
    __syncwarp();
  }
}

// ---- scheduled forward: chunk-parallel compositing in three passes
//
// Per pixel, front-to-back compositing over a list is a product of (1 - alpha)
// factors and a sum of colours weighted by the running product, so chunks of
// K entries can be composited independently from T = 1 and combined:
// C += T C_c, T *= T_c.  The early stop is the only order-dependent decision:
// a pixel whose (T T_c) would fall below T_MIN, or whose chunk stopped on its
// own, stops inside that chunk, which is then walked again from the true
// incoming state.
//   pass 1 (chunk jobs):   partial (T_c, C_c, last_c | stop) of every chunk;
//   pass 2 (list warps):   combine in order, find each pixel's stop chunk c*,
//                          write the checkpoints in front of chunks <= c*,
//                          finish the pixels that never stop;
//   pass 3 (chunk jobs):   walk chunk c* again for the pixels that stop there,
//                          write their final state and remaining checkpoints.
// Per pixel the blended entries and the stop decision are those of the
// sequential walk; the combine changes only the rounding order of T and C.
constexpr uint32_t STOP_BIT = 0x80000000u;  // chunk partial: the pixel stopped inside the chunk
constexpr uint32_t REWALK_BIT = 0x80000000u;  // n_contrib between passes 2 and 3: stop chunk pending,
                                             // the stop chunk c* in the bits below it

// The warp's pixel of (list o, block w) and its geometry.
template <int BW>
struct PixelOf {
  int u, tile, tx, ty, px, py, pix_local;
  bool inside;
  uint32_t wbits;  // the 4x4 blocks of the warp's pixels
  __device__ __forceinline__ PixelOf(const uint32_t* __restrict__ order, int o, int w, int n_tiles, int TX, int W,
                                     int H) {
    uint32_t f = order[o];
    u = (int)(f / (uint32_t)n_tiles);
    tile = (int)(f % (uint32_t)n_tiles);
    tx = tile % TX;
    ty = tile / TX;
    constexpr int BH = 32 / BW, NWX = TILE / BW;
    int lane = threadIdx.x & 31;
    px = tx * TILE + (w % NWX) * BW + (lane % BW);
    py = ty * TILE + (w / NWX) * BH + (lane / BW);
    pix_local = (py - ty * TILE) * TILE + (px - tx * TILE);
    inside = px < W && py < H;
    wbits = warp_block_bits<BW>(w);
  }
};

// Pass 1: job (list o, chunk c, block w) composites entries [c K, min((c+1) K, L))
// from T = 1.  A list of one chunk is final here.  Otherwise chunk 0's state
// (exact: nothing lies in front of it) goes to img (colour without
// background), final_T and n_contrib (| STOP_BIT), chunk c >= 1's partial to
// checkpoint slot c - 1 and chunk_last.
template <int BW>
__global__ void __launch_bounds__(32) k_render_fwd_m(const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ order,
                                                           const uint32_t* __restrict__ job_base,
                                                           const uint32_t* __restrict__ jobs, int K, int NT,
                                                           float4* __restrict__ ckpt,
                                                           uint32_t* __restrict__ chunk_last,
                                                           const uint32_t* __restrict__ vals,
                                                           const uint16_t* __restrict__ masks,
                                                           const float4* __restrict__ xy,
                                                           const float4* __restrict__ conic_op,
                                                           const float4* __restrict__ rgb, int W, int H, int TX,
                                                           int n_tiles, float bg0, float bg1, float bg2,
                                                           float* __restrict__ img, float* __restrict__ final_T,
                                                           uint32_t* __restrict__ n_contrib,
    uint32_t* __restrict__ ticket) {
  __shared__ Rec s_rec[32];
  // the resident warps take the (chunk job, pixel block) units from a ticket counter (zeroed before
  // the launch), the next ticket fetched while a unit runs: no block of a grid sized for the capacity
  // sits idle, and units of very different cost still spread as they finish
  const uint32_t total = job_base[NT] * 8u;
  auto job = [&](uint32_t vb) {
    uint32_t jid = vb >> 3;
    int w = (int)(vb & 7u);
    int o = (int)jobs[2 * (int64_t)jid], ch = (int)jobs[2 * (int64_t)jid + 1];
    PixelOf<BW> P(order, o, w, n_tiles, TX, W, H);
    int nch = (int)(job_base[o + 1] - job_base[o]);
    uint2 rg = ranges[(int64_t)P.u * n_tiles + P.tile];
    int L = (int)(rg.y - rg.x);
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    int last = 0;
    bool done = !P.inside;
    walk_fwd(vals, masks, xy, conic_op, rgb, rg.x, ch * K, min(ch * K + K, L), P.wbits, (float)(P.tx * TILE),
             (float)(P.ty * TILE), (float)(P.px - P.tx * TILE), (float)(P.py - P.ty * TILE), s_rec, T, c0, c1, c2,
             last, done);
    if (!P.inside) return;
    int64_t plane = (int64_t)W * H;
    int64_t pix = (int64_t)P.py * W + P.px;
    float* im = img + (int64_t)P.u * 3 * plane;
    if (nch == 1 || ch == 0) {
      bool fin = nch == 1;
      im[pix] = fin ? c0 + T * bg0 : c0;
      im[plane + pix] = fin ? c1 + T * bg1 : c1;
      im[2 * plane + pix] = fin ? c2 + T * bg2 : c2;
      final_T[(int64_t)P.u * plane + pix] = T;
      n_contrib[(int64_t)P.u * plane + pix] = (uint32_t)last | (!fin && done ? STOP_BIT : 0u);
    } else {
      int64_t slot = ((int64_t)job_base[o] - o + ch - 1) * TILE_PIX + P.pix_local;
      ckpt[slot] = make_float4(T, c0, c1, c2);
      chunk_last[slot] = (uint32_t)last | (done ? STOP_BIT : 0u);
    }
  };
  const bool lead = (threadIdx.x & 31) == 0;
  uint32_t vb = __shfl_sync(0xffffffffu, lead ? atomicAdd(ticket, 1u) : 0u, 0);
  while (vb < total) {
    uint32_t nxt = lead ? atomicAdd(ticket, 1u) : 0u;
    job(vb);
    vb = __shfl_sync(0xffffffffu, nxt, 0);
  }
}

// Pass 2: one warp per (list, block) in tile order.  Empty lists give the
// background.  For lists of several chunks, the state in front of chunk c is
// (T, C); the chunk's partial is applied when it shows no stop and
// T T_c >= T_MIN (then no entry of the chunk can stop the pixel), and
// otherwise chunk c is the pixel's stop chunk c*.  T in front of each
// boundary up to c* goes to chunk_last (the backward's checkpoints take it
// from there).  Pixels that never stop are final here; pixels with c* >= 1
// leave their state in front of c* in img / final_T, (c* | REWALK_BIT) in
// n_contrib and their last contributing position in chunk_last at c*'s slot
// for pass 3.  The per-chunk loads are issued CB chunks at a time: for lists
// of hundreds of chunks the walk is otherwise one load latency per chunk.
constexpr int CB = 4;

// The combine of one pixel (pass 2), for a list of nch >= 2 chunks; cstar
// receives the pixel's stop chunk (-1: none, or a stop inside chunk 0).
template <int BW>
__device__ __forceinline__ void combine_pixel(const PixelOf<BW>& P, int o, int nch, int64_t plane, int64_t pix,
                                              float* im, float* fT, uint32_t* nc, float4* __restrict__ ckpt,
                                              uint32_t* __restrict__ chunk_last,
                                              const uint32_t* __restrict__ job_base, float bg0, float bg1, float bg2,
                                              int& cstar) {
  float c0 = im[pix], c1 = im[plane + pix], c2 = im[2 * plane + pix];
  float T = fT[pix];
  uint32_t lw0 = nc[pix];
  int last = (int)(lw0 & ~STOP_BIT);
  bool done = (lw0 & STOP_BIT) != 0u;  // a stop in chunk 0 is exact
  int64_t cp0 = (int64_t)job_base[o] - o;
  float4* cpp = ckpt + cp0 * TILE_PIX + P.pix_local;       // slot of boundary b: cpp[(b - 1) * TILE_PIX]
  uint32_t* clp = chunk_last + cp0 * TILE_PIX + P.pix_local;
  for (int cb = 1; cb < nch && cstar < 0; cb += CB) {
    uint32_t lwv[CB];
    float4 ptv[CB];
    #pragma unroll
    for (int q = 0; q < CB; ++q) {
      int c = cb + q;
      if (c < nch) {
        lwv[q] = clp[(int64_t)(c - 1) * TILE_PIX];
        if (!done) ptv[q] = cpp[(int64_t)(c - 1) * TILE_PIX];
      }
    }
    #pragma unroll
    for (int q = 0; q < CB; ++q) {
      int c = cb + q;
      if (c >= nch || cstar >= 0) break;
      clp[(int64_t)(c - 1) * TILE_PIX] = __float_as_uint(T);  // T in front of chunk c (final once done)
      if (done) continue;
      float4 pt = ptv[q];
      float Tn = T * pt.x;
      if ((lwv[q] & STOP_BIT) == 0u && !(Tn < T_MIN)) {
        c0 += T * pt.y; c1 += T * pt.z; c2 += T * pt.w;
        T = Tn;
        uint32_t lc = lwv[q] & ~STOP_BIT;
        if (lc) last = (int)lc;
      } else {
        cstar = c;  // pass 3 walks chunk c for this pixel and writes the rest
      }
    }
  }
  if (cstar >= 1) {
    // boundaries in front of the stop chunk: S_b = A_b + B_b S_c* (pass 3 knows S_c*)
    float A0 = 0.f, A1 = 0.f, A2 = 0.f, B = 1.f;
    for (int bb = cstar - 1; bb >= 1; bb -= CB) {
      float4 ptv[CB];
      #pragma unroll
      for (int q = 0; q < CB; ++q)
        if (bb - q >= 1) ptv[q] = cpp[(int64_t)(bb - q - 1) * TILE_PIX];
      #pragma unroll
      for (int q = 0; q < CB; ++q) {
        if (bb - q < 1) break;
        float4 pt = ptv[q];
        A0 = pt.y + pt.x * A0; A1 = pt.z + pt.x * A1; A2 = pt.w + pt.x * A2;
        B = pt.x * B;
        cpp[(int64_t)(bb - q - 1) * TILE_PIX] = make_float4(B, A0, A1, A2);
      }
    }
    im[pix] = c0; im[plane + pix] = c1; im[2 * plane + pix] = c2;
    fT[pix] = T;
    clp[(int64_t)(cstar - 1) * TILE_PIX] = (uint32_t)last;  // pass 3 reads it and puts T back
    nc[pix] = (uint32_t)cstar | REWALK_BIT;
  } else {
    // checkpoint b: (T in front of chunk b, colour behind boundary b per unit T there), the chunks
    // from b to the stop composited back to front over the background (a pixel that stopped in
    // chunk 0 has the background behind every boundary)
    int stop_at = done ? 0 : nch;
    float S0 = bg0, S1 = bg1, S2 = bg2;
    for (int bb = nch - 1; bb >= 1; bb -= CB) {
      float4 ptv[CB];
      uint32_t tv[CB];
      #pragma unroll
      for (int q = 0; q < CB; ++q) {
        int b = bb - q;
        if (b >= 1) {
          if (b <= stop_at) ptv[q] = cpp[(int64_t)(b - 1) * TILE_PIX];
          tv[q] = clp[(int64_t)(b - 1) * TILE_PIX];
        }
      }
      #pragma unroll
      for (int q = 0; q < CB; ++q) {
        int b = bb - q;
        if (b < 1) break;
        if (b <= stop_at) {
          float4 pt = ptv[q];
          S0 = pt.y + pt.x * S0; S1 = pt.z + pt.x * S1; S2 = pt.w + pt.x * S2;
        }
        cpp[(int64_t)(b - 1) * TILE_PIX] = make_float4(__uint_as_float(tv[q]), S0, S1, S2);
      }
    }
    im[pix] = c0 + T * bg0;
    im[plane + pix] = c1 + T * bg1;
    im[2 * plane + pix] = c2 + T * bg2;
    fT[pix] = T;
    nc[pix] = (uint32_t)last;
  }
}

template <int BW>
__global__ void __launch_bounds__(32) k_render_fwd_combine(const uint2* __restrict__ ranges,
                                                                 const uint32_t* __restrict__ order,
                                                                 const uint32_t* __restrict__ job_base, int K,
                                                                 float4* __restrict__ ckpt,
                                                                 uint32_t* __restrict__ chunk_last, int W, int H,
                                                                 int TX, int n_tiles, float bg0, float bg1, float bg2,
                                                                 float* __restrict__ img, float* __restrict__ final_T,
                                                                 uint32_t* __restrict__ n_contrib,
                                                                 uint32_t* __restrict__ queue, uint32_t qcap) {
  int o = (int)(blockIdx.x >> 3), w = (int)(blockIdx.x & 7u);
  int nch = (int)(job_base[o + 1] - job_base[o]);
  if (nch == 1) return;
  PixelOf<BW> P(order, o, w, n_tiles, TX, W, H);
  int64_t plane = (int64_t)W * H;
  int64_t pix = (int64_t)P.py * W + P.px;
  float* im = img + (int64_t)P.u * 3 * plane;
  float* fT = final_T + (int64_t)P.u * plane;
  uint32_t* nc = n_contrib + (int64_t)P.u * plane;
  if (nch == 0) {  // the whole warp returns here
    if (P.inside) {
      im[pix] = bg0; im[plane + pix] = bg1; im[2 * plane + pix] = bg2;
      fT[pix] = 1.f;
      nc[pix] = 0u;
    }
    return;
  }
  int cstar = -1;
  if (P.inside) combine_pixel(P, o, nch, plane, pix, im, fT, nc, ckpt, chunk_last, job_base, bg0, bg1, bg2, cstar);
  // queue the units pass 3 walks: one (stop chunk, pixel block) per distinct stop chunk of the warp's pixels
  int key = cstar >= 1 ? cstar : -1;
  unsigned peers = __match_any_sync(0xffffffffu, key);
  if (key >= 1 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    uint32_t slot = atomicAdd(queue + qcap, 1u);
    queue[slot] = ((job_base[o] + (uint32_t)key) << 3) | (uint32_t)w;
  }
}

// Pass 3: the units pass 2 queued, (list o, chunk c, block w) with some pixel
// of block w stopping in chunk c: walks chunk c again for those pixels from
// the state pass 2 left, and writes their final image, final_T, n_contrib and
// the checkpoints after c (final state).  A resident grid takes the queued
// units from a ticket counter (zeroed before the launch), so no block is
// launched for a chunk in which nothing stops.  Bounded to 64 registers (32
// resident warps per SM, the one-warp block limit): the body needs ~114 and
// spills ~200 bytes of its checkpoint loops, which costs less than the
// occupancy it gains (forward 1.69 -> 1.63 ms at 10M/1080p).
template <int BW>
__global__ void __launch_bounds__(32, 32) k_render_fwd_stop(const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ order,
                                                              const uint32_t* __restrict__ job_base,
                                                              const uint32_t* __restrict__ jobs, int K,
                                                              float4* __restrict__ ckpt,
                                                              uint32_t* __restrict__ chunk_last,
                                                              const uint32_t* __restrict__ vals,
                                                              const uint16_t* __restrict__ masks,
                                                              const float4* __restrict__ xy,
                                                              const float4* __restrict__ conic_op,
                                                              const float4* __restrict__ rgb, int W, int H, int TX,
                                                              int n_tiles, float bg0, float bg1, float bg2,
                                                              float* __restrict__ img, float* __restrict__ final_T,
                                                              uint32_t* __restrict__ n_contrib,
                                                              const uint32_t* __restrict__ queue, uint32_t qcap,
                                                              uint32_t* __restrict__ ticket) {
  __shared__ Rec s_rec[32];
  const uint32_t total = queue[qcap];
  auto job = [&](uint32_t ent) {
  uint32_t jid = ent >> 3;
  int o = (int)jobs[2 * (int64_t)jid], ch = (int)jobs[2 * (int64_t)jid + 1];
  if (ch == 0) return;
  int nch = (int)(job_base[o + 1] - job_base[o]);
  int w = (int)(ent & 7u);
  PixelOf<BW> P(order, o, w, n_tiles, TX, W, H);
  uint2 rg = ranges[(int64_t)P.u * n_tiles + P.tile];
  int L = (int)(rg.y - rg.x);
  int64_t plane = (int64_t)W * H;
  int64_t pix = (int64_t)P.py * W + P.px;
  float* im = img + (int64_t)P.u * 3 * plane;
  float* fT = final_T + (int64_t)P.u * plane;
  uint32_t* nc = n_contrib + (int64_t)P.u * plane;
  bool mine = false;
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  int last = 0;
  int64_t cp0 = (int64_t)job_base[o] - o;
  if (P.inside) {
    uint32_t lw = nc[pix];
    mine = (lw & REWALK_BIT) != 0u && (int)(lw & ~REWALK_BIT) == ch;
    if (mine) {
      last = (int)chunk_last[(cp0 + ch - 1) * TILE_PIX + P.pix_local];  // left there by pass 2
      c0 = im[pix]; c1 = im[plane + pix]; c2 = im[2 * plane + pix];
      T = fT[pix];
    }
  }
  // only the 4x4 pixel blocks of this warp's walking pixels: records whose block mask misses them
  // cannot reach those pixels
  uint32_t my_block = mine ? 1u << (4 * ((P.py - P.ty * TILE) >> 2) + ((P.px - P.tx * TILE) >> 2)) : 0u;
  uint32_t wbits = __reduce_or_sync(0xffffffffu, my_block);
  if (!wbits) return;
  bool done = !mine;
  // walk chunk c* (and, should the pixel not stop there after all, the chunks after it), keeping each
  // walked chunk's partial and the T in front of it; chunks behind the stop get the identity partial
  int c = ch;
  for (; c < nch; ++c) {
    LocalAcc la = {1.f, 0.f, 0.f, 0.f};
    float Tin = T;
    walk_fwd<true>(vals, masks, xy, conic_op, rgb, rg.x, c * K, min(c * K + K, L), wbits, (float)(P.tx * TILE),
                   (float)(P.ty * TILE), (float)(P.px - P.tx * TILE), (float)(P.py - P.ty * TILE), s_rec, T, c0, c1,
                   c2, last, done, &la);
    if (mine) {
      int64_t slot = (cp0 + c - 1) * TILE_PIX + P.pix_local;
      ckpt[slot] = make_float4(la.t, la.c0, la.c1, la.c2);
      chunk_last[slot] = __float_as_uint(Tin);
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  if (!mine) return;
  // checkpoints: (T in front of boundary b, colour behind it per unit T), composited back to front
  float4* cpp = ckpt + cp0 * TILE_PIX + P.pix_local;  // slot of boundary b: cpp[(b - 1) * TILE_PIX]
  const uint32_t* clp = chunk_last + cp0 * TILE_PIX + P.pix_local;
  for (int b = nch - 1; b > c; --b)
    cpp[(int64_t)(b - 1) * TILE_PIX] = make_float4(T, bg0, bg1, bg2);  // behind the stop: final state
  float S0 = bg0, S1 = bg1, S2 = bg2;
  for (int bb = min(c, nch - 1); bb >= ch; bb -= CB) {  // walked chunks, back to front
    float4 ptv[CB];
    uint32_t tv[CB];
    #pragma unroll
    for (int q = 0; q < CB; ++q)
      if (bb - q >= ch) { ptv[q] = cpp[(int64_t)(bb - q - 1) * TILE_PIX]; tv[q] = clp[(int64_t)(bb - q - 1) * TILE_PIX]; }
    #pragma unroll
    for (int q = 0; q < CB; ++q) {
      if (bb - q < ch) break;
      float4 pt = ptv[q];
      S0 = pt.y + pt.x * S0; S1 = pt.z + pt.x * S1; S2 = pt.w + pt.x * S2;
      cpp[(int64_t)(bb - q - 1) * TILE_PIX] = make_float4(__uint_as_float(tv[q]), S0, S1, S2);
    }
  }
  for (int bb = 1; bb < ch; bb += CB) {  // in front of c*: S_b = A_b + B_b S_c* as left by pass 2
    float4 abv[CB];
    uint32_t tv[CB];
    #pragma unroll
    for (int q = 0; q < CB; ++q)
      if (bb + q < ch) { abv[q] = cpp[(int64_t)(bb + q - 1) * TILE_PIX]; tv[q] = clp[(int64_t)(bb + q - 1) * TILE_PIX]; }
    #pragma unroll
    for (int q = 0; q < CB; ++q) {
      if (bb + q >= ch) break;
      float4 ab = abv[q];
      cpp[(int64_t)(bb + q - 1) * TILE_PIX] = make_float4(__uint_as_float(tv[q]), ab.y + ab.x * S0,
                                                          ab.z + ab.x * S1, ab.w + ab.x * S2);
    }
  }
  im[pix] = c0 + T * bg0;
  im[plane + pix] = c1 + T * bg1;
  im[2 * plane + pix] = c2 + T * bg2;
  fT[pix] = T;
  nc[pix] = (uint32_t)last;
  };
  const bool lead = (threadIdx.x & 31) == 0;
  uint32_t e = __shfl_sync(0xffffffffu, lead ? atomicAdd(ticket, 1u) : 0u, 0);
  while (e < total) {
    uint32_t nxt = lead ? atomicAdd(ticket, 1u) : 0u;
    job(queue[e]);
    e = __shfl_sync(0xffffffffu, nxt, 0);
  }
}


// Forward walking whole lists: one warp per (list, pixel block) in tile order
// composites its list chunk after chunk and stores (T, C) of each pixel in
// front of every interior chunk boundary (the backward's checkpoints); after
// an early exit the remaining checkpoints hold the final state.  No work
// follows a block's last stop, which suits renders whose pixels mostly stop
// near the front of their lists (opaque, trained scenes).
template <int BW>
__global__ void __launch_bounds__(32) k_render_fwd_seq(const uint2* __restrict__ ranges,
                                                             const uint32_t* __restrict__ order,
                                                             const uint32_t* __restrict__ job_base, int K,
                                                             float4* __restrict__ ckpt,
                                                             uint32_t* __restrict__ chunk_last,
                                                             const uint32_t* __restrict__ vals,
                                                             const uint16_t* __restrict__ masks,
                                                             const float4* __restrict__ xy,
                                                             const float4* __restrict__ conic_op,
                                                             const float4* __restrict__ rgb, int W, int H, int TX,
                                                             int n_tiles, float bg0, float bg1, float bg2,
                                                             float* __restrict__ img, float* __restrict__ final_T,
                                                             uint32_t* __restrict__ n_contrib) {
  __shared__ Rec s_rec[32];
  int o = (int)(blockIdx.x >> 3), w = (int)(blockIdx.x & 7u);
  PixelOf<BW> P(order, o, w, n_tiles, TX, W, H);
  uint2 rg = ranges[(int64_t)P.u * n_tiles + P.tile];
  int L = (int)(rg.y - rg.x);
  int nch = (int)(job_base[o + 1] - job_base[o]);
  int64_t cp0 = (int64_t)job_base[o] - o;
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  int last = 0;
  bool done = !P.inside;
  for (int c = 0; c < max(nch, 1); ++c) {
    LocalAcc la = {1.f, 0.f, 0.f, 0.f};
    float Tin = T;
    walk_fwd<true>(vals, masks, xy, conic_op, rgb, rg.x, c * K, min(c * K + K, L), P.wbits, (float)(P.tx * TILE),
                   (float)(P.ty * TILE), (float)(P.px - P.tx * TILE), (float)(P.py - P.ty * TILE), s_rec, T, c0, c1,
                   c2, last, done, &la);
    if (c > 0 && P.inside) {  // the chunk's partial and the T in front of it
      int64_t slot = (cp0 + c - 1) * TILE_PIX + P.pix_local;
      ckpt[slot] = make_float4(la.t, la.c0, la.c1, la.c2);
      chunk_last[slot] = __float_as_uint(Tin);
    }
  }
  if (P.inside) {
    // checkpoints: (T in front of boundary b, colour behind it per unit T), composited back to front
    float4* cpp = ckpt + cp0 * TILE_PIX + P.pix_local;  // slot of boundary b: cpp[(b - 1) * TILE_PIX]
    const uint32_t* clp = chunk_last + cp0 * TILE_PIX + P.pix_local;
    float S0 = bg0, S1 = bg1, S2 = bg2;
    for (int bb = nch - 1; bb >= 1; bb -= CB) {
      float4 ptv[CB];
      uint32_t tv[CB];
      #pragma unroll
      for (int q = 0; q < CB; ++q)
        if (bb - q >= 1) { ptv[q] = cpp[(int64_t)(bb - q - 1) * TILE_PIX]; tv[q] = clp[(int64_t)(bb - q - 1) * TILE_PIX]; }
      #pragma unroll
      for (int q = 0; q < CB; ++q) {
        if (bb - q < 1) break;
        float4 pt = ptv[q];
        S0 = pt.y + pt.x * S0; S1 = pt.z + pt.x * S1; S2 = pt.w + pt.x * S2;
        cpp[(int64_t)(bb - q - 1) * TILE_PIX] = make_float4(__uint_as_float(tv[q]), S0, S1, S2);
      }
    }
    int64_t plane = (int64_t)W * H;
    int64_t pix = (int64_t)P.py * W + P.px;
    float* im = img + (int64_t)P.u * 3 * plane;
    im[pix] = c0 + T * bg0;
    im[plane + pix] = c1 + T * bg1;
    im[2 * plane + pix] = c2 + T * bg2;
    final_T[(int64_t)P.u * plane + pix] = T;
    n_contrib[(int64_t)P.u * plane + pix] = (uint32_t)last;
  }
}

// Contributing lanes up to which the scheduled backward skips the warp
// reduction of a record's nine gradient values and lets each lane issue its
// own vector atomics.  L2 absorbs these well: at 1M and 10M Gaussians per
// 1080p view every threshold from 3 to 32 was faster than the one below it;
// 16 keeps the same-address atomics of a record bounded for large splats.
constexpr int DIRECT_LANES = 16;

// Position and conic terms of one (pixel, record) pair's gradient from the
// pixel offset (dx, dy), dp = o G dL/dalpha and the conic (A, B, C):
// v = (dx, dy | dA, dB, dC) in the order add_lane expects.
__device__ __forceinline__ void pos_conic_terms(float dx, float dy, float dp, float A, float B, float Cc, float* v) {
  v[2] = -0.5f * dx * dx * dp;
  v[3] = -dx * dy * dp;
  v[4] = -0.5f * dy * dy * dp;
  v[0] = -(A * dx + B * dy) * dp;
  v[1] = -(Cc * dy + B * dx) * dp;
}

// Ring of deferred (pixel, record) pairs of the scheduled backward, per warp.
constexpr int QCAP = 64;

// Lanes 0..count-1 finish entries head .. head + count - 1 of the ring: the
// position and conic terms, then the record's three vector atomics.
__device__ __forceinline__ void bwd_queue_flush(const float4* s_q, int head, int count, int lane, float* dxy,
                                                float* dco, float* drgb) {
  if (lane < count) {
    int e = (head + lane) & (QCAP - 1);
    float4 a = s_q[e], b = s_q[QCAP + e], c = s_q[2 * QCAP + e];
    float v[5];
    pos_conic_terms(a.x, a.y, a.z, b.x, b.y, b.z, v);
    int64_t pr = (int64_t)__float_as_uint(b.w);
    atomic_add2(dxy + 2 * pr, v[0], v[1]);
    atomic_add4(dco + 4 * pr, v[2], v[3], v[4], a.w);
    atomic_add4(drgb + 4 * pr, c.x, c.y, c.z, 0.f);
  }
}

// Backward over chunk jobs: job (list, chunk c, pixel block) replays entries
// [c K, min((c + 1) K, L)) of the list back to front.  It starts from the
// forward's checkpoint at the chunk's end (T in front of it and the colour
// behind it per unit T), or from final_T and the background for the last
// chunk.  Headers two rounds ahead, hit records one round ahead, as in the
// forward.  QUEUE (float accumulation) defers the gradient terms of sparse
// hits to a per-warp ring; the deterministic mode (fixed != NULL) runs
// without it.
template <int BW, bool QUEUE>
__global__ void __launch_bounds__(32, 32) k_render_bwd_m(const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ order,
                                                           const uint32_t* __restrict__ job_base,
                                                           const uint32_t* __restrict__ jobs, int K,
                                                           const float4* __restrict__ ckpt,
                                                           const uint32_t* __restrict__ vals,
                                                           const uint16_t* __restrict__ masks,
                                                           const float4* __restrict__ xy,
                                                           const float4* __restrict__ conic_op,
                                                           const float4* __restrict__ rgb, int W, int H, int TX,
                                                           int n_tiles, int NT, float bg0, float bg1, float bg2,
                                                           const float* __restrict__ img,
                                                           const float* __restrict__ final_T,
                                                           const uint32_t* __restrict__ n_contrib,
                                                           const float* __restrict__ dimg,
                                                           const float* __restrict__ dLdT, float* __restrict__ dxy,
                                                           float* __restrict__ dco, float* __restrict__ drgb,
                                                           unsigned long long* __restrict__ fixed,
    uint32_t* __restrict__ ticket) {
  const unsigned FULL = 0xffffffffu;
  __shared__ Rec s_rec[32];
  // the resident warps take the (chunk job, pixel block) units from a ticket counter (zeroed before
  // the launch), the next ticket fetched while a unit runs: no block of a grid sized for the capacity
  // sits idle, and units of very different cost still spread as they finish
  const uint32_t total = job_base[NT] * 8u;
  auto job = [&](uint32_t vb) {
    uint32_t jid = vb >> 3;
    int w = (int)(vb & 7u);
    int o = (int)jobs[2 * (int64_t)jid], ch = (int)jobs[2 * (int64_t)jid + 1];
    uint32_t f = order[o];
    int u = (int)(f / (uint32_t)n_tiles), tile = (int)(f % (uint32_t)n_tiles);
    int nch = (int)(job_base[o + 1] - job_base[o]);
    int tx = tile % TX, ty = tile / TX;
    constexpr int BH = 32 / BW, NWX = TILE / BW;
    int lane = threadIdx.x & 31;
    int px = tx * TILE + (w % NWX) * BW + (lane % BW), py = ty * TILE + (w / NWX) * BH + (lane / BW);
    uint32_t wbits = warp_block_bits<BW>(w);
    bool inside = px < W && py < H;
    float tox = (float)(tx * TILE), toy = (float)(ty * TILE);  // origin of the staged record positions
    float lx = (float)(px - tx * TILE), ly = (float)(py - ty * TILE);
    uint2 rg = ranges[(int64_t)u * n_tiles + tile];
    int L = (int)(rg.y - rg.x);
    int cbeg = ch * K, cend = min(cbeg + K, L);
    int64_t plane = (int64_t)W * H;
    int64_t pix = (int64_t)py * W + px;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, S0 = bg0, S1 = bg1, S2 = bg2;
    float qT = 0.f;  // dL/dT_final x T_final: a blended entry adds -qT / (1 - alpha) to dL/dalpha
    int last = 0;
    if (inside) {
      last = (int)n_contrib[(int64_t)u * plane + pix];
      const float* d = dimg + (int64_t)u * 3 * plane;
      g0 = d[pix]; g1 = d[plane + pix]; g2 = d[2 * plane + pix];
      if (dLdT) qT = dLdT[(int64_t)u * plane + pix] * final_T[(int64_t)u * plane + pix];
      if (ch + 1 < nch && last > cbeg) {
        // the forward's checkpoint at the chunk's end: T there and the colour behind it per unit T
        int pix_local = (py - ty * TILE) * TILE + (px - tx * TILE);
        float4 cp = ckpt[((int64_t)job_base[o] - o + ch) * TILE_PIX + pix_local];
        T = cp.x;
        S0 = cp.y; S1 = cp.z; S2 = cp.w;
      } else {
        T = final_T[(int64_t)u * plane + pix];
      }
    }
    // entries this warp replays: [cbeg, min(cend, max over its pixels of last))
    int n = min(__reduce_max_sync(FULL, last), cend);
    Rec* my = &s_rec[0];
    int q = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    bool h1 = false;
    uint32_t p1 = 0;
    float4 m1 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 co1 = make_float4(0.f, 0.f, 0.f, 0.f), cc1 = co1;
    uint32_t mk2 = 0, pk2 = 0;
    {
      int k = n - 32 + lane;
      if (n > cbeg && k >= cbeg) {
        uint32_t mk = masks[rg.x + k];
        if (mk & wbits) {
          p1 = vals[rg.x + k];
          h1 = true; m1 = xy[p1]; co1 = conic_op[p1]; cc1 = rgb[p1];
        }
      }
      int k2 = n - 64 + lane;
      if (n - 32 > cbeg && k2 >= cbeg) { mk2 = masks[rg.x + k2]; pk2 = vals[rg.x + k2]; }
    }
    // QUEUE: pairs of hits with at most DIRECT_LANES contributing lanes go to a ring of
    // (dx, dy, dp, dopacity | A, B, C, id | dr, dg, db) entries; every 32 entries all
    // lanes finish one pair each (conic and position terms, vector atomics).  The
    // per-pixel state (T, colour behind) is still updated at the hit in list order.
    __shared__ float4 s_q[QUEUE ? 3 * QCAP : 1];
    int qh = 0, qt = 0;  // ring head and tail (warp-uniform)
    for (int top = n; top > cbeg; top -= 32) {
      int base = top - 32;
      bool hit = h1;
      uint32_t p = p1;
      float4 m = m1;
      float4 co = co1, c = cc1;
      h1 = (mk2 & wbits) != 0;
      if (h1) { p1 = pk2; m1 = xy[pk2]; co1 = conic_op[pk2]; cc1 = rgb[pk2]; }
      int k2 = top - 96 + lane;
      mk2 = 0;
      if (top - 64 > cbeg && k2 >= cbeg) { mk2 = masks[rg.x + k2]; pk2 = vals[rg.x + k2]; }
      unsigned mask = __ballot_sync(FULL, hit);
      const float rx = rel_pos(m.x, m.z, tox), ry = rel_pos(m.y, m.w, toy);
      if (hit) {
        my[lane].a = make_float4(rx, ry, co.x, co.y);
        my[lane].b = make_float4(co.z, co.w, c.w, __uint_as_float(p));
        my[lane].c = c;
      }
      __syncwarp();
      if (QUEUE && __popc(mask) >= HIT_LISTS_BWD) {
        // per-lane hit lists, back to front: bit j of `mine` = hit j's alpha box reaches this lane's
        // pixel and the entry lies in front of the pixel's last contribution; every pair goes to the ring
        uint32_t mine = transpose32(hit ? hit_lanes(rx, ry, co, (float)((w % NWX) * BW), (float)((w / NWX) * BH), BW)
                                        : 0u);
        const int upto = last - base;
        mine &= upto >= 32 ? 0xffffffffu : (upto > 0 ? (1u << upto) - 1u : 0u);
        while (__any_sync(FULL, mine != 0u)) {
          const bool act = mine != 0u;
          const int j = act ? 31 - __clz(mine) : 0;
          if (act) mine &= ~(1u << j);
          bool contrib = false;
          float dx = 0.f, dy = 0.f, dp = 0.f, v5 = 0.f, v6 = 0.f, v7 = 0.f, v8 = 0.f;
          float4 ra = my[j].a, rb = my[j].b;
          if (act) {
            dx = ra.x - lx; dy = ra.y - ly;
            float power = splat_power(ra.z, ra.w, rb.x, dx, dy);
            if (power <= 0.f && power >= rb.z) {
              float G = __expf(power);
              float araw = rb.y * G;
              bool clamped = araw > ALPHA_MAX;
              float alpha = clamped ? ALPHA_MAX : araw;
              if (alpha >= ALPHA_MIN) {
                contrib = true;
                float4 rc = my[j].c;
                T = __fdividef(T, 1.f - alpha);
                float wgt = alpha * T;
                v6 = wgt * g0; v7 = wgt * g1; v8 = wgt * g2;
                float dalpha = T * ((rc.x - S0) * g0 + (rc.y - S1) * g1 + (rc.z - S2) * g2);
                if (qT != 0.f) dalpha -= __fdividef(qT, 1.f - alpha);
                S0 = alpha * rc.x + (1.f - alpha) * S0;
                S1 = alpha * rc.y + (1.f - alpha) * S1;
                S2 = alpha * rc.z + (1.f - alpha) * S2;
                if (!clamped) {
                  v5 = G * dalpha;
                  dp = araw * dalpha;
                }
              }
            }
          }
          unsigned cm = __ballot_sync(FULL, contrib);
          if (!cm) continue;
          if (contrib) {
            int e = (qt + __popc(cm & ((1u << lane) - 1u))) & (QCAP - 1);
            s_q[e] = make_float4(dx, dy, dp, v5);
            s_q[QCAP + e] = make_float4(ra.z, ra.w, rb.x, rb.w);
            s_q[2 * QCAP + e] = make_float4(v6, v7, v8, 0.f);
          }
          qt += __popc(cm);
          if (qt - qh >= 32) {
            __syncwarp();
            bwd_queue_flush(s_q, qh, 32, lane, dxy, dco, drgb);
            qh += 32;
            __syncwarp();
          }
        }
        mask = 0u;  // every hit of the round is done
      }
      while (mask) {
        int j = 31 - __clz(mask);
        mask &= ~(1u << j);
        int pos = base + j;
        bool contrib = false;
        float dx = 0.f, dy = 0.f, dp = 0.f, v5 = 0.f, v6 = 0.f, v7 = 0.f, v8 = 0.f;
        float4 ra = my[j].a, rb = my[j].b;
        if (pos < last) {
          dx = ra.x - lx; dy = ra.y - ly;
          float power = splat_power(ra.z, ra.w, rb.x, dx, dy);
          if (power <= 0.f && power >= rb.z) {
            float G = __expf(power);
            float araw = rb.y * G;
            bool clamped = araw > ALPHA_MAX;
            float alpha = clamped ? ALPHA_MAX : araw;
            if (alpha >= ALPHA_MIN) {
              contrib = true;
              float4 rc = my[j].c;
              T = __fdividef(T, 1.f - alpha);
              float wgt = alpha * T;
              v6 = wgt * g0; v7 = wgt * g1; v8 = wgt * g2;
              float dalpha = T * ((rc.x - S0) * g0 + (rc.y - S1) * g1 + (rc.z - S2) * g2);
              if (qT != 0.f) dalpha -= __fdividef(qT, 1.f - alpha);
              S0 = alpha * rc.x + (1.f - alpha) * S0;
              S1 = alpha * rc.y + (1.f - alpha) * S1;
              S2 = alpha * rc.z + (1.f - alpha) * S2;
              if (!clamped) {  // a clamped alpha passes no gradient to opacity, conic or position
                v5 = G * dalpha;
                dp = araw * dalpha;
              }
            }
          }
        }
        unsigned cm = __ballot_sync(FULL, contrib);
        if (!cm) continue;
        int nc = __popc(cm);
        if (QUEUE && nc <= DIRECT_LANES) {
          if (contrib) {
            int e = (qt + __popc(cm & ((1u << lane) - 1u))) & (QCAP - 1);
            s_q[e] = make_float4(dx, dy, dp, v5);
            s_q[QCAP + e] = make_float4(ra.z, ra.w, rb.x, rb.w);
            s_q[2 * QCAP + e] = make_float4(v6, v7, v8, 0.f);
          }
          qt += nc;
          if (qt - qh >= 32) {
            __syncwarp();
            bwd_queue_flush(s_q, qh, 32, lane, dxy, dco, drgb);
            qh += 32;
            __syncwarp();
          }
          continue;
        }
        int64_t pr = (int64_t)__float_as_uint(rb.w);
        float v[9];
        pos_conic_terms(dx, dy, dp, ra.z, ra.w, rb.x, v);
        v[5] = v5; v[6] = v6; v[7] = v7; v[8] = v8;
        // fixed point: nine scalar int64 atomics per lane, so reduce unless one lane contributes
        if (nc <= (fixed ? 1 : DIRECT_LANES)) {
          // few contributing lanes (small splats): each issues its own three vector
          // atomics, which costs fewer instructions and atomic operations than a reduction
          if (contrib) add_lane(dxy, dco, drgb, fixed, pr, v);
        } else {
          float tot = reduce8(v, lane);
          float e8 = v[8];
          #pragma unroll
          for (int oo = 16; oo > 0; oo >>= 1) e8 += __shfl_xor_sync(FULL, e8, oo);
          if ((lane & 3) == 0) {
            add_one(dxy, dco, drgb, fixed, pr, q, tot);
          } else if (lane == 1) {
            add_one(dxy, dco, drgb, fixed, pr, 8, e8);
          }
        }
      }
      __syncwarp();
    }
    if (QUEUE && qt > qh) bwd_queue_flush(s_q, qh, qt - qh, lane, dxy, dco, drgb);
  };
  const bool lead = (threadIdx.x & 31) == 0;
  uint32_t vb = __shfl_sync(0xffffffffu, lead ? atomicAdd(ticket, 1u) : 0u, 0);
  while (vb < total) {
    uint32_t nxt = lead ? atomicAdd(ticket, 1u) : 0u;
    job(vb);
    vb = __shfl_sync(0xffffffffu, nxt, 0);
  }
}

// Tile order: heaviest lists first (counting sort of (unit, tile) by the
// bit length of the list length; order within a class is arbitrary and the
// blend results do not depend on it).
__global__ void k_order_hist(const uint2* __restrict__ ranges, int n, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s[33];
  if (threadIdx.x < 33) s[threadIdx.x] = 0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    uint2 r = ranges[i];
    uint32_t len = r.y - r.x;
    atomicAdd(&s[32 - __clz(len)], 1u);  // class 0: empty; class c: 2^(c-1) <= len < 2^c
  }
  __syncthreads();
  if (threadIdx.x < 33 && s[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_order_scatter(const uint2* __restrict__ ranges, int n, const uint32_t* __restrict__ hist,
                                uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_base[33];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int c = 32; c >= 0; --c) { s_base[c] = acc; acc += hist[c]; }  // heavy classes first
  }
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint2 r = ranges[i];
  int c = 32 - __clz(r.y - r.x);
  order[s_base[c] + atomicAdd(&cursor[c], 1u)] = (uint32_t)i;
}

// Work counters of one rendered view (diagnostic, outside any timed region):
// counts[0] = blended (pixel, record) pairs (records before n_contrib whose
// alpha reaches 1/255); counts[1] = (pixel, list entry) pairs the sequential
// front-to-back walk evaluates, up to and including the entry that stops the
// pixel; counts[2] = sum of n_contrib, the entries the reverse replay walks
// per pixel; counts[3], counts[4] = the pairs of counts[1] and counts[2]
// whose block mask reaches the pixel's 4x4 block (0 without masks): the
// (pixel, entry) pairs a walk that skips masked-out records must evaluate.
__global__ void __launch_bounds__(TILE_PIX) k_blend_pairs(const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ vals,
                                                          const float4* __restrict__ xy,
                                                          const float4* __restrict__ conic_op, int W, int H, int TX,
                                                          int n_tiles, const uint32_t* __restrict__ n_contrib,
                                                          const uint16_t* __restrict__ masks,
                                                          unsigned long long* __restrict__ counts) {
  int tile = blockIdx.x, u = blockIdx.y;
  int tx = tile % TX, ty = tile / TX;
  int px = tx * TILE + (threadIdx.x & 15), py = ty * TILE + (threadIdx.x >> 4);
  const uint32_t blk = 1u << (4 * ((threadIdx.x >> 4) >> 2) + ((threadIdx.x & 15) >> 2));
  unsigned long long c = 0, visited = 0, replay = 0, m_visited = 0, m_replay = 0;
  if (px < W && py < H) {
    uint2 rg = ranges[(int64_t)u * n_tiles + tile];
    int L = (int)(rg.y - rg.x);
    int last = (int)n_contrib[(int64_t)u * W * H + (int64_t)py * W + px];
    replay = (unsigned long long)last;
    float T = 1.f;
    int j = 0;
    for (; j < L; ++j) {
      bool in_mask = masks && (masks[rg.x + j] & blk);
      m_visited += in_mask ? 1 : 0;
      m_replay += (in_mask && j < last) ? 1 : 0;
      uint32_t p = vals[rg.x + j];
      float4 m = xy[p];
      float4 co = conic_op[p];
      float dx = rel_pos(m.x, m.z, (float)(tx * TILE)) - (float)(px - tx * TILE);
      float dy = rel_pos(m.y, m.w, (float)(ty * TILE)) - (float)(py - ty * TILE);
      float power = splat_power(co.x, co.y, co.z, dx, dy);
      if (power > 0.f) continue;
      float alpha = fminf(ALPHA_MAX, co.w * __expf(power));
      if (alpha < ALPHA_MIN) continue;
      if (j < last) ++c;
      float tT = T * (1.f - alpha);
      if (tT < T_MIN) break;
      T = tT;
    }
    visited = (unsigned long long)min(j + 1, L);
    // the remaining entries up to n_contrib count for the replay (none after a stop, which ends the list)
    for (int k = j + 1; k < min(last, L); ++k) m_replay += (masks && (masks[rg.x + k] & blk)) ? 1 : 0;
  }
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    visited += __shfl_xor_sync(0xffffffffu, visited, o);
    replay += __shfl_xor_sync(0xffffffffu, replay, o);
    m_visited += __shfl_xor_sync(0xffffffffu, m_visited, o);
    m_replay += __shfl_xor_sync(0xffffffffu, m_replay, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(&counts[0], c);
    if (visited) atomicAdd(&counts[1], visited);
    if (replay) atomicAdd(&counts[2], replay);
    if (m_visited) atomicAdd(&counts[3], m_visited);
    if (m_replay) atomicAdd(&counts[4], m_replay);
  }
}

// Deterministic mode: the int64 fixed-point sums back to the float screen-space gradients.
__global__ void k_fixed_to_grad2d(const unsigned long long* __restrict__ fixed, int64_t P, float* __restrict__ dxy,
                                  float* __restrict__ dco, float* __restrict__ drgb) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float g[9];
  #pragma unroll
  for (int q = 0; q < 9; ++q) g[q] = __ll2float_rn((long long)fixed[9 * p + q]) * (1.0f / FIX_SCALE);
  reinterpret_cast<float2*>(dxy)[p] = make_float2(g[0], g[1]);
  reinterpret_cast<float4*>(dco)[p] = make_float4(g[2], g[3], g[4], g[5]);
  reinterpret_cast<float4*>(drgb)[p] = make_float4(g[6], g[7], g[8], 0.f);
}

// Grid of a one-warp kernel whose blocks take units of work from a ticket counter: as many blocks as
// stay resident on the device, at most one per unit.
template <typename K>
unsigned resident_grid(K kernel, int64_t units) {
  int dev = 0, sms = 0, per = 0;
  if (units < 1) return 1u;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 32, 0) != cudaSuccess || sms < 1 || per < 1)
    return (unsigned)units;
  int64_t g = (int64_t)sms * per;
  return (unsigned)(g < units ? g : units);
}

// The ticket word of the scheduled blend kernels: the jobs array's last entry, which no job uses
// (a list of L entries has ceil(L / K) < L / K + 1 jobs, so there are fewer than max_jobs - 1).
inline uint32_t* sched_ticket(const gs_schedule* sched) {
  return sched->jobs + 2 * (sched->max_jobs - 1);
}

}  // namespace

int gs_render_fwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                       int width, int height, const float* bg, float* img, float* final_T, uint32_t* n_contrib,
                       int variant, const gs_schedule* sched, cudaStream_t s) {
  if (!proj || !proj->xy || !proj->conic_op || !proj->rgb || !sorted_vals || !ranges || !bg || !img ||
      !final_T || !n_contrib || n_units < 1 || n_units > GS_MAX_UNITS || width <= 0 || height <= 0 ||
      variant < 0 || variant > 2)
    return GS_ERR_INVALID;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  dim3 grid(TX * TY * n_units);
  // the re-walk queue holds at most one entry per (chunk job, pixel block); its count follows it
  const uint32_t qcap = sched ? (uint32_t)(8 * sched->max_jobs) : 0u;
#define GS_FWD(BW)                                                                                                  \
  if (sched && sched->walk_whole_lists) {                                                                          \
    k_render_fwd_seq<BW><<<dim3(grid.x * 8), 32, 0, s>>>(                                                           \
        (const uint2*)ranges, sched->tile_order, sched->job_base, sched->chunk, (float4*)sched->checkpoints,        \
        sched->chunk_last, sorted_vals, sched->block_masks, (const float4*)proj->xy, (const float4*)proj->conic_op,                    \
        (const float4*)proj->rgb, width, height, TX, TX * TY, bg[0], bg[1], bg[2], img, final_T, n_contrib);        \
  } else if (sched) {                                                                                               \
    if (cudaMemsetAsync(sched_ticket(sched), 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;          \
    k_render_fwd_m<BW><<<dim3(resident_grid(k_render_fwd_m<BW>, sched->max_jobs * 8)), 32, 0, s>>>(                 \
        (const uint2*)ranges, sched->tile_order, sched->job_base, sched->jobs, sched->chunk, (int)grid.x,            \
        (float4*)sched->checkpoints, sched->chunk_last, sorted_vals, sched->block_masks, (const float4*)proj->xy,   \
        (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height, TX, TX * TY, bg[0], bg[1], bg[2],  \
        img, final_T, n_contrib, sched_ticket(sched));                                                              \
    if (cudaMemsetAsync(sched->stop_queue + qcap, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;     \
    k_render_fwd_combine<BW><<<dim3(grid.x * 8), 32, 0, s>>>(                                                       \
        (const uint2*)ranges, sched->tile_order, sched->job_base, sched->chunk, (float4*)sched->checkpoints,        \
        sched->chunk_last, width, height, TX, TX * TY, bg[0], bg[1], bg[2], img, final_T, n_contrib,               \
        sched->stop_queue, qcap);                                                                                   \
    if (cudaMemsetAsync(sched_ticket(sched), 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;          \
    k_render_fwd_stop<BW><<<dim3(resident_grid(k_render_fwd_stop<BW>, (int64_t)qcap)), 32, 0, s>>>(                 \
        (const uint2*)ranges, sched->tile_order, sched->job_base, sched->jobs, sched->chunk,                        \
        (float4*)sched->checkpoints, sched->chunk_last, sorted_vals, sched->block_masks, (const float4*)proj->xy,    \
        (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height, TX, TX * TY, bg[0], bg[1], bg[2],  \
        img, final_T, n_contrib, sched->stop_queue, qcap, sched_ticket(sched));                                     \
  } else                                                                                                            \
    k_render_fwd<BW><<<grid, TILE_PIX, 0, s>>>((const uint2*)ranges, nullptr, sorted_vals, (const float4*)proj->xy, \
                                               (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height, \
                                               TX, TX * TY, bg[0], bg[1], bg[2], img, final_T, n_contrib)
  if (variant == 0) { GS_FWD(8); } else if (variant == 1) { GS_FWD(16); } else { GS_FWD(4); }
#undef GS_FWD
  return gs_check_launch();
}

GS_API int gs_render_fwd(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                         int width, int height, const float* bg, float* img, float* final_T, uint32_t* n_contrib,
                         int variant, const gs_schedule* sched, gs_stream_t stream) {
  GS_RANGE("gs_render_fwd");
  return gs_render_fwd_impl(proj, sorted_vals, ranges, n_units, width, height, bg, img, final_T, n_contrib, variant,
                            sched, (cudaStream_t)stream);
}

int gs_blend_bwd_impl(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                      int width, int height, const float* bg, const float* final_T, const uint32_t* n_contrib,
                      const float* dL_dimg, const float* dL_dT, const gs_grad2d* g2d, int64_t n_proj, int variant,
                      const gs_schedule* sched, const float* img, cudaStream_t s) {
  if (!proj || !proj->xy || !proj->conic_op || !proj->rgb || !sorted_vals || !ranges || !bg || !final_T ||
      !n_contrib || !dL_dimg || !g2d || !g2d->dxy || !g2d->dconic_op || !g2d->drgb || n_units < 1 || (sched && !img) ||
      n_units > GS_MAX_UNITS || width <= 0 || height <= 0 || n_proj < 0 || variant < 0 || variant > 2)
    return GS_ERR_INVALID;
  unsigned long long* fixed = g2d->fixed;
  if (fixed) {
    if (cudaMemsetAsync(fixed, 0, sizeof(unsigned long long) * 9 * (size_t)n_proj, s) != cudaSuccess)
      return GS_ERR_CUDA;
  } else if (cudaMemsetAsync(g2d->dxy, 0, sizeof(float) * 2 * (size_t)n_proj, s) != cudaSuccess ||
             cudaMemsetAsync(g2d->dconic_op, 0, sizeof(float) * 4 * (size_t)n_proj, s) != cudaSuccess ||
             cudaMemsetAsync(g2d->drgb, 0, sizeof(float) * 4 * (size_t)n_proj, s) != cudaSuccess) {
    return GS_ERR_CUDA;
  }
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  dim3 grid(TX * TY * n_units);
#define GS_BWD(BW)                                                                                                   \
  if (sched)                                                                                                         \
    {                                                                                                              \
      if (cudaMemsetAsync(sched_ticket(sched), 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;        \
      auto kb = fixed ? k_render_bwd_m<BW, false> : k_render_bwd_m<BW, true>;                                      \
      kb<<<dim3(resident_grid(kb, sched->max_jobs * 8)), 32, 0, s>>>(                                               \
          (const uint2*)ranges, sched->tile_order, sched->job_base, sched->jobs, sched->chunk,                       \
          (const float4*)sched->checkpoints, sorted_vals, sched->block_masks, (const float4*)proj->xy,               \
          (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height, TX, TX * TY, TX * TY * n_units,   \
          bg[0], bg[1], bg[2],                                                                                       \
          img, final_T, n_contrib, dL_dimg, dL_dT, g2d->dxy, g2d->dconic_op, g2d->drgb, fixed,                       \
          sched_ticket(sched));                                                                                      \
    }                                                                                                              \
  else                                                                                                               \
    k_render_bwd<BW><<<grid, TILE_PIX, 0, s>>>((const uint2*)ranges, nullptr, sorted_vals, (const float4*)proj->xy, \
                                               (const float4*)proj->conic_op, (const float4*)proj->rgb, width, height,  \
                                               TX, TX * TY, bg[0], bg[1], bg[2], final_T, n_contrib, dL_dimg, dL_dT,    \
                                               g2d->dxy, g2d->dconic_op, g2d->drgb, fixed)
  if (variant == 0) { GS_BWD(8); } else if (variant == 1) { GS_BWD(16); } else { GS_BWD(4); }
#undef GS_BWD
  if (fixed && n_proj > 0)
    k_fixed_to_grad2d<<<(unsigned)((n_proj + 255) / 256), 256, 0, s>>>(fixed, n_proj, g2d->dxy, g2d->dconic_op,
                                                                       g2d->drgb);
  return gs_check_launch();
}

GS_API int gs_blend_pairs(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges, int n_units,
                          int width, int height, const uint32_t* n_contrib, const uint16_t* block_masks,
                          unsigned long long* d_count, gs_stream_t stream) {
  GS_RANGE("gs_blend_pairs");
  if (!proj || !proj->xy || !proj->conic_op || !sorted_vals || !ranges || !n_contrib || !d_count || n_units < 1 ||
      n_units > GS_MAX_UNITS || width <= 0 || height <= 0)
    return GS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_count, 0, 5 * sizeof(unsigned long long), s) != cudaSuccess) return GS_ERR_CUDA;
  int TX = (width + TILE - 1) / TILE, TY = (height + TILE - 1) / TILE;
  k_blend_pairs<<<dim3(TX * TY, n_units), TILE_PIX, 0, s>>>((const uint2*)ranges, sorted_vals, (const float4*)proj->xy,
                                                            (const float4*)proj->conic_op, width, height, TX, TX * TY,
                                                            n_contrib, block_masks, d_count);
  return gs_check_launch();
}

// Heaviest-first order of the (unit, tile) blocks from the tile ranges.
// ws: 2 x 33 uint32 of scratch.
int gs_tile_order_impl(const uint32_t* ranges, int n, uint32_t* ws, uint32_t* order, cudaStream_t s) {
  if (cudaMemsetAsync(ws, 0, sizeof(uint32_t) * 66, s) != cudaSuccess) return GS_ERR_CUDA;
  unsigned nb = (unsigned)((n + 255) / 256);
  k_order_hist<<<nb, 256, 0, s>>>((const uint2*)ranges, n, ws);
  k_order_scatter<<<nb, 256, 0, s>>>((const uint2*)ranges, n, ws, ws + 33, order);
  return gs_check_launch();
}
