// FP64 CPU oracle for the differentiable tile-based Gaussian-splat rasterizer.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
// it exists so that tests, the smoke check and the bench's CPU baseline can
// check the CUDA library against a plain, slow, obviously-correct definition.
// It shares no code, header, table or constant generator with the CUDA path.
//
// The paper (Sec. I-II) trains 3D Gaussian Splatting [Kerbl et al.] per data
// partition and merges the splats for the final render (Sec. II, "Global
// Reconstruction").  It does not restate the rasterizer, so every step below
// is the standard EWA-splatting / 3D-GS definition with the readings fixed in
// the design notes (dilation 0.3 px^2, near plane 0.2, J clamp 1.3 tan(fov/2),
// 3-sigma radius, 16x16 tiles, alpha clamp 0.99, skip below 1/255, stop before
// transmittance would fall below 1e-4).
//
// Everything is templated on the scalar type so that the same forward code
// runs on doubles and on forward-mode dual numbers (exact directional
// derivatives); discrete decisions (culling, rectangles, skips, clamps, the
// stop) are always taken on the real part.
//
// Parity pins for each function live in tests/test_oracle_*.py.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual fabs(Dual a) { return a.v > 0 ? a : (a.v < 0 ? -a : Dual(0.0, 0.0)); }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double tan_(double x) { return x; }
inline double tan_(const Dual& x) { return x.d; }
using std::exp;
using std::sqrt;
using std::log;
using std::fabs;

// ---------------------------------------------------------------- camera
// Camera block layout (doubles): R[9] row-major, t[3], fx, fy, cx, cy,
// tan_fovx, tan_fovy, campos[3], znear, W, H   (24 values).
struct Cam {
  double R[9], t[3], fx, fy, cx, cy, tanx, tany, campos[3], znear;
  int W, H;
};
static Cam load_cam(const double* c) {
  Cam k;
  for (int i = 0; i < 9; ++i) k.R[i] = c[i];
  for (int i = 0; i < 3; ++i) k.t[i] = c[9 + i];
  k.fx = c[12]; k.fy = c[13]; k.cx = c[14]; k.cy = c[15];
  k.tanx = c[16]; k.tany = c[17];
  for (int i = 0; i < 3; ++i) k.campos[i] = c[18 + i];
  k.znear = c[21];
  k.W = (int)c[22]; k.H = (int)c[23];
  return k;
}

static const int TILE = 16;
static const double DILATION = 0.3;     // low-pass added to the 2D covariance (px^2)
static const double ALPHA_MAX = 0.99;   // alpha clamp
static const double ALPHA_MIN = 1.0 / 255.0;  // skip threshold
static const double T_MIN = 1e-4;       // transmittance stop threshold
static const double JCLAMP = 1.3;       // x/z, y/z clamp inside J, in units of tan(fov/2)
static const double LAMBDA_FLOOR = 0.1; // floor under the discriminant sqrt

// floor(a / 16) for integer a (rounds toward -inf)
static inline int floordiv16(long long a) {
  long long q = a / TILE;
  if ((a % TILE) != 0 && a < 0) --q;
  return (int)q;
}
static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Tile rectangle of a splat centred at (u, v) with integer radius r:
// [x0, x1) x [y0, y1) with x0 = floor((u - r)/16), x1 = floor((u + r + 15)/16),
// clamped to the tile grid.  floor(u) enters only through floor((.)/16), so
// computing with floor(u) is exact.
static inline void tile_rect(double u, double v, int r, int TX, int TY, int rect[4]) {
  long long fu = (long long)std::floor(u), fv = (long long)std::floor(v);
  rect[0] = clampi(floordiv16(fu - r), 0, TX);
  rect[1] = clampi(floordiv16(fv - r), 0, TY);
  rect[2] = clampi(floordiv16(fu + r + TILE - 1), 0, TX);
  rect[3] = clampi(floordiv16(fv + r + TILE - 1), 0, TY);
}

// ---------------------------------------------------------------- real spherical harmonics
// Real SH with the Condon-Shortley phase, ordered m = -l..l, index l^2 + l + m:
//   m = 0 : N_l^0 P_l(z)
//   m > 0 : sqrt(2) N_l^m (-1)^m  P_l^(m)(z) Re((x + i y)^m)
//   m < 0 : sqrt(2) N_l^|m| (-1)^|m| P_l^(|m|)(z) Im((x + i y)^|m|)
// where P_l^(m) is the m-th derivative of the Legendre polynomial P_l and
// N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  On the unit sphere,
// (1 - z^2)^(m/2) cos(m phi) = Re((x + i y)^m), which makes this the textbook
// associated-Legendre definition written as a polynomial in (x, y, z).
struct ShTables {
  double poly[4][4][4];  // poly[l][m][k]: coefficient of z^k in d^m P_l / dz^m
  double N[4][4];
  ShTables() {
    double P[4][4] = {{0}};
    P[0][0] = 1.0;
    P[1][1] = 1.0;
    for (int l = 1; l < 3; ++l)  // Bonnet: (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1}
      for (int k = 0; k < 4; ++k) {
        double a = (k > 0) ? (2 * l + 1) * P[l][k - 1] : 0.0;
        P[l + 1][k] = (a - l * P[l - 1][k]) / (l + 1);
      }
    for (int l = 0; l < 4; ++l) {
      double cur[4];
      for (int k = 0; k < 4; ++k) cur[k] = P[l][k];
      for (int m = 0; m <= l; ++m) {
        for (int k = 0; k < 4; ++k) poly[l][m][k] = cur[k];
        double nxt[4] = {0, 0, 0, 0};
        for (int k = 1; k < 4; ++k) nxt[k - 1] = k * cur[k];
        for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
      }
    }
    auto fact = [](int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; };
    for (int l = 0; l < 4; ++l)
      for (int m = 0; m <= l; ++m)
        N[l][m] = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - m) / fact(l + m));
  }
};
static const ShTables& sh_tables() { static ShTables t; return t; }

template <class S>
void sh_basis(int deg, S x, S y, S z, S* out) {
  const ShTables& T = sh_tables();
  for (int l = 0; l <= deg; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      S p = S(0.0);
      S zp = S(1.0);
      for (int k = 0; k + am <= l; ++k) {  // degree of d^m P_l is l - m
        p = p + T.poly[l][am][k] * zp;
        zp = zp * z;
      }
      S re = S(1.0), im = S(0.0);  // (x + i y)^am
      for (int j = 0; j < am; ++j) {
        S nre = re * x - im * y;
        S nim = re * y + im * x;
        re = nre; im = nim;
      }
      double sgn = (am % 2) ? -1.0 : 1.0;
      S v;
      if (m == 0) v = T.N[l][0] * p;
      else if (m > 0) v = std::sqrt(2.0) * T.N[l][am] * sgn * p * re;
      else v = std::sqrt(2.0) * T.N[l][am] * sgn * p * im;
      out[l * l + l + m] = v;
    }
  }
}

// ---------------------------------------------------------------- quaternion
// Rotation of the unit quaternion q / |q| = (w, x, y, z): the matrix of
// v -> q v q*.
template <class S>
void quat_to_rot(const S q[4], S R[9]) {
  S n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z); R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y); R[7] = 2.0 * (y * z + w * x); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// ---------------------------------------------------------------- projection
// The list order is decided on the depth key: the camera-space z of the mean
// rounded to float32 (the key is stored as a float32 bit pattern).  Here z is
// evaluated in FP64 from the (float32-representable) inputs, whose products are
// exact in FP64, and rounded once.
static inline double depth_key(double z) { return (double)(float)z; }

// Float32 error model of the discrete decisions (diagnostics only: the FP64
// decisions are the oracle's results).  A decision is "unstable" when it
// changes as the continuous quantity it is taken on moves by a bound on the
// error a float32 evaluation of the same formula can make, u = 2^-24:
//   z (near cull):  8 u (|r20 x| + |r21 y| + |r22 z| + |t2|)  (four terms, a few roundings each);
//   pixel u, v:     computed as float pairs (hi + lo, ~2^-44 relative): 2^-40 [ f (s_t / z + |t_x| s_z / z^2)
//                   + |u| ] with s_t, s_z the sums of the terms' magnitudes of t_x and z;
//   3 sqrt(lambda): relative 4 u (33 + mid / sqrt(max(0.1, disc))): a, b, c carry absolute errors
//                   up to ~30 u lambda_max (sums of products of a PSD form, which cancel for thin
//                   splats seen edge-on), and disc = mid^2 - det loses ~4 u mid^2 to its own roundings;
//                   half of lambda's relative error reaches the square root; the factor 4 is slack.
enum { UNSTABLE_CULL = 1, UNSTABLE_RADIUS = 2, UNSTABLE_RECT = 4 };

template <class S>
struct Proj {
  S x, y;        // pixel-space mean
  S A, B, C;     // conic = inverse of the dilated 2D covariance [[a, b], [b, c]]
  S op;          // opacity
  S col[3];      // RGB after the +0.5 offset and the clamp at 0
  S depth;       // float32 sort key (camera-space z), see depth_key
  int radius;    // 0 = culled
  int unstable;  // UNSTABLE_* bits: decisions a float32 evaluation may take the other way
  int rect[4];
  int tiles;
  int clamp;     // bit c set if channel c was clamped to 0
  // covariance before inversion, kept for pins
  S a, b, c;
};

// One Gaussian seen by one camera: EWA projection (Zwicker et al.), the 3D-GS
// 2D covariance Sigma2D = J W Sigma3D W^T J^T + 0.3 I, its inverse, the 3-sigma
// radius and tile rectangle, SH colour and sigmoid opacity.
template <class S>
Proj<S> project_one(const S mu[3], const S ls[3], const S q[4], S logit, const S* sh, int deg,
                    const Cam& cam) {
  Proj<S> P;
  P.radius = 0; P.tiles = 0; P.clamp = 0; P.unstable = 0;
  P.rect[0] = P.rect[1] = P.rect[2] = P.rect[3] = 0;
  const double* R = cam.R;
  S t[3];
  for (int i = 0; i < 3; ++i) t[i] = R[3 * i] * mu[0] + R[3 * i + 1] * mu[1] + R[3 * i + 2] * mu[2] + cam.t[i];
  P.depth = S(depth_key(val(t[2])));
  const double U32 = std::ldexp(1.0, -24);
  double tsum[3];
  for (int i = 0; i < 3; ++i)
    tsum[i] = std::fabs(R[3 * i] * val(mu[0])) + std::fabs(R[3 * i + 1] * val(mu[1])) +
              std::fabs(R[3 * i + 2] * val(mu[2])) + std::fabs(cam.t[i]);
  double ez = 8.0 * U32 * tsum[2];
  if (std::fabs(val(t[2]) - cam.znear) <= ez) P.unstable |= UNSTABLE_CULL;
  if (val(t[2]) <= cam.znear) return P;

  // Sigma3D = (Rq S)(Rq S)^T
  S Rq[9];
  quat_to_rot(q, Rq);
  S s[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
  S M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * s[j];
  S Sig[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Sig[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];

  // Jacobian of the perspective map at t, with x/z and y/z clamped to
  // +-1.3 tan(fov/2) (a clamped ratio is a constant of the map).
  double limx = JCLAMP * cam.tanx, limy = JCLAMP * cam.tany;
  S xz = t[0] / t[2], yz = t[1] / t[2];
  if (val(xz) < -limx) xz = S(-limx);
  if (val(xz) > limx) xz = S(limx);
  if (val(yz) < -limy) yz = S(-limy);
  if (val(yz) > limy) yz = S(limy);
  S J00 = cam.fx / t[2], J02 = -cam.fx * xz / t[2];
  S J11 = cam.fy / t[2], J12 = -cam.fy * yz / t[2];
  // T2 = J W (W = camera rotation)
  S T2[6];
  for (int j = 0; j < 3; ++j) {
    T2[j] = J00 * R[j] + J02 * R[6 + j];
    T2[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
  }
  S Cv[4] = {S(0.0), S(0.0), S(0.0), S(0.0)};  // T2 Sig T2^T
  for (int r = 0; r < 2; ++r)
    for (int cc = 0; cc < 2; ++cc) {
      S acc = S(0.0);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc = acc + T2[3 * r + i] * Sig[3 * i + j] * T2[3 * cc + j];
      Cv[2 * r + cc] = acc;
    }
  S a = Cv[0] + DILATION, b = Cv[1], c = Cv[3] + DILATION;
  P.a = a; P.b = b; P.c = c;
  S det = a * c - b * b;
  if (val(det) <= 0.0) return P;
  P.A = c / det;
  P.B = -b / det;
  P.C = a / det;
  double mid = 0.5 * (val(a) + val(c));
  double lam = mid + std::sqrt(std::max(LAMBDA_FLOOR, mid * mid - val(det)));
  int radius = (int)std::ceil(3.0 * std::sqrt(lam));
  P.x = cam.fx * t[0] / t[2] + cam.cx;
  P.y = cam.fy * t[1] / t[2] + cam.cy;
  int TX = (cam.W + TILE - 1) / TILE, TY = (cam.H + TILE - 1) / TILE;
  tile_rect(val(P.x), val(P.y), radius, TX, TY, P.rect);
  int tiles = (P.rect[2] - P.rect[0]) * (P.rect[3] - P.rect[1]);
  {
    // stability of the radius and of the rectangle (see the error model above)
    double tz = val(t[2]);
    double eps_r = 4.0 * U32 * (33.0 + mid / std::sqrt(std::max(LAMBDA_FLOOR, mid * mid - val(det))));
    double r3 = 3.0 * std::sqrt(lam);
    int rlo = (int)std::ceil(r3 * (1.0 - eps_r)), rhi = (int)std::ceil(r3 * (1.0 + eps_r));
    if (rlo != radius || rhi != radius) P.unstable |= UNSTABLE_RADIUS;
    double f[2] = {cam.fx, cam.fy}, pix[2] = {val(P.x), val(P.y)};
    double e[2];
    for (int k = 0; k < 2; ++k) {
      e[k] = std::ldexp(1.0, -40) * (std::fabs(f[k]) * (tsum[k] / tz + std::fabs(val(t[k])) * tsum[2] / (tz * tz)) +
                                     std::fabs(pix[k]));
    }
    for (int sx = -1; sx <= 1; sx += 2)
      for (int sy = -1; sy <= 1; sy += 2)
        for (int rr = rlo; rr <= rhi; ++rr) {
          int q[4];
          tile_rect(pix[0] + sx * e[0], pix[1] + sy * e[1], rr, TX, TY, q);
          if (q[0] != P.rect[0] || q[1] != P.rect[1] || q[2] != P.rect[2] || q[3] != P.rect[3])
            P.unstable |= UNSTABLE_RECT;
        }
  }
  if (radius == 0 || tiles == 0) return P;
  P.radius = radius;
  P.tiles = tiles;

  // view-dependent colour
  S d[3] = {mu[0] - cam.campos[0], mu[1] - cam.campos[1], mu[2] - cam.campos[2]};
  S dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  S Y[16];
  sh_basis(deg, d[0] / dn, d[1] / dn, d[2] / dn, Y);
  int nc = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    S acc = S(0.5);
    for (int k = 0; k < nc; ++k) acc = acc + Y[k] * sh[3 * k + ch];
    if (val(acc) < 0.0) { acc = S(0.0); P.clamp |= 1 << ch; }
    P.col[ch] = acc;
  }
  P.op = 1.0 / (1.0 + exp(-logit));
  return P;
}

// ---------------------------------------------------------------- binning
struct Lists {
  std::vector<int> idx;    // Gaussian index of each instance, sorted by (tile, depth, index)
  std::vector<int> tile;   // tile of each instance
  std::vector<int> start, end;  // per tile [start, end)
};

// Duplicate each visible Gaussian once per covered tile (rows, then columns),
// then order the instances by (tile, depth, Gaussian index).
static void bin_and_sort(int n, const double* x, const double* y, const int* radius,
                         const double* depth, int W, int H, Lists& L, int* tie_tiles) {
  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  struct E { int tile; double depth; int idx; };
  std::vector<E> es;
  for (int i = 0; i < n; ++i) {
    if (radius[i] <= 0) continue;
    int r[4];
    tile_rect(x[i], y[i], radius[i], TX, TY, r);
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) es.push_back({ty * TX + tx, depth[i], i});
  }
  std::sort(es.begin(), es.end(), [](const E& a, const E& b) {
    if (a.tile != b.tile) return a.tile < b.tile;
    if (a.depth != b.depth) return a.depth < b.depth;
    return a.idx < b.idx;
  });
  L.idx.resize(es.size());
  L.tile.resize(es.size());
  L.start.assign(TX * TY, 0);
  L.end.assign(TX * TY, 0);
  for (size_t k = 0; k < es.size(); ++k) {
    L.idx[k] = es[k].idx;
    L.tile[k] = es[k].tile;
    if (k == 0 || es[k - 1].tile != es[k].tile) L.start[es[k].tile] = (int)k;
    if (k + 1 == es.size() || es[k + 1].tile != es[k].tile) L.end[es[k].tile] = (int)k + 1;
    // equal keys: the order comes from the index (deterministic on both sides);
    // recorded for diagnostics only
    if (tie_tiles && k > 0 && es[k - 1].tile == es[k].tile && es[k - 1].depth == es[k].depth)
      tie_tiles[es[k].tile] = 1;
  }
}

// ---------------------------------------------------------------- blending
// Front-to-back compositing of one pixel over its tile's list.
// For each entry: power = -(A dx^2 + C dy^2)/2 - B dx dy with d = mean - pixel;
// skip if power > 0; alpha = min(0.99, o e^power); skip if alpha < 1/255;
// if T (1 - alpha) < 1e-4 the entry is not blended and the pixel stops;
// otherwise C += alpha T c, T *= (1 - alpha).  Finally C += T bg.
// Also records the smallest relative distance of any decision to its threshold.
template <class S>
struct PixelOut {
  S col[3];
  S T;
  int n_contrib;
  double margin;
  // diagnostics of the early-stop decision: its smallest relative distance to T_MIN over the
  // entries tested, and a bound on the relative error a float32 evaluation accumulates in T
  // over the blended entries (1e-6 per factor, times 1 / (1 - alpha) for near-opaque ones)
  double stop_margin;
  double t_err;
};

template <class S>
PixelOut<S> blend_pixel(int px, int py, const int* list, int len, const Proj<S>* P,
                        const double bg[3], std::vector<int>* blended = nullptr,
                        std::vector<S>* Ts = nullptr) {
  PixelOut<S> o;
  o.col[0] = o.col[1] = o.col[2] = S(0.0);
  S T = S(1.0);
  int last = 0;
  double margin = std::numeric_limits<double>::infinity();
  double stop_margin = std::numeric_limits<double>::infinity(), t_err = 0.0;
  for (int k = 0; k < len; ++k) {
    const Proj<S>& g = P[list[k]];
    S dx = g.x - (double)px, dy = g.y - (double)py;
    S power = -0.5 * (g.A * dx * dx + g.C * dy * dy) - g.B * dx * dy;
    // power <= 0 for a positive-definite conic; its sign can only be decided
    // differently under cancellation, so the margin is relative to the terms
    double terms = 0.5 * (std::fabs(val(g.A)) * val(dx) * val(dx) + std::fabs(val(g.C)) * val(dy) * val(dy)) +
                   std::fabs(val(g.B) * val(dx) * val(dy));
    if (terms > 0.0) margin = std::min(margin, std::fabs(val(power)) / terms);
    if (val(power) > 0.0) continue;
    S G = exp(power);
    S araw = g.op * G;
    margin = std::min(margin, std::fabs(val(araw) - ALPHA_MAX) / ALPHA_MAX);
    S alpha = (val(araw) > ALPHA_MAX) ? S(ALPHA_MAX) : araw;
    margin = std::min(margin, std::fabs(val(alpha) - ALPHA_MIN) / ALPHA_MIN);
    if (val(alpha) < ALPHA_MIN) continue;
    S testT = T * (1.0 - alpha);
    margin = std::min(margin, std::fabs(val(testT) - T_MIN) / T_MIN);
    stop_margin = std::min(stop_margin, std::fabs(val(testT) - T_MIN) / T_MIN);
    if (val(testT) < T_MIN) break;
    t_err += 1e-6 / (1.0 - val(alpha));
    for (int ch = 0; ch < 3; ++ch) o.col[ch] = o.col[ch] + g.col[ch] * alpha * T;
    if (blended) blended->push_back(k);
    if (Ts) Ts->push_back(T);
    T = testT;
    last = k + 1;
  }
  for (int ch = 0; ch < 3; ++ch) o.col[ch] = o.col[ch] + T * bg[ch];
  o.T = T;
  o.n_contrib = last;
  o.margin = margin;
  o.stop_margin = stop_margin;
  o.t_err = t_err;
  return o;
}

template <class S>
void render_image(const Lists& L, const Proj<S>* P, int W, int H, const double bg[3], S* img,
                  S* finalT, int* ncontrib, double* margin, double* stop_margin = nullptr,
                  double* t_err = nullptr) {
  int TX = (W + TILE - 1) / TILE;
#pragma omp parallel for schedule(dynamic, 4)
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tile = (py / TILE) * TX + px / TILE;
      int s = L.start[tile], e = L.end[tile];
      PixelOut<S> o = blend_pixel(px, py, L.idx.data() + s, e - s, P, bg);
      size_t p = (size_t)py * W + px;
      for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + p] = o.col[ch];
      if (finalT) finalT[p] = o.T;
      if (ncontrib) ncontrib[p] = o.n_contrib;
      if (margin) margin[p] = o.margin;
      if (stop_margin) stop_margin[p] = o.stop_margin;
      if (t_err) t_err[p] = o.t_err;
    }
}

// ---------------------------------------------------------------- loss
// SSIM window: separable normalised Gaussian, 11 taps, sigma 1.5.
static void ssim_window(double g[11]) {
  double s = 0;
  for (int k = 0; k < 11; ++k) { g[k] = std::exp(-(k - 5.0) * (k - 5.0) / (2.0 * 1.5 * 1.5)); s += g[k]; }
  for (int k = 0; k < 11; ++k) g[k] /= s;
}

// zero-padded "same" 2D convolution with the separable window
template <class S>
void conv_same(const S* in, S* out, int W, int H, const double g[11]) {
  std::vector<S> tmp((size_t)W * H);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      S acc = S(0.0);
      for (int k = -5; k <= 5; ++k) {
        int xx = x + k;
        if (xx >= 0 && xx < W) acc = acc + g[k + 5] * in[(size_t)y * W + xx];
      }
      tmp[(size_t)y * W + x] = acc;
    }
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      S acc = S(0.0);
      for (int k = -5; k <= 5; ++k) {
        int yy = y + k;
        if (yy >= 0 && yy < H) acc = acc + g[k + 5] * tmp[(size_t)yy * W + x];
      }
      out[(size_t)y * W + x] = acc;
    }
}

static const double SSIM_C1 = 0.01 * 0.01, SSIM_C2 = 0.03 * 0.03;

// loss = (1 - lam) * masked L1 + lam * (1 - masked SSIM), both averaged over
// the 3 channels and the mask pixels.  lam = 0 gives the plain masked L1.
template <class S>
S loss_value(const S* img, const double* gt, const unsigned char* mask, int W, int H, double lam) {
  size_t np = (size_t)W * H;
  double msum = 0;
  for (size_t p = 0; p < np; ++p) msum += mask[p] ? 1.0 : 0.0;
  if (msum == 0.0) return S(0.0);
  S l1 = S(0.0);
  for (int ch = 0; ch < 3; ++ch)
    for (size_t p = 0; p < np; ++p)
      if (mask[p]) l1 = l1 + fabs(img[ch * np + p] - gt[ch * np + p]);
  l1 = l1 / (3.0 * msum);
  if (lam == 0.0) return l1;
  double g[11];
  ssim_window(g);
  S ssum = S(0.0);
  std::vector<S> x(np), y(np), xx(np), yy(np), xy(np), mx(np), my(np), sxx(np), syy(np), sxy(np);
  for (int ch = 0; ch < 3; ++ch) {
    for (size_t p = 0; p < np; ++p) {
      x[p] = img[ch * np + p];
      y[p] = S(gt[ch * np + p]);
      xx[p] = x[p] * x[p]; yy[p] = y[p] * y[p]; xy[p] = x[p] * y[p];
    }
    conv_same(x.data(), mx.data(), W, H, g);
    conv_same(y.data(), my.data(), W, H, g);
    conv_same(xx.data(), sxx.data(), W, H, g);
    conv_same(yy.data(), syy.data(), W, H, g);
    conv_same(xy.data(), sxy.data(), W, H, g);
    for (size_t p = 0; p < np; ++p) {
      if (!mask[p]) continue;
      S vx = sxx[p] - mx[p] * mx[p], vy = syy[p] - my[p] * my[p], cxy = sxy[p] - mx[p] * my[p];
      S s = ((2.0 * mx[p] * my[p] + SSIM_C1) * (2.0 * cxy + SSIM_C2)) /
            ((mx[p] * mx[p] + my[p] * my[p] + SSIM_C1) * (vx + vy + SSIM_C2));
      ssum = ssum + s;
    }
  }
  S ssim = ssum / (3.0 * msum);
  return (1.0 - lam) * l1 + lam * (1.0 - ssim);
}

// Hand-derived gradient of loss_value with respect to the image.
static double loss_grad(const double* img, const double* gt, const unsigned char* mask, int W, int H,
                        double lam, double* dimg) {
  size_t np = (size_t)W * H;
  double msum = 0;
  for (size_t p = 0; p < np; ++p) msum += mask[p] ? 1.0 : 0.0;
  for (size_t p = 0; p < 3 * np; ++p) dimg[p] = 0.0;
  if (msum == 0.0) return 0.0;
  double l1 = 0;
  double w1 = (1.0 - lam) / (3.0 * msum);
  for (int ch = 0; ch < 3; ++ch)
    for (size_t p = 0; p < np; ++p)
      if (mask[p]) {
        double d = img[ch * np + p] - gt[ch * np + p];
        l1 += std::fabs(d);
        dimg[ch * np + p] = w1 * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0));
      }
  l1 /= 3.0 * msum;
  if (lam == 0.0) return l1;
  double g[11];
  ssim_window(g);
  double ssum = 0;
  std::vector<double> x(np), y(np), xx(np), yy(np), xy(np), mx(np), my(np), sxx(np), syy(np),
      sxy(np), dmu(np), dexx(np), dexy(np), cmu(np), cexx(np), cexy(np);
  double wp = -lam / (3.0 * msum);  // d loss / d S_p for mask pixels
  for (int ch = 0; ch < 3; ++ch) {
    for (size_t p = 0; p < np; ++p) {
      x[p] = img[ch * np + p]; y[p] = gt[ch * np + p];
      xx[p] = x[p] * x[p]; yy[p] = y[p] * y[p]; xy[p] = x[p] * y[p];
    }
    conv_same(x.data(), mx.data(), W, H, g);
    conv_same(y.data(), my.data(), W, H, g);
    conv_same(xx.data(), sxx.data(), W, H, g);
    conv_same(yy.data(), syy.data(), W, H, g);
    conv_same(xy.data(), sxy.data(), W, H, g);
    for (size_t p = 0; p < np; ++p) {
      dmu[p] = dexx[p] = dexy[p] = 0.0;
      if (!mask[p]) continue;
      double ux = mx[p], uy = my[p];
      double vx = sxx[p] - ux * ux, vy = syy[p] - uy * uy, cxy = sxy[p] - ux * uy;
      double A1 = 2 * ux * uy + SSIM_C1, A2 = 2 * cxy + SSIM_C2;
      double B1 = ux * ux + uy * uy + SSIM_C1, B2 = vx + vy + SSIM_C2;
      double s = A1 * A2 / (B1 * B2);
      ssum += s;
      // S as a function of (mu_x, E[x^2], E[xy]) with the y statistics fixed
      dmu[p] = wp * s * (2 * uy / A1 - 2 * ux / B1 - 2 * uy / A2 + 2 * ux / B2);
      dexx[p] = wp * s * (-1.0 / B2);
      dexy[p] = wp * s * (2.0 / A2);
    }
    // adjoint of the zero-padded same convolution with a symmetric window is itself
    conv_same(dmu.data(), cmu.data(), W, H, g);
    conv_same(dexx.data(), cexx.data(), W, H, g);
    conv_same(dexy.data(), cexy.data(), W, H, g);
    for (size_t p = 0; p < np; ++p)
      dimg[ch * np + p] += cmu[p] + 2.0 * x[p] * cexx[p] + y[p] * cexy[p];
  }
  double ssim = ssum / (3.0 * msum);
  return (1.0 - lam) * l1 + lam * (1.0 - ssim);
}

// ---------------------------------------------------------------- parameter access
struct Params {
  int n, deg;
  const double *means, *ls, *quats, *logit, *sh;
};
static inline int n_coeffs(int deg) { return (deg + 1) * (deg + 1); }
static inline int n_params(int deg) { return 11 + 3 * n_coeffs(deg); }

// Parameter vector of Gaussian i in the order: mean(3), log-scale(3), quat(4),
// logit opacity(1), SH coefficients (coefficient-major, channel-minor).
static void gather_params(const Params& p, int i, double* out) {
  for (int k = 0; k < 3; ++k) out[k] = p.means[3 * i + k];
  for (int k = 0; k < 3; ++k) out[3 + k] = p.ls[3 * i + k];
  for (int k = 0; k < 4; ++k) out[6 + k] = p.quats[4 * i + k];
  out[10] = p.logit[i];
  int nsh = 3 * n_coeffs(p.deg);
  for (int k = 0; k < nsh; ++k) out[11 + k] = p.sh[(size_t)nsh * i + k];
}

template <class S>
Proj<S> project_vec(const S* v, int deg, const Cam& cam) {
  return project_one<S>(v, v + 3, v + 6, v[10], v + 11, deg, cam);
}

static void project_all(const Params& p, const Cam& cam, std::vector<Proj<double>>& out) {
  out.resize(p.n);
  int np = n_params(p.deg);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < p.n; ++i) {
    std::vector<double> v(np);
    gather_params(p, i, v.data());
    out[i] = project_vec<double>(v.data(), p.deg, cam);
  }
}

static void split_proj(const std::vector<Proj<double>>& P, std::vector<double>& x, std::vector<double>& y,
                       std::vector<int>& r, std::vector<double>& d) {
  size_t n = P.size();
  x.resize(n); y.resize(n); r.resize(n); d.resize(n);
  for (size_t i = 0; i < n; ++i) { x[i] = P[i].x; y[i] = P[i].y; r[i] = P[i].radius; d[i] = P[i].depth; }
}

}  // namespace orc

using namespace orc;

extern "C" {

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// Real SH basis values for unit directions: out[n][(deg+1)^2].
void orc_sh_basis(int n, int deg, const double* dirs, double* out) {
  int nc = n_coeffs(deg);
  for (int i = 0; i < n; ++i) {
    double Y[16];
    sh_basis<double>(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    for (int k = 0; k < nc; ++k) out[(size_t)nc * i + k] = Y[k];
  }
}

void orc_quat_to_rot(int n, const double* q, double* R) {
  for (int i = 0; i < n; ++i) quat_to_rot<double>(q + 4 * i, R + 9 * i);
}

// Per-Gaussian projection for one camera.  Outputs are per Gaussian:
// xy[2], conic[3] (A, B, C), opacity, rgb[3], clamp bits, depth, radius,
// rect[4], tiles touched, cov2d[3] (a, b, c before inversion), unstable (UNSTABLE_*
// bits of the float32 error model).
void orc_project(int n, int deg, const double* means, const double* ls, const double* quats,
                 const double* logit, const double* sh, const double* camv, double* xy, double* conic,
                 double* opacity, double* rgb, int* clampbits, double* depth, int* radius, int* rect,
                 int* tiles, double* cov2d, int* unstable) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  std::vector<Proj<double>> P;
  project_all(p, cam, P);
  for (int i = 0; i < n; ++i) {
    const Proj<double>& g = P[i];
    bool vis = g.radius > 0;
    xy[2 * i] = vis ? g.x : 0; xy[2 * i + 1] = vis ? g.y : 0;
    conic[3 * i] = vis ? g.A : 0; conic[3 * i + 1] = vis ? g.B : 0; conic[3 * i + 2] = vis ? g.C : 0;
    opacity[i] = vis ? g.op : 0;
    for (int c = 0; c < 3; ++c) rgb[3 * i + c] = vis ? g.col[c] : 0;
    clampbits[i] = vis ? g.clamp : 0;
    depth[i] = g.depth;
    radius[i] = g.radius;
    for (int k = 0; k < 4; ++k) rect[4 * i + k] = vis ? g.rect[k] : 0;
    tiles[i] = g.tiles;
    if (unstable) unstable[i] = g.unstable;
    if (cov2d) {
      bool has = val(g.depth) > cam.znear;
      cov2d[3 * i] = has ? g.a : 0; cov2d[3 * i + 1] = has ? g.b : 0; cov2d[3 * i + 2] = has ? g.c : 0;
    }
  }
}

// Binning + sort of given screen-space means, radii and depths (e.g. the
// CUDA path's own float32 values, for the bit-exact list comparison).
// Returns the instance count; fills idx/tile (capacity cap) and ranges[2*ntiles].
long long orc_bin(int n, const double* xy, const int* radius, const double* depth, int W, int H,
                  long long cap, int* out_idx, int* out_tile, int* ranges, int* tie_tiles) {
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; ++i) { x[i] = xy[2 * i]; y[i] = xy[2 * i + 1]; }
  Lists L;
  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  if (tie_tiles) std::memset(tie_tiles, 0, sizeof(int) * TX * TY);
  bin_and_sort(n, x.data(), y.data(), radius, depth, W, H, L, tie_tiles);
  long long I = (long long)L.idx.size();
  for (long long k = 0; k < I && k < cap; ++k) { out_idx[k] = L.idx[k]; out_tile[k] = L.tile[k]; }
  for (int t = 0; t < TX * TY; ++t) { ranges[2 * t] = L.start[t]; ranges[2 * t + 1] = L.end[t]; }
  return I;
}

// Full forward render of one view: project -> bin/sort -> blend.
// img[3][H][W], finalT[H][W], ncontrib[H][W], margin[H][W] (smallest relative
// distance of any blend decision to its threshold), tie_tiles[ntiles].
void orc_render(int n, int deg, const double* means, const double* ls, const double* quats,
                const double* logit, const double* sh, const double* camv, const double* bg,
                double* img, double* finalT, int* ncontrib, double* margin, int* tie_tiles,
                double* stop_margin, double* t_err) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  std::vector<Proj<double>> P;
  project_all(p, cam, P);
  std::vector<double> x, y, d;
  std::vector<int> r;
  split_proj(P, x, y, r, d);
  Lists L;
  int TX = (cam.W + TILE - 1) / TILE, TY = (cam.H + TILE - 1) / TILE;
  if (tie_tiles) std::memset(tie_tiles, 0, sizeof(int) * TX * TY);
  bin_and_sort(n, x.data(), y.data(), r.data(), d.data(), cam.W, cam.H, L, tie_tiles);
  render_image<double>(L, P.data(), cam.W, cam.H, bg, img, finalT, ncontrib, margin, stop_margin, t_err);
}

// Brute-force render used as a pin of the tile path: each pixel independently
// collects every visible Gaussian whose tile rectangle contains the pixel's
// tile, stable-sorts them by depth (index order breaks ties) and blends.
void orc_render_bruteforce(int n, int deg, const double* means, const double* ls, const double* quats,
                           const double* logit, const double* sh, const double* camv, const double* bg,
                           double* img, double* finalT, int* ncontrib) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  std::vector<Proj<double>> P;
  project_all(p, cam, P);
  int W = cam.W, H = cam.H;
#pragma omp parallel for schedule(dynamic, 4)
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tx = px / TILE, ty = py / TILE;
      std::vector<int> cand;
      for (int i = 0; i < n; ++i)
        if (P[i].radius > 0 && tx >= P[i].rect[0] && tx < P[i].rect[2] && ty >= P[i].rect[1] &&
            ty < P[i].rect[3])
          cand.push_back(i);
      std::stable_sort(cand.begin(), cand.end(),
                       [&](int a, int b) { return P[a].depth < P[b].depth; });
      PixelOut<double> o = blend_pixel(px, py, cand.data(), (int)cand.size(), P.data(), bg);
      size_t q = (size_t)py * W + px;
      for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + q] = o.col[ch];
      finalT[q] = o.T;
      ncontrib[q] = o.n_contrib;
    }
}

double orc_loss(const double* img, const double* gt, const unsigned char* mask, int W, int H,
                double lam, double* dimg) {
  if (dimg) return loss_grad(img, gt, mask, W, H, lam, dimg);
  return loss_value<double>(img, gt, mask, W, H, lam);
}

// Directional derivative of the loss along the image direction dir (dual numbers).
double orc_loss_dir(const double* img, const double* dir, const double* gt, const unsigned char* mask,
                    int W, int H, double lam) {
  size_t np = (size_t)3 * W * H;
  std::vector<Dual> x(np);
  for (size_t k = 0; k < np; ++k) x[k] = Dual(img[k], dir[k]);
  return loss_value<Dual>(x.data(), gt, mask, W, H, lam).d;
}

// Screen-space gradients of the loss for one view, by reverse replay of the
// blend: per visible Gaussian dL/d(x, y), dL/d(A, B, C), dL/d opacity and
// dL/d rgb.  dimg is dL/dimage [3][H][W]; dT (may be NULL) is dL/dT_final
// [H][W], the gradient of a loss term on the pixels' final transmittance.
void orc_render_backward(int n, int deg, const double* means, const double* ls, const double* quats,
                         const double* logit, const double* sh, const double* camv, const double* bg,
                         const double* dimg, const double* dT, double* dxy, double* dconic, double* dop,
                         double* drgb) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  std::vector<Proj<double>> P;
  project_all(p, cam, P);
  std::vector<double> x, y, d;
  std::vector<int> r;
  split_proj(P, x, y, r, d);
  Lists L;
  bin_and_sort(n, x.data(), y.data(), r.data(), d.data(), cam.W, cam.H, L, nullptr);
  int W = cam.W, H = cam.H, TX = (W + TILE - 1) / TILE;
  size_t np = (size_t)W * H;
  std::memset(dxy, 0, sizeof(double) * 2 * n);
  std::memset(dconic, 0, sizeof(double) * 3 * n);
  std::memset(dop, 0, sizeof(double) * n);
  std::memset(drgb, 0, sizeof(double) * 3 * n);
  // serial over pixels: plain accumulation, no atomics
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tile = (py / TILE) * TX + px / TILE;
      const int* list = L.idx.data() + L.start[tile];
      int len = L.end[tile] - L.start[tile];
      std::vector<int> blended;
      std::vector<double> Ts;
      PixelOut<double> o = blend_pixel(px, py, list, len, P.data(), bg, &blended, &Ts);
      size_t q = (size_t)py * W + px;
      double g[3] = {dimg[q], dimg[np + q], dimg[2 * np + q]};
      // T_final is the product of (1 - alpha_k) over the blended entries, so its derivative with
      // respect to one entry's alpha_i is -T_final / (1 - alpha_i)
      double gT = dT ? dT[q] : 0.0;
      // colour of everything behind entry k, seen through entry k's own gap
      double behind[3] = {bg[0], bg[1], bg[2]};
      for (int b = (int)blended.size() - 1; b >= 0; --b) {
        int j = list[blended[b]];
        const Proj<double>& G = P[j];
        double Ti = Ts[b];
        double dx = G.x - px, dy = G.y - py;
        double power = -0.5 * (G.A * dx * dx + G.C * dy * dy) - G.B * dx * dy;
        double e = std::exp(power);
        double araw = G.op * e;
        bool clamped = araw > ALPHA_MAX;
        double alpha = clamped ? ALPHA_MAX : araw;
        double dalpha = 0;
        for (int ch = 0; ch < 3; ++ch) {
          drgb[3 * j + ch] += alpha * Ti * g[ch];
          dalpha += Ti * (G.col[ch] - behind[ch]) * g[ch];
          behind[ch] = alpha * G.col[ch] + (1.0 - alpha) * behind[ch];
        }
        dalpha += gT * (-o.T / (1.0 - alpha));
        if (clamped) continue;
        dop[j] += e * dalpha;
        double dpow = araw * dalpha;
        dconic[3 * j] += -0.5 * dx * dx * dpow;
        dconic[3 * j + 1] += -dx * dy * dpow;
        dconic[3 * j + 2] += -0.5 * dy * dy * dpow;
        dxy[2 * j] += -(G.A * dx + G.B * dy) * dpow;
        dxy[2 * j + 1] += -(G.C * dy + G.B * dx) * dpow;
      }
    }
}

// Parameter gradients from screen-space gradients: the Jacobian of the
// per-Gaussian projection is taken column by column with dual numbers (one
// pass per parameter), so no derivative is derived by hand here.
// grads: [n][n_params(deg)] in gather_params order.
void orc_project_backward(int n, int deg, const double* means, const double* ls, const double* quats,
                          const double* logit, const double* sh, const double* camv, const double* dxy,
                          const double* dconic, const double* dop, const double* drgb, double* grads) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  int np = n_params(deg);
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; ++i) {
    std::vector<double> v(np);
    gather_params(p, i, v.data());
    std::vector<Dual> dv(np);
    double* gout = grads + (size_t)np * i;
    Proj<double> base = project_vec<double>(v.data(), deg, cam);
    if (base.radius == 0) {
      for (int k = 0; k < np; ++k) gout[k] = 0.0;
      continue;
    }
    for (int k = 0; k < np; ++k) {
      for (int j = 0; j < np; ++j) dv[j] = Dual(v[j], j == k ? 1.0 : 0.0);
      Proj<Dual> P = project_vec<Dual>(dv.data(), deg, cam);
      double acc = dxy[2 * i] * P.x.d + dxy[2 * i + 1] * P.y.d + dconic[3 * i] * P.A.d +
                   dconic[3 * i + 1] * P.B.d + dconic[3 * i + 2] * P.C.d + dop[i] * P.op.d;
      for (int ch = 0; ch < 3; ++ch) acc += drgb[3 * i + ch] * P.col[ch].d;
      gout[k] = acc;
    }
  }
}

// Loss of one view and its exact directional derivative along a parameter
// tangent (all params in gather_params order, tangent likewise), by running
// projection, blending and loss on dual numbers.  Returns the loss value;
// *dloss receives the directional derivative.
double orc_loss_params_dir(int n, int deg, const double* means, const double* ls, const double* quats,
                           const double* logit, const double* sh, const double* tangent,
                           const double* camv, const double* bg, const double* gt,
                           const unsigned char* mask, double lam, double* dloss) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  int np = n_params(deg);
  std::vector<Proj<Dual>> P(n);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    std::vector<double> v(np);
    gather_params(p, i, v.data());
    std::vector<Dual> dv(np);
    for (int k = 0; k < np; ++k) dv[k] = Dual(v[k], tangent[(size_t)np * i + k]);
    P[i] = project_vec<Dual>(dv.data(), deg, cam);
  }
  std::vector<double> x(n), y(n), d(n);
  std::vector<int> r(n);
  for (int i = 0; i < n; ++i) { x[i] = P[i].x.v; y[i] = P[i].y.v; r[i] = P[i].radius; d[i] = P[i].depth.v; }
  Lists L;
  bin_and_sort(n, x.data(), y.data(), r.data(), d.data(), cam.W, cam.H, L, nullptr);
  size_t npx = (size_t)cam.W * cam.H;
  std::vector<Dual> img(3 * npx);
  render_image<Dual>(L, P.data(), cam.W, cam.H, bg, img.data(), nullptr, nullptr, nullptr);
  Dual l = loss_value<Dual>(img.data(), gt, mask, cam.W, cam.H, lam);
  if (dloss) *dloss = l.d;
  return l.v;
}

// Background-opacity penalty of one view (a variant of the mask of Sec. II,
// "Image Rendering and Masking"): lam times the mean of the rendered opacity
// 1 - T_final over the pixels outside the mask (0 when there are none).
// dT (may be NULL) receives dpenalty/dT_final [H][W].
double orc_bg_penalty(const double* finalT, const unsigned char* mask, int W, int H, double lam, double* dT) {
  size_t np = (size_t)W * H;
  size_t nb = 0;
  double acc = 0.0;
  for (size_t q = 0; q < np; ++q)
    if (!mask[q]) { acc += 1.0 - finalT[q]; ++nb; }
  if (dT)
    for (size_t q = 0; q < np; ++q) dT[q] = (!mask[q] && nb) ? -lam / (double)nb : 0.0;
  return nb ? lam * acc / (double)nb : 0.0;
}

// The penalty of one view and its exact directional derivative along a
// parameter tangent (dual numbers through projection and blending, as
// orc_loss_params_dir).  Returns the penalty; *dpen receives the derivative.
double orc_penalty_params_dir(int n, int deg, const double* means, const double* ls, const double* quats,
                              const double* logit, const double* sh, const double* tangent, const double* camv,
                              const double* bg, const unsigned char* mask, double lam, double* dpen) {
  Cam cam = load_cam(camv);
  Params p{n, deg, means, ls, quats, logit, sh};
  int np = n_params(deg);
  std::vector<Proj<Dual>> P(n);
  for (int i = 0; i < n; ++i) {
    std::vector<double> v(np);
    gather_params(p, i, v.data());
    std::vector<Dual> dv(np);
    for (int k = 0; k < np; ++k) dv[k] = Dual(v[k], tangent[(size_t)np * i + k]);
    P[i] = project_vec<Dual>(dv.data(), deg, cam);
  }
  std::vector<double> x(n), y(n), d(n);
  std::vector<int> r(n);
  for (int i = 0; i < n; ++i) { x[i] = P[i].x.v; y[i] = P[i].y.v; r[i] = P[i].radius; d[i] = P[i].depth.v; }
  Lists L;
  bin_and_sort(n, x.data(), y.data(), r.data(), d.data(), cam.W, cam.H, L, nullptr);
  size_t npx = (size_t)cam.W * cam.H;
  std::vector<Dual> img(3 * npx), T(npx);
  render_image<Dual>(L, P.data(), cam.W, cam.H, bg, img.data(), T.data(), nullptr, nullptr);
  Dual acc(0.0, 0.0);
  size_t nb = 0;
  for (size_t q = 0; q < npx; ++q)
    if (!mask[q]) { acc = acc + (Dual(1.0, 0.0) - T[q]); ++nb; }
  if (!nb) { if (dpen) *dpen = 0.0; return 0.0; }
  if (dpen) *dpen = lam * acc.d / (double)nb;
  return lam * acc.v / (double)nb;
}

// Textbook Adam with bias correction, one step t >= 1, per-element learning rate.
void orc_adam(long long n, double* p, const double* g, double* m, double* v, const double* lr,
              double beta1, double beta2, double eps, int t) {
  double bc1 = 1.0 - std::pow(beta1, t), bc2 = 1.0 - std::pow(beta2, t);
  for (long long i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    double mh = m[i] / bc1, vh = v[i] / bc2;
    p[i] -= lr[i] * mh / (std::sqrt(vh) + eps);
  }
}

// Exact k nearest neighbours by brute force (self excluded), ordered by
// (distance, index).  dist is the Euclidean distance.
void orc_knn(int n, const double* pts, int k, int* idx, double* dist) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; ++i) {
    std::vector<std::pair<double, int>> c;
    c.reserve(n);
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = pts[3 * j] - pts[3 * i], dy = pts[3 * j + 1] - pts[3 * i + 1], dz = pts[3 * j + 2] - pts[3 * i + 2];
      c.push_back({dx * dx + dy * dy + dz * dz, j});
    }
    int kk = std::min(k, (int)c.size());
    std::partial_sort(c.begin(), c.begin() + kk, c.end());
    for (int a = 0; a < k; ++a) {
      idx[(size_t)k * i + a] = a < kk ? c[a].second : -1;
      dist[(size_t)k * i + a] = a < kk ? std::sqrt(c[a].first) : INFINITY;
    }
  }
}

// Ghost filter of the merge: keep Gaussian i of partition k iff its mean lies
// in partition k's owned box [lo, hi) (a box side with closed_hi set is closed).
void orc_owned(int n, const double* means, const int* part_of, const double* boxes,
               const int* closed_hi, unsigned char* keep) {
  for (int i = 0; i < n; ++i) {
    int k = part_of[i];
    const double* b = boxes + 6 * k;
    bool in = true;
    for (int a = 0; a < 3; ++a) {
      double x = means[3 * i + a];
      bool hi_ok = closed_hi[3 * k + a] ? (x <= b[3 + a]) : (x < b[3 + a]);
      in = in && (x >= b[a]) && hi_ok;
    }
    keep[i] = in ? 1 : 0;
  }
}

}  // extern "C"
