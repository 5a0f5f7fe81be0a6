// FP64 CPU oracle for the learned initialiser: kNN geometry features and the
// 3-layer MLP that maps them to initial scale, rotation and opacity.
//
// TEST INFRASTRUCTURE ONLY (see gs_oracle.cpp).  Shares no code with the CUDA
// library.
//
// The network: X[n][112] -> relu(X W1 + b1)[64] -> relu(. W2 + b2)[64] -> . W3 + b3 [8]
// with every GEMM operand rounded to bfloat16 (round to nearest even) and the
// products accumulated exactly (here in FP64; the CUDA path accumulates in
// FP32).  Activations are rounded to bf16 where they become the next GEMM's
// operand.  Loss: mean squared error over the 8 outputs.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace orc_mlp {

// Round a double to the nearest bfloat16 value (8 significant bits), ties to
// even, by scaling to the bf16 grid of the value's binade.
static double bf16(double x) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  int e;
  std::frexp(x, &e);  // |x| in [2^(e-1), 2^e)
  double ulp = std::ldexp(1.0, e - 8);
  double q = x / ulp;
  double r = std::nearbyint(q);  // default rounding mode: to nearest, ties to even
  return r * ulp;
}

static const int KIN = 112, HID = 64, KOUT = 8, KNN = 16;

}  // namespace orc_mlp

using namespace orc_mlp;

extern "C" {

double orc_bf16_round(double x) { return bf16(x); }

void orc_bf16_round_array(long long n, const double* x, double* out) {
  for (long long k = 0; k < n; ++k) out[k] = bf16(x[k]);
}

// Features of point i from its 16 nearest neighbours (sorted by distance):
// [0, 48)   neighbour offsets (p_j - p_i) divided by the mean neighbour distance
// [48, 96)  neighbour unit normals
// [96, 99)  own unit normal
// [99, 112) zero padding
void orc_mlp_features(int n, const double* pts, const double* nrm, const int* knn_idx,
                      const double* knn_dist, double* X) {
  for (int i = 0; i < n; ++i) {
    double* x = X + (size_t)KIN * i;
    for (int k = 0; k < KIN; ++k) x[k] = 0.0;
    double dbar = 0;
    for (int a = 0; a < KNN; ++a) dbar += knn_dist[(size_t)KNN * i + a];
    dbar /= KNN;
    if (!(dbar > 1e-12)) dbar = 1e-12;
    for (int a = 0; a < KNN; ++a) {
      int j = knn_idx[(size_t)KNN * i + a];
      for (int c = 0; c < 3; ++c) {
        x[3 * a + c] = (pts[3 * j + c] - pts[3 * i + c]) / dbar;
        x[48 + 3 * a + c] = nrm[3 * j + c];
      }
    }
    for (int c = 0; c < 3; ++c) x[96 + c] = nrm[3 * i + c];
  }
}

// Forward pass.  H1, H2 are the post-ReLU activations before their bf16
// rounding; Y the outputs; A1, A2 (may be NULL) the pre-activations.
void orc_mlp_forward_full(int n, const double* X, const double* W1, const double* b1, const double* W2,
                          const double* b2, const double* W3, const double* b3, double* H1, double* H2,
                          double* Y, double* A1, double* A2) {
  std::vector<double> w1(KIN * HID), w2(HID * HID), w3(HID * KOUT);
  for (int k = 0; k < KIN * HID; ++k) w1[k] = bf16(W1[k]);
  for (int k = 0; k < HID * HID; ++k) w2[k] = bf16(W2[k]);
  for (int k = 0; k < HID * KOUT; ++k) w3[k] = bf16(W3[k]);
  for (int i = 0; i < n; ++i) {
    double xb[KIN], h1b[HID], h2b[HID];
    for (int k = 0; k < KIN; ++k) xb[k] = bf16(X[(size_t)KIN * i + k]);
    for (int o = 0; o < HID; ++o) {
      double acc = 0;
      for (int k = 0; k < KIN; ++k) acc += xb[k] * w1[k * HID + o];
      acc += b1[o];
      if (A1) A1[(size_t)HID * i + o] = acc;
      double h = acc > 0 ? acc : 0.0;
      H1[(size_t)HID * i + o] = h;
      h1b[o] = bf16(h);
    }
    for (int o = 0; o < HID; ++o) {
      double acc = 0;
      for (int k = 0; k < HID; ++k) acc += h1b[k] * w2[k * HID + o];
      acc += b2[o];
      if (A2) A2[(size_t)HID * i + o] = acc;
      double h = acc > 0 ? acc : 0.0;
      H2[(size_t)HID * i + o] = h;
      h2b[o] = bf16(h);
    }
    for (int o = 0; o < KOUT; ++o) {
      double acc = 0;
      for (int k = 0; k < HID; ++k) acc += h2b[k] * w3[k * KOUT + o];
      Y[(size_t)KOUT * i + o] = acc + b3[o];
    }
  }
}

void orc_mlp_forward(int n, const double* X, const double* W1, const double* b1, const double* W2,
                     const double* b2, const double* W3, const double* b3, double* H1, double* H2,
                     double* Y) {
  orc_mlp_forward_full(n, X, W1, b1, W2, b2, W3, b3, H1, H2, Y, nullptr, nullptr);
}

// Loss L = sum (Y - T)^2 / (8 n) and its weight gradients, by the chain rule
// written out layer by layer.  The back-propagated signals are rounded to
// bf16 where they become GEMM operands (dY, dH2, dH1), and the bias gradients
// sum those rounded signals.  ReLU passes the gradient where the pre-activation
// was > 0.  Returns L.
double orc_mlp_backward(int n, const double* X, const double* W1, const double* b1, const double* W2,
                        const double* b2, const double* W3, const double* b3, const double* T,
                        double* dW1, double* db1, double* dW2, double* db2, double* dW3, double* db3) {
  std::vector<double> H1((size_t)n * HID), H2((size_t)n * HID), Y((size_t)n * KOUT);
  orc_mlp_forward(n, X, W1, b1, W2, b2, W3, b3, H1.data(), H2.data(), Y.data());
  std::vector<double> w2(HID * HID), w3(HID * KOUT);
  for (int k = 0; k < HID * HID; ++k) w2[k] = bf16(W2[k]);
  for (int k = 0; k < HID * KOUT; ++k) w3[k] = bf16(W3[k]);
  std::memset(dW1, 0, sizeof(double) * KIN * HID);
  std::memset(dW2, 0, sizeof(double) * HID * HID);
  std::memset(dW3, 0, sizeof(double) * HID * KOUT);
  std::memset(db1, 0, sizeof(double) * HID);
  std::memset(db2, 0, sizeof(double) * HID);
  std::memset(db3, 0, sizeof(double) * KOUT);
  double L = 0;
  double scale = 1.0 / (8.0 * n);
  for (int i = 0; i < n; ++i) {
    double dy[KOUT], dh2[HID], dh1[HID], xb[KIN], h1b[HID], h2b[HID];
    for (int k = 0; k < KIN; ++k) xb[k] = bf16(X[(size_t)KIN * i + k]);
    for (int k = 0; k < HID; ++k) { h1b[k] = bf16(H1[(size_t)HID * i + k]); h2b[k] = bf16(H2[(size_t)HID * i + k]); }
    for (int o = 0; o < KOUT; ++o) {
      double e = Y[(size_t)KOUT * i + o] - T[(size_t)KOUT * i + o];
      L += e * e;
      dy[o] = bf16(2.0 * e * scale);
    }
    for (int o = 0; o < KOUT; ++o) {
      db3[o] += dy[o];
      for (int k = 0; k < HID; ++k) dW3[k * KOUT + o] += h2b[k] * dy[o];
    }
    for (int k = 0; k < HID; ++k) {
      double acc = 0;
      for (int o = 0; o < KOUT; ++o) acc += dy[o] * w3[k * KOUT + o];
      dh2[k] = bf16(H2[(size_t)HID * i + k] > 0 ? acc : 0.0);
    }
    for (int o = 0; o < HID; ++o) {
      db2[o] += dh2[o];
      for (int k = 0; k < HID; ++k) dW2[k * HID + o] += h1b[k] * dh2[o];
    }
    for (int k = 0; k < HID; ++k) {
      double acc = 0;
      for (int o = 0; o < HID; ++o) acc += dh2[o] * w2[k * HID + o];
      dh1[k] = bf16(H1[(size_t)HID * i + k] > 0 ? acc : 0.0);
    }
    for (int o = 0; o < HID; ++o) {
      db1[o] += dh1[o];
      for (int k = 0; k < KIN; ++k) dW1[k * HID + o] += xb[k] * dh1[o];
    }
  }
  return L * scale;
}

// Initial Gaussian parameters from the kNN distances (and optionally the MLP
// outputs Y [n][8]): log-scale log(max(d3, 1e-7)) (+ Y[0:3]), rotation
// identity (or Y[3:7]), logit opacity logit_default (or Y[7]); a Gaussian whose
// outputs are non-finite or whose rotation has norm <= 1e-6 keeps the plain
// values.  d3 = mean of the first three neighbour distances.
void orc_init_gaussians(int n, const double* knn_dist, int k, const double* Y, double logit_default,
                        double* log_scales, double* quats, double* logit) {
  for (int i = 0; i < n; ++i) {
    double d3 = (knn_dist[(size_t)k * i] + knn_dist[(size_t)k * i + 1] + knn_dist[(size_t)k * i + 2]) / 3.0;
    double ls = std::log(d3 > 1e-7 ? d3 : 1e-7);
    double q[4] = {1, 0, 0, 0};
    double s[3] = {ls, ls, ls};
    double lo = logit_default;
    if (Y) {
      const double* y = Y + (size_t)KOUT * i;
      bool ok = true;
      for (int c = 0; c < KOUT; ++c) ok = ok && std::isfinite(y[c]);
      double qn = std::sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
      if (ok && qn > 1e-6) {
        for (int c = 0; c < 3; ++c) s[c] = ls + y[c];
        for (int c = 0; c < 4; ++c) q[c] = y[3 + c];
        lo = y[7];
      }
    }
    for (int c = 0; c < 3; ++c) log_scales[3 * i + c] = s[c];
    for (int c = 0; c < 4; ++c) quats[4 * i + c] = q[c];
    logit[i] = lo;
  }
}

}  // extern "C"
