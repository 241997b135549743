/*
 * Oracle of the learned predictor and the residual codec mode.  TEST
 * INFRASTRUCTURE ONLY (see tera_oracle.h).  Not in the paper: the paper's
 * difference is taken against the previous record (Sec. 2.3); here a small
 * MLP predicts each agent's next position from its recent motion, and the
 * position words carry the integer difference of the bit patterns instead.
 *
 * MLP 8 -> 64 -> 64 -> 3, ReLU on the hidden layers.  Parameters (4931
 * floats): W1[64][8], b1[64], W2[64][64], b2[64], W3[3][64], b3[3].
 * Inference (float32): for each neuron j, acc = b[j]; for k ascending,
 * acc = fmaf(W[j][k], in[k], acc); hidden outputs relu(v) = (v > 0 ? v : 0).
 * Training reference (float64): the same network in double precision, MSE
 * loss (1/n) sum_i sum_a (o_ia - y_ia)^2, analytic gradient, plain SGD.
 *
 * Per reference slot a history record of 48 bytes travels with the reference
 * on both sides:  u64 xp[3] (bits of the position one iteration before the
 * reference's) | u32 d2[3] (bits of (float)(xp - the position before it)) |
 * u32 n (valid steps: 0, 1, 2) | u64 zero.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tera_oracle.h"

#define IN 8
#define H 64
#define OUT 3
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + H * IN)
#define OFF_W2 (OFF_B1 + H)
#define OFF_B2 (OFF_W2 + H * H)
#define OFF_W3 (OFF_B2 + H)
#define OFF_B3 (OFF_W3 + OUT * H)
#define NPARAM (OFF_B3 + OUT)

int or_mlp_nparam(void) { return NPARAM; }

static float relu_f(float v) { return v > 0.0f ? v : 0.0f; }
static double relu_d(double v) { return v > 0.0 ? v : 0.0; }

void or_mlp_infer_f32(const float* p, const float* in, float* out) {
  float h1[H], h2[H];
  for (int j = 0; j < H; ++j) {
    float acc = p[OFF_B1 + j];
    for (int k = 0; k < IN; ++k) acc = fmaf(p[OFF_W1 + j * IN + k], in[k], acc);
    h1[j] = relu_f(acc);
  }
  for (int j = 0; j < H; ++j) {
    float acc = p[OFF_B2 + j];
    for (int k = 0; k < H; ++k) acc = fmaf(p[OFF_W2 + j * H + k], h1[k], acc);
    h2[j] = relu_f(acc);
  }
  for (int j = 0; j < OUT; ++j) {
    float acc = p[OFF_B3 + j];
    for (int k = 0; k < H; ++k) acc = fmaf(p[OFF_W3 + j * H + k], h2[k], acc);
    out[j] = acc;
  }
}

/* Loss over n samples and (optionally) its gradient, all in float64. */
double or_mlp_loss_grad_f64(const double* p, const double* X, const double* Y, int64_t n,
                            double* grad) {
  if (grad) memset(grad, 0, sizeof(double) * NPARAM);
  double loss = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double* x = X + i * IN;
    const double* y = Y + i * OUT;
    double z1[H], a1[H], z2[H], a2[H], o[OUT];
    for (int j = 0; j < H; ++j) {
      double acc = p[OFF_B1 + j];
      for (int k = 0; k < IN; ++k) acc += p[OFF_W1 + j * IN + k] * x[k];
      z1[j] = acc;
      a1[j] = relu_d(acc);
    }
    for (int j = 0; j < H; ++j) {
      double acc = p[OFF_B2 + j];
      for (int k = 0; k < H; ++k) acc += p[OFF_W2 + j * H + k] * a1[k];
      z2[j] = acc;
      a2[j] = relu_d(acc);
    }
    for (int j = 0; j < OUT; ++j) {
      double acc = p[OFF_B3 + j];
      for (int k = 0; k < H; ++k) acc += p[OFF_W3 + j * H + k] * a2[k];
      o[j] = acc;
    }
    double go[OUT];
    for (int j = 0; j < OUT; ++j) {
      const double e = o[j] - y[j];
      loss += e * e;
      go[j] = 2.0 * e / (double)n;  /* d loss / d o */
    }
    if (!grad) continue;
    double g2[H], g1[H];
    for (int k = 0; k < H; ++k) g2[k] = 0.0;
    for (int j = 0; j < OUT; ++j) {
      grad[OFF_B3 + j] += go[j];
      for (int k = 0; k < H; ++k) {
        grad[OFF_W3 + j * H + k] += go[j] * a2[k];
        g2[k] += go[j] * p[OFF_W3 + j * H + k];
      }
    }
    for (int k = 0; k < H; ++k) g2[k] = z2[k] > 0.0 ? g2[k] : 0.0;  /* through relu */
    for (int k = 0; k < H; ++k) g1[k] = 0.0;
    for (int j = 0; j < H; ++j) {
      grad[OFF_B2 + j] += g2[j];
      for (int k = 0; k < H; ++k) {
        grad[OFF_W2 + j * H + k] += g2[j] * a1[k];
        g1[k] += g2[j] * p[OFF_W2 + j * H + k];
      }
    }
    for (int k = 0; k < H; ++k) g1[k] = z1[k] > 0.0 ? g1[k] : 0.0;
    for (int j = 0; j < H; ++j) {
      grad[OFF_B1 + j] += g1[j];
      for (int k = 0; k < IN; ++k) grad[OFF_W1 + j * IN + k] += g1[j] * x[k];
    }
  }
  return loss / (double)n;
}

void or_mlp_sgd_f64(double* p, const double* grad, double lr) {
  for (int i = 0; i < NPARAM; ++i) p[i] -= lr * grad[i];
}

/* One SGD step with global-norm clipping (the predictor's training rule, not
 * in the paper): with |g| the Euclidean norm of the whole gradient,
 * c = clip / |g| when clip > 0 and |g| > clip, else c = 1; p -= lr * c * g. */
void or_mlp_sgd_clip_f64(double* p, const double* grad, double lr, double clip) {
  double ss = 0.0;
  for (int i = 0; i < NPARAM; ++i) ss += grad[i] * grad[i];
  double norm = sqrt(ss);
  double c = (clip > 0.0 && norm > clip) ? clip / norm : 1.0;
  for (int i = 0; i < NPARAM; ++i) p[i] -= lr * c * grad[i];
}

/* ---------- features, history, residual ---------- */

static uint64_t rd64(const uint8_t* b) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)b[i] << (8 * i);
  return v;
}
static uint32_t rd32(const uint8_t* b) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)b[i] << (8 * i);
  return v;
}
static void wr64(uint8_t* b, uint64_t v) {
  for (int i = 0; i < 8; ++i) b[i] = (uint8_t)(v >> (8 * i));
}
static void wr32(uint8_t* b, uint32_t v) {
  for (int i = 0; i < 4; ++i) b[i] = (uint8_t)(v >> (8 * i));
}
static double as_d(uint64_t u) {
  double d;
  memcpy(&d, &u, 8);
  return d;
}
static uint64_t bits_d(double d) {
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
}
static float as_f(uint32_t u) {
  float f;
  memcpy(&f, &u, 4);
  return f;
}
static uint32_t bits_f(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

uint64_t or_zigzag(uint64_t d) { return (d << 1) ^ (uint64_t)((int64_t)d >> 63); }
uint64_t or_unzigzag(uint64_t z) { return (z >> 1) ^ (0 - (z & 1)); }

/* Cell of a position: floor((v - lo) / w) on each axis, in binary64. */
static void cell_of(const uint8_t* rec, const double lo[3], double w, int64_t c[3]) {
  for (int a = 0; a < 3; ++a) c[a] = (int64_t)floor((as_d(rd64(rec + 8 * (a + 1))) - lo[a]) / w);
}

/* Neighbour count of each reference slot: records of the same reference in
 * the same cell (the slot itself included). */
void or_cell_counts(const uint8_t* ref, uint64_t r, const double lo[3], double w,
                    uint32_t* count) {
  int64_t* cells = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(r ? r : 1));
  for (uint64_t j = 0; j < r; ++j) cell_of(ref + j * 64, lo, w, cells + 3 * j);
  for (uint64_t j = 0; j < r; ++j) {
    uint32_t c = 0;
    for (uint64_t k = 0; k < r; ++k)
      if (cells[3 * k] == cells[3 * j] && cells[3 * k + 1] == cells[3 * j + 1] &&
          cells[3 * k + 2] == cells[3 * j + 2])
        ++c;
    count[j] = c;
  }
  free(cells);
}

/* Features of reference slot j; returns 1 when the slot is predictable
 * (two steps of history and all features finite). */
int or_features(const uint8_t* rec, const uint8_t* hist, uint32_t ncount, float* f) {
  if (rd32(hist + 36) < 2) return 0;
  for (int a = 0; a < 3; ++a) {
    const double x1 = as_d(rd64(rec + 8 * (a + 1)));  /* x_{t-1} */
    const double x2 = as_d(rd64(hist + 8 * a));       /* x_{t-2} */
    f[a] = (float)(x1 - x2);
    f[3 + a] = as_f(rd32(hist + 24 + 4 * a));         /* (float)(x_{t-2} - x_{t-3}) */
  }
  f[6] = (float)(as_d(rd64(rec + 32)) / 10.0);
  f[7] = (float)ncount * 0.03125f;
  for (int i = 0; i < IN; ++i)
    if (!isfinite(f[i])) return 0;
  return 1;
}

/* Predicted position bits of slot j (3 words); returns 0 when the slot is
 * not predictable (no history, a non-finite feature or output). */
int or_predict(const float* params, const uint8_t* rec, const uint8_t* hist, uint32_t ncount,
               uint64_t* pred_bits) {
  float f[IN], o[OUT];
  if (!or_features(rec, hist, ncount, f)) return 0;
  or_mlp_infer_f32(params, f, o);
  for (int a = 0; a < OUT; ++a)
    if (!isfinite(o[a])) return 0;
  for (int a = 0; a < 3; ++a)
    pred_bits[a] = bits_d(as_d(rd64(rec + 8 * (a + 1))) + (double)o[a]);
  return 1;
}

/* History of a new reference entry made from slot (rec, hist) of the old one;
 * hist == NULL makes the entry of a new record. */
void or_hist_next(const uint8_t* rec, const uint8_t* hist, uint8_t* out) {
  memset(out, 0, 48);
  if (!rec || !hist) return;
  const uint32_t n = rd32(hist + 36);
  for (int a = 0; a < 3; ++a) {
    const uint64_t x1 = rd64(rec + 8 * (a + 1));
    wr64(out + 8 * a, x1);
    if (n >= 1) wr32(out + 24 + 4 * a, bits_f((float)(as_d(x1) - as_d(rd64(hist + 8 * a)))));
  }
  wr32(out + 36, n + 1 > 2 ? 2 : n + 1);
}

/* Training sample of a matched slot: features and target displacement
 * (float)(x_t - x_{t-1}); returns 0 when the slot is not predictable. */
int or_sample(const uint8_t* cur, const uint8_t* rec, const uint8_t* hist, uint32_t ncount,
              float* x, float* y) {
  if (!or_features(rec, hist, ncount, x)) return 0;
  for (int a = 0; a < 3; ++a)
    y[a] = (float)(as_d(rd64(cur + 8 * (a + 1))) - as_d(rd64(rec + 8 * (a + 1))));
  return 1;
}
