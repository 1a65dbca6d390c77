/* CPU oracle of the learned-closure network: a multilayer perceptron
 * 15 -> 128 -> 128 -> 3 with GELU (tanh form, Hendrycks & Gimpel) on the two
 * hidden layers, mean-squared-error loss, and Adam (Kingma & Ba).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite and the benchmark's
 * CPU-baseline leg, never by the product path.  It shares no code with the
 * CUDA library.  Plain FP64 loops; with bf16 != 0 the inputs, weights and
 * hidden activations are rounded to bfloat16 (nearest even) before every
 * product, at the points where the GPU kernels round them.
 *
 * Parameter layout (flat, FP64): W1[128][15], b1[128], W2[128][128], b2[128],
 * W3[3][128], b3[3]  (row = output unit).
 * Pinned by tests/test_oracle_mlp.py against torch's CPU autograd and Adam.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#define NI 15
#define NH 128
#define NO 3
#define NPARAM (NH * NI + NH + NH * NH + NH + NO * NH + NO)

static double bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static double gelu(double z) {
  const double c = 0.7978845608028654;  /* sqrt(2/pi) */
  return 0.5 * z * (1.0 + tanh(c * (z + 0.044715 * z * z * z)));
}
static double gelu_d(double z) {
  const double c = 0.7978845608028654;
  double th = tanh(c * (z + 0.044715 * z * z * z));
  return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * c * (1.0 + 3.0 * 0.044715 * z * z);
}

int mlp_nparam(void) { return NPARAM; }

/* loss = mean over samples and outputs of (y - t)^2; grad (NPARAM) = d loss / d params
 * (grad may be NULL); y (n x 3) may be NULL. */
double mlp_forward_backward(const double *P, const double *X, const double *T, int n, int bf, double *y_out,
                            double *grad) {
  const double *W1 = P, *b1 = W1 + NH * NI, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH, *b3 = W3 + NO * NH;
  double *g = grad;
  if (g) memset(g, 0, sizeof(double) * NPARAM);
  double *gW1 = g, *gb1 = g ? g + NH * NI : 0, *gW2 = g ? gb1 + NH : 0, *gb2 = g ? gW2 + NH * NH : 0,
         *gW3 = g ? gb2 + NH : 0, *gb3 = g ? gW3 + NO * NH : 0;
  double loss = 0.0;
  double x[NI], z1[NH], a1[NH], z2[NH], a2[NH], y[NO], dy[NO], da2[NH], dz2[NH], da1[NH], dz1[NH];
  for (int s = 0; s < n; ++s) {
    for (int i = 0; i < NI; ++i) x[i] = bf ? bf16(X[s * NI + i]) : X[s * NI + i];
    for (int h = 0; h < NH; ++h) {
      double acc = 0.0;
      for (int i = 0; i < NI; ++i) acc += (bf ? bf16(W1[h * NI + i]) : W1[h * NI + i]) * x[i];
      z1[h] = acc + b1[h];
      a1[h] = gelu(z1[h]);
      if (bf) a1[h] = bf16(a1[h]);
    }
    for (int h = 0; h < NH; ++h) {
      double acc = 0.0;
      for (int k = 0; k < NH; ++k) acc += (bf ? bf16(W2[h * NH + k]) : W2[h * NH + k]) * a1[k];
      z2[h] = acc + b2[h];
      a2[h] = gelu(z2[h]);
      if (bf) a2[h] = bf16(a2[h]);
    }
    for (int o = 0; o < NO; ++o) {
      double acc = 0.0;
      for (int k = 0; k < NH; ++k) acc += (bf ? bf16(W3[o * NH + k]) : W3[o * NH + k]) * a2[k];
      y[o] = acc + b3[o];
      if (y_out) y_out[s * NO + o] = y[o];
      double d = y[o] - T[s * NO + o];
      loss += d * d;
      dy[o] = 2.0 * d / ((double)n * NO);
    }
    if (!g) continue;
    /* backward: the same bf16 roundings of the operands as the forward pass */
    double dyb[NO];
    for (int o = 0; o < NO; ++o) {
      dyb[o] = bf ? bf16(dy[o]) : dy[o];
      gb3[o] += dy[o];
      for (int k = 0; k < NH; ++k) gW3[o * NH + k] += dyb[o] * a2[k];
    }
    for (int k = 0; k < NH; ++k) {
      double acc = 0.0;
      for (int o = 0; o < NO; ++o) acc += dyb[o] * (bf ? bf16(W3[o * NH + k]) : W3[o * NH + k]);
      da2[k] = acc;
      dz2[k] = da2[k] * gelu_d(z2[k]);
    }
    for (int h = 0; h < NH; ++h) {
      double d = bf ? bf16(dz2[h]) : dz2[h];
      gb2[h] += dz2[h];
      for (int k = 0; k < NH; ++k) gW2[h * NH + k] += d * a1[k];
    }
    for (int k = 0; k < NH; ++k) {
      double acc = 0.0;
      for (int h = 0; h < NH; ++h) acc += (bf ? bf16(dz2[h]) : dz2[h]) * (bf ? bf16(W2[h * NH + k]) : W2[h * NH + k]);
      da1[k] = acc;
      dz1[k] = da1[k] * gelu_d(z1[k]);
    }
    for (int h = 0; h < NH; ++h) {
      double d = bf ? bf16(dz1[h]) : dz1[h];
      gb1[h] += dz1[h];
      for (int i = 0; i < NI; ++i) gW1[h * NI + i] += d * x[i];
    }
  }
  return loss / ((double)n * NO);
}

/* one Adam step (Kingma & Ba): t is the 1-based step number */
void mlp_adam(double *P, const double *grad, double *m, double *v, int t, double lr, double b1, double b2,
              double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int k = 0; k < NPARAM; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * grad[k];
    v[k] = b2 * v[k] + (1.0 - b2) * grad[k] * grad[k];
    double mh = m[k] / c1, vh = v[k] / c2;
    P[k] -= lr * mh / (sqrt(vh) + eps);
  }
}
