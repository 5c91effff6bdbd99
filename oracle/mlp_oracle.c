/*
 * mlp_oracle.c -- FP64 oracle of the seed network (learned IK seeds).
 *
 * TEST INFRASTRUCTURE ONLY.  The paper has no learned component; this network
 * is the learned-seed pattern added around its LM solver: a multilayer
 * perceptron maps a target pose (position plus the 6-D rotation made of the
 * first two columns of R) to K joint-space proposals, and its output head maps
 * each proposal into the joint limits with q = mid + half * tanh(y).
 *
 * Parameter layout (one contiguous double array): for every layer l,
 * W_l [d_{l+1}][d_l] row-major followed by b_l [d_{l+1}].  Hidden layers use
 * SiLU(x) = x / (1 + exp(-x)); the last layer is linear.
 *
 * Loss of one sample with label q*: e_k = |q_k - q*|^2, L = min_k e_k +
 * mu * mean_k e_k (ties in the min go to the lowest k); the batch loss is the
 * mean over samples.  The AdamW step follows Loshchilov & Hutter (decoupled
 * weight decay) with bias-corrected moments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double silu(double x) { return x / (1.0 + exp(-x)); }
static double dsilu(double x) {
  double s = 1.0 / (1.0 + exp(-x));
  return s * (1.0 + x * (1.0 - s));
}

static long n_params(int n_layers, const int32_t* dims) {
  long n = 0;
  for (int l = 0; l < n_layers; ++l) n += (long)dims[l + 1] * dims[l] + dims[l + 1];
  return n;
}

/* Forward pass of M samples; y_out [M][dims[n_layers]] (pre-head outputs). */
int32_t or_mlp_forward(int32_t n_layers, const int32_t* dims, const double* params, int32_t M,
                       const double* x, double* y_out) {
  int maxd = 0;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] > maxd) maxd = dims[l];
  double* a = (double*)malloc(sizeof(double) * maxd);
  double* z = (double*)malloc(sizeof(double) * maxd);
  for (int m = 0; m < M; ++m) {
    memcpy(a, x + (long)m * dims[0], sizeof(double) * dims[0]);
    const double* P = params;
    for (int l = 0; l < n_layers; ++l) {
      const int di = dims[l], dout = dims[l + 1];
      const double* W = P;
      const double* b = P + (long)dout * di;
      for (int o = 0; o < dout; ++o) {
        double s = b[o];
        for (int i = 0; i < di; ++i) s += W[(long)o * di + i] * a[i];
        z[o] = s;
      }
      P += (long)dout * di + dout;
      for (int o = 0; o < dout; ++o) a[o] = (l + 1 < n_layers) ? silu(z[o]) : z[o];
    }
    memcpy(y_out + (long)m * dims[n_layers], a, sizeof(double) * dims[n_layers]);
  }
  free(a);
  free(z);
  return 0;
}

/* x rounded to BF16 (8 significant bits, round to nearest, ties to even):
 * x = m 2^e with 1/2 <= |m| < 1, and m 2^8 rounded to an integer. */
static double round_bf16(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  const double m = frexp(x, &e);
  return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* Exported for the pins. */
void or_round_bf16(int64_t n, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) y[i] = round_bf16(x[i]);
}

/* The forward pass at the precision the seed network runs in: every layer's
 * operands are BF16 (the weights and the inputs are given BF16-rounded; each
 * hidden layer's SiLU output is rounded to BF16 before it enters the next
 * layer), sums and SiLU in FP64.  y_out [M][d_L] pre-head outputs; scale_out
 * (optional) [M][d_L]: sum_i |W_oi| |a_i| + |b_o| of the output layer, the
 * magnitude that rounding differences in its inputs are relative to. */
int32_t or_mlp_forward_bf16(int32_t n_layers, const int32_t* dims, const double* params, int32_t M,
                            const double* x, double* y_out, double* scale_out) {
  int maxd = 0;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] > maxd) maxd = dims[l];
  double* a = (double*)malloc(sizeof(double) * maxd);
  double* z = (double*)malloc(sizeof(double) * maxd);
  for (int m = 0; m < M; ++m) {
    memcpy(a, x + (long)m * dims[0], sizeof(double) * dims[0]);
    const double* P = params;
    for (int l = 0; l < n_layers; ++l) {
      const int di = dims[l], dout = dims[l + 1];
      const double* W = P;
      const double* b = P + (long)dout * di;
      const int last = l + 1 == n_layers;
      for (int o = 0; o < dout; ++o) {
        double s = b[o], mag = fabs(b[o]);
        for (int i = 0; i < di; ++i) {
          s += W[(long)o * di + i] * a[i];
          mag += fabs(W[(long)o * di + i]) * fabs(a[i]);
        }
        z[o] = s;
        if (last && scale_out) scale_out[(long)m * dout + o] = mag;
      }
      P += (long)dout * di + dout;
      for (int o = 0; o < dout; ++o) a[o] = last ? z[o] : round_bf16(silu(z[o]));
    }
    memcpy(y_out + (long)m * dims[n_layers], a, sizeof(double) * dims[n_layers]);
  }
  free(a);
  free(z);
  return 0;
}

/*
 * Loss and gradient over M samples.  The last layer has K * n outputs; the
 * head maps output (k, i) to q = mid_i + half_i tanh(y), mid/half from the
 * limits lo/hi [n].  grad_out has the parameter layout; q_out (optional)
 * [M][K][n]; returns the mean loss in *loss_out.
 */
int32_t or_mlp_loss_grad(int32_t n_layers, const int32_t* dims, const double* params, int32_t M,
                         const double* x, const double* q_star, int32_t K, int32_t n,
                         const double* lo, const double* hi, double mu, double* grad_out,
                         double* q_out, double* loss_out) {
  if (dims[n_layers] != K * n) return 1;
  const long np = n_params(n_layers, dims);
  memset(grad_out, 0, sizeof(double) * np);
  int width = 0;
  for (int l = 0; l <= n_layers; ++l) width += dims[l];
  /* per-layer pre-activations z_l and activations a_l (a_0 = x) */
  double* zs = (double*)malloc(sizeof(double) * width);
  double* as = (double*)malloc(sizeof(double) * width);
  long* off = (long*)malloc(sizeof(long) * (n_layers + 1));
  long* poff = (long*)malloc(sizeof(long) * n_layers);
  off[0] = 0;
  for (int l = 0; l < n_layers; ++l) off[l + 1] = off[l] + dims[l];
  poff[0] = 0;
  for (int l = 1; l < n_layers; ++l) poff[l] = poff[l - 1] + (long)dims[l] * dims[l - 1] + dims[l];
  int maxd = 0;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] > maxd) maxd = dims[l];
  double* g = (double*)malloc(sizeof(double) * maxd);
  double* gp = (double*)malloc(sizeof(double) * maxd);
  double* e = (double*)malloc(sizeof(double) * K);
  double loss = 0;
  for (int m = 0; m < M; ++m) {
    /* forward */
    memcpy(as + off[0], x + (long)m * dims[0], sizeof(double) * dims[0]);
    for (int l = 0; l < n_layers; ++l) {
      const int di = dims[l], dout = dims[l + 1];
      const double* W = params + poff[l];
      const double* b = W + (long)dout * di;
      for (int o = 0; o < dout; ++o) {
        double s = b[o];
        for (int i = 0; i < di; ++i) s += W[(long)o * di + i] * as[off[l] + i];
        zs[off[l + 1] + o] = s;
        as[off[l + 1] + o] = (l + 1 < n_layers) ? silu(s) : s;
      }
    }
    /* head and loss */
    const double* y = as + off[n_layers];
    const double* qs = q_star + (long)m * n;
    int best = 0;
    double mean = 0;
    for (int k = 0; k < K; ++k) {
      double s = 0;
      for (int i = 0; i < n; ++i) {
        double mid = 0.5 * (lo[i] + hi[i]), half = 0.5 * (hi[i] - lo[i]);
        double q = mid + half * tanh(y[k * n + i]);
        if (q_out) q_out[((long)m * K + k) * n + i] = q;
        s += (q - qs[i]) * (q - qs[i]);
      }
      e[k] = s;
      mean += s / K;
      if (s < e[best]) best = k;
    }
    loss += e[best] + mu * mean;
    /* dL/dy */
    for (int k = 0; k < K; ++k) {
      double w = (k == best ? 1.0 : 0.0) + mu / K;
      for (int i = 0; i < n; ++i) {
        double half = 0.5 * (hi[i] - lo[i]);
        double t = tanh(y[k * n + i]);
        double q = 0.5 * (lo[i] + hi[i]) + half * t;
        g[k * n + i] = w * 2.0 * (q - qs[i]) * half * (1.0 - t * t) / M;
      }
    }
    /* backward through the layers */
    for (int l = n_layers - 1; l >= 0; --l) {
      const int di = dims[l], dout = dims[l + 1];
      const double* W = params + poff[l];
      double* gW = grad_out + poff[l];
      double* gb = gW + (long)dout * di;
      if (l + 1 < n_layers)
        for (int o = 0; o < dout; ++o) g[o] *= dsilu(zs[off[l + 1] + o]);
      for (int o = 0; o < dout; ++o) {
        gb[o] += g[o];
        for (int i = 0; i < di; ++i) gW[(long)o * di + i] += g[o] * as[off[l] + i];
      }
      if (l > 0) {
        for (int i = 0; i < di; ++i) {
          double s = 0;
          for (int o = 0; o < dout; ++o) s += W[(long)o * di + i] * g[o];
          gp[i] = s;
        }
        memcpy(g, gp, sizeof(double) * di);
      }
    }
  }
  *loss_out = loss / M;
  free(zs); free(as); free(off); free(poff); free(g); free(gp); free(e);
  return 0;
}

/* One AdamW step on n parameters (bias-corrected moments, decoupled decay). */
void or_adamw(int64_t n, double* p, const double* grad, double* m, double* v, double lr,
              double beta1, double beta2, double eps, double wd, int64_t step) {
  const double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * (mh / (sqrt(vh) + eps) + wd * p[i]);
  }
}
