// pk_math.cuh -- FP32 device math for the kinematic LM kernels (sm_103a).
//
// Rigid transforms, the SE(3) logarithm, the blocks of the inverse SE(3) left
// Jacobian, and register-resident packed Cholesky.  Everything is written for
// one thread owning one problem: small fixed-size arrays that the compiler
// keeps in registers once the loops are unrolled.
//
// Conventions: a transform is 3x4 row-major [R | t]; twists are [rho; omega].
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace pk {

// sin and cos of an angle in radians: Cody-Waite reduction x = k pi/2 + r
// with pi/2 split into a float head and tail (two FMAs; exact enough for the
// few-radian joint angles of the LM iterates), then the Taylor series of sin
// and cos on |r| <= pi/4 (truncated after r^9 / 9! and r^10 / 10!:
// truncation below 2e-9), and the quadrant from k mod 4.  A few FMAs instead
// of a general library routine keeps one LM iteration of one thread short.
__device__ __forceinline__ void sincos_rad(float x, float* s, float* c) {
  const float kf = rintf(x * 0.636619772367581343f);  // 2 / pi
  float r = fmaf(-kf, 1.57079637050628662f, x);       // pi/2 rounded to float
  r = fmaf(-kf, -4.37113900018624283e-8f, r);         // pi/2 - (its float)
  const float r2 = r * r;
  const float sp = fmaf(r2, fmaf(r2, fmaf(r2, fmaf(r2, 2.75573192e-6f, -1.98412698e-4f), 8.33333333e-3f),
                                 -1.66666667e-1f), 1.f) * r;
  const float cp = fmaf(r2, fmaf(r2, fmaf(r2, fmaf(r2, fmaf(r2, -2.75573192e-7f, 2.48015873e-5f), -1.38888889e-3f),
                                           4.16666667e-2f), -0.5f), 1.f);
  const int q = (int)kf & 3;
  const float ss = (q & 1) ? cp : sp, cc = (q & 1) ? sp : cp;
  *s = (q & 2) ? -ss : ss;
  *c = ((q + 1) & 2) ? -cc : cc;
}

struct Rt {
  float r[9];  // row-major rotation
  float t[3];
};

__device__ __forceinline__ void rt_load(const float* __restrict__ p, Rt& a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) a.r[i * 3 + j] = p[i * 4 + j];
    a.t[i] = p[i * 4 + 3];
  }
}

__device__ __forceinline__ void rt_store(float* __restrict__ p, const Rt& a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) p[i * 4 + j] = a.r[i * 3 + j];
    p[i * 4 + 3] = a.t[i];
  }
}

__device__ __forceinline__ void rt_identity(Rt& a) {
#pragma unroll
  for (int i = 0; i < 9; ++i) a.r[i] = (i % 4 == 0) ? 1.f : 0.f;
  a.t[0] = a.t[1] = a.t[2] = 0.f;
}

// c = a * b
__device__ __forceinline__ void rt_mul(const Rt& a, const Rt& b, Rt& c) {
  Rt o;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      o.r[i * 3 + j] = fmaf(a.r[i * 3 + 0], b.r[0 * 3 + j],
                            fmaf(a.r[i * 3 + 1], b.r[1 * 3 + j], a.r[i * 3 + 2] * b.r[2 * 3 + j]));
    o.t[i] = fmaf(a.r[i * 3 + 0], b.t[0], fmaf(a.r[i * 3 + 1], b.t[1], fmaf(a.r[i * 3 + 2], b.t[2], a.t[i])));
  }
  c = o;
}

// a.t += a.R * d  (compose with a pure translation)
__device__ __forceinline__ void rt_translate(Rt& a, const float* d) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
    a.t[i] = fmaf(a.r[i * 3 + 0], d[0], fmaf(a.r[i * 3 + 1], d[1], fmaf(a.r[i * 3 + 2], d[2], a.t[i])));
}

__device__ __forceinline__ void rt_inv(const Rt& a, Rt& c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.r[i * 3 + j] = a.r[j * 3 + i];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    c.t[i] = -(c.r[i * 3 + 0] * a.t[0] + c.r[i * 3 + 1] * a.t[1] + c.r[i * 3 + 2] * a.t[2]);
}

__device__ __forceinline__ void mat_vec(const float* r, const float* x, float* y) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = fmaf(r[i * 3 + 0], x[0], fmaf(r[i * 3 + 1], x[1], r[i * 3 + 2] * x[2]));
}

__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
  c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
  c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
  c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

// Revolute joint motion applied on the right: R <- R * Rot(a, q).
// With u = R a (the joint axis seen from the frame R is expressed in),
// R Rot(a, q) = cos(q) R + sin(q) [u]x R + (1 - cos(q)) u a^T, column by column.
__device__ __forceinline__ void rot_joint(float* r, const float* u, const float* a, float s, float c) {
  const float omc = 1.f - c;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float x = r[k], y = r[3 + k], z = r[6 + k];
    const float cx = fmaf(u[1], z, -u[2] * y);
    const float cy = fmaf(u[2], x, -u[0] * z);
    const float cz = fmaf(u[0], y, -u[1] * x);
    const float ak = omc * a[k];
    r[k] = fmaf(c, x, fmaf(s, cx, ak * u[0]));
    r[3 + k] = fmaf(c, y, fmaf(s, cy, ak * u[1]));
    r[6 + k] = fmaf(c, z, fmaf(s, cz, ak * u[2]));
  }
}

// ---------------------------------------------------------------------------
// SE(3) logarithm and the inverse left Jacobian.
//
// beta(t) = (1 - (t/2) cot(t/2)) / t^2 is the W^2 coefficient of both V^-1
// (the translation part of log) and the SO(3) inverse left Jacobian.  The
// inverse SE(3) left Jacobian is I - ad/2 + c2 ad^2 + c4 ad^4 (the odd part of
// x/(e^x-1) is exactly -x/2; the even part is interpolated on the spectrum
// {0, +-i t} of ad).  Its blocks are
//   A = I - W/2 + beta W^2,
//   B = -P/2 + beta (W P + P W) + c4 (W^2 P W + W P W^2),   P = [rho]x, W = [omega]x,
// with c4 = (beta + cot(t/2)/(4t) - csc^2(t/2)/8) / t^2.  Both coefficients
// cancel catastrophically in FP32 near 0, so their Bernoulli-number series are
// used below t = 1 (beta) and t = 2 (c4).
__device__ __forceinline__ float co_beta(float t, float s, float c) {
  if (t < 1.f) {
    const float t2 = t * t;
    return fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 2.08767569878681e-08f, 8.267195767195768e-07f),
                                  3.306878306878307e-05f),
                         1.388888888888889e-03f),
                0.08333333333333333f);
  }
  return (1.f - 0.5f * t * s / (1.f - c)) / (t * t);
}

__device__ __forceinline__ float co_c4(float t, float s, float c, float beta) {
  if (t < 2.f) {
    const float y = t * t;
    float p = -1.9573818287022555e-15f;
    p = fmaf(p, y, -6.868849645022276e-14f);
    p = fmaf(p, y, -2.372776207425808e-12f);
    p = fmaf(p, y, -8.029521918410807e-11f);
    p = fmaf(p, y, -2.6420950693437467e-09f);
    p = fmaf(p, y, -8.35070279514724e-08f);
    p = fmaf(p, y, -2.48015873015873e-06f);
    p = fmaf(p, y, -6.613756613756614e-05f);
    p = fmaf(p, y, -1.388888888888889e-03f);
    return p;
  }
  const float omc = 1.f - c;
  return (beta + s / (4.f * t * omc) - 0.25f / omc) / (t * t);
}

// log of a rotation: omega (3) and its angle.  The axis comes from the
// symmetric part when cos(t) < -0.99, where the skew part loses precision.
__device__ __forceinline__ float so3_log(const float* R, float* w) {
  float c = 0.5f * (R[0] + R[4] + R[8] - 1.f);
  c = fminf(1.f, fmaxf(-1.f, c));
  const float v0 = 0.5f * (R[7] - R[5]);
  const float v1 = 0.5f * (R[2] - R[6]);
  const float v2 = 0.5f * (R[3] - R[1]);
  const float s = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
  const float th = atan2f(s, c);
  if (c < -0.99f) {
    const float d0 = R[0] - c, d1 = R[4] - c, d2 = R[8] - c;
    float a0, a1, a2;
    if (d0 >= d1 && d0 >= d2) {
      a0 = d0; a1 = 0.5f * (R[1] + R[3]); a2 = 0.5f * (R[2] + R[6]);
    } else if (d1 >= d2) {
      a0 = 0.5f * (R[1] + R[3]); a1 = d1; a2 = 0.5f * (R[5] + R[7]);
    } else {
      a0 = 0.5f * (R[2] + R[6]); a1 = 0.5f * (R[5] + R[7]); a2 = d2;
    }
    float k = rsqrtf(fmaf(a0, a0, fmaf(a1, a1, a2 * a2)));
    if (a0 * v0 + a1 * v1 + a2 * v2 < 0.f) k = -k;
    k *= th;
    w[0] = k * a0; w[1] = k * a1; w[2] = k * a2;
  } else {
    const float k = (th < 1e-4f) ? fmaf(th * th, 1.f / 6.f, 1.f) : th / s;
    w[0] = k * v0; w[1] = k * v1; w[2] = k * v2;
  }
  return th;
}

// Inverse left-Jacobian blocks A (3x3) and B (3x3) at xi = [rho; omega].
__device__ __forceinline__ void se3_jlinv_blocks(const float* rho, const float* w, float th,
                                                 float* A, float* B) {
  float s, c;
  sincos_rad(th, &s, &c);
  const float be = co_beta(th, s, c);
  const float c4 = co_c4(th, s, c, be);
  float W[9] = {0.f, -w[2], w[1], w[2], 0.f, -w[0], -w[1], w[0], 0.f};
  float P[9] = {0.f, -rho[2], rho[1], rho[2], 0.f, -rho[0], -rho[1], rho[0], 0.f};
  float WW[9], WP[9], PW[9], WPW[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      WW[i * 3 + j] = W[i * 3] * W[j] + W[i * 3 + 1] * W[3 + j] + W[i * 3 + 2] * W[6 + j];
      WP[i * 3 + j] = W[i * 3] * P[j] + W[i * 3 + 1] * P[3 + j] + W[i * 3 + 2] * P[6 + j];
      PW[i * 3 + j] = P[i * 3] * W[j] + P[i * 3 + 1] * W[3 + j] + P[i * 3 + 2] * W[6 + j];
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      WPW[i * 3 + j] = WP[i * 3] * W[j] + WP[i * 3 + 1] * W[3 + j] + WP[i * 3 + 2] * W[6 + j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // W^2 P W = W (W P W);  W P W^2 = (W P W) W
      const float t1 = W[i * 3] * WPW[j] + W[i * 3 + 1] * WPW[3 + j] + W[i * 3 + 2] * WPW[6 + j];
      const float t2 = WPW[i * 3] * W[j] + WPW[i * 3 + 1] * W[3 + j] + WPW[i * 3 + 2] * W[6 + j];
      const int k = i * 3 + j;
      A[k] = (i == j ? 1.f : 0.f) - 0.5f * W[k] + be * WW[k];
      B[k] = -0.5f * P[k] + be * (WP[k] + PW[k]) + c4 * (t1 + t2);
    }
}

// SE(3) log of E: xi = [rho; omega]; returns the rotation angle.
// rho = V^-1 t = t - omega x t / 2 + beta omega x (omega x t).
__device__ __forceinline__ float se3_log(const Rt& E, float* xi) {
  float w[3];
  const float th = so3_log(E.r, w);
  float s, c;
  sincos_rad(th, &s, &c);
  const float be = co_beta(th, s, c);
  float wt[3], wwt[3];
  cross3(w, E.t, wt);
  cross3(w, wt, wwt);
#pragma unroll
  for (int i = 0; i < 3; ++i) xi[i] = fmaf(be, wwt[i], fmaf(-0.5f, wt[i], E.t[i]));
  xi[3] = w[0]; xi[4] = w[1]; xi[5] = w[2];
  return th;
}

// ---------------------------------------------------------------------------
// Packed lower-triangular storage: element (i, j), j <= i, at i(i+1)/2 + j.
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// In-place Cholesky of a packed SPD matrix.  The diagonal slots receive the
// RECIPROCAL of L's diagonal so that the triangular solves multiply instead
// of divide.  Returns false on a non-positive or non-finite pivot.
//
// Column by column (right-looking) with one column of lookahead: once column
// j is scaled, pivot j+1 takes its last update and its rsqrt is issued before
// the rest of the trailing update, whose independent FMAs then cover the
// rsqrt's latency (a warp issues in order, so the order of the code is the
// order of the waits).  Every entry still sees the row-by-row form's FMAs in
// the same order, a_ij - l_i0 l_j0 - l_i1 l_j1 - ... (k ascending), then one
// multiply by 1 / l_jj, so the factor is bit for bit the same.
template <int N>
__device__ __forceinline__ bool chol_packed(float* L) {
  float d = L[0];
  bool ok = (d > 0.f) & (d < INFINITY);
  float inv = rsqrtf(d);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    L[tri(j, j)] = inv;
#pragma unroll
    for (int i = j + 1; i < N; ++i) L[tri(i, j)] *= inv;
    if (j + 1 < N) {
      d = fmaf(-L[tri(j + 1, j)], L[tri(j + 1, j)], L[tri(j + 1, j + 1)]);
      ok = ok & (d > 0.f) & (d < INFINITY);
      inv = rsqrtf(d);
#pragma unroll
      for (int k = j + 1; k < N; ++k)
#pragma unroll
        for (int i = k; i < N; ++i)
          if (i > j + 1 || k > j + 1) L[tri(i, k)] = fmaf(-L[tri(i, j)], L[tri(k, j)], L[tri(i, k)]);
    }
  }
  return ok;
}

// Solve L L^T x = b in place (b -> x), with L from chol_packed.
template <int N>
__device__ __forceinline__ void chol_solve_packed(const float* L, float* b) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float x = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) x = fmaf(-L[tri(i, k)], b[k], x);
    b[i] = x * L[tri(i, i)];
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    float x = b[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) x = fmaf(-L[tri(k, i)], b[k], x);
    b[i] = x * L[tri(i, i)];
  }
}

}  // namespace pk
