/*
 * pk_oracle.c -- FP64 CPU oracle: forward kinematics, SE(3) log / Jacobians,
 * the IK residuals and their analytic Jacobian, and the Levenberg-Marquardt
 * multi-start solve.
 *
 * TEST INFRASTRUCTURE ONLY (see pk_oracle.h).  Plain, unblocked, unfused code
 * in the order the paper states the method:
 *   - forward kinematics T_base<-i = FK(q)_i over fixed / revolute / prismatic
 *     joints (Sec. III-B);
 *   - joint pose cost log(T_target^-1 T_base<-i), joint limit cost
 *     max(0, q - q_upper) + max(0, q_lower - q), joint regularisation q - q_reg
 *     (Sec. III-C), each weighted;
 *   - Levenberg-Marquardt on the sum of squared residuals (Sec. III-A).
 * The readings where the paper is silent (residual ordering [rho; omega],
 * damping D = I, nu = 2, strict-decrease acceptance, rest pose = middle of the
 * limits) are the ones listed in the design notes.
 */
#ifndef _GNU_SOURCE
#define _GNU_SOURCE
#endif
#include "pk_oracle.h"

#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* 3-vectors, 3x3 matrices (row-major), rigid transforms (3x4 row-major) */

static void v3_cross(const double* a, const double* b, double* c) {
  double x = a[1] * b[2] - a[2] * b[1];
  double y = a[2] * b[0] - a[0] * b[2];
  double z = a[0] * b[1] - a[1] * b[0];
  c[0] = x; c[1] = y; c[2] = z;
}
static double v3_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double v3_norm(const double* a) { return sqrt(v3_dot(a, a)); }

static void m3_mul(const double* A, const double* B, double* C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[k * 3 + j];
      T[i * 3 + j] = s;
    }
  memcpy(C, T, sizeof T);
}
static void m3_vec(const double* A, const double* x, double* y) {
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = A[i * 3] * x[0] + A[i * 3 + 1] * x[1] + A[i * 3 + 2] * x[2];
  y[0] = t[0]; y[1] = t[1]; y[2] = t[2];
}
static void m3_hat(const double* v, double* M) {
  M[0] = 0;     M[1] = -v[2]; M[2] = v[1];
  M[3] = v[2];  M[4] = 0;     M[5] = -v[0];
  M[6] = -v[1]; M[7] = v[0];  M[8] = 0;
}
static void m3_eye(double* M) { memset(M, 0, 9 * sizeof(double)); M[0] = M[4] = M[8] = 1; }

static void tf_rot(const double* T, double* R) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i * 3 + j] = T[i * 4 + j];
}
static void tf_trans(const double* T, double* t) { t[0] = T[3]; t[1] = T[7]; t[2] = T[11]; }
static void tf_make(const double* R, const double* t, double* T) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) T[i * 4 + j] = R[i * 3 + j];
    T[i * 4 + 3] = t[i];
  }
}
static void tf_mul(const double* A, const double* B, double* C) {
  double Ra[9], Rb[9], ta[3], tb[3], R[9], t[3];
  tf_rot(A, Ra); tf_rot(B, Rb); tf_trans(A, ta); tf_trans(B, tb);
  m3_mul(Ra, Rb, R);
  m3_vec(Ra, tb, t);
  t[0] += ta[0]; t[1] += ta[1]; t[2] += ta[2];
  tf_make(R, t, C);
}
static void tf_inv(const double* A, double* C) {
  double R[9], Rt[9], t[3], ti[3];
  tf_rot(A, R); tf_trans(A, t);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rt[i * 3 + j] = R[j * 3 + i];
  m3_vec(Rt, t, ti);
  ti[0] = -ti[0]; ti[1] = -ti[1]; ti[2] = -ti[2];
  tf_make(Rt, ti, C);
}

/* Rodrigues: R = I + sin(th) K + (1 - cos(th)) K^2, K = hat(axis). */
static void rodrigues(const double* a, double th, double* R) {
  double K[9], K2[9];
  m3_hat(a, K);
  m3_mul(K, K, K2);
  double s = sin(th), c = 1.0 - cos(th);
  m3_eye(R);
  for (int i = 0; i < 9; ++i) R[i] += s * K[i] + c * K2[i];
}

/* ------------------------------------------------------------------ */
/* Robot model (Sec. III-B)                                             */

static int is_mimic(const or_robot* rb, int j) { return rb->mimic && rb->mimic[j] >= 0; }

int32_t or_n_dof(const or_robot* rb) {
  int32_t n = 0;
  for (int j = 0; j < rb->n_joints; ++j) n += rb->type[j] != OR_JOINT_FIXED && !is_mimic(rb, j);
  return n;
}

/* Variable driving joint j (-1 for fixed joints), with the joint value
 * mult * q[var] + off. */
static int joint_var(const or_robot* rb, int j, double* mult, double* off) {
  *mult = 1.0;
  *off = 0.0;
  if (rb->type[j] == OR_JOINT_FIXED) return -1;
  int src = j;
  if (is_mimic(rb, j)) {
    src = rb->mimic[j];
    *mult = rb->mimic_mult[j];
    *off = rb->mimic_off[j];
  }
  int v = 0;
  for (int i = 0; i < src; ++i) v += rb->type[i] != OR_JOINT_FIXED && !is_mimic(rb, i);
  return v;
}

int32_t or_n_residuals(const or_robot* rb, const or_target_spec* ts) {
  int32_t m = 0;
  for (int k = 0; k < ts->n_targets; ++k)
    m += (ts->kinds && ts->kinds[k] == OR_TARGET_POSITION) ? 3 : 6;
  return m + 2 * or_n_dof(rb) + rb->n_pairs;
}

/* Eq. 1 activation (trajopt_oracle.c). */
double or_coll_activation(double d, double eta, double* df);

/* T_j = T_parent(j) * origin_j * X_j(q_j) for j in index order. */
void or_fk(const or_robot* rb, const double* q, double* T_out) {
  for (int j = 0; j < rb->n_joints; ++j) {
    double X[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    const double* a = rb->axis + 3 * j;
    double mult, off;
    const int v = joint_var(rb, j, &mult, &off);
    if (rb->type[j] == OR_JOINT_REVOLUTE) {
      double R[9], z[3] = {0, 0, 0};
      rodrigues(a, mult * q[v] + off, R);
      tf_make(R, z, X);
    } else if (rb->type[j] == OR_JOINT_PRISMATIC) {
      double d = mult * q[v] + off;
      X[3] = a[0] * d; X[7] = a[1] * d; X[11] = a[2] * d;
    }
    double L[12];
    tf_mul(rb->origin + 12 * j, X, L);
    if (rb->parent[j] < 0)
      memcpy(T_out + 12 * j, L, sizeof L);
    else
      tf_mul(T_out + 12 * rb->parent[j], L, T_out + 12 * j);
  }
}

/* ------------------------------------------------------------------ */
/* SO(3) / SE(3)                                                         */

/* log of a rotation matrix; the axis is taken from the symmetric part when the
 * angle is within 1e-3 of pi, where the skew part carries no precision. */
static void so3_log(const double* R, double* w) {
  double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  if (c > 1) c = 1;
  if (c < -1) c = -1;
  double v[3] = {0.5 * (R[7] - R[5]), 0.5 * (R[2] - R[6]), 0.5 * (R[3] - R[1])};
  double s = v3_norm(v);
  double th = atan2(s, c);
  if (th < 1e-8) {
    double k = 1.0 + th * th / 6.0;
    w[0] = k * v[0]; w[1] = k * v[1]; w[2] = k * v[2];
  } else if (M_PI - th < 1e-3) {
    double S[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S[i * 3 + j] = 0.5 * (R[i * 3 + j] + R[j * 3 + i]) - (i == j ? c : 0.0);
    int i = 0;
    if (S[4] > S[0]) i = 1;
    if (S[8] > S[i * 4]) i = 2;
    double scale = 1.0 / sqrt(S[i * 4] * (1.0 - c));
    double a[3] = {S[0 * 3 + i] * scale, S[1 * 3 + i] * scale, S[2 * 3 + i] * scale};
    double na = v3_norm(a);
    a[0] /= na; a[1] /= na; a[2] /= na;
    if (v3_dot(a, v) < 0) { a[0] = -a[0]; a[1] = -a[1]; a[2] = -a[2]; }
    w[0] = th * a[0]; w[1] = th * a[1]; w[2] = th * a[2];
  } else {
    double k = th / s;
    w[0] = k * v[0]; w[1] = k * v[1]; w[2] = k * v[2];
  }
}

/* Coefficients of the SO(3) left Jacobian family, with Taylor series below
 * 0.1 rad where the closed forms lose digits to cancellation.
 *   a = (1 - cos t) / t^2,   b = (t - sin t) / t^3,
 *   beta = (1 - (t/2) cot(t/2)) / t^2   (inverse left Jacobian),
 *   a2 = (t^2 + 2 cos t - 2) / (2 t^4),  a3 = (2t - 3 sin t + t cos t) / (2 t^5). */
static double co_a(double t) {
  if (t < 0.1) { double t2 = t * t; return 0.5 - t2 / 24.0 + t2 * t2 / 720.0 - t2 * t2 * t2 / 40320.0; }
  return (1.0 - cos(t)) / (t * t);
}
static double co_b(double t) {
  if (t < 0.1) { double t2 = t * t; return 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0 - t2 * t2 * t2 / 362880.0; }
  return (t - sin(t)) / (t * t * t);
}
static double co_beta(double t) {
  if (t < 0.1) { double t2 = t * t; return 1.0 / 12.0 + t2 / 720.0 + t2 * t2 / 30240.0 + t2 * t2 * t2 / 1209600.0; }
  return (1.0 - 0.5 * t * sin(t) / (1.0 - cos(t))) / (t * t);
}
static double co_a2(double t) {
  if (t < 0.1) { double t2 = t * t; return 1.0 / 24.0 - t2 / 720.0 + t2 * t2 / 40320.0 - t2 * t2 * t2 / 3628800.0; }
  return (t * t + 2.0 * cos(t) - 2.0) / (2.0 * t * t * t * t);
}
static double co_a3(double t) {
  if (t < 0.1) { double t2 = t * t; return 1.0 / 120.0 - t2 / 2520.0 + t2 * t2 / 120960.0; }
  return (2.0 * t - 3.0 * sin(t) + t * cos(t)) / (2.0 * t * t * t * t * t);
}

/* SO(3) left Jacobian J = I + a W + b W^2 and its inverse I - W/2 + beta W^2. */
static void so3_jl(const double* w, double* J) {
  double W[9], W2[9], t = v3_norm(w), a = co_a(t), b = co_b(t);
  m3_hat(w, W); m3_mul(W, W, W2); m3_eye(J);
  for (int i = 0; i < 9; ++i) J[i] += a * W[i] + b * W2[i];
}
static void so3_jlinv(const double* w, double* J) {
  double W[9], W2[9], t = v3_norm(w), be = co_beta(t);
  m3_hat(w, W); m3_mul(W, W, W2); m3_eye(J);
  for (int i = 0; i < 9; ++i) J[i] += -0.5 * W[i] + be * W2[i];
}

/* The off-diagonal block Q(rho, phi) of the SE(3) left Jacobian (Barfoot). */
static void se3_Q(const double* rho, const double* phi, double* Q) {
  double t = v3_norm(phi);
  double P[9], W[9], WP[9], PW[9], WPW[9], WW[9], WWP[9], PWW[9], WPWW[9], WWPW[9];
  m3_hat(rho, P); m3_hat(phi, W);
  m3_mul(W, P, WP); m3_mul(P, W, PW); m3_mul(WP, W, WPW);
  m3_mul(W, W, WW); m3_mul(WW, P, WWP); m3_mul(P, WW, PWW);
  m3_mul(WPW, W, WPWW); m3_mul(W, WPW, WWPW);
  double c1 = co_b(t), c2 = co_a2(t), c3 = co_a3(t);
  for (int i = 0; i < 9; ++i)
    Q[i] = 0.5 * P[i] + c1 * (WP[i] + PW[i] + WPW[i]) + c2 * (WWP[i] + PWW[i] - 3.0 * WPW[i]) +
           c3 * (WPWW[i] + WWPW[i]);
}

void or_se3_log(const double* T, double* xi) {
  double R[9], t[3], w[3], Vi[9];
  tf_rot(T, R); tf_trans(T, t);
  so3_log(R, w);
  so3_jlinv(w, Vi);
  m3_vec(Vi, t, xi);
  xi[3] = w[0]; xi[4] = w[1]; xi[5] = w[2];
}

void or_se3_exp(const double* xi, double* T) {
  double R[9], V[9], t[3], th = v3_norm(xi + 3);
  if (th > 0) {
    double a[3] = {xi[3] / th, xi[4] / th, xi[5] / th};
    rodrigues(a, th, R);
  } else {
    m3_eye(R);
  }
  so3_jl(xi + 3, V);
  m3_vec(V, xi, t);
  tf_make(R, t, T);
}

void or_se3_jl(const double* xi, double* J) {
  double Jr[9], Q[9];
  so3_jl(xi + 3, Jr);
  se3_Q(xi, xi + 3, Q);
  memset(J, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      J[i * 6 + j] = Jr[i * 3 + j];
      J[(i + 3) * 6 + j + 3] = Jr[i * 3 + j];
      J[i * 6 + j + 3] = Q[i * 3 + j];
    }
}

/* [[Ji, -Ji Q Ji], [0, Ji]] with Ji the SO(3) inverse left Jacobian. */
void or_se3_jlinv(const double* xi, double* J) {
  double Ji[9], Q[9], T1[9], B[9];
  so3_jlinv(xi + 3, Ji);
  se3_Q(xi, xi + 3, Q);
  m3_mul(Ji, Q, T1);
  m3_mul(T1, Ji, B);
  memset(J, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      J[i * 6 + j] = Ji[i * 3 + j];
      J[(i + 3) * 6 + j + 3] = Ji[i * 3 + j];
      J[i * 6 + j + 3] = -B[i * 3 + j];
    }
}

/* Adjoint of T = (R, t) acting on a twist [v; w]: [R v + t x (R w); R w]. */
static void se3_adjoint_apply(const double* T, const double* xi, double* out) {
  double R[9], t[3], Rv[3], Rw[3], c[3];
  tf_rot(T, R); tf_trans(T, t);
  m3_vec(R, xi, Rv);
  m3_vec(R, xi + 3, Rw);
  v3_cross(t, Rw, c);
  out[0] = Rv[0] + c[0]; out[1] = Rv[1] + c[1]; out[2] = Rv[2] + c[2];
  out[3] = Rw[0]; out[4] = Rw[1]; out[5] = Rw[2];
}

/* ------------------------------------------------------------------ */
/* Residuals and analytic Jacobian (Sec. III-C)                          */

static int is_ancestor_or_self(const or_robot* rb, int j, int link) {
  for (int l = link; l >= 0; l = rb->parent[l])
    if (l == j) return 1;
  return 0;
}

void or_ik_residual(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts,
                    const double* targets, const double* q, double* r, double* J) {
  const int n = rb->n_joints, nd = or_n_dof(rb), m = or_n_residuals(rb, ts);
  double* T = (double*)malloc(sizeof(double) * 12 * n);
  int* var = (int*)malloc(sizeof(int) * n);
  double* mult = (double*)malloc(sizeof(double) * n);
  or_fk(rb, q, T);
  for (int j = 0; j < n; ++j) {
    double off;
    var[j] = joint_var(rb, j, &mult[j], &off);
  }
  if (J) memset(J, 0, sizeof(double) * m * nd);
  int row = 0;
  for (int k = 0; k < ts->n_targets; ++k) {
    const int link = ts->links[k];
    const double* Tt = targets + 12 * k;
    const double* Tl = T + 12 * link;
    if (!ts->kinds || ts->kinds[k] == OR_TARGET_POSE) {
      /* r = w (.) log(T_target^-1 T_link) */
      double Ti[12], E[12], xi[6], Jli[36];
      const double w[6] = {p->w_pos, p->w_pos, p->w_pos, p->w_rot, p->w_rot, p->w_rot};
      tf_inv(Tt, Ti);
      tf_mul(Ti, Tl, E);
      or_se3_log(E, xi);
      for (int i = 0; i < 6; ++i) r[row + i] = w[i] * xi[i];
      if (J) {
        or_se3_jlinv(xi, Jli);
        for (int j = 0; j < n; ++j) {
          if (var[j] < 0 || !is_ancestor_or_self(rb, j, link)) continue;
          /* world twist of joint j: revolute [p x w; w], prismatic [d; 0] */
          double Rj[9], pj[3], ax[3], tw[6], eta[6];
          tf_rot(T + 12 * j, Rj); tf_trans(T + 12 * j, pj);
          m3_vec(Rj, rb->axis + 3 * j, ax);
          if (rb->type[j] == OR_JOINT_REVOLUTE) {
            v3_cross(pj, ax, tw);
            tw[3] = ax[0]; tw[4] = ax[1]; tw[5] = ax[2];
          } else {
            tw[0] = ax[0]; tw[1] = ax[1]; tw[2] = ax[2];
            tw[3] = tw[4] = tw[5] = 0;
          }
          se3_adjoint_apply(Ti, tw, eta);
          for (int i = 0; i < 6; ++i) {
            double s = 0;
            for (int l = 0; l < 6; ++l) s += Jli[i * 6 + l] * eta[l];
            J[(row + i) * nd + var[j]] += mult[j] * w[i] * s;  /* a mimic joint adds to its source's column */
          }
        }
      }
      row += 6;
    } else {
      /* r = w_pos (p_link - p_target), world frame */
      double pl[3], pt[3];
      tf_trans(Tl, pl); tf_trans(Tt, pt);
      for (int i = 0; i < 3; ++i) r[row + i] = p->w_pos * (pl[i] - pt[i]);
      if (J) {
        for (int j = 0; j < n; ++j) {
          if (var[j] < 0 || !is_ancestor_or_self(rb, j, link)) continue;
          double Rj[9], pj[3], ax[3], col[3];
          tf_rot(T + 12 * j, Rj); tf_trans(T + 12 * j, pj);
          m3_vec(Rj, rb->axis + 3 * j, ax);
          if (rb->type[j] == OR_JOINT_REVOLUTE) {
            double d[3] = {pl[0] - pj[0], pl[1] - pj[1], pl[2] - pj[2]};
            v3_cross(ax, d, col);
          } else {
            col[0] = ax[0]; col[1] = ax[1]; col[2] = ax[2];
          }
          for (int i = 0; i < 3; ++i) J[(row + i) * nd + var[j]] += mult[j] * p->w_pos * col[i];
        }
      }
      row += 3;
    }
  }
  /* self collision (Sec. III-C, Eq. 1): per sphere pair, w_self f(d, eta)
   * with d = |c_a - c_b| - r_a - r_b and the sphere centres moving with
   * their frames */
  const int prow = m - rb->n_pairs;
  for (int pidx = 0; pidx < rb->n_pairs; ++pidx) {
    const int sa = rb->pairs[2 * pidx], sb = rb->pairs[2 * pidx + 1];
    const int ja = rb->sph_joint[sa], jb = rb->sph_joint[sb];
    double ca[3], cb[3], R[9], t[3];
    tf_rot(T + 12 * ja, R); tf_trans(T + 12 * ja, t);
    m3_vec(R, rb->sph_centre + 3 * sa, ca);
    for (int i = 0; i < 3; ++i) ca[i] += t[i];
    tf_rot(T + 12 * jb, R); tf_trans(T + 12 * jb, t);
    m3_vec(R, rb->sph_centre + 3 * sb, cb);
    for (int i = 0; i < 3; ++i) cb[i] += t[i];
    double diff[3] = {ca[0] - cb[0], ca[1] - cb[1], ca[2] - cb[2]};
    const double dist = v3_norm(diff);
    const double d = dist - rb->sph_radius[sa] - rb->sph_radius[sb];
    double df = 0;
    const double f = or_coll_activation(d, p->eta_self, &df);
    r[prow + pidx] = p->w_self * f;
    if (J && dist > 1e-12) {
      double nh[3] = {diff[0] / dist, diff[1] / dist, diff[2] / dist};
      for (int j = 0; j < n; ++j) {
        if (var[j] < 0) continue;
        const int ina = is_ancestor_or_self(rb, j, ja), inb = is_ancestor_or_self(rb, j, jb);
        if (!ina && !inb) continue;
        double Rj[9], pj[3], ax[3], va[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
        tf_rot(T + 12 * j, Rj); tf_trans(T + 12 * j, pj);
        m3_vec(Rj, rb->axis + 3 * j, ax);
        /* velocity of a point x moved by joint j: revolute w x (x - p_j), prismatic w */
        if (rb->type[j] == OR_JOINT_REVOLUTE) {
          double da[3] = {ca[0] - pj[0], ca[1] - pj[1], ca[2] - pj[2]};
          double db[3] = {cb[0] - pj[0], cb[1] - pj[1], cb[2] - pj[2]};
          if (ina) v3_cross(ax, da, va);
          if (inb) v3_cross(ax, db, vb);
        } else {
          if (ina) { va[0] = ax[0]; va[1] = ax[1]; va[2] = ax[2]; }
          if (inb) { vb[0] = ax[0]; vb[1] = ax[1]; vb[2] = ax[2]; }
        }
        const double dd = nh[0] * (va[0] - vb[0]) + nh[1] * (va[1] - vb[1]) + nh[2] * (va[2] - vb[2]);
        J[(prow + pidx) * nd + var[j]] += mult[j] * p->w_self * df * dd;
      }
    }
  }
  /* joint limit hinge and rest pose (middle of the limits) of every variable,
   * with its own joint's limits (a mimic joint's limits are not enforced) */
  for (int j = 0; j < n; ++j) {
    if (var[j] < 0 || is_mimic(rb, j)) continue;
    const int v = var[j];
    const double lo = rb->lower[j], hi = rb->upper[j], qv = q[v];
    double h = 0, dh = 0;
    if (qv > hi) { h += qv - hi; dh = 1; }
    if (qv < lo) { h += lo - qv; dh = -1; }
    r[row + v] = p->w_limit * h;
    r[row + nd + v] = p->w_rest * (qv - 0.5 * (lo + hi));
    if (J) {
      J[(row + v) * nd + v] = p->w_limit * dh;
      J[(row + nd + v) * nd + v] = p->w_rest;
    }
  }
  free(T);
  free(var);
  free(mult);
}

void or_ik_errors(const or_robot* rb, const or_target_spec* ts, const double* targets,
                  const double* q, double* pos_err, double* rot_err) {
  double* T = (double*)malloc(sizeof(double) * 12 * rb->n_joints);
  or_fk(rb, q, T);
  double pe = 0, re = 0;
  for (int k = 0; k < ts->n_targets; ++k) {
    const double* Tt = targets + 12 * k;
    const double* Tl = T + 12 * ts->links[k];
    double d[3] = {Tl[3] - Tt[3], Tl[7] - Tt[7], Tl[11] - Tt[11]};
    double e = v3_norm(d);
    if (!(e <= pe)) pe = e;
    if (!ts->kinds || ts->kinds[k] == OR_TARGET_POSE) {
      double Ra[9], Rb[9], Rat[9], Rd[9], w[3];
      tf_rot(Tt, Ra); tf_rot(Tl, Rb);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rat[i * 3 + j] = Ra[j * 3 + i];
      m3_mul(Rat, Rb, Rd);
      so3_log(Rd, w);
      double a = v3_norm(w);
      if (!(a <= re)) re = a;
    }
  }
  *pos_err = pe;
  *rot_err = re;
  free(T);
}

/* ------------------------------------------------------------------ */
/* Dense Cholesky                                                        */

int32_t or_cholesky_solve(int32_t n, const double* A, const double* b, double* x) {
  double* L = (double*)calloc((size_t)n * n, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * n);
  int32_t rc = 0;
  for (int j = 0; j < n && rc == 0; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0) || !isfinite(d)) { rc = 1; break; }
    L[j * n + j] = sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / L[j * n + j];
    }
  }
  if (rc == 0) {
    for (int i = 0; i < n; ++i) {
      double s = b[i];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
      x[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i)
      if (!isfinite(x[i])) rc = 1;
  }
  free(L);
  free(y);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Levenberg-Marquardt on one (target, seed) problem (Sec. III-A)       */

/* Gauss-Newton normal equations A = J^T J, g = J^T r of an m x nd Jacobian
 * (row-major).  A is symmetric: its lower triangle is summed and mirrored. */
void or_normal_equations(int32_t m, int32_t nd, const double* J, const double* r, double* A, double* g) {
  for (int a = 0; a < nd; ++a) {
    double s = 0;
    for (int i = 0; i < m; ++i) s += J[i * nd + a] * r[i];
    g[a] = s;
    for (int b = 0; b <= a; ++b) {
      double t = 0;
      for (int i = 0; i < m; ++i) t += J[i * nd + a] * J[i * nd + b];
      A[a * nd + b] = t;
      A[b * nd + a] = t;
    }
  }
}

typedef struct {
  double cost, pos_err, rot_err, margin;
  int32_t iters, status;
} lm_result;

static double half_sq(const double* r, int m) {
  double s = 0;
  for (int i = 0; i < m; ++i) s += r[i] * r[i];
  return 0.5 * s;
}

static int converged(const or_ik_params* p, double pe, double re) {
  return pe <= p->tol_pos && re <= p->tol_rot;
}

/* One LM run (Sec. III-A) from `seed` with damping lambda_init (the LM state
 * of an earlier run, or p->lambda0 when negative); the damping after the last
 * iteration goes to *lambda_out when given.  trace / lam_trace (optional,
 * n_trace entries each) receive q and the damping after iterations
 * 1..n_trace; entries past the last iteration repeat the final state. */
static void lm_problem(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts,
                       const double* targets, const double* seed, double* q, lm_result* res,
                       int n_trace, double* trace, double* lam_trace, double lambda_init,
                       double* lambda_out) {
  const int nd = or_n_dof(rb), m = or_n_residuals(rb, ts);
  double* r = (double*)malloc(sizeof(double) * m);
  double* rt = (double*)malloc(sizeof(double) * m);
  double* J = (double*)malloc(sizeof(double) * m * nd);
  double* A = (double*)malloc(sizeof(double) * nd * nd);
  double* g = (double*)malloc(sizeof(double) * nd);
  double* ng = (double*)malloc(sizeof(double) * nd);
  double* dq = (double*)malloc(sizeof(double) * nd);
  double* qt = (double*)malloc(sizeof(double) * nd);
  memcpy(q, seed, sizeof(double) * nd);
  res->margin = INFINITY;
  or_ik_residual(rb, p, ts, targets, q, r, NULL);
  double f = half_sq(r, m), pe, re;
  double lambda = lambda_init >= 0 ? lambda_init : p->lambda0;
  int it = 0, conv = 0;
  if (!isfinite(f)) {
    res->cost = f; res->pos_err = NAN; res->rot_err = NAN;
    res->iters = 0; res->status = OR_P_NONFINITE;
    for (int t = 0; t < n_trace; ++t) {
      if (trace) memcpy(trace + t * nd, q, sizeof(double) * nd);
      if (lam_trace) lam_trace[t] = lambda;
    }
    goto done;
  }
  or_ik_errors(rb, ts, targets, q, &pe, &re);
  conv = converged(p, pe, re);
  if (!(p->early_exit && conv)) {
    while (it < p->max_iters) {
      ++it;
      /* normal equations (J^T J + lambda I) dq = -J^T r */
      or_ik_residual(rb, p, ts, targets, q, r, J);
      or_normal_equations(m, nd, J, r, A, g);
      for (int a = 0; a < nd; ++a) {
        A[a * nd + a] += lambda;
        ng[a] = -g[a];
      }
      int accepted = 0;
      if (or_cholesky_solve(nd, A, ng, dq) == 0) {
        for (int a = 0; a < nd; ++a) qt[a] = q[a] + dq[a];
        or_ik_residual(rb, p, ts, targets, qt, rt, NULL);
        double ft = half_sq(rt, m);
        if (it <= n_trace && f > 0) {
          double mg = fabs(ft - f) / f;
          if (mg < res->margin) res->margin = mg;
        }
        if (ft < f) {
          accepted = 1;
          memcpy(q, qt, sizeof(double) * nd);
          f = ft;
        }
      }
      if (accepted) {
        lambda = lambda / p->nu;
        if (lambda < p->lambda_min) lambda = p->lambda_min;
        or_ik_errors(rb, ts, targets, q, &pe, &re);
        conv = converged(p, pe, re);
      } else {
        lambda = lambda * p->nu;
        if (lambda > p->lambda_max) lambda = p->lambda_max;
      }
      if (it <= n_trace && trace) memcpy(trace + (it - 1) * nd, q, sizeof(double) * nd);
      if (it <= n_trace && lam_trace) lam_trace[it - 1] = lambda;
      if (p->early_exit && conv) break;
    }
  }
  for (int t = it; t < n_trace; ++t) {
    if (trace) memcpy(trace + t * nd, q, sizeof(double) * nd);
    if (lam_trace) lam_trace[t] = lambda;
  }
  or_ik_errors(rb, ts, targets, q, &pe, &re);
  res->cost = f; res->pos_err = pe; res->rot_err = re; res->iters = it;
  res->status = converged(p, pe, re) ? OR_P_CONVERGED : OR_P_MAX_ITERS;
  if (lambda_out) *lambda_out = lambda;
done:
  free(r); free(rt); free(J); free(A); free(g); free(ng); free(dq); free(qt);
}

/* ------------------------------------------------------------------ */
/* Multi-start driver over a thread pool                                 */

typedef struct {
  const or_robot* rb;
  const or_ik_params* p;
  const or_target_spec* ts;
  int32_t batch, n_seeds, nd, n_trace;
  const double* targets;
  const double* seeds;
  double* q_all;
  lm_result* res;
  double* trace;
  long next;
} pool_ctx;

static void* pool_worker(void* arg) {
  pool_ctx* c = (pool_ctx*)arg;
  const long P = (long)c->batch * c->n_seeds;
  const int k = c->ts->n_targets;
  for (;;) {
    long i = __atomic_fetch_add(&c->next, 1, __ATOMIC_RELAXED);
    if (i >= P) break;
    long b = i / c->n_seeds;
    lm_problem(c->rb, c->p, c->ts, c->targets + b * 12 * k, c->seeds + i * c->nd,
               c->q_all + i * c->nd, &c->res[i], c->n_trace,
               c->trace ? c->trace + i * (long)c->n_trace * c->nd : NULL, NULL, -1.0, NULL);
  }
  return NULL;
}

int32_t or_host_cores(void) {
  cpu_set_t set;
  if (sched_getaffinity(0, sizeof set, &set) == 0) {
    int n = CPU_COUNT(&set);
    if (n > 0) return n;
  }
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

int32_t or_ik_solve(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts,
                    int32_t batch, int32_t n_seeds, const double* targets, const double* seeds,
                    double* q_out, double* err_out, int32_t* iters_out, int32_t* status_out,
                    double* per_problem, int32_t n_trace, double* trace, double* margin,
                    int32_t n_threads) {
  const int nd = or_n_dof(rb);
  const long P = (long)batch * n_seeds;
  if (n_threads <= 0) n_threads = or_host_cores();
  if (n_threads > P) n_threads = (int)(P > 0 ? P : 1);
  pool_ctx c = {rb, p, ts, batch, n_seeds, nd, trace ? n_trace : 0, targets, seeds,
                (double*)malloc(sizeof(double) * (P > 0 ? P : 1) * nd),
                (lm_result*)malloc(sizeof(lm_result) * (P > 0 ? P : 1)), trace, 0};
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, pool_worker, &c);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  for (int32_t b = 0; b < batch; ++b) {
    int best = -1;
    for (int s = 0; s < n_seeds; ++s) {
      const lm_result* x = &c.res[(long)b * n_seeds + s];
      if (best < 0) { best = s; continue; }
      const lm_result* y = &c.res[(long)b * n_seeds + best];
      int xc = x->status == OR_P_CONVERGED, yc = y->status == OR_P_CONVERGED;
      double xf = isfinite(x->cost) ? x->cost : INFINITY, yf = isfinite(y->cost) ? y->cost : INFINITY;
      if (xc > yc || (xc == yc && xf < yf)) best = s;
    }
    if (best < 0) continue;
    const long i = (long)b * n_seeds + best;
    memcpy(q_out + (long)b * nd, c.q_all + i * nd, sizeof(double) * nd);
    err_out[2 * b] = c.res[i].pos_err;
    err_out[2 * b + 1] = c.res[i].rot_err;
    iters_out[b] = c.res[i].iters;
    status_out[b] = c.res[i].status;
  }
  for (long i = 0; i < P; ++i) {
    if (per_problem) {
      double* o = per_problem + i * (nd + 5);
      memcpy(o, c.q_all + i * nd, sizeof(double) * nd);
      o[nd] = c.res[i].cost; o[nd + 1] = c.res[i].pos_err; o[nd + 2] = c.res[i].rot_err;
      o[nd + 3] = c.res[i].iters; o[nd + 4] = c.res[i].status;
    }
    if (margin) margin[i] = c.res[i].margin;
  }
  free(c.q_all);
  free(c.res);
  return n_threads;
}

int32_t or_lm_run(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts, const double* targets,
                  const double* seed, double lambda_init, int32_t n_trace, double* q_trace, double* lam_trace,
                  double* q_out, double* res_out) {
  lm_result res;
  double lam = 0;
  lm_problem(rb, p, ts, targets, seed, q_out, &res, n_trace, q_trace, lam_trace, lambda_init, &lam);
  res_out[0] = res.cost; res_out[1] = res.pos_err; res_out[2] = res.rot_err;
  res_out[3] = res.iters; res_out[4] = res.status; res_out[5] = lam;
  return res.status;
}

/* ------------------------------------------------------------------ */
/* IK-Beam (Sec. V-C): every target starts from n_seeds seeds; all of them
 * take steps1 LM iterations; the `keep` seeds with the lowest cost (ties: the
 * lower seed index; a non-finite cost ranks last) continue from their LM state
 * (configuration and damping) for steps2 more iterations; the result is the
 * best of those (converged first, then lowest cost, then lowest seed index). */

typedef struct {
  const or_robot* rb;
  const or_ik_params* p;
  const or_target_spec* ts;
  int32_t batch, n_seeds, steps1, keep, steps2, nd;
  const double* targets;
  const double* seeds;
  double* q_out;
  double* err_out;
  int32_t* iters_out;
  int32_t* status_out;
  int32_t* kept_out;
  long next;
} beam_ctx;

static double rank_cost(double f) { return isfinite(f) ? f : INFINITY; }

static void beam_target(beam_ctx* c, long b) {
  const int nd = c->nd, S = c->n_seeds, k = c->ts->n_targets;
  const double* tg = c->targets + b * 12 * k;
  or_ik_params p1 = *c->p, p2 = *c->p;
  p1.max_iters = c->steps1;
  p2.max_iters = c->steps2;
  double* q1 = (double*)malloc(sizeof(double) * S * nd);
  double* lam1 = (double*)malloc(sizeof(double) * S);
  lm_result* r1 = (lm_result*)malloc(sizeof(lm_result) * S);
  int* taken = (int*)calloc(S, sizeof(int));
  double* q2 = (double*)malloc(sizeof(double) * nd);
  /* phase 1: every seed */
  for (int s = 0; s < S; ++s)
    lm_problem(c->rb, &p1, c->ts, tg, c->seeds + (b * S + s) * nd, q1 + s * nd, &r1[s], 0, NULL, NULL, -1.0,
               &lam1[s]);
  /* selection and phase 2 */
  int best_s = -1, best_conv = 0, best_it = 0, best_status = 0;
  double best_f = INFINITY, best_pe = NAN, best_re = NAN;
  double* best_q = (double*)malloc(sizeof(double) * nd);
  for (int r = 0; r < c->keep && r < S; ++r) {
    int sel = -1;
    for (int s = 0; s < S; ++s) {
      if (taken[s]) continue;
      if (sel < 0 || rank_cost(r1[s].cost) < rank_cost(r1[sel].cost)) sel = s;
    }
    taken[sel] = 1;
    if (c->kept_out) c->kept_out[b * c->keep + r] = sel;
    lm_result r2;
    if (r1[sel].status == OR_P_NONFINITE) {
      memcpy(q2, q1 + sel * nd, sizeof(double) * nd);
      r2 = r1[sel];
      r2.iters = 0;
    } else {
      lm_problem(c->rb, &p2, c->ts, tg, q1 + sel * nd, q2, &r2, 0, NULL, NULL, lam1[sel], NULL);
    }
    const int conv = r2.status == OR_P_CONVERGED;
    const double f = rank_cost(r2.cost);
    if (best_s < 0 || conv > best_conv || (conv == best_conv && (f < best_f || (f == best_f && sel < best_s)))) {
      best_s = sel; best_conv = conv; best_f = f; best_pe = r2.pos_err; best_re = r2.rot_err;
      best_it = r1[sel].iters + r2.iters; best_status = r2.status;
      memcpy(best_q, q2, sizeof(double) * nd);
    }
  }
  memcpy(c->q_out + b * nd, best_q, sizeof(double) * nd);
  c->err_out[2 * b] = best_pe;
  c->err_out[2 * b + 1] = best_re;
  c->iters_out[b] = best_it;
  c->status_out[b] = best_status;
  free(q1); free(lam1); free(r1); free(taken); free(q2); free(best_q);
}

static void* beam_worker(void* arg) {
  beam_ctx* c = (beam_ctx*)arg;
  for (;;) {
    long b = __atomic_fetch_add(&c->next, 1, __ATOMIC_RELAXED);
    if (b >= c->batch) break;
    beam_target(c, b);
  }
  return NULL;
}

int32_t or_ik_beam(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts, int32_t batch,
                   int32_t n_seeds, int32_t steps1, int32_t keep, int32_t steps2, const double* targets,
                   const double* seeds, double* q_out, double* err_out, int32_t* iters_out,
                   int32_t* status_out, int32_t* kept_out, int32_t n_threads) {
  if (n_threads <= 0) n_threads = or_host_cores();
  if (n_threads > batch) n_threads = batch > 0 ? batch : 1;
  beam_ctx c = {rb, p, ts, batch, n_seeds, steps1, keep, steps2, or_n_dof(rb), targets, seeds,
                q_out, err_out, iters_out, status_out, kept_out, 0};
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, beam_worker, &c);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  return n_threads;
}
