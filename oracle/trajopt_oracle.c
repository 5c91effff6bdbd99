/*
 * trajopt_oracle.c -- FP64 oracle of collision-aware trajectory optimisation.
 *
 * TEST INFRASTRUCTURE ONLY.  Variables: T joint configurations q_0..q_{T-1}
 * (Sec. III-B "q_t").  Residuals, each weighted (Sec. III-C):
 *   start      w_s (q_0 - q_start)                                  7 rows
 *   goal pose  [w_gp rho; w_gr omega] = log(T_goal^-1 FK(q_{T-1}))   6 rows
 *   velocity   w_v (q_t - q_{t-1}),           t = 1..T-1  (smoothness cost)
 *   accel.     w_a (q_{t+1} - 2 q_t + q_{t-1}), t = 1..T-2 (finite-difference
 *              acceleration, the 3-point stencil)
 *   limits     w_l hinge(q_t)                 every t
 *   collision  w_c f(d, eta) per (link sphere, obstacle) and (sphere, plane),
 *              f the activation of Eq. 1 (d <= 0 takes the linear branch)
 * Link j carries S spheres with centres p_j + (s + 1/2)/S (p_{j+1} - p_j)
 * (p_j the origin of joint frame j, p_n the tool frame) and given radii; the
 * first link's spheres are not tested against the plane.  The solver is LM on
 * the sum of squared residuals (Sec. III-A) with the same rules as the IK
 * oracle, a fixed iteration count, and either a dense Cholesky of the full
 * normal matrix or a block-banded one (the normal matrix is block
 * pentadiagonal in t).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pk_oracle.h"

typedef struct {
  double w_start, w_goal_pos, w_goal_rot, w_vel, w_acc, w_limit, w_coll, eta;
  double lambda0, lambda_min, lambda_max, nu;
  int32_t iters;
  int32_t banded; /* 1: block-banded Cholesky, 0: dense */
  /* extensions (0 = off): velocity-limit hinge w_vlimit max(0, |q_t - q_{t-1}|
   * - v_max) (Sec. III-C, dt = 1) and swept-sphere collision between t and
   * t+1, w_swept f(d, eta) with d the distance from an obstacle sphere to the
   * capsule swept by a link sphere (Sec. IV-A continuous collision) */
  double w_vlimit, v_max, w_swept;
  /* five-point stencils (Sec. III-C smoothness; 0 = off): acceleration
   * (-q_{t+2} + 16 q_{t+1} - 30 q_t + 16 q_{t-1} - q_{t-2}) / 12 and jerk
   * (q_{t+2} - 2 q_{t+1} + 2 q_{t-1} - q_{t-2}) / 2 for t = 2..T-3 (dt = 1);
   * they widen the block band of the normal matrix from 2 to 4 */
  double w_acc5, w_jerk;
} or_traj_params;

typedef struct {
  int32_t S;             /* spheres per link */
  const double* radii;   /* [n_dof][S] */
  int32_t n_obs;
  const double* obs;     /* [n_obs][4] centre, radius */
  const double* plane;   /* [4] unit normal, offset h: signed distance n.c - h */
} or_traj_scene;

/* Eq. 1 activation and its derivative. */
double or_coll_activation(double d, double eta, double* df) {
  if (d <= 0) {
    if (df) *df = -1.0;
    return -d + 0.5 * eta;
  }
  if (d < eta) {
    if (df) *df = -(eta - d) / eta;
    return 0.5 / eta * (eta - d) * (eta - d);
  }
  if (df) *df = 0.0;
  return 0.0;
}

int32_t or_traj_n_residuals(const or_robot* rb, const or_traj_scene* sc, int32_t T) {
  const int n = or_n_dof(rb);
  return n + 6 + n * (T - 1) + n * (T - 2 > 0 ? T - 2 : 0) + n * T + T * n * sc->S * (sc->n_obs + 1) +
         n * (T - 1) + (T - 1) * n * sc->S * sc->n_obs + 2 * n * (T - 4 > 0 ? T - 4 : 0);
}

/* Row width of the row-sparse Jacobian: a swept-sphere row touches two
 * timesteps. */
#define KW (2 * n)

/* Row-sparse Jacobian: every row has at most KW = 2n nonzeros; row i keeps
 * its column indices in Jc[i][0..KW) (-1 = unused) and values in Jv[i][0..KW). */
#define SETJ(row_, col_, val_)                                     \
  do {                                                             \
    if (Jc) {                                                      \
      int* c_ = Jc + (size_t)(row_) * KW;                          \
      double* v_ = Jv + (size_t)(row_) * KW;                       \
      int k_ = 0;                                                  \
      while (k_ < KW && c_[k_] >= 0 && c_[k_] != (col_)) ++k_;     \
      c_[k_] = (col_);                                             \
      v_[k_] = (val_);                                             \
    }                                                              \
  } while (0)

/* All residual rows and (optionally) the row-sparse Jacobian.
 * Row order: start, goal, velocity (t = 1..), acceleration (t = 1..T-2),
 * limits (t-major), collisions (t, link, sphere, [obstacles..., plane]). */
void or_traj_residual_sparse(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T,
                             const double* x, const double* q_start, const double* goal, double* r, int* Jc,
                             double* Jv) {
  const int n = or_n_dof(rb), nj = rb->n_joints;
  const int m = or_traj_n_residuals(rb, sc, T);
  if (Jc)
    for (size_t i = 0; i < (size_t)m * KW; ++i) Jc[i] = -1;
  int row = 0;
  /* start */
  for (int i = 0; i < n; ++i, ++row) {
    r[row] = p->w_start * (x[i] - q_start[i]);
    SETJ(row, i, p->w_start);
  }
  /* goal pose at t = T-1, through the IK residual of one pose target on the last frame */
  {
    or_ik_params ip;
    memset(&ip, 0, sizeof ip);
    ip.w_pos = p->w_goal_pos;
    ip.w_rot = p->w_goal_rot;
    int32_t link = nj - 1;
    or_target_spec ts = {1, &link, NULL};
    const int mi = or_n_residuals(rb, &ts);
    double* ri = (double*)malloc(sizeof(double) * mi);
    double* Ji = (double*)malloc(sizeof(double) * mi * n);
    or_ik_residual(rb, &ip, &ts, goal, x + (size_t)(T - 1) * n, ri, Ji);
    for (int i = 0; i < 6; ++i, ++row) {
      r[row] = ri[i];
      for (int a = 0; a < n; ++a) SETJ(row, (T - 1) * n + a, Ji[i * n + a]);
    }
    free(ri);
    free(Ji);
  }
  /* velocity */
  for (int t = 1; t < T; ++t)
    for (int i = 0; i < n; ++i, ++row) {
      r[row] = p->w_vel * (x[t * n + i] - x[(t - 1) * n + i]);
      SETJ(row, t * n + i, p->w_vel);
      SETJ(row, (t - 1) * n + i, -p->w_vel);
    }
  /* acceleration */
  for (int t = 1; t + 1 < T; ++t)
    for (int i = 0; i < n; ++i, ++row) {
      r[row] = p->w_acc * (x[(t + 1) * n + i] - 2 * x[t * n + i] + x[(t - 1) * n + i]);
      SETJ(row, (t + 1) * n + i, p->w_acc);
      SETJ(row, t * n + i, -2 * p->w_acc);
      SETJ(row, (t - 1) * n + i, p->w_acc);
    }
  /* limits */
  {
    int v = 0;
    for (int t = 0; t < T; ++t) {
      v = 0;
      for (int j = 0; j < nj; ++j) {
        if (rb->type[j] == OR_JOINT_FIXED) continue;
        const double q = x[t * n + v], lo = rb->lower[j], hi = rb->upper[j];
        double h = 0, dh = 0;
        if (q > hi) { h = q - hi; dh = 1; }
        if (q < lo) { h = lo - q; dh = -1; }
        r[row + v] = p->w_limit * h;
        SETJ(row + v, t * n + v, p->w_limit * dh);
        ++v;
      }
      row += n;
    }
  }
  /* collisions: frames of the movable joints and the tool (serial chain) */
  double* Tf = (double*)malloc(sizeof(double) * 12 * nj);
  int* jidx = (int*)malloc(sizeof(int) * (n + 1));
  {
    int v = 0;
    for (int j = 0; j < nj; ++j)
      if (rb->type[j] != OR_JOINT_FIXED) jidx[v++] = j;
    jidx[n] = nj - 1; /* tool frame closes the last link */
  }
  for (int t = 0; t < T; ++t) {
    or_fk(rb, x + (size_t)t * n, Tf);
    for (int l = 0; l < n; ++l) {
      const double* pa = Tf + 12 * jidx[l];
      const double* pb = Tf + 12 * jidx[l + 1];
      for (int s = 0; s < sc->S; ++s) {
        const double al = (s + 0.5) / sc->S;
        double c[3] = {pa[3] + al * (pb[3] - pa[3]), pa[7] + al * (pb[7] - pa[7]),
                       pa[11] + al * (pb[11] - pa[11])};
        const double rad = sc->radii[l * sc->S + s];
        for (int o = 0; o <= sc->n_obs; ++o, ++row) {
          double d, nrm[3];
          if (o < sc->n_obs) {
            const double* ob = sc->obs + 4 * o;
            double v3[3] = {c[0] - ob[0], c[1] - ob[1], c[2] - ob[2]};
            double len = sqrt(v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2]);
            d = len - rad - ob[3];
            nrm[0] = v3[0] / len; nrm[1] = v3[1] / len; nrm[2] = v3[2] / len;
          } else {
            if (l == 0) { r[row] = 0; continue; } /* first link not tested against the plane */
            nrm[0] = sc->plane[0]; nrm[1] = sc->plane[1]; nrm[2] = sc->plane[2];
            d = nrm[0] * c[0] + nrm[1] * c[1] + nrm[2] * c[2] - sc->plane[3] - rad;
          }
          double df;
          r[row] = p->w_coll * or_coll_activation(d, p->eta, &df);
          if (Jc && df != 0.0) {
            /* d(c)/d(q_i) = w_i x (c - p_i) for the joints of links 0..l */
            for (int i = 0; i <= l; ++i) {
              const double* Ti = Tf + 12 * jidx[i];
              double Ri[9] = {Ti[0], Ti[1], Ti[2], Ti[4], Ti[5], Ti[6], Ti[8], Ti[9], Ti[10]};
              const double* a = rb->axis + 3 * jidx[i];
              double w[3] = {Ri[0] * a[0] + Ri[1] * a[1] + Ri[2] * a[2], Ri[3] * a[0] + Ri[4] * a[1] + Ri[5] * a[2],
                             Ri[6] * a[0] + Ri[7] * a[1] + Ri[8] * a[2]};
              double dc[3];
              if (rb->type[jidx[i]] == OR_JOINT_REVOLUTE) {
                double e[3] = {c[0] - Ti[3], c[1] - Ti[7], c[2] - Ti[11]};
                dc[0] = w[1] * e[2] - w[2] * e[1];
                dc[1] = w[2] * e[0] - w[0] * e[2];
                dc[2] = w[0] * e[1] - w[1] * e[0];
              } else {
                /* a prismatic joint translates both ends of the link */
                dc[0] = w[0]; dc[1] = w[1]; dc[2] = w[2];
              }
              SETJ(row, t * n + i, p->w_coll * df * (nrm[0] * dc[0] + nrm[1] * dc[1] + nrm[2] * dc[2]));
            }
          }
        }
      }
    }
  }
  /* velocity-limit hinge per (t >= 1, joint): w_vlimit max(0, |q_t - q_{t-1}| - v_max) */
  for (int t = 1; t < T; ++t)
    for (int i = 0; i < n; ++i, ++row) {
      if (!(p->w_vlimit > 0)) { r[row] = 0; continue; } /* hinge off */
      const double v = x[t * n + i] - x[(t - 1) * n + i];
      const double h = fabs(v) - p->v_max;
      if (h > 0) {
        const double sg = v > 0 ? 1.0 : -1.0;
        r[row] = p->w_vlimit * h;
        SETJ(row, t * n + i, p->w_vlimit * sg);
        SETJ(row, (t - 1) * n + i, -p->w_vlimit * sg);
      } else {
        r[row] = 0;
      }
    }
  /* swept spheres: the capsule from c(t) to c(t+1) of every link sphere
   * against every obstacle sphere; d = |o - p| - r - r_o with p the capsule
   * axis point closest to the obstacle centre o (parameter u in [0, 1]);
   * dd/dc(t) = (1 - u) n and dd/dc(t+1) = u n, n = (p - o) / |p - o| */
  double* Tf2 = (double*)malloc(sizeof(double) * 12 * nj);
  if (!(p->w_swept > 0)) {
    /* swept rows off: every row is w_swept * f = 0 */
    for (int i = 0; i < (T - 1) * n * sc->S * sc->n_obs; ++i, ++row) r[row] = 0;
  }
  for (int t = 0; t + 1 < T && p->w_swept > 0; ++t) {
    or_fk(rb, x + (size_t)t * n, Tf);
    or_fk(rb, x + (size_t)(t + 1) * n, Tf2);
    for (int l = 0; l < n; ++l) {
      for (int s = 0; s < sc->S; ++s) {
        const double al = (s + 0.5) / sc->S;
        double c0[3], c1[3];
        {
          const double* pa = Tf + 12 * jidx[l];
          const double* pb = Tf + 12 * jidx[l + 1];
          const double* qa = Tf2 + 12 * jidx[l];
          const double* qb = Tf2 + 12 * jidx[l + 1];
          for (int i = 0; i < 3; ++i) {
            const int k = 4 * i + 3;
            c0[i] = pa[k] + al * (pb[k] - pa[k]);
            c1[i] = qa[k] + al * (qb[k] - qa[k]);
          }
        }
        const double rad = sc->radii[l * sc->S + s];
        for (int o = 0; o < sc->n_obs; ++o, ++row) {
          const double* ob = sc->obs + 4 * o;
          double e[3] = {c1[0] - c0[0], c1[1] - c0[1], c1[2] - c0[2]};
          const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
          double u = ee > 0 ? ((ob[0] - c0[0]) * e[0] + (ob[1] - c0[1]) * e[1] + (ob[2] - c0[2]) * e[2]) / ee : 0.0;
          u = u < 0 ? 0 : (u > 1 ? 1 : u);
          double pnt[3] = {c0[0] + u * e[0], c0[1] + u * e[1], c0[2] + u * e[2]};
          double v3[3] = {pnt[0] - ob[0], pnt[1] - ob[1], pnt[2] - ob[2]};
          const double len = sqrt(v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2]);
          const double d = len - rad - ob[3];
          double df;
          const double fa = p->w_swept > 0 ? or_coll_activation(d, p->eta, &df) : 0.0;
          r[row] = p->w_swept * fa;
          if (!Jc || p->w_swept <= 0 || df == 0.0 || len <= 0) continue;
          const double nrm[3] = {v3[0] / len, v3[1] / len, v3[2] / len};
          for (int side = 0; side < 2; ++side) {
            const double* TT = side ? Tf2 : Tf;
            const double* c = side ? c1 : c0;
            const double sc_ = side ? u : 1.0 - u;
            const int tt = t + side;
            for (int i = 0; i <= l; ++i) {
              const double* Ti = TT + 12 * jidx[i];
              const double* a = rb->axis + 3 * jidx[i];
              double w[3] = {Ti[0] * a[0] + Ti[1] * a[1] + Ti[2] * a[2], Ti[4] * a[0] + Ti[5] * a[1] + Ti[6] * a[2],
                             Ti[8] * a[0] + Ti[9] * a[1] + Ti[10] * a[2]};
              double dc[3];
              if (rb->type[jidx[i]] == OR_JOINT_REVOLUTE) {
                double ev[3] = {c[0] - Ti[3], c[1] - Ti[7], c[2] - Ti[11]};
                dc[0] = w[1] * ev[2] - w[2] * ev[1];
                dc[1] = w[2] * ev[0] - w[0] * ev[2];
                dc[2] = w[0] * ev[1] - w[1] * ev[0];
              } else {
                dc[0] = w[0]; dc[1] = w[1]; dc[2] = w[2];
              }
              SETJ(row, tt * n + i, p->w_swept * df * sc_ * (nrm[0] * dc[0] + nrm[1] * dc[1] + nrm[2] * dc[2]));
            }
          }
        }
      }
    }
  }
  free(Tf2);
  /* five-point acceleration and jerk rows, t = 2..T-3 */
  {
    static const double ca[5] = {-1.0 / 12, 16.0 / 12, -30.0 / 12, 16.0 / 12, -1.0 / 12}; /* q_{t-2} .. q_{t+2} */
    static const double cj[5] = {-0.5, 1.0, 0.0, -1.0, 0.5};
    for (int kind = 0; kind < 2; ++kind) {
      const double* c = kind ? cj : ca;
      const double w = kind ? p->w_jerk : p->w_acc5;
      for (int t = 2; t + 2 < T; ++t)
        for (int i = 0; i < n; ++i, ++row) {
          if (w == 0.0) { r[row] = 0; continue; } /* stencil off */
          double v = 0;
          for (int k = 0; k < 5; ++k) v += c[k] * x[(t - 2 + k) * n + i];
          r[row] = w * v;
          if (w != 0.0)
            for (int k = 0; k < 5; ++k)
              if (c[k] != 0.0) SETJ(row, (t - 2 + k) * n + i, w * c[k]);
        }
    }
  }
  free(Tf);
  free(jidx);
}

/* Dense form of the same residual (small problems; J [m][T*n] row-major). */
void or_traj_residual(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T,
                      const double* x, const double* q_start, const double* goal, double* r, double* J) {
  const int n = or_n_dof(rb), N = T * n, m = or_traj_n_residuals(rb, sc, T);
  int* Jc = J ? (int*)malloc(sizeof(int) * (size_t)m * KW) : NULL;
  double* Jv = J ? (double*)malloc(sizeof(double) * (size_t)m * KW) : NULL;
  or_traj_residual_sparse(rb, p, sc, T, x, q_start, goal, r, Jc, Jv);
  if (J) {
    memset(J, 0, sizeof(double) * (size_t)m * N);
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < KW && Jc[(size_t)i * KW + k] >= 0; ++k)
        J[(size_t)i * N + Jc[(size_t)i * KW + k]] = Jv[(size_t)i * KW + k];
  }
  free(Jc);
  free(Jv);
}

/* Normal equations (J^T J [N][N] dense, J^T r [N]) and cost 1/2 |r|^2, formed
 * row by row from the dense Jacobian of or_traj_residual. */
static double traj_normal(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T,
                          const double* x, const double* qs, const double* goal, double* A, double* g) {
  const int n = or_n_dof(rb), N = T * n, m = or_traj_n_residuals(rb, sc, T);
  double* r = (double*)malloc(sizeof(double) * m);
  int* Jc = A ? (int*)malloc(sizeof(int) * (size_t)m * KW) : NULL;
  double* Jv = A ? (double*)malloc(sizeof(double) * (size_t)m * KW) : NULL;
  or_traj_residual_sparse(rb, p, sc, T, x, qs, goal, r, Jc, Jv);
  double f = 0;
  for (int i = 0; i < m; ++i) f += r[i] * r[i];
  if (A) {
    /* J^T J and J^T r, one row's outer product at a time; J^T J is
     * symmetric, so its lower triangle is summed and mirrored at the end */
    memset(A, 0, sizeof(double) * (size_t)N * N);
    memset(g, 0, sizeof(double) * N);
    for (int i = 0; i < m; ++i) {
      const int* c = Jc + (size_t)i * KW;
      const double* v = Jv + (size_t)i * KW;
      for (int u = 0; u < KW && c[u] >= 0; ++u) {
        g[c[u]] += v[u] * r[i];
        for (int w = 0; w < KW && c[w] >= 0; ++w)
          if (c[w] <= c[u]) A[(size_t)c[u] * N + c[w]] += v[u] * v[w];
      }
    }
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < a; ++b) A[(size_t)b * N + a] = A[(size_t)a * N + b];
    free(Jc);
    free(Jv);
  }
  free(r);
  return 0.5 * f;
}

/* Block-banded Cholesky of an SPD matrix with blocks (t, t'), |t - t'| <= B,
 * of size n: the block diagonals are factored step by step in t.  L is
 * written into a dense [N][N] array (zero outside the band).  Returns 0 on
 * success. */
int32_t or_banded_cholesky_b(int32_t T, int32_t n, int32_t B, const double* A, double* L) {
  const int N = T * n;
  memset(L, 0, sizeof(double) * (size_t)N * N);
  for (int t = 0; t < T; ++t) {
    const int c0 = (t >= B ? t - B : 0) * n; /* first column of the band in block row t */
    for (int i = t * n; i < (t + 1) * n; ++i) {
      for (int j = c0; j <= i; ++j) {
        double s = A[(size_t)i * N + j];
        /* L[i][k] and L[j][k] are both inside the band only from column k0 on */
        const int cj = (j / n >= B ? j / n - B : 0) * n;
        const int k0 = cj > c0 ? cj : c0;
        for (int k = k0; k < j; ++k) s -= L[(size_t)i * N + k] * L[(size_t)j * N + k];
        if (i == j) {
          if (!(s > 0) || !isfinite(s)) return 1;
          L[(size_t)i * N + i] = sqrt(s);
        } else {
          L[(size_t)i * N + j] = s / L[(size_t)j * N + j];
        }
      }
    }
  }
  return 0;
}

/* The band-2 case (the three-point stencils). */
int32_t or_banded_cholesky(int32_t T, int32_t n, const double* A, double* L) {
  return or_banded_cholesky_b(T, n, 2, A, L);
}

static int dense_cholesky(int N, const double* A, double* L) {
  memset(L, 0, sizeof(double) * (size_t)N * N);
  for (int j = 0; j < N; ++j) {
    double d = A[(size_t)j * N + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * N + k] * L[(size_t)j * N + k];
    if (!(d > 0) || !isfinite(d)) return 1;
    L[(size_t)j * N + j] = sqrt(d);
    for (int i = j + 1; i < N; ++i) {
      double s = A[(size_t)i * N + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * N + k] * L[(size_t)j * N + k];
      L[(size_t)i * N + j] = s / L[(size_t)j * N + j];
    }
  }
  return 0;
}

static void chol_solve(int N, const double* L, const double* b, double* x) {
  double* y = (double*)malloc(sizeof(double) * N);
  for (int i = 0; i < N; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * N + k] * y[k];
    y[i] = s / L[(size_t)i * N + i];
  }
  for (int i = N - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < N; ++k) s -= L[(size_t)k * N + i] * x[k];
    x[i] = s / L[(size_t)i * N + i];
  }
  free(y);
}

/* The same substitutions with a block-banded factor (blocks of n, B block
 * sub-diagonals): only the band of L enters the sums. */
static void chol_solve_band(int N, int n, int B, const double* L, const double* b, double* x) {
  double* y = (double*)malloc(sizeof(double) * N);
  for (int i = 0; i < N; ++i) {
    const int k0 = (i / n >= B ? i / n - B : 0) * n;
    double s = b[i];
    for (int k = k0; k < i; ++k) s -= L[(size_t)i * N + k] * y[k];
    y[i] = s / L[(size_t)i * N + i];
  }
  for (int i = N - 1; i >= 0; --i) {
    const int k1 = (i / n + B + 1) * n < N ? (i / n + B + 1) * n : N;
    double s = y[i];
    for (int k = i + 1; k < k1; ++k) s -= L[(size_t)k * N + i] * x[k];
    x[i] = s / L[(size_t)i * N + i];
  }
  free(y);
}

/* Exported for the pins: normal matrix, gradient and cost at x. */
double or_traj_normal(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T,
                      const double* x, const double* qs, const double* goal, double* A, double* g) {
  return traj_normal(rb, p, sc, T, x, qs, goal, A, g);
}

/* LM on one trajectory: x [T][n] in/out; trace (optional) [iters][T][n] and
 * lam_trace (optional) [iters]: x and the damping after every iteration. */
static double traj_lm(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T,
                      double* x, const double* qs, const double* goal, double* trace, double* margin,
                      double* lam_trace) {
  const int n = or_n_dof(rb), N = T * n;
  double* A = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* Al = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* L = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* g = (double*)malloc(sizeof(double) * N);
  double* ng = (double*)malloc(sizeof(double) * N);
  double* dx = (double*)malloc(sizeof(double) * N);
  double* xt = (double*)malloc(sizeof(double) * N);
  double lambda = p->lambda0;
  double f = traj_normal(rb, p, sc, T, x, qs, goal, A, g);
  if (margin) *margin = INFINITY;
  for (int it = 0; it < p->iters; ++it) {
    memcpy(Al, A, sizeof(double) * (size_t)N * N);
    for (int i = 0; i < N; ++i) {
      Al[(size_t)i * N + i] += lambda;
      ng[i] = -g[i];
    }
    const int band = (p->w_acc5 != 0.0 || p->w_jerk != 0.0) ? 4 : 2;
    const int rc = p->banded ? or_banded_cholesky_b(T, n, band, Al, L) : dense_cholesky(N, Al, L);
    int accepted = 0;
    if (rc == 0) {
      if (p->banded)
        chol_solve_band(N, n, band, L, ng, dx);
      else
        chol_solve(N, L, ng, dx);
      for (int i = 0; i < N; ++i) xt[i] = x[i] + dx[i];
      const double ft = traj_normal(rb, p, sc, T, xt, qs, goal, NULL, NULL);
      if (margin && it < 5 && f > 0 && fabs(ft - f) / f < *margin) *margin = fabs(ft - f) / f;
      if (ft < f) {
        accepted = 1;
        memcpy(x, xt, sizeof(double) * N);
        f = traj_normal(rb, p, sc, T, x, qs, goal, A, g);
      }
    }
    if (accepted) {
      lambda /= p->nu;
      if (lambda < p->lambda_min) lambda = p->lambda_min;
    } else {
      lambda *= p->nu;
      if (lambda > p->lambda_max) lambda = p->lambda_max;
    }
    if (trace) memcpy(trace + (size_t)it * N, x, sizeof(double) * N);
    if (lam_trace) lam_trace[it] = lambda;
  }
  free(A); free(Al); free(L); free(g); free(ng); free(dx); free(xt);
  return f;
}

typedef struct {
  const or_robot* rb;
  const or_traj_params* p;
  const or_traj_scene* sc;
  int32_t batch, T, n;
  double* x;
  const double* qs;
  const double* goals;
  double* cost;
  double* trace;
  double* margin;
  long next;
} traj_pool;

static void* traj_worker(void* arg) {
  traj_pool* c = (traj_pool*)arg;
  for (;;) {
    long b = __atomic_fetch_add(&c->next, 1, __ATOMIC_RELAXED);
    if (b >= c->batch) break;
    const size_t N = (size_t)c->T * c->n;
    c->cost[b] = traj_lm(c->rb, c->p, c->sc, c->T, c->x + b * N, c->qs + b * c->n, c->goals + b * 12,
                         c->trace ? c->trace + b * (size_t)c->p->iters * N : NULL,
                         c->margin ? c->margin + b : NULL, NULL);
  }
  return NULL;
}

/* Batched LM over trajectories (x [batch][T][n] in/out, q_start [batch][n],
 * goals [batch][12]); returns the number of threads used. */
int32_t or_traj_solve(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t batch,
                      int32_t T, double* x, const double* q_start, const double* goals, double* cost,
                      double* trace, double* margin, int32_t n_threads) {
  if (n_threads <= 0) n_threads = or_host_cores();
  if (n_threads > batch) n_threads = batch > 0 ? batch : 1;
  traj_pool c = {rb, p, sc, batch, T, or_n_dof(rb), x, q_start, goals, cost, trace, margin, 0};
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, traj_worker, &c);
  for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
  free(th);
  return n_threads;
}

/* One trajectory's LM run with its x and damping after every iteration, for
 * the pins of the damping schedule; returns the final cost. */
double or_traj_lm_run(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T, double* x,
                      const double* q_start, const double* goal, double* trace, double* lam_trace) {
  return traj_lm(rb, p, sc, T, x, q_start, goal, trace, NULL, lam_trace);
}
