/*
 * flops_traj.cpp -- the trajectory oracle (trajopt_oracle.c, unchanged)
 * compiled with the counting double of flopcount.hpp, and the census of its
 * work per LM unit.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY.  Units of one trajectory LM
 * iteration: a candidate evaluation (residuals and cost), a normal-equation
 * build at an accepted point (the Jacobian rows' share of the residual pass
 * and the banded J^T J, J^T r) and a damped solve (lambda on the diagonal,
 * the block-banded Cholesky of Sec. III-A's normal equations, both
 * substitutions, the trial step).
 */
#include "flopcount.hpp"

#define double or_fd
extern "C" {
#include "trajopt_oracle.c"
}

extern "C" {

void orf_reset(void);
void orf_read(int64_t* out);

/* out[0..1] evaluation, out[2..3] build, out[4..5] solve (FLOPs, special) at
 * trajectory x [T][n] with damping lambda. */
void orf_traj_units(const or_robot* rb, const or_traj_params* p, const or_traj_scene* sc, int32_t T,
                    const double* x, const double* q_start, const double* goal, double lambda, int64_t* out) {
  const int n = or_n_dof(rb), N = T * n;
  const int band = (p->w_acc5 != 0.0 || p->w_jerk != 0.0) ? 4 : 2;
  double* A = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* L = (double*)malloc(sizeof(double) * (size_t)N * N);
  double* g = (double*)malloc(sizeof(double) * N);
  double* dx = (double*)malloc(sizeof(double) * N);
  int64_t c0[2], c1[2];
  orf_reset();
  (void)traj_normal(rb, p, sc, T, x, q_start, goal, NULL, NULL);
  orf_read(c0);
  out[0] = c0[0]; out[1] = c0[1];
  orf_reset();
  (void)traj_normal(rb, p, sc, T, x, q_start, goal, A, g);
  orf_read(c1);
  out[2] = c1[0] - c0[0]; out[3] = c1[1] - c0[1];
  for (int i = 0; i < N; ++i) g[i] = -g[i];
  orf_reset();
  or_fc.skip_zeros = 0;
  for (int i = 0; i < N; ++i) A[(size_t)i * N + i] += lambda;
  const int rc = or_banded_cholesky_b(T, n, band, A, L);
  if (rc == 0) {
    chol_solve_band(N, n, band, L, g, dx);
    for (int i = 0; i < N; ++i) dx[i] = x[i] + dx[i];
  }
  or_fc.skip_zeros = 1;
  orf_read(c1);
  out[4] = rc == 0 ? c1[0] : -1;
  out[5] = c1[1];
  free(A); free(L); free(g); free(dx);
}

}  // extern "C"
