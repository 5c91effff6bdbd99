/*
 * flops_pk.cpp -- the IK oracle (pk_oracle.c, unchanged) compiled with the
 * counting double of flopcount.hpp, and the census of its work per LM unit.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY: the benchmark's roofline takes
 * its algorithmic FLOPs per unit from here.  The units are the ones a solver
 * counts while it runs: a candidate evaluation (FK, residuals, cost), a
 * normal-equation build at an accepted point (Jacobian, J^T J, J^T r, the
 * convergence errors) and a damped solve (lambda on the diagonal, Cholesky,
 * both substitutions, the trial step).
 */
#include "flopcount.hpp"

thread_local or_flop_counts or_fc = {0, 0, 1};

#define double or_fd
extern "C" {
#include "pk_oracle.c"
}

extern "C" {

void orf_reset(void) { or_fc.flops = 0; or_fc.special = 0; }

void orf_read(int64_t* out) { out[0] = or_fc.flops; out[1] = or_fc.special; }

/* FLOPs and special operations of the three LM units at configuration q:
 *   out[0..1] evaluation: or_ik_residual without Jacobian + 1/2 |r|^2
 *   out[2..3] build: Jacobian (residual with J minus residual without),
 *             or_normal_equations, and the convergence errors (or_ik_errors
 *             minus its own FK)
 *   out[4..5] solve: lambda added to the diagonal, or_cholesky_solve, q + dq */
void orf_ik_units(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts, const double* targets,
                  const double* q, double lambda, int64_t* out) {
  const int nd = or_n_dof(rb), m = or_n_residuals(rb, ts);
  double* r = (double*)malloc(sizeof(double) * m);
  double* J = (double*)malloc(sizeof(double) * m * nd);
  double* A = (double*)malloc(sizeof(double) * nd * nd);
  double* g = (double*)malloc(sizeof(double) * nd);
  double* dq = (double*)malloc(sizeof(double) * nd);
  double* T = (double*)malloc(sizeof(double) * 12 * rb->n_joints);
  int64_t c0[2], c1[2];
  double pe, re;
  /* evaluation */
  orf_reset();
  or_ik_residual(rb, p, ts, targets, q, r, NULL);
  (void)half_sq(r, m);
  orf_read(c0);
  out[0] = c0[0]; out[1] = c0[1];
  /* build */
  orf_reset();
  or_ik_residual(rb, p, ts, targets, q, r, J);
  orf_read(c1);
  int64_t jac = c1[0] - c0[0] + (int64_t)0, jac_s = c1[1] - c0[1];
  /* half_sq is not part of the residual call: add it back to the difference */
  orf_reset();
  (void)half_sq(r, m);
  orf_read(c1);
  jac += c1[0]; jac_s += c1[1];
  orf_reset();
  or_normal_equations(m, nd, J, r, A, g);
  or_ik_errors(rb, ts, targets, q, &pe, &re);
  orf_read(c1);
  int64_t b = c1[0], b_s = c1[1];
  orf_reset();
  or_fk(rb, q, T);
  orf_read(c1);
  out[2] = jac + b - c1[0];
  out[3] = jac_s + b_s - c1[1];
  /* solve */
  for (int a = 0; a < nd; ++a) g[a] = -g[a];
  orf_reset();
  or_fc.skip_zeros = 0;
  for (int a = 0; a < nd; ++a) A[a * nd + a] += lambda;
  const int rc = or_cholesky_solve(nd, A, g, dq);
  for (int a = 0; a < nd; ++a) dq[a] = q[a] + dq[a];
  or_fc.skip_zeros = 1;
  orf_read(c1);
  out[4] = rc == 0 ? c1[0] : -1;
  out[5] = c1[1];
  free(r); free(J); free(A); free(g); free(dq); free(T);
}

}  // extern "C"
