/*
 * pk_oracle.h -- FP64 CPU oracle for the batched Levenberg-Marquardt kinematic
 * optimiser of "PyRoki: A Modular Toolkit for Robot Kinematic Optimization"
 * (arXiv 2505.03728).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the parity authority for the CUDA
 * path; only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, constant or helper with the
 * CUDA library: every formula here is written out again from the paper
 * (Sec. III-A solver, Sec. III-B variables, Sec. III-C costs, Eq. 1) and from
 * textbook Lie-group identities.
 *
 * Conventions
 *   - A rigid transform is 12 doubles, 3x4 row-major [R | t].
 *   - A twist is [rho; omega] (translation part first).
 *   - Joint types: 0 fixed, 1 revolute, 2 prismatic.  Joint j's parent is
 *     parent[j] < j (or -1 for the base).  Movable joints own one variable
 *     each, numbered in joint order ("dof index"), except mimic joints, which
 *     follow another joint's variable.
 *   - Target kinds: 0 full pose (6 residual rows), 1 position only (3 rows).
 *   - Residual rows: the targets' rows, then one limit-hinge and one rest row per
 *     variable, then one self-collision row per sphere pair.
 */
#ifndef PK_ORACLE_H
#define PK_ORACLE_H
#include <stdint.h>

#define OR_JOINT_FIXED 0
#define OR_JOINT_REVOLUTE 1
#define OR_JOINT_PRISMATIC 2
#define OR_TARGET_POSE 0
#define OR_TARGET_POSITION 1

/* per-problem status codes */
#define OR_P_CONVERGED 0
#define OR_P_MAX_ITERS 1
#define OR_P_NONFINITE 2

typedef struct {
  int32_t n_joints;
  const int32_t* parent; /* [n_joints] */
  const int32_t* type;   /* [n_joints] */
  const double* axis;    /* [n_joints][3] unit vector, joint frame */
  const double* origin;  /* [n_joints][12] parent frame -> joint frame */
  const double* lower;   /* [n_joints] (ignored for fixed joints) */
  const double* upper;   /* [n_joints] */
  /* Mimic joints (Sec. III-B): joint j with mimic[j] = s >= 0 has no variable
   * of its own; its value is mimic_mult[j] * q(s) + mimic_off[j].  NULL = no
   * mimic joints. */
  const int32_t* mimic;      /* [n_joints] source joint or -1 */
  const double* mimic_mult;  /* [n_joints] */
  const double* mimic_off;   /* [n_joints] */
  /* Self-collision model (Sec. III-C): spheres riding on joint frames and the
   * sphere pairs whose signed distance enters the self-collision cost. */
  int32_t n_spheres;
  const int32_t* sph_joint;   /* [n_spheres] frame each sphere rides on */
  const double* sph_centre;   /* [n_spheres][3] in that frame */
  const double* sph_radius;   /* [n_spheres] */
  int32_t n_pairs;
  const int32_t* pairs;       /* [n_pairs][2] sphere indices */
} or_robot;

typedef struct {
  double w_pos, w_rot;     /* pose residual weights (translation / rotation rows) */
  double w_limit, w_rest;  /* joint-limit hinge weight, rest-pose weight */
  double lambda0, lambda_min, lambda_max, nu;
  double tol_pos, tol_rot; /* success thresholds: metres, radians */
  int32_t max_iters;
  int32_t early_exit;      /* 1: stop once the tolerances are met */
  double w_self, eta_self; /* self-collision weight and buffer distance (Eq. 1) */
} or_ik_params;

typedef struct {
  int32_t n_targets;       /* k */
  const int32_t* links;    /* [k] joint frame each target constrains */
  const int32_t* kinds;    /* [k] OR_TARGET_* (NULL = all pose) */
} or_target_spec;

int32_t or_n_dof(const or_robot* rb);
int32_t or_n_residuals(const or_robot* rb, const or_target_spec* ts);

/* FK of every joint frame: T_out[n_joints][12] (base <- joint j after motion). */
void or_fk(const or_robot* rb, const double* q, double* T_out);

/* SE(3) / SO(3) helpers (exported for the pins). */
void or_se3_log(const double* T, double* xi);
void or_se3_exp(const double* xi, double* T);
void or_se3_jl(const double* xi, double* J);     /* 6x6 row-major left Jacobian */
void or_se3_jlinv(const double* xi, double* J);  /* 6x6 row-major inverse */

/* IK residual r[m] and analytic Jacobian J[m][n_dof] (J may be NULL). */
void or_ik_residual(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts,
                    const double* targets, const double* q, double* r, double* J);

/* pose errors: max over targets of |p - p*| and of the rotation angle */
void or_ik_errors(const or_robot* rb, const or_target_spec* ts, const double* targets,
                  const double* q, double* pos_err, double* rot_err);

/* Gauss-Newton normal equations A = J^T J [nd][nd], g = J^T r [nd] of the
 * m x nd row-major Jacobian J. */
void or_normal_equations(int32_t m, int32_t nd, const double* J, const double* r, double* A, double* g);

/* Cholesky solve of the SPD system A x = b (n x n row-major). Returns 0 on success. */
int32_t or_cholesky_solve(int32_t n, const double* A, const double* b, double* x);

/*
 * Multi-start LM over batch targets x n_seeds seeds.
 *   targets [batch][k][12], seeds [batch][n_seeds][n_dof]
 *   q_out [batch][n_dof] best seed (converged first, then lowest cost, then lowest index)
 *   err_out [batch][2], iters_out [batch], status_out [batch]
 *   per_problem (optional, [batch*n_seeds][n_dof + 5]): q, cost, pos_err, rot_err,
 *       iters, status of every seed.
 *   trace (optional, [batch*n_seeds][n_trace][n_dof]): q after iteration 1..n_trace.
 *   margin (optional, [batch*n_seeds]): min over the first n_trace iterations of
 *       |f_trial - f| / f, used to flag accept/reject near-ties.
 * n_threads <= 0 uses every online core.  Returns the number of threads used.
 */
int32_t or_ik_solve(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts,
                    int32_t batch, int32_t n_seeds, const double* targets, const double* seeds,
                    double* q_out, double* err_out, int32_t* iters_out, int32_t* status_out,
                    double* per_problem, int32_t n_trace, double* trace, double* margin,
                    int32_t n_threads);

/*
 * One LM run (Sec. III-A) of a single (target set, seed) problem, for the pins
 * of the damping schedule.  lambda_init < 0 starts from p->lambda0.
 *   q_trace [n_trace][n_dof], lam_trace [n_trace] (either may be NULL): q and
 *     the damping after iterations 1..n_trace (the final state repeated past
 *     the last iteration);
 *   q_out [n_dof]; res_out [6] = cost, pos_err, rot_err, iterations, status,
 *     final damping.
 * Returns the status.
 */
int32_t or_lm_run(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts, const double* targets,
                  const double* seed, double lambda_init, int32_t n_trace, double* q_trace, double* lam_trace,
                  double* q_out, double* res_out);

/*
 * IK-Beam (Sec. V-C) over batch targets with n_seeds seeds each: steps1 LM
 * iterations on every seed, then the `keep` lowest-cost seeds (ties: lower
 * seed index; non-finite costs last) continue from their configuration and
 * damping for steps2 iterations; the best of those (converged first, then
 * lowest cost, then lowest seed index) is returned.  p->max_iters is ignored;
 * p->early_exit applies to both phases.  iters_out = phase-1 + phase-2
 * iterations of the returned seed; kept_out (optional, [batch][keep]) the
 * kept seed indices in selection order.
 */
int32_t or_ik_beam(const or_robot* rb, const or_ik_params* p, const or_target_spec* ts, int32_t batch,
                   int32_t n_seeds, int32_t steps1, int32_t keep, int32_t steps2, const double* targets,
                   const double* seeds, double* q_out, double* err_out, int32_t* iters_out,
                   int32_t* status_out, int32_t* kept_out, int32_t n_threads);

/* Host cores available to this process (affinity mask, else online CPUs). */
int32_t or_host_cores(void);

#endif
