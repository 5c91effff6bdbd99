/*
 * pk.h -- C ABI of libpk, the GB300 (sm_103a) batched kinematic optimiser.
 *
 * The library solves many independent robot-kinematics least-squares problems
 * with Levenberg-Marquardt (LM), following "PyRoki: A Modular Toolkit for
 * Robot Kinematic Optimization" (arXiv 2505.03728):
 *   - variables: one joint configuration q per problem, forward kinematics
 *     T_base<-i = FK(q)_i over fixed, revolute and prismatic joints (Sec. III-B);
 *   - costs, each weighted (Sec. III-C): joint pose cost
 *     log(T_target^-1 T_base<-i) in R^6 ordered [rho; omega], joint limit cost
 *     max(0, q - q_upper) + max(0, q_lower - q), joint regularisation
 *     q - q_rest with q_rest the middle of the limits;
 *   - solver: LM on the sum of squared residuals with analytic Jacobians
 *     (Sec. III-A and Sec. V-C): (J^T J + lambda I) dq = -J^T r, a trial step is
 *     kept iff it strictly lowers the cost; lambda /= nu on acceptance and
 *     lambda *= nu on rejection, clamped to [lambda_min, lambda_max].
 *
 * Conventions shared by every entry point
 *   - Transforms are 12 floats, 3x4 row-major [R | t]; lengths in metres,
 *     angles in radians.
 *   - Pointers named d_* are DEVICE pointers owned by the caller; all other
 *     pointers are host pointers, read during the call only.
 *   - Every call that takes a stream only enqueues work on it (cudaStream_t,
 *     NULL = the legacy default stream) and returns without synchronising.
 *     Argument errors are detected on the host and returned synchronously,
 *     with nothing enqueued.  Per-problem numerical trouble is reported in the
 *     per-problem status output, never by a trap.
 *   - No C++ exception crosses this interface.  pk_last_error() returns a
 *     thread-local description of the last non-PK_OK status.
 *   - Robot handles are immutable after creation and may be used from several
 *     threads and streams at once.
 */
#ifndef PK_H
#define PK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PK_OK = 0,
  PK_ERR_INVALID_ARG = 1,
  PK_ERR_CUDA = 2,
  PK_ERR_OOM = 3,
  PK_ERR_TIMEOUT = 4,
  PK_ERR_UNSUPPORTED = 5
} pk_status;

typedef enum { PK_JOINT_FIXED = 0, PK_JOINT_REVOLUTE = 1, PK_JOINT_PRISMATIC = 2 } pk_joint_type;

/* Pose targets give 6 residual rows, position targets 3 (world-frame
 * difference of the frame origin), Sec. III-C joint pose cost. */
typedef enum { PK_TARGET_POSE = 0, PK_TARGET_POSITION = 1 } pk_target_kind;

/* Per-problem status codes written by the solvers. */
enum {
  PK_P_CONVERGED = 0, /* final pose within tol_pos / tol_rot for every target */
  PK_P_MAX_ITERS = 1, /* iteration cap reached without meeting the tolerances */
  PK_P_NONFINITE = 2, /* the cost at the seed was not finite (e.g. NaN target) */
  PK_P_CANCELLED = 3  /* stopped because a sibling seed of the same target converged */
};

typedef struct pk_robot pk_robot;

/* LM settings.  Weights multiply residuals (the cost is 1/2 sum r^2). */
typedef struct {
  float w_pos;           /* translation rows of the pose residual (default 1)   */
  float w_rot;           /* rotation rows of the pose residual (default 0.5)    */
  float w_limit;         /* joint-limit hinge (default 10)                      */
  float w_rest;          /* rest-pose regularisation (default 1e-3)             */
  float lambda0;         /* initial damping (default 1e-2)                      */
  float lambda_min;      /* default 1e-10                                       */
  float lambda_max;      /* default 1e10                                        */
  float nu;              /* damping factor, > 1 (default 2)                     */
  float tol_pos;         /* success threshold, metres (default 1e-3)            */
  float tol_rot;         /* success threshold, radians (default 0.5 deg)        */
  int32_t max_iters;     /* LM iterations per seed; a rejected step counts      */
  int32_t early_exit;    /* 1: a seed stops as soon as it meets the tolerances  */
  int32_t cancel_siblings; /* 1: all seeds of a target stop once one converged  */
  int32_t reserved;      /* must be 0                                           */
  float w_self;          /* self-collision weight (Sec. III-C; 0 = off, default)  */
  float eta_self;        /* its buffer distance eta of Eq. 1, metres (0.02)      */
} pk_ik_params;

/* Fills *p with the defaults listed above (max_iters 50, early_exit 1,
 * cancel_siblings 0). */
void pk_ik_params_default(pk_ik_params* p);

/*
 * pk_robot_create -- kinematic tree (Sec. III-B: fixed, revolute and prismatic
 * joints; T_j = T_parent(j) * origin_j * X_j(q_j)).
 *   n_joints  1..64
 *   parent    [n_joints], parent[j] in [-1, j-1]; -1 = attached to the base
 *   type      [n_joints], pk_joint_type
 *   axis      [n_joints][3], joint axis in the joint frame (normalised here;
 *             must be non-zero for movable joints)
 *   origin    [n_joints][12], parent frame -> joint frame before motion
 *             (rotation part must be orthonormal to 1e-4)
 *   lower, upper [n_joints], limits of movable joints (lower <= upper);
 *             ignored for fixed joints
 *   tool      [12] or NULL: when given, appended as one more fixed joint
 *             whose parent is joint n_joints-1
 * Movable joints own one variable each, numbered in joint order.
 * All pointers are host pointers, copied.  Returns PK_ERR_INVALID_ARG on a
 * malformed tree, PK_ERR_CUDA / PK_ERR_OOM if the device copy fails.
 */
pk_status pk_robot_create(int32_t n_joints, const int32_t* parent, const int32_t* type,
                          const float* axis, const float* origin, const float* lower,
                          const float* upper, const float* tool, pk_robot** out);
void pk_robot_destroy(pk_robot* robot);
/*
 * Mimic joints (Sec. III-B, the coupled joints of robot hands): movable joint
 * `joint` gives up its own variable and follows movable joint `source`'s:
 * value = multiplier * q_source + offset.  Variables are renumbered (the
 * movable joints that are not mimics, in joint order), so pk_robot_n_dof()
 * drops by one; the mimic joint's own limits are not enforced (its source's
 * are).  A source may not itself be a mimic, a mimic may not be a source, and
 * a joint is made a mimic once.
 * Robots with mimic joints run on the warp-per-problem path (up to 4 mimics
 * per variable); the serial-chain kernels and trajectory optimisation refuse
 * them (PK_ERR_UNSUPPORTED).  Synchronous (updates the device copy); call it
 * before any solve that uses the robot.
 */
pk_status pk_robot_set_mimic(pk_robot* robot, int32_t joint, int32_t source, float multiplier, float offset);
/*
 * Self-collision model (Sec. III-C): spheres riding on joint frames and the
 * sphere pairs that must stay apart.  With params->w_self > 0, every pair adds
 * the residual w_self f(d, eta_self) of Eq. 1, d = |c_a - c_b| - r_a - r_b
 * (rows after the limit and rest rows), and the solve runs on the
 * warp-per-problem path.
 *   n_spheres 0..64: joint [n] (frame each sphere rides on), centre [n][3]
 *   (in that frame), radius [n] (>= 0); n_pairs 0..64: pairs [n_pairs][2]
 *   (distinct sphere indices).  Host pointers, copied; replaces any earlier
 *   model; synchronous.
 */
pk_status pk_robot_set_spheres(pk_robot* robot, int32_t n_spheres, const int32_t* joint, const float* centre,
                               const float* radius, int32_t n_pairs, const int32_t* pairs);
int32_t pk_robot_n_joints(const pk_robot* robot);
int32_t pk_robot_n_dof(const pk_robot* robot);

/*
 * pk_fk -- forward kinematics of every joint frame (Sec. III-B).
 *   d_q      [batch][n_dof]
 *   d_T_out  [batch][n_joints][12]
 */
pk_status pk_fk(const pk_robot* robot, int32_t batch, const float* d_q, float* d_T_out,
                void* stream);

/*
 * pk_ik_residual -- weighted residual vector and analytic Jacobian at given
 * configurations (Sec. III-C costs; the Jacobian of the pose rows is
 * Jl^-1(r) Ad(T_target^-1) xi_j for every movable ancestor j).
 * Supported: serial chains with one target on the last frame (k = 1), n_dof <= 8.
 *   d_targets [batch][k][12], d_q [batch][n_dof]
 *   d_r_out   [batch][m], m = 6 (or 3) + 2 n_dof, rows: pose, limit, rest
 *   d_J_out   [batch][m][n_dof] row-major, or NULL
 */
pk_status pk_ik_residual(const pk_robot* robot, const pk_ik_params* params, int32_t k,
                         const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                         const float* d_targets, const float* d_q, float* d_r_out, float* d_J_out,
                         void* stream);

/*
 * Scratch that pk_ik_solve needs for (batch, n_seeds): a work-queue head, one
 * cancellation flag per target and one result record per seed.
 */
size_t pk_ik_workspace_bytes(const pk_robot* robot, int32_t batch, int32_t n_seeds);

/*
 * pk_ik_solve -- multi-start LM inverse kinematics (Sec. III-A, Sec. IV-A).
 * Each target is solved from n_seeds seeds independently; the returned seed is
 * the best one: converged first, then lowest cost, then lowest seed index.
 *   k, target_links, target_kinds  host [k]; kinds may be NULL (all pose)
 *   d_targets  [batch][k][12]
 *   d_seeds    [batch][n_seeds][n_dof]
 *   d_q_out    [batch][n_dof]     best seed's final configuration
 *   d_err_out  [batch][2]         its position error (m) and rotation error (rad),
 *                                 max over targets
 *   d_iters_out [batch]           its LM iteration count
 *   d_status_out [batch]          its PK_P_* status
 *   d_workspace, workspace_bytes  caller scratch of at least
 *                                 pk_ik_workspace_bytes() bytes, 256-byte aligned;
 *                                 NULL makes the call allocate it stream-ordered
 *                                 (cudaMallocAsync / cudaFreeAsync).
 * batch == 0 is a no-op.  The workspace must not be shared by calls that can
 * overlap on the GPU.
 * Kernels: a serial chain (n_dof <= 8) with one target on a frame after its
 * last movable joint runs one problem per thread; any other tree with up to 32
 * movable joints, 64 joints and 8 targets runs one problem per warp
 * (PK_ERR_UNSUPPORTED beyond that).
 */
pk_status pk_ik_solve(const pk_robot* robot, const pk_ik_params* params, int32_t k,
                      const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                      int32_t n_seeds, const float* d_targets, const float* d_seeds,
                      float* d_q_out, float* d_err_out, int32_t* d_iters_out,
                      int32_t* d_status_out, void* d_workspace, size_t workspace_bytes,
                      void* stream);

/*
 * pk_ik_solve_noalloc -- pk_ik_solve for callers that cannot allocate device
 * memory while they run: real-time control loops that must not allocate on
 * their hot path (cudaMalloc can block for an unbounded time) and plugin hosts
 * whose device memory belongs to another allocator.  The paper has no
 * counterpart; this entry point only changes where the solver's scratch lives.
 *   Arguments, outputs and results are those of pk_ik_solve, without the
 *   workspace.  The scratch is a 32 MiB array in the library's own device
 *   memory (held on every GPU that loads the library until the process
 *   exits); a (batch, n_seeds) whose pk_ik_workspace_bytes() exceeds it is
 *   rejected with PK_ERR_INVALID_ARG and nothing is enqueued (about 690,000
 *   seeds in total for a 7-DoF chain).
 *   No cudaMalloc, cudaFree or other allocating call is made.  The argument
 *   checks of pk_ik_solve run first (a bad argument is reported as such, and
 *   batch == 0 returns PK_OK before anything else); the size limit comes
 *   next.  Every call outside stream capture looks up the array's device
 *   address on the current device (set-up; a lookup allocates nothing and
 *   stays valid after a device or context reset); a call made while `stream`
 *   is being captured uses the address of the last call outside capture, so
 *   make the first call on each device before any stream capture.
 *   All calls on a device share the one array, and it keeps the last call's
 *   contents; each call clears what must start at zero.  Calls that can
 *   overlap on the GPU (different streams, or threads) race on the array and
 *   must be serialised by the caller.
 */
pk_status pk_ik_solve_noalloc(const pk_robot* robot, const pk_ik_params* params, int32_t k,
                              const int32_t* target_links, const int32_t* target_kinds,
                              int32_t batch, int32_t n_seeds, const float* d_targets,
                              const float* d_seeds, float* d_q_out, float* d_err_out,
                              int32_t* d_iters_out, int32_t* d_status_out, void* stream);

/*
 * Scratch that pk_ik_solve_split needs for (batch, n_seeds): the
 * pk_ik_workspace_bytes() layout plus one index and one damping value per
 * (target, seed) problem.
 */
size_t pk_ik_split_workspace_bytes(const pk_robot* robot, int32_t batch, int32_t n_seeds);

/*
 * pk_ik_solve_split -- pk_ik_solve (Sec. III-A, Sec. IV-A) in two launches, so
 * that the iterations of the few slow problems can overlap other work.  Same
 * arguments, outputs and results as pk_ik_solve, plus:
 *   split_iters   >= 1: the first launch, on `stream`, carries every problem
 *                 up to this many LM iterations; a problem still running then
 *                 (not converged, not cancelled by a converged sibling) is
 *                 suspended: its configuration, iteration count and damping
 *                 stay in the workspace.
 *   tail_ctas     >= 0: 128-thread blocks of the second launch, which resumes
 *                 the suspended problems and runs them to the end (0: the full
 *                 persistent grid).  A few blocks leave the rest of the GPU to
 *                 work queued on `stream` behind the first launch (e.g. the
 *                 next batch's seed inference).
 *   tail_stream   the second launch and the best-seed selection run here,
 *                 ordered after the first launch by an event; the outputs are
 *                 complete in tail_stream's order.  tail_stream == stream runs
 *                 everything on one stream.
 *   d_workspace   required (not NULL), pk_ik_split_workspace_bytes() bytes,
 *                 256-byte aligned; it is in use until tail_stream passes the
 *                 call, so a call that overlaps it needs another workspace.
 * A resumed problem re-evaluates its cost, Jacobian and normal matrix at its
 * saved configuration and continues with its saved damping, which is what the
 * single launch holds at that point: without sibling cancellation the results
 * equal pk_ik_solve's bit for bit.  Robots served by the one-problem-per-warp
 * tree kernel run in one launch on `stream`, and tail_stream waits for it.
 * Under CUDA graph capture, join tail_stream back into the capturing stream
 * before the capture ends.
 */
pk_status pk_ik_solve_split(const pk_robot* robot, const pk_ik_params* params, int32_t k,
                            const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                            int32_t n_seeds, const float* d_targets, const float* d_seeds, float* d_q_out,
                            float* d_err_out, int32_t* d_iters_out, int32_t* d_status_out, void* d_workspace,
                            size_t workspace_bytes, int32_t split_iters, int32_t tail_ctas, void* stream,
                            void* tail_stream);

/*
 * IK-Beam (Sec. V-C) -- the paper's benchmark IK schedule: every target starts
 * from n_seeds seeds, all of which take steps1 LM iterations; the `keep` seeds
 * with the lowest cost (ties: lower seed index; a non-finite cost ranks last)
 * continue from their LM state -- configuration and damping -- for steps2
 * more iterations, and the best of those is returned (converged first, then
 * lowest cost, then lowest seed index).  The paper's schedule is 64 seeds,
 * 6 iterations, keep 4, 10 iterations (pk_ik_beam_params_default).
 */
typedef struct {
  int32_t n_seeds;  /* seeds per target, keep..1024 */
  int32_t steps1;   /* LM iterations on every seed, >= 0 */
  int32_t keep;     /* seeds that continue, 1..32 */
  int32_t steps2;   /* LM iterations on the kept seeds, >= 0 */
} pk_ik_beam_params;

void pk_ik_beam_params_default(pk_ik_beam_params* beam);
/* Scratch bytes of pk_ik_beam_solve for `batch` targets (0 on bad arguments). */
size_t pk_ik_beam_workspace_bytes(const pk_robot* robot, int32_t batch, const pk_ik_beam_params* beam);
/*
 *   params     LM weights, damping rules and tolerances as pk_ik_solve;
 *              max_iters and cancel_siblings are ignored (the beam fixes the
 *              iteration counts and runs every seed of the first round);
 *              early_exit applies to both rounds.
 *   k, target_links, target_kinds  one target on a frame after the last
 *              movable joint of a serial chain with 1..8 movable joints
 *              (PK_ERR_UNSUPPORTED otherwise)
 *   d_targets  [batch][1][12], 16-byte aligned
 *   d_seeds    [batch][n_seeds][n_dof]
 *   d_q_out [batch][n_dof], d_err_out [batch][2], d_status_out [batch]: as
 *              pk_ik_solve; d_iters_out [batch]: first-round + second-round
 *              iterations of the returned seed
 *   d_kept_out [batch][keep] or NULL: the kept seed indices, lowest cost first
 *   d_workspace, workspace_bytes  caller scratch of at least
 *              pk_ik_beam_workspace_bytes() bytes, 256-byte aligned, or NULL
 *              (stream-ordered allocation); pk_ik_workspace_stats() on it
 *              reports the work of both rounds.
 * Enqueues two memsets and four kernels on `stream`; batch == 0 is a no-op.
 */
pk_status pk_ik_beam_solve(const pk_robot* robot, const pk_ik_params* params, const pk_ik_beam_params* beam,
                           int32_t k, const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                           const float* d_targets, const float* d_seeds, float* d_q_out, float* d_err_out,
                           int32_t* d_iters_out, int32_t* d_status_out, int32_t* d_kept_out, void* d_workspace,
                           size_t workspace_bytes, void* stream);

/*
 * Uneven batches (plans).  Several problem sets -- each its own robot, target
 * set, batch size and seeds -- are solved together.  Schedule variants 0 and 1
 * run ONE persistent kernel launch: every warp drains the sets in turn, serial
 * chains of 6 or 7 movable joints one problem per thread and other trees one
 * problem per warp, so warps that finish the expensive sets fall through to
 * the cheap ones (variant 1 caps registers for three 128-thread blocks per SM).
 * With every set on the warp path (chains_as_trees = 1) the launch uses a
 * kernel without the per-thread chain path, at the tree kernel's 128
 * registers (variant 1: four 128-thread blocks per SM).  Variants 2 and 3 run each set's own specialised kernel (the pk_ik_solve
 * kernels), one after another (2) or on forked streams so that their tails
 * overlap (3).  A plan fixes its buffers at creation; its first run captures
 * the whole solve (workspace reset, the LM kernels, one best-seed reduction
 * per set) into a CUDA graph and every run launches that graph.  The LM rules
 * and outputs are those of pk_ik_solve, per set.
 */
typedef struct pk_ik_plan pk_ik_plan;

typedef struct {
  const pk_robot* robot;
  int32_t k;                   /* targets, 1..8 */
  const int32_t* target_links; /* host [k] */
  const int32_t* target_kinds; /* host [k] or NULL (all pose) */
  int32_t batch, n_seeds;
  const float* d_targets;      /* [batch][k][12], 16-byte aligned */
  const float* d_seeds;        /* [batch][n_seeds][n_dof] */
  float* d_q_out;              /* [batch][n_dof] */
  float* d_err_out;            /* [batch][2] */
  int32_t* d_iters_out;        /* [batch] */
  int32_t* d_status_out;       /* [batch] */
} pk_ik_problem_set;

/* 1..8 sets; allocates the plan's workspace (cudaMalloc).  A schedule tuned
 * earlier in this process for the same device and plan signature (robots,
 * target counts, power-of-two batch buckets, seeds) is reused. */
pk_status pk_ik_plan_create(const pk_ik_params* params, int32_t n_sets, const pk_ik_problem_set* sets,
                            pk_ik_plan** out);
void pk_ik_plan_destroy(pk_ik_plan* plan);
/* Enqueue one solve as a CUDA-graph launch on `stream`. */
pk_status pk_ik_plan_run(pk_ik_plan* plan, void* stream);
/* The same work launched kernel by kernel (no graph). */
pk_status pk_ik_plan_run_eager(pk_ik_plan* plan, void* stream);
/* Autotuner: times every candidate schedule (variant 0..3 as above, block
 * size 64/128/256 for the persistent variants, chain sets on the thread or the
 * warp path, largest-work-first or given set order) with
 * `reps` timed runs each after a warm-up, keeps the fastest (returned in
 * *best_ms, milliseconds per solve) and caches it.  Synchronous; it runs the
 * plan's solve many times, overwriting its outputs. */
pk_status pk_ik_plan_autotune(pk_ik_plan* plan, int32_t reps, void* stream, float* best_ms);
/* Read or force the schedule (block 64, 128 or 256; variant 0..3; variant 1
 * takes blocks of at most 128; grid is 0 for variants 2 and 3). */
pk_status pk_ik_plan_schedule(const pk_ik_plan* plan, int32_t* block, int32_t* grid, int32_t* chains_as_trees,
                              int32_t* given_order, int32_t* variant);
pk_status pk_ik_plan_set_schedule(pk_ik_plan* plan, int32_t block, int32_t chains_as_trees, int32_t given_order,
                                  int32_t variant);
/* Work counters of the last run (as pk_ik_workspace_stats; synchronous). */
pk_status pk_ik_plan_stats(const pk_ik_plan* plan, int64_t* stats_out);

/*
 * Work counters of the last pk_ik_solve that ran with this caller workspace
 * (read back with a synchronous copy, so call it after the solve has been
 * enqueued; it waits for the device).  stats_out (host, [4]):
 *   [0] candidate evaluations (FK + residuals + cost, seeds included)
 *   [1] normal-equation builds (Jacobian, J^T J, J^T r)
 *   [2] damped solves (Cholesky + triangular solves)
 *   [3] problems finished
 */
pk_status pk_ik_workspace_stats(const void* d_workspace, int64_t* stats_out);
/* The same for a pk_ik_solve_split workspace, stats_out [8]: [0..4) the first
 * launch (problems finished there, suspended ones not counted), [4..8) the
 * second launch (the resumed problems). */
pk_status pk_ik_split_workspace_stats(const void* d_workspace, int64_t* stats_out);

/*
 * Kernel timing trace.  While enabled, every solver kernel launch is bracketed
 * by CUDA events recorded on its own stream.  pk_trace_enable() clears the
 * trace.  pk_trace_summary() waits for the recorded events and returns the
 * summed duration (ms) and the count of traced launches of one kernel family:
 * "ik_lm" (fused LM kernel), "ik_reduce" (best-seed reduction).
 */
pk_status pk_trace_enable(int32_t enable);
pk_status pk_trace_summary(const char* kernel, double* total_ms, int64_t* launches);

/*
 * Collision-aware trajectory optimisation (Sec. IV-A, Sec. III-C costs): the
 * variables are T configurations q_0 .. q_{T-1} of a serial chain; the
 * residuals, each weighted, are the start configuration, the goal pose
 * log(T_goal^-1 FK(q_{T-1})) on the last frame, velocity q_t - q_{t-1} and
 * acceleration q_{t+1} - 2 q_t + q_{t-1} (smoothness), joint-limit hinges, and
 * the world collision cost w_c f(d, eta) of Eq. 1 for every (link sphere,
 * obstacle sphere) and (link sphere, plane) pair, d the signed distance
 * (d <= 0 takes the linear branch).  Link j carries S spheres centred at
 * p_j + (s + 1/2)/S (p_{j+1} - p_j), p_j the origin of joint frame j and p_n
 * the tool frame; the first link's spheres are not tested against the plane.
 * LM with the rules of pk_ik_solve for a fixed number of iterations; the
 * block-pentadiagonal normal matrix is factored by a block-banded Cholesky.
 */
enum { PK_T_OK = 0, PK_T_GOAL_MISSED = 1, PK_T_COLLISION = 2 }; /* status bits */

typedef struct {
  float w_start;      /* default 100 */
  float w_goal_pos;   /* default 100 (the goal is held like the start) */
  float w_goal_rot;   /* default 50 */
  float w_vel;        /* default 1 */
  float w_acc;        /* default 1 */
  float w_limit;      /* default 10 */
  float w_coll;       /* default 10 */
  float eta;          /* collision margin, metres (default 0.02) */
  float lambda0, lambda_min, lambda_max, nu; /* as pk_ik_params */
  float tol_pos, tol_rot; /* goal success thresholds (1 mm, 0.5 deg) */
  int32_t iters;      /* LM iterations (default 50) */
  int32_t reserved;   /* must be 0 */
  /* extensions, off by default: velocity-limit hinge (Sec. III-C, dt = 1)
   * w_vlimit max(0, |q_t - q_{t-1}| - v_max) per joint, and swept-sphere
   * collision between t and t+1 (Sec. IV-A): w_swept f(d, eta) with d the
   * distance from each obstacle sphere to the capsule a link sphere sweeps */
  float w_vlimit;     /* default 0 */
  float v_max;        /* rad (or m) per timestep, default 0.1 */
  float w_swept;      /* default 0 */
  /* five-point stencils (Sec. III-C smoothness, dt = 1), off by default: for
   * t = 2..T-3 and every joint, acceleration
   * w_acc5 (-q_{t+2} + 16 q_{t+1} - 30 q_t + 16 q_{t-1} - q_{t-2}) / 12 and jerk
   * w_jerk (q_{t+2} - 2 q_{t+1} + 2 q_{t-1} - q_{t-2}) / 2.  Either one nonzero
   * widens the normal matrix to four block sub-diagonals. */
  float w_acc5;       /* default 0 */
  float w_jerk;       /* default 0 */
} pk_trajopt_params;

void pk_trajopt_params_default(pk_trajopt_params* p);

/*
 * pk_trajopt_solve -- batch of trajectories of one serial chain (6 or 7 movable
 * joints, the goal on the last frame).
 *   T                  3..64 timesteps
 *   d_q_start [batch][n], d_goal [batch][12], d_q_init [batch][T][n]
 *   spheres_per_link   1..4;  d_radii [n][spheres_per_link]
 *   n_obs 0..64;  d_obs [n_obs][4] centre, radius (shared by the batch)
 *   plane              host [4]: unit normal and offset h (distance n.c - h)
 *   d_q_out [batch][T][n], d_cost_out [batch] (1/2 sum r^2),
 *   d_status_out [batch]: PK_T_* bits (goal missed, any sphere penetrating)
 */
pk_status pk_trajopt_solve(const pk_robot* robot, const pk_trajopt_params* params, int32_t batch, int32_t T,
                           const float* d_q_start, const float* d_goal, const float* d_q_init,
                           int32_t spheres_per_link, const float* d_radii, int32_t n_obs, const float* d_obs,
                           const float* plane, float* d_q_out, float* d_cost_out, int32_t* d_status_out,
                           void* stream);

/*
 * pk_ik_select_clear -- collision-free goal configurations by IK (Sec. IV-A:
 * the start and goal configurations of a trajectory are found by IK and must
 * be collision-free).  Runs after pk_ik_solve on the same workspace and
 * (batch, n_seeds), on the same stream, and re-chooses each target's answer
 * from that solve's per-seed results: among the converged seeds, the lowest
 * cost whose link spheres clear every obstacle sphere and the plane by
 * `margin` (sphere model and plane rule of pk_trajopt_solve); if none is
 * clear, the lowest-cost converged seed; if none converged, the lowest cost.
 * Ties go to the lower seed index.  Run the solve with cancel_siblings = 0 so
 * that every seed runs to its end (a cancelled seed is not a candidate).
 *   robot              serial chain with 6 or 7 movable joints
 *   d_workspace        the workspace the preceding pk_ik_solve used
 *   spheres_per_link   1..4;  d_radii [n][spheres_per_link]
 *   n_obs 0..64;  d_obs [n_obs][4] centre, radius (16-byte aligned)
 *   plane              host [4]: unit normal and offset h
 *   margin             metres (the clearance a sphere must keep)
 *   outputs as pk_ik_solve: d_q_out [batch][n], d_err_out [batch][2],
 *   d_iters_out [batch], d_status_out [batch] (caller-owned device buffers).
 * Argument errors return synchronously with nothing enqueued.
 */
pk_status pk_ik_select_clear(const pk_robot* robot, int32_t batch, int32_t n_seeds, const void* d_workspace,
                             int32_t spheres_per_link, const float* d_radii, int32_t n_obs, const float* d_obs,
                             const float* plane, float margin, float* d_q_out, float* d_err_out,
                             int32_t* d_iters_out, int32_t* d_status_out, void* stream);

/*
 * pk_trajopt_interpolate -- the initial trajectory of Sec. IV-A: start and
 * goal configurations (the goal found by IK) joined by linear interpolation
 * in joint space, q_t = (1 - s_t) q_start + s_t q_goal, s_t = t / (T - 1)
 * (s_0 = 0 when T = 1).
 *   d_q_start, d_q_goal [batch][n]; d_q_out [batch][T][n] (caller-owned
 *   device buffers).  batch >= 0, T >= 1, n >= 1, batch * T * n < 2^31;
 *   argument errors return PK_ERR_INVALID_ARG with nothing enqueued.
 */
pk_status pk_trajopt_interpolate(int32_t batch, int32_t T, int32_t n, const float* d_q_start,
                                 const float* d_q_goal, float* d_q_out, void* stream);

/*
 * pk_trajopt_normal -- the normal equations of the same problem at given
 * trajectories d_q [batch][T][n]: full diagonal blocks of J^T J
 * d_D_out [batch][T][n][n] (smoothness included), the first sub-diagonal
 * blocks (t, t-1) d_E_out [batch][T][n][n] (NULL: not written; block 0 is
 * zero), J^T r d_g_out [batch][T][n] and the cost d_cost_out [batch].  The
 * blocks further from the diagonal come from the smoothness rows alone and are
 * scalar multiples of I: w_acc^2 I at offset 2 when w_acc5 = w_jerk = 0.
 */
pk_status pk_trajopt_normal(const pk_robot* robot, const pk_trajopt_params* params, int32_t batch, int32_t T,
                            const float* d_q_start, const float* d_goal, const float* d_q,
                            int32_t spheres_per_link, const float* d_radii, int32_t n_obs, const float* d_obs,
                            const float* plane, float* d_D_out, float* d_E_out, float* d_g_out, float* d_cost_out,
                            void* stream);

/*
 * Learned seeds.  The paper's solver starts from given seeds; a seed network
 * adds the learned-seed pattern around it: a SiLU MLP maps target poses to K
 * joint-space proposals that the LM solver (pk_ik_solve) refines.  It runs on
 * the BF16 tensor cores (tcgen05, FP32 accumulation) for inference and
 * training, with FP32 master weights and AdamW.
 *   Features of one target pose: its position then the first two columns of its
 *   rotation, [t0 t1 t2 r00 r10 r20 r01 r11 r21]; k targets give 9k inputs.
 *   Head: q = (lower + upper)/2 + (upper - lower)/2 * tanh(y) per joint.
 *   Loss per sample with label q*: min_k |q_k - q*|^2 + mu * mean_k |q_k - q*|^2.
 *   Training data: uniform random in-limit configurations (drawn on the device by
 *   a counter-based SplitMix64 generator keyed by seed and step) and the
 *   forward kinematics of the target frames.
 * A net is used by one stream at a time (it owns its activation buffers).
 */
typedef struct pk_seednet pk_seednet;

typedef struct {
  int32_t epochs;          /* default 8 */
  int32_t batch;           /* samples per step, >= 128 (default 8192) */
  int32_t steps_per_epoch; /* default 1220 (~10M samples per epoch) */
  float lr;                /* peak learning rate, cosine schedule (default 1e-3) */
  float weight_decay;      /* AdamW decoupled decay (default 1e-4) */
  float beta1, beta2, eps; /* AdamW moments (0.9, 0.999, 1e-8) */
  float mu;                /* weight of the mean term of the loss (default 0.01) */
  int32_t refine_every;    /* LM-refined labels: a pk_seednet_refine round after every
                              refine_every epochs but the last (0: off, default) */
  uint64_t seed;           /* training-data generator key (default 500) */
  int32_t refine_n;        /* targets per refinement round (default 65536) */
  int32_t refine_iters;    /* LM iterations of a round (default 20) */
  float pool_frac;         /* share of every batch drawn from the label pool once it
                              holds a round (0..1, default 0.5) */
  int32_t first_epoch;     /* a call runs epochs first_epoch .. last_epoch - 1 of the
                              `epochs`-long schedule (learning rate, refinement rounds):
                              stop with last_epoch, save, load, resume with first_epoch
                              (default 0) */
  int32_t last_epoch;      /* 0: epochs (default 0) */
} pk_train_params;

void pk_train_params_default(pk_train_params* p);

/* k target frames (target_links, host [k]), K proposals, `depth` hidden layers
 * of `width` (a multiple of 256) units; weights initialised from `seed`. */
pk_status pk_seednet_create(const pk_robot* robot, int32_t k, const int32_t* target_links, int32_t K,
                            int32_t width, int32_t depth, uint64_t seed, pk_seednet** out);
void pk_seednet_destroy(pk_seednet* net);

/* Parameter count and FP32 copies in the layout: per layer W [out][in] row-major
 * then b [out] (host buffers).  set_params also resets the AdamW state. */
int64_t pk_seednet_n_params(const pk_seednet* net);
pk_status pk_seednet_get_params(const pk_seednet* net, float* host_params, int64_t n);
pk_status pk_seednet_set_params(pk_seednet* net, const float* host_params, int64_t n);

/* Training checkpoint.  pk_seednet_save writes the network and its whole
 * training state to a file at `path` (host path, host byte order): a small
 * header with the network's shape, the FP32 parameters in the get_params
 * layout, the AdamW step count (also the training-data generator's counter),
 * the AdamW first and second moments, and the LM-refined label pool.
 * pk_seednet_load reads such a file into a network of the same shape and
 * restores all of it, so that pk_seednet_train continues (first_epoch) where
 * the saved run stopped; files of the earlier parameters-only format load
 * their parameters and reset the AdamW state, as set_params.  Synchronous.
 * PK_ERR_INVALID_ARG if the file cannot be opened, written or fully read, is
 * not such a file, or holds a network of another shape (the network is then
 * unchanged). */
pk_status pk_seednet_save(const pk_seednet* net, const char* path);
pk_status pk_seednet_load(pk_seednet* net, const char* path);

/* Pre-head outputs d_y_out [batch][K * n_dof] (FP32) for d_targets [batch][k][12]. */
pk_status pk_seednet_forward(pk_seednet* net, int32_t batch, const float* d_targets, float* d_y_out,
                             void* stream);

/* Seeds d_seeds_out [batch][K][n_dof] for d_targets [batch][k][12]: the layout
 * pk_ik_solve takes.  Widths 256 and 512 with K * n_dof <= 256 run as one
 * kernel (features, every layer and the head, activations kept on chip);
 * other shapes, or the environment variable PK_SEEDNET_FUSED=0, use the
 * layer-by-layer GEMMs.  Both give the same seeds.  PK_MLP_STAGES (2..3) and
 * PK_MLP_GRID (CTAs) cap the fused kernel's weight ring and grid, for tuning. */
pk_status pk_seednet_infer(pk_seednet* net, int32_t batch, const float* d_targets, float* d_seeds_out,
                           void* stream);

/* Synchronises `stream` and reports a device-side failure recorded by earlier
 * asynchronous calls on this network (pk_seednet_infer, pk_seednet_forward):
 * a tensor-core pipeline wait that ran out its bound returns PK_ERR_TIMEOUT
 * (the record is cleared).  PK_OK otherwise. */
pk_status pk_seednet_check(pk_seednet* net, void* stream);

/* Mean loss and gradient (host, parameter layout above) of one batch with
 * labels d_qstar [batch][n_dof], mu = 0.01.  Synchronous. */
pk_status pk_seednet_loss_grad(pk_seednet* net, int32_t batch, const float* d_targets,
                               const float* d_qstar, float* host_loss, float* host_grad, void* stream);

/* One AdamW step on one given batch at learning rate lr.  Synchronous. */
pk_status pk_seednet_train_step(pk_seednet* net, const pk_train_params* params, int32_t batch,
                                const float* d_targets, const float* d_qstar, float lr, void* stream);

/* Full training run on generated data; host_loss [epochs] (or NULL) receives the
 * mean loss of every epoch.  Synchronous.  PK_ERR_TIMEOUT if a tensor-core
 * pipeline wait expired (the kernels bound every wait). */
pk_status pk_seednet_train(pk_seednet* net, const pk_train_params* params, float* host_loss, void* stream);

/*
 * One LM refinement round of the label pool: n fresh targets (forward
 * kinematics of uniform in-limit configurations, a generator keyed by `seed`
 * and the round), K proposals each from the network, pk_ik_solve from them
 * (max_iters, early exit, sibling cancellation), and the pool becomes those n
 * targets with the LM solution as label where it converged, the drawn
 * configuration elsewhere.  Training then draws pool_frac of every batch from
 * the pool.  The robot handle given to pk_seednet_create must still exist.
 * Synchronous; *n_converged (optional) receives the converged count.
 */
pk_status pk_seednet_refine(pk_seednet* net, int32_t n, int32_t max_iters, uint64_t seed, int32_t* n_converged,
                            void* stream);
/* Copy the pool: d_targets_out [n][k][12], d_labels_out [n][n_dof], with n (host)
 * = its size (0 before the first round; nothing is copied then).  Both buffers
 * NULL: only the size is returned. */
pk_status pk_seednet_pool(const pk_seednet* net, float* d_targets_out, float* d_labels_out, int32_t* n_out,
                          void* stream);

/*
 * Index checks.  The paper has no counterpart: these serve testing.  The
 * library built with -DPK_DEBUG_BOUNDS (libpk_debug.so, from
 * paper_2505_03728_gb300/build.py with debug_bounds=True) checks the indices
 * its kernels derive from run-time data (queue claims and resumed records,
 * tree joint, parent and target lists, kept and chosen seeds, obstacle
 * indices) and skips an access whose index is out of range, recording the
 * first such failure; nothing traps.  The default build compiles the checks
 * out.
 *
 * pk_debug_bounds_enabled: 1 in the checked build, 0 otherwise.
 * pk_debug_bounds_take: synchronizes the device; *code receives the first
 *   failed check since the last call, (site << 48) | (bound << 24) | index
 *   (bound clipped to 2^24 - 1, index to 2^24 - 2, a negative index as
 *   2^24 - 1), 0 if none, and the record is cleared.  Sites: 1 chain queue
 *   record index, 2 chain queue target index, 3 tree record index, 4 tree
 *   joint, parent or variable index, 5 tree target link or variable joint,
 *   6 best-seed record,
 *   7 IK-Beam kept seed, 8 trajectory obstacle, 9 collision-free seed
 *   record, 15 the self-test.
 *   PK_ERR_UNSUPPORTED (and *code = 0) in the default build.
 * pk_debug_bounds_selftest: enqueues on `stream` one check that fails at site
 *   15 with index n against bound n, in a kernel that addresses nothing with
 *   it, so that the status path itself can be tested.  PK_ERR_UNSUPPORTED in
 *   the default build.
 */
int32_t pk_debug_bounds_enabled(void);
pk_status pk_debug_bounds_take(uint64_t* code);
pk_status pk_debug_bounds_selftest(int32_t n, void* stream);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* pk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PK_H */
