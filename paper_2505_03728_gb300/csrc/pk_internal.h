// pk_internal.h -- host-side types shared by the libpk translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pk.h"

struct pk_robot {
  int32_t n_joints = 0, n_dof = 0;
  std::vector<int32_t> parent, type, var;  // var[j]: variable index or -1
  std::vector<float> axis, origin, lower, upper;
  std::vector<int32_t> mimic;     // source joint of a mimic joint, else -1
  std::vector<float> mult, offs;  // joint value = mult * q[var] + offs
  bool has_mimic = false;
  std::vector<int32_t> sph_joint, pairs;  // self-collision spheres and pairs
  std::vector<float> sph;                 // [n_spheres][4]: centre, radius
  int n_spheres = 0, n_pairs = 0;
  // Device copy for the generic (tree) kernels, see RobotDev.
  void* d_blob = nullptr;
  int device = 0;
};

namespace pk {

constexpr int kMaxJoints = 64;
constexpr int kMaxSpheres = 64;
constexpr int kMaxPairs = 64;
constexpr int kMaxDevices = 64;
constexpr int kMaxChainDof = 8;

// Device-side robot layout (one contiguous allocation per robot handle).
struct RobotDev {
  int32_t n_joints, n_dof;
  int32_t parent[kMaxJoints];
  int32_t type[kMaxJoints];
  int32_t var[kMaxJoints];
  float axis[kMaxJoints][3];
  float origin[kMaxJoints][12];
  float lower[kMaxJoints], upper[kMaxJoints];
  float mult[kMaxJoints], offs[kMaxJoints];  // joint value = mult * q[var] + offs (mimic joints)
  int32_t own[kMaxJoints];                   // 1: the joint owns its variable (not a mimic)
  uint64_t subtree[kMaxJoints];              // bit l: joint l is joint j or one of its descendants
  int32_t n_spheres, n_pairs;                // self-collision model
  int32_t sph_joint[kMaxSpheres];
  float sph[kMaxSpheres][4];                 // centre in the joint frame, radius
  int32_t pair[kMaxPairs][2];
};

// Serial chain folded so that every fixed joint is merged into the next
// movable joint's origin and the fixed joints after the last movable joint
// form the tool transform.
struct ChainHost {
  int n;                      // movable joints
  float o_r[kMaxChainDof][9];  // origin rotations
  float o_t[kMaxChainDof][3];  // origin translations
  float a[kMaxChainDof][3];    // axes (unit)
  float tool_r[9], tool_t[3];
  float lo[kMaxChainDof], hi[kMaxChainDof];
  uint32_t prism, orot, toolrot;
};

// Device-ready LM settings.
struct LmParams {
  float w_pos, w_rot, w_limit, w_rest;
  float w_self = 0.f, eta_self = 0.02f;  // self-collision (tree path)
  float lambda0, lambda_min, lambda_max, nu;
  float tol_pos, tol_rot;
  int32_t max_iters, early_exit, cancel, pos_only;
  // Chain path only: per-problem initial damping (NULL: lambda0) and the
  // damping after the last iteration (NULL: not written), indexed like the
  // records; used to continue an LM run in a later launch (IK-Beam).
  const float* lam_in = nullptr;
  float* lam_out = nullptr;
  // Chain path only, two-launch solve.  suspend_at > 0: a problem still
  // running after that many iterations (not converged, not cancelled) writes
  // its record with status kStatusSuspended and its iteration count, its
  // damping to lam_sus[pid], and appends pid to resume_ids (*resume_n counts).
  // resume_in != NULL: the launch takes its problems from resume_in[0 ..
  // *resume_n) and continues each one from its record and lam_sus.
  int32_t suspend_at = 0;
  int32_t* resume_n = nullptr;
  int32_t* resume_ids = nullptr;
  const int32_t* resume_in = nullptr;
  float* lam_sus = nullptr;
};

// Record status of a problem suspended between the two launches of a split
// solve (never returned: the second launch rewrites every such record).
constexpr int kStatusSuspended = 15;

// Scratch layout of the IK solve.
struct IkWorkspace {
  unsigned long long* stats;  // [4] work counters, [4..8) the split solve's second launch (zeroed per call)
  int32_t* head;   // work-queue head (1 int, zeroed per call)
  int32_t* flags;  // [batch] converged-sibling flags (zeroed per call)
  float* rec;      // [batch * n_seeds][rec_stride] per-seed results
  // split solve only (ik_split_workspace_bytes): second queue head and the
  // suspended-problem count (zeroed per call), suspended problem indices and
  // their damping
  int32_t* head2 = nullptr;
  int32_t* resume_n = nullptr;
  int32_t* resume_ids = nullptr;
  float* lam_sus = nullptr;
};

size_t ik_workspace_bytes(int n_dof, long batch, long n_seeds);
void ik_workspace_carve(void* base, int n_dof, long batch, long n_seeds, IkWorkspace* ws,
                        size_t* zero_bytes);
size_t ik_split_workspace_bytes(int n_dof, long batch, long n_seeds);
void ik_split_workspace_carve(void* base, int n_dof, long batch, long n_seeds, IkWorkspace* ws,
                              size_t* zero_bytes);
int ik_rec_stride(int n_dof);

// Launchers (ik_chain.cu).  Return a cudaError_t from the launch.
// d_q == NULL: records only, no best-seed reduction.
cudaError_t launch_chain_lm(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                            const float* d_seeds, int batch, int n_seeds, IkWorkspace ws,
                            float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                            cudaStream_t stream);
cudaError_t launch_ik_reduce(const float* rec, int n_dof, int batch, int n_seeds, float* d_q, float* d_err,
                             int32_t* d_iters, int32_t* d_status, cudaStream_t stream);
// Two-launch chain solve: every problem runs up to split_iters iterations on
// `stream`; the ones still running are finished on `tail` (tail_ctas blocks,
// 0: a full grid) after `ev`, recorded on `stream` behind the first launch,
// then the best-seed reduction runs on `tail`.
cudaError_t launch_chain_lm_split(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                  const float* d_seeds, int batch, int n_seeds, IkWorkspace ws, int split_iters,
                                  int tail_ctas, float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                                  cudaStream_t stream, cudaStream_t tail, cudaEvent_t ev);
struct TreeInfo;
bool build_tree_info(const pk_robot* rb, int k, const int32_t* links, const int32_t* kinds, TreeInfo* ti);
cudaError_t launch_tree_lm(const pk_robot* rb, const TreeInfo& ti, const LmParams& lp, const float* d_targets,
                           const float* d_seeds, int batch, int n_seeds, IkWorkspace ws, float* d_q, float* d_err,
                           int32_t* d_iters, int32_t* d_status, cudaStream_t stream);
cudaError_t launch_chain_residual(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                  const float* d_q, int batch, float* d_r, float* d_J,
                                  cudaStream_t stream);
cudaError_t launch_fk(const RobotDev* d_robot, int n_joints, int n_dof, int batch, const float* d_q,
                      float* d_T, cudaStream_t stream);

// IK-Beam (ik_beam.cu): byte offsets of the two rounds' scratch in one buffer.
struct BeamWorkspace {
  size_t bytes1, ws1_off, lam1_off, ws2_off, seeds2_off, lam2_off, it1_off, kept_off, total;
  char* base;
};
void beam_layout(int n_dof, long batch, int S1, int keep, BeamWorkspace* w, char* base);
cudaError_t launch_beam(const ChainHost& ch, const LmParams& lp, int steps1, int steps2, const float* d_targets,
                        const float* d_seeds, int batch, int S1, int keep, const BeamWorkspace& w,
                        int32_t* d_kept_out, float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                        cudaStream_t st);

// Uneven multi-robot batches in one persistent launch (ik_chain.cu, ik_plan.cu).
constexpr int kMaxSegs = 8;

struct MultiSeg {
  int32_t kind;     // 0: chain (thread per problem), 1: tree (warp per problem)
  int32_t n;        // movable joints
  int32_t slot;     // constants slot (chain n-specific array or tree array)
  int32_t pos_only;
  int32_t batch, n_seeds, P;
  const float* targets;
  const float* seeds;
  int32_t* head;
  int32_t* flags;
  float* rec;
  const RobotDev* rb;
};

// chains: some segment runs on the thread-per-problem chain path (false
// selects the instantiation without it)
cudaError_t launch_ik_multi(const void* host_params, int variant, bool chains, int block, int grid,
                            cudaStream_t st);
size_t ik_multi_params_size();
void* ik_multi_params_new();
void ik_multi_params_free(void* p);
// Fill slot `slot` of the chain (n = 6, 7) or tree constants and segment `s`.
bool ik_multi_set_chain(void* p, int slot, const ChainHost& ch);
void ik_multi_set_tree(void* p, int slot, const struct TreeInfo& ti);
void ik_multi_set_seg(void* p, int s, const MultiSeg& seg);
void ik_multi_set_common(void* p, int n_segs, const LmParams& lp, unsigned long long* stats);
int ik_multi_max_blocks_per_sm(int block, int variant, bool chains);  // sets the smem attribute; 0 = not launchable

// Trajectory optimisation (trajopt.cu).
constexpr int kTrajMaxT = 64;
constexpr int kTrajMaxObs = 64;
constexpr int kTrajMaxS = 4;

struct TrajParamsDev {
  float w_start, w_goal_pos, w_goal_rot, w_vel, w_acc, w_limit, w_coll, eta;
  float lambda0, lambda_min, lambda_max, nu, tol_pos, tol_rot;
  int32_t iters, T, S, n_obs;
  float plane[4];
  float w_vlimit, v_max, w_swept, w_acc5, w_jerk;
};

cudaError_t launch_trajopt(const ChainHost& ch, const TrajParamsDev& tp, int batch, const float* q_start,
                           const float* goals, const float* q_init, const float* radii, const float* obs,
                           float* q_out, float* cost_out, int32_t* status_out, float* D_out, float* E_out,
                           float* g_out, cudaStream_t st);

// Linear interpolation of trajectories [batch][T][n] between q_start and
// q_goal [batch][n] (trajopt.cu).
cudaError_t launch_interpolate(int batch, int T, int n, const float* q_start, const float* q_goal, float* q_out,
                               cudaStream_t st);

// Best seed per target preferring converged seeds whose link spheres clear a
// scene by `margin` (trajopt.cu); rec: the per-seed records of a chain solve.
cudaError_t launch_select_clear(const ChainHost& ch, const float* rec, int batch, int n_seeds, int S,
                                const float* radii, int n_obs, const float* obs, const float* plane, float margin,
                                float* q_out, float* err_out, int32_t* iters_out, int32_t* status_out,
                                cudaStream_t st);

// Folds a serial chain ending at frame `link` (false if it is not one).
bool fold_chain_quiet(const pk_robot* rb, int link, ChainHost* ch);

// Records a thread-local error message (pk_last_error) and returns s.
pk_status set_error(pk_status s, const char* msg);

// The argument checks of pk_ik_solve (everything but the workspace); *empty
// is set when batch == 0 (nothing to do).
pk_status ik_check_args(const pk_robot* rb, const pk_ik_params* params, int32_t k, const int32_t* target_links,
                        const int32_t* target_kinds, int32_t batch, int32_t n_seeds, const float* d_targets,
                        const float* d_seeds, float* d_q_out, float* d_err_out, int32_t* d_iters_out,
                        int32_t* d_status_out, bool* empty);

// Kernel timing trace (pk_api.cu): brackets a launch with events when enabled.
struct TraceScope {
  TraceScope(const char* name, cudaStream_t s);
  ~TraceScope();
  void* slot;
  cudaStream_t stream;
};


// ---------------------------------------------------------------------------
// Index checks (PK_DEBUG_BOUNDS builds).  PK_IN_BOUNDS(i, n, site) is true
// when 0 <= i < n.  In a build compiled with -DPK_DEBUG_BOUNDS a failed check
// also records the first failure since the last read as
//   (site << 48) | (min(n, 2^24 - 1) << 24) | min(i, 2^24 - 2)   (i < 0: 2^24 - 1)
// in a status word, and the caller skips the access that the index was for;
// nothing traps.  Without device-code linking every translation unit has its
// own word, so each registers a reader that pk_debug_bounds_take() calls.  In
// other builds the macro is the constant `true`.
using BoundsReader = unsigned long long (*)();
bool bounds_register(BoundsReader reader);
unsigned long long bounds_take_all();

// Check sites (the `site` field of a recorded failure).
enum BoundsSite : int {
  kSiteChainClaimPid = 1,    // chain queue: record index of a claimed or resumed problem
  kSiteChainClaimTgt = 2,    // chain queue: target index
  kSiteTreeClaimPid = 3,     // tree kernel: record index of a claimed problem
  kSiteTreeParent = 4,       // tree FK: joint, parent or variable index
  kSiteTreeLink = 5,         // tree targets: target link / variable joint
  kSiteReduceRec = 6,        // best-seed selection: record index
  kSiteBeamKeep = 7,         // IK-Beam: kept seed index
  kSiteTrajSphere = 8,       // trajectory collisions: obstacle index of a screened pair
  kSiteSelectClear = 9,      // collision-free seed choice: record index
  kSiteSelfTest = 15,        // pk_debug_bounds_selftest
};

}  // namespace pk

#if defined(__CUDACC__) && defined(PK_DEBUG_BOUNDS)
static __device__ unsigned long long g_pk_bounds;
static unsigned long long pk_bounds_take_local() {
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_pk_bounds, sizeof(v)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_pk_bounds, &z, sizeof(z));
  return v;
}
static const bool pk_bounds_registered = pk::bounds_register(&pk_bounds_take_local);
namespace pk {
__device__ __forceinline__ bool in_bounds_check(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  const unsigned long long nb = n < 0 ? 0ull : (n > 0xffffffll ? 0xffffffull : (unsigned long long)n);
  const unsigned long long ib = i < 0 ? 0xffffffull : (i > 0xfffffell ? 0xfffffeull : (unsigned long long)i);
  atomicCAS(&g_pk_bounds, 0ull, ((unsigned long long)(site & 0x7fff) << 48) | (nb << 24) | ib);
  return false;
}
}  // namespace pk
#define PK_IN_BOUNDS(i, n, site) (::pk::in_bounds_check((long long)(i), (long long)(n), (site)))
#else
#define PK_IN_BOUNDS(i, n, site) true
#endif
