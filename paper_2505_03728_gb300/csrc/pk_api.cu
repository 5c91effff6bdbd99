// pk_api.cu -- the C ABI of libpk: argument checking, robot handles, scratch
// layout and kernel dispatch.  No C++ exception leaves this file.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include <cmath>

#include "pk_internal.h"
#include "ik_tree.cuh"

namespace {

thread_local std::string g_last_error;

pk_status fail(pk_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

pk_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? PK_ERR_OOM : PK_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

bool finite_all(const float* p, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(p[i])) return false;
  return true;
}

bool rotation_ok(const float* T) {
  // T is 3x4 row-major; check R^T R = I to 1e-4
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0;
      for (int i = 0; i < 3; ++i) s += (double)T[i * 4 + a] * T[i * 4 + b];
      if (fabs(s - (a == b ? 1.0 : 0.0)) > 1e-4) return false;
    }
  return true;
}

bool is_identity_rot(const float* r9) {
  for (int i = 0; i < 9; ++i)
    if (r9[i] != ((i % 4 == 0) ? 1.f : 0.f)) return false;
  return true;
}

// 3x4 row-major compose: C = A * B (double accumulation for the host folds).
void compose(const float* A, const float* B, float* C) {
  float o[12];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += (double)A[i * 4 + k] * B[k * 4 + j];
      o[i * 4 + j] = (float)s;
    }
    double t = A[i * 4 + 3];
    for (int k = 0; k < 3; ++k) t += (double)A[i * 4 + k] * B[k * 4 + 3];
    o[i * 4 + 3] = (float)t;
  }
  memcpy(C, o, sizeof o);
}

pk_status check_params(const pk_ik_params* p) {
  if (!p) return fail(PK_ERR_INVALID_ARG, "params is NULL");
  if (!(p->nu > 1.f) || !isfinite(p->nu)) return fail(PK_ERR_INVALID_ARG, "nu must be > 1");
  if (!(p->lambda0 > 0.f) || !(p->lambda_min > 0.f) || !(p->lambda_max >= p->lambda_min))
    return fail(PK_ERR_INVALID_ARG, "lambda0, lambda_min must be > 0 and lambda_max >= lambda_min");
  if (p->max_iters < 0) return fail(PK_ERR_INVALID_ARG, "max_iters must be >= 0");
  if (!(p->w_pos >= 0.f) || !(p->w_rot >= 0.f) || !(p->w_limit >= 0.f) || !(p->w_rest >= 0.f))
    return fail(PK_ERR_INVALID_ARG, "weights must be >= 0");
  if (!(p->tol_pos >= 0.f) || !(p->tol_rot >= 0.f))
    return fail(PK_ERR_INVALID_ARG, "tolerances must be >= 0");
  if (p->reserved != 0) return fail(PK_ERR_INVALID_ARG, "reserved must be 0");
  if (!(p->w_self >= 0.f) || !isfinite(p->w_self) || (p->w_self > 0.f && !(p->eta_self > 0.f)))
    return fail(PK_ERR_INVALID_ARG, "w_self must be >= 0 (and eta_self > 0 when it is used)");
  return PK_OK;
}

// The self-collision rows are in play (tree path only).
bool self_collision(const pk_robot* rb, const pk_ik_params* p) { return p->w_self > 0.f && rb->n_pairs > 0; }

pk::LmParams lm_params(const pk_ik_params* p, bool pos_only) {
  pk::LmParams l;
  l.w_pos = p->w_pos; l.w_rot = p->w_rot; l.w_limit = p->w_limit; l.w_rest = p->w_rest;
  l.lambda0 = p->lambda0; l.lambda_min = p->lambda_min; l.lambda_max = p->lambda_max; l.nu = p->nu;
  l.tol_pos = p->tol_pos; l.tol_rot = pos_only ? INFINITY : p->tol_rot;
  l.max_iters = p->max_iters; l.early_exit = p->early_exit != 0; l.cancel = p->cancel_siblings != 0;
  l.pos_only = pos_only;
  l.w_self = p->w_self;
  l.eta_self = p->eta_self;
  return l;
}

// Fold a serial chain ending at frame `link` into the kernel's canonical form.
pk_status fold_chain(const pk_robot* rb, int link, pk::ChainHost* ch) {
  if (rb->has_mimic) return fail(PK_ERR_UNSUPPORTED, "chains with mimic joints run on the tree path");
  for (int j = 0; j < rb->n_joints; ++j)
    if (rb->parent[j] != j - 1)
      return fail(PK_ERR_UNSUPPORTED, "the fused IK kernel needs a serial chain (parent[j] == j-1)");
  for (int j = link + 1; j < rb->n_joints; ++j)
    if (rb->type[j] != PK_JOINT_FIXED)
      return fail(PK_ERR_UNSUPPORTED, "the target must be on or after the last movable joint");
  if (rb->n_dof < 1 || rb->n_dof > pk::kMaxChainDof)
    return fail(PK_ERR_UNSUPPORTED, "serial-chain IK supports 1..%d movable joints (got %d)",
                pk::kMaxChainDof, rb->n_dof);
  memset(ch, 0, sizeof *ch);
  float pend[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  int v = 0;
  for (int j = 0; j <= link; ++j) {
    float o[12];
    compose(pend, &rb->origin[12 * j], o);
    if (rb->type[j] == PK_JOINT_FIXED) {
      memcpy(pend, o, sizeof o);
      continue;
    }
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) ch->o_r[v][r * 3 + c] = o[r * 4 + c];
      ch->o_t[v][r] = o[r * 4 + 3];
      ch->a[v][r] = rb->axis[3 * j + r];
    }
    if (!is_identity_rot(ch->o_r[v])) ch->orot |= 1u << v;
    if (rb->type[j] == PK_JOINT_PRISMATIC) ch->prism |= 1u << v;
    ch->lo[v] = rb->lower[j];
    ch->hi[v] = rb->upper[j];
    ++v;
    const float I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    memcpy(pend, I, sizeof I);
  }
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) ch->tool_r[r * 3 + c] = pend[r * 4 + c];
    ch->tool_t[r] = pend[r * 4 + 3];
  }
  ch->toolrot = is_identity_rot(ch->tool_r) ? 0u : 1u;
  ch->n = v;
  return PK_OK;
}

pk_status check_targets(const pk_robot* rb, int32_t k, const int32_t* links, const int32_t* kinds,
                        bool* pos_only) {
  if (k < 1) return fail(PK_ERR_INVALID_ARG, "k must be >= 1");
  if (!links) return fail(PK_ERR_INVALID_ARG, "target_links is NULL");
  for (int i = 0; i < k; ++i) {
    if (links[i] < 0 || links[i] >= rb->n_joints)
      return fail(PK_ERR_INVALID_ARG, "target_links[%d] = %d out of range", i, links[i]);
    if (kinds && kinds[i] != PK_TARGET_POSE && kinds[i] != PK_TARGET_POSITION)
      return fail(PK_ERR_INVALID_ARG, "target_kinds[%d] = %d invalid", i, kinds[i]);
  }
  *pos_only = kinds && kinds[0] == PK_TARGET_POSITION;
  return PK_OK;
}

// True when the thread-per-problem chain kernel serves this (robot, target).
bool chain_eligible(const pk_robot* rb, int32_t k, const int32_t* links) {
  if (k != 1 || rb->n_dof < 1 || rb->n_dof > pk::kMaxChainDof || rb->has_mimic) return false;
  for (int j = 0; j < rb->n_joints; ++j)
    if (rb->parent[j] != j - 1) return false;
  for (int j = links[0] + 1; j < rb->n_joints; ++j)
    if (rb->type[j] != PK_JOINT_FIXED) return false;
  return true;
}

}  // namespace

namespace pk {

pk_status set_error(pk_status s, const char* msg) { return fail(s, "%s", msg); }

bool fold_chain_quiet(const pk_robot* rb, int link, ChainHost* ch) {
  const std::string keep = g_last_error;
  const bool ok = fold_chain(rb, link, ch) == PK_OK;
  g_last_error = keep;
  return ok;
}

size_t ik_workspace_bytes(int n_dof, long batch, long n_seeds) {
  const size_t head = 256;
  const size_t flags = (((size_t)batch * 4) + 255) & ~(size_t)255;
  const size_t rec = (size_t)batch * n_seeds * ik_rec_stride(n_dof) * sizeof(float);
  return head + flags + ((rec + 255) & ~(size_t)255);
}

void ik_workspace_carve(void* base, int n_dof, long batch, long n_seeds, IkWorkspace* ws,
                        size_t* zero_bytes) {
  char* p = (char*)base;
  const size_t flags = (((size_t)batch * 4) + 255) & ~(size_t)255;
  ws->stats = (unsigned long long*)p;
  ws->head = (int32_t*)(p + 64);
  ws->flags = (int32_t*)(p + 256);
  ws->rec = (float*)(p + 256 + flags);
  *zero_bytes = 256 + flags;
  (void)n_dof;
  (void)n_seeds;
}

// The split solve's workspace: the plain one, then the suspended problems'
// indices and damping (one int and one float per problem); its second queue
// head and suspended count sit in the zeroed head area.
size_t ik_split_workspace_bytes(int n_dof, long batch, long n_seeds) {
  const size_t P = (size_t)batch * n_seeds;
  return ik_workspace_bytes(n_dof, batch, n_seeds) + 2 * (((P * 4) + 255) & ~(size_t)255);
}

void ik_split_workspace_carve(void* base, int n_dof, long batch, long n_seeds, IkWorkspace* ws,
                              size_t* zero_bytes) {
  ik_workspace_carve(base, n_dof, batch, n_seeds, ws, zero_bytes);
  char* p = (char*)base;
  const size_t P = (size_t)batch * n_seeds;
  const size_t ids = ik_workspace_bytes(n_dof, batch, n_seeds);
  ws->resume_n = (int32_t*)(p + 128);
  ws->head2 = (int32_t*)(p + 192);
  ws->resume_ids = (int32_t*)(p + ids);
  ws->lam_sus = (float*)(p + ids + (((P * 4) + 255) & ~(size_t)255));
}

// ---------------------------------------------------------------------------
// Kernel timing trace: a pool of event pairs, one per traced launch.

namespace {
struct TraceRec {
  std::string name;
  cudaEvent_t start, stop;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRec*> g_trace;  // recorded launches
std::vector<TraceRec*> g_trace_free;
}  // namespace

TraceScope::TraceScope(const char* name, cudaStream_t s) : slot(nullptr), stream(s) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_on) return;
  TraceRec* r = nullptr;
  if (!g_trace_free.empty()) {
    r = g_trace_free.back();
    g_trace_free.pop_back();
  } else {
    r = new (std::nothrow) TraceRec;
    if (!r) return;
    if (cudaEventCreate(&r->start) != cudaSuccess || cudaEventCreate(&r->stop) != cudaSuccess) {
      delete r;
      return;
    }
  }
  r->name = name;
  cudaEventRecord(r->start, s);
  slot = r;
}

TraceScope::~TraceScope() {
  if (!slot) return;
  TraceRec* r = (TraceRec*)slot;
  cudaEventRecord(r->stop, stream);
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace.push_back(r);
}

}  // namespace pk

namespace pk {

static std::vector<BoundsReader>& bounds_readers() {
  static std::vector<BoundsReader> readers;
  return readers;
}
// Called from each translation unit's static initialisation (library load).
bool bounds_register(BoundsReader reader) {
  bounds_readers().push_back(reader);
  return true;
}
// The first recorded failure over the translation units (each record cleared).
unsigned long long bounds_take_all() {
  unsigned long long first = 0;
  for (BoundsReader r : bounds_readers()) {
    const unsigned long long v = r();
    if (v && !first) first = v;
  }
  return first;
}

#ifdef PK_DEBUG_BOUNDS
// One check that fails (i = n against the bound n) so that the status path can
// be exercised; the index addresses nothing.
__global__ void bounds_selftest_kernel(int n) { (void)PK_IN_BOUNDS(n, n, kSiteSelfTest); }
#endif

}  // namespace pk

extern "C" {

pk_status pk_trace_enable(int32_t enable) {
  std::lock_guard<std::mutex> lk(pk::g_trace_mu);
  for (auto* r : pk::g_trace) pk::g_trace_free.push_back(r);
  pk::g_trace.clear();
  pk::g_trace_on = enable != 0;
  return PK_OK;
}

pk_status pk_trace_summary(const char* kernel, double* total_ms, int64_t* launches) {
  if (!kernel || !total_ms || !launches) return fail(PK_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(pk::g_trace_mu);
  double ms = 0;
  int64_t n = 0;
  for (auto* r : pk::g_trace) {
    if (r->name != kernel) continue;
    cudaError_t e = cudaEventSynchronize(r->stop);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r->start, r->stop);
    if (e != cudaSuccess) return cuda_fail(e, "pk_trace_summary");
    ms += t;
    ++n;
  }
  *total_ms = ms;
  *launches = n;
  return PK_OK;
}

int32_t pk_debug_bounds_enabled(void) {
#ifdef PK_DEBUG_BOUNDS
  return 1;
#else
  return 0;
#endif
}

pk_status pk_debug_bounds_take(uint64_t* code) {
  if (!code) return fail(PK_ERR_INVALID_ARG, "code is NULL");
  *code = 0;
#ifdef PK_DEBUG_BOUNDS
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "pk_debug_bounds_take");
  *code = pk::bounds_take_all();
  return PK_OK;
#else
  return fail(PK_ERR_UNSUPPORTED, "this library was built without PK_DEBUG_BOUNDS");
#endif
}

pk_status pk_debug_bounds_selftest(int32_t n, void* stream) {
#ifdef PK_DEBUG_BOUNDS
  if (n < 0) return fail(PK_ERR_INVALID_ARG, "n must be >= 0");
  pk::bounds_selftest_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_debug_bounds_selftest");
#else
  (void)n;
  (void)stream;
  return fail(PK_ERR_UNSUPPORTED, "this library was built without PK_DEBUG_BOUNDS");
#endif
}

void pk_trajopt_params_default(pk_trajopt_params* p) {
  if (!p) return;
  p->w_start = 100.f;
  p->w_goal_pos = 100.f;
  p->w_goal_rot = 50.f;
  p->w_vel = 1.f;
  p->w_acc = 1.f;
  p->w_limit = 10.f;
  p->w_coll = 10.f;
  p->eta = 0.02f;
  p->lambda0 = 1e-2f;
  p->lambda_min = 1e-10f;
  p->lambda_max = 1e10f;
  p->nu = 2.f;
  p->tol_pos = 1e-3f;
  p->tol_rot = 0.5f * 3.14159265358979f / 180.f;
  p->iters = 50;
  p->reserved = 0;
  p->w_vlimit = 0.f;
  p->v_max = 0.1f;
  p->w_swept = 0.f;
  p->w_acc5 = 0.f;
  p->w_jerk = 0.f;
}

static pk_status trajopt_common(const pk_robot* rb, const pk_trajopt_params* p, int32_t batch, int32_t T,
                                const float* d_q_start, const float* d_goal, const float* d_q,
                                int32_t S, const float* d_radii, int32_t n_obs, const float* d_obs,
                                const float* plane, float* d_q_out, float* d_cost_out, int32_t* d_status_out,
                                float* d_D_out, float* d_E_out, float* d_g_out, void* stream) {
  if (!rb || !p) return fail(PK_ERR_INVALID_ARG, "robot or params is NULL");
  if (!(p->nu > 1.f) || !(p->lambda0 > 0.f) || !(p->lambda_min > 0.f) || !(p->lambda_max >= p->lambda_min))
    return fail(PK_ERR_INVALID_ARG, "invalid damping parameters");
  if (p->iters < 0 || p->reserved != 0) return fail(PK_ERR_INVALID_ARG, "iters must be >= 0, reserved 0");
  if (!(p->eta > 0.f)) return fail(PK_ERR_INVALID_ARG, "eta must be > 0");
  if (!(p->w_vlimit >= 0.f) || !(p->v_max >= 0.f) || !(p->w_swept >= 0.f))
    return fail(PK_ERR_INVALID_ARG, "w_vlimit, v_max and w_swept must be >= 0");
  if (!(p->w_acc5 >= 0.f) || !(p->w_jerk >= 0.f)) return fail(PK_ERR_INVALID_ARG, "w_acc5 and w_jerk must be >= 0");
  if (T < 3 || T > pk::kTrajMaxT) return fail(PK_ERR_INVALID_ARG, "T must be in 3..%d", pk::kTrajMaxT);
  if (S < 1 || S > pk::kTrajMaxS) return fail(PK_ERR_INVALID_ARG, "spheres_per_link must be in 1..%d", pk::kTrajMaxS);
  if (n_obs < 0 || n_obs > pk::kTrajMaxObs) return fail(PK_ERR_INVALID_ARG, "n_obs must be in 0..%d", pk::kTrajMaxObs);
  if (!plane || !finite_all(plane, 4)) return fail(PK_ERR_INVALID_ARG, "plane must be 4 finite floats");
  if (batch < 0) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  pk::ChainHost ch;
  pk_status s = fold_chain(rb, rb->n_joints - 1, &ch);
  if (s != PK_OK) return s;
  if (ch.n != 6 && ch.n != 7) return fail(PK_ERR_UNSUPPORTED, "trajectory optimisation supports 6 or 7 movable joints");
  if (batch == 0) return PK_OK;
  if (!d_q_start || !d_goal || !d_q || !d_radii || (n_obs > 0 && !d_obs) || !d_cost_out)
    return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  pk::TrajParamsDev tp;
  tp.w_start = p->w_start; tp.w_goal_pos = p->w_goal_pos; tp.w_goal_rot = p->w_goal_rot;
  tp.w_vel = p->w_vel; tp.w_acc = p->w_acc; tp.w_limit = p->w_limit; tp.w_coll = p->w_coll; tp.eta = p->eta;
  tp.lambda0 = p->lambda0; tp.lambda_min = p->lambda_min; tp.lambda_max = p->lambda_max; tp.nu = p->nu;
  tp.tol_pos = p->tol_pos; tp.tol_rot = p->tol_rot;
  tp.iters = p->iters; tp.T = T; tp.S = S; tp.n_obs = n_obs;
  for (int i = 0; i < 4; ++i) tp.plane[i] = plane[i];
  tp.w_vlimit = p->w_vlimit; tp.v_max = p->v_max; tp.w_swept = p->w_swept;
  tp.w_acc5 = p->w_acc5; tp.w_jerk = p->w_jerk;
  cudaError_t e = pk::launch_trajopt(ch, tp, batch, d_q_start, d_goal, d_q, d_radii, d_obs, d_q_out, d_cost_out,
                                     d_status_out, d_D_out, d_E_out, d_g_out, (cudaStream_t)stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "trajectory optimisation launch");
}

pk_status pk_trajopt_solve(const pk_robot* rb, const pk_trajopt_params* p, int32_t batch, int32_t T,
                           const float* d_q_start, const float* d_goal, const float* d_q_init, int32_t S,
                           const float* d_radii, int32_t n_obs, const float* d_obs, const float* plane,
                           float* d_q_out, float* d_cost_out, int32_t* d_status_out, void* stream) {
  if (batch > 0 && (!d_q_out || !d_status_out)) return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  return trajopt_common(rb, p, batch, T, d_q_start, d_goal, d_q_init, S, d_radii, n_obs, d_obs, plane, d_q_out,
                        d_cost_out, d_status_out, nullptr, nullptr, nullptr, stream);
}

pk_status pk_ik_select_clear(const pk_robot* rb, int32_t batch, int32_t n_seeds, const void* d_workspace,
                             int32_t S, const float* d_radii, int32_t n_obs, const float* d_obs, const float* plane,
                             float margin, float* d_q_out, float* d_err_out, int32_t* d_iters_out,
                             int32_t* d_status_out, void* stream) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  if (batch < 0 || n_seeds < 1) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0 and n_seeds >= 1");
  if (S < 1 || S > pk::kTrajMaxS) return fail(PK_ERR_INVALID_ARG, "spheres_per_link must be in 1..%d", pk::kTrajMaxS);
  if (n_obs < 0 || n_obs > pk::kTrajMaxObs) return fail(PK_ERR_INVALID_ARG, "n_obs must be in 0..%d", pk::kTrajMaxObs);
  if (!plane || !finite_all(plane, 4) || !std::isfinite(margin))
    return fail(PK_ERR_INVALID_ARG, "plane must be 4 finite floats and margin finite");
  pk::ChainHost ch;
  pk_status s = fold_chain(rb, rb->n_joints - 1, &ch);
  if (s != PK_OK) return s;
  if (ch.n != 6 && ch.n != 7) return fail(PK_ERR_UNSUPPORTED, "clearance selection supports 6 or 7 movable joints");
  if (batch == 0) return PK_OK;
  if (!d_workspace || !d_radii || (n_obs > 0 && !d_obs) || !d_q_out || !d_err_out || !d_iters_out || !d_status_out)
    return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  if (((uintptr_t)d_obs & 15) != 0) return fail(PK_ERR_INVALID_ARG, "d_obs must be 16-byte aligned");
  pk::IkWorkspace ws;
  size_t zero_bytes = 0;
  pk::ik_workspace_carve(const_cast<void*>(d_workspace), rb->n_dof, batch, n_seeds, &ws, &zero_bytes);
  cudaError_t e = pk::launch_select_clear(ch, ws.rec, batch, n_seeds, S, d_radii, n_obs, d_obs, plane, margin, d_q_out,
                                          d_err_out, d_iters_out, d_status_out, (cudaStream_t)stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_ik_select_clear launch");
}

pk_status pk_trajopt_interpolate(int32_t batch, int32_t T, int32_t n, const float* d_q_start,
                                 const float* d_q_goal, float* d_q_out, void* stream) {
  if (batch < 0 || T < 1 || n < 1) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0, T and n >= 1");
  if ((long long)batch * T * n > 0x7fffffffLL) return fail(PK_ERR_INVALID_ARG, "batch * T * n exceeds 2^31");
  if (batch == 0) return PK_OK;
  if (!d_q_start || !d_q_goal || !d_q_out) return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  cudaError_t e = pk::launch_interpolate(batch, T, n, d_q_start, d_q_goal, d_q_out, (cudaStream_t)stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_trajopt_interpolate launch");
}

pk_status pk_trajopt_normal(const pk_robot* rb, const pk_trajopt_params* p, int32_t batch, int32_t T,
                            const float* d_q_start, const float* d_goal, const float* d_q, int32_t S,
                            const float* d_radii, int32_t n_obs, const float* d_obs, const float* plane,
                            float* d_D_out, float* d_E_out, float* d_g_out, float* d_cost_out, void* stream) {
  if (batch > 0 && (!d_D_out || !d_g_out)) return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  return trajopt_common(rb, p, batch, T, d_q_start, d_goal, d_q, S, d_radii, n_obs, d_obs, plane, nullptr,
                        d_cost_out, nullptr, d_D_out, d_E_out, d_g_out, stream);
}

pk_status pk_ik_workspace_stats(const void* d_workspace, int64_t* stats_out) {
  if (!d_workspace || !stats_out) return fail(PK_ERR_INVALID_ARG, "NULL argument");
  unsigned long long h[4];
  cudaError_t e = cudaMemcpy(h, d_workspace, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "pk_ik_workspace_stats");
  for (int i = 0; i < 4; ++i) stats_out[i] = (int64_t)h[i];
  return PK_OK;
}

pk_status pk_ik_split_workspace_stats(const void* d_workspace, int64_t* stats_out) {
  if (!d_workspace || !stats_out) return fail(PK_ERR_INVALID_ARG, "NULL argument");
  unsigned long long h[8];
  cudaError_t e = cudaMemcpy(h, d_workspace, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "pk_ik_split_workspace_stats");
  for (int i = 0; i < 8; ++i) stats_out[i] = (int64_t)h[i];
  return PK_OK;
}


void pk_ik_params_default(pk_ik_params* p) {
  if (!p) return;
  p->w_pos = 1.f;
  p->w_rot = 0.5f;
  p->w_limit = 10.f;
  p->w_rest = 1e-3f;
  p->lambda0 = 1e-2f;
  p->lambda_min = 1e-10f;
  p->lambda_max = 1e10f;
  p->nu = 2.f;
  p->tol_pos = 1e-3f;
  p->tol_rot = 0.5f * 3.14159265358979f / 180.f;
  p->max_iters = 50;
  p->early_exit = 1;
  p->cancel_siblings = 0;
  p->reserved = 0;
  p->w_self = 0.f;
  p->eta_self = 0.02f;
}

const char* pk_last_error(void) { return g_last_error.c_str(); }

// Device copy of the robot (RobotDev) from the host description.
static cudaError_t upload_robot(const pk_robot* rb) {
  pk::RobotDev h;
  memset(&h, 0, sizeof h);
  h.n_joints = rb->n_joints;
  h.n_dof = rb->n_dof;
  for (int j = 0; j < rb->n_joints; ++j) {
    h.parent[j] = rb->parent[j];
    h.type[j] = rb->type[j];
    h.var[j] = rb->var[j];
    memcpy(h.axis[j], &rb->axis[3 * j], 3 * sizeof(float));
    memcpy(h.origin[j], &rb->origin[12 * j], 12 * sizeof(float));
    h.lower[j] = rb->lower[j];
    h.upper[j] = rb->upper[j];
    h.mult[j] = rb->mult[j];
    h.offs[j] = rb->offs[j];
    h.own[j] = rb->type[j] != PK_JOINT_FIXED && rb->mimic[j] < 0;
  }
  for (int l = 0; l < rb->n_joints; ++l)  // l lies in the subtree of each of its ancestors
    for (int j = l; j >= 0; j = rb->parent[j]) h.subtree[j] |= 1ull << l;
  h.n_spheres = rb->n_spheres;
  h.n_pairs = rb->n_pairs;
  for (int i = 0; i < rb->n_spheres; ++i) {
    h.sph_joint[i] = rb->sph_joint[i];
    for (int c = 0; c < 4; ++c) h.sph[i][c] = rb->sph[4 * i + c];
  }
  for (int i = 0; i < rb->n_pairs; ++i) {
    h.pair[i][0] = rb->pairs[2 * i];
    h.pair[i][1] = rb->pairs[2 * i + 1];
  }
  return cudaMemcpy(rb->d_blob, &h, sizeof h, cudaMemcpyHostToDevice);
}

pk_status pk_robot_create(int32_t n_joints, const int32_t* parent, const int32_t* type,
                          const float* axis, const float* origin, const float* lower,
                          const float* upper, const float* tool, pk_robot** out) {
  if (!out) return fail(PK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  const int total = n_joints + (tool ? 1 : 0);
  if (n_joints < 1 || total > pk::kMaxJoints)
    return fail(PK_ERR_INVALID_ARG, "n_joints must be in 1..%d (including the tool)", pk::kMaxJoints);
  if (!parent || !type || !axis || !origin || !lower || !upper)
    return fail(PK_ERR_INVALID_ARG, "NULL robot array");
  pk_robot* rb = new (std::nothrow) pk_robot;
  if (!rb) return fail(PK_ERR_OOM, "host allocation failed");
  rb->n_joints = total;
  rb->parent.resize(total);
  rb->type.resize(total);
  rb->var.resize(total);
  rb->axis.resize(3 * total);
  rb->origin.resize(12 * total);
  rb->lower.resize(total);
  rb->upper.resize(total);
  int nd = 0;
  for (int j = 0; j < total; ++j) {
    const bool is_tool = j == n_joints;
    const int32_t pj = is_tool ? n_joints - 1 : parent[j];
    const int32_t tj = is_tool ? PK_JOINT_FIXED : type[j];
    const float* o = is_tool ? tool : origin + 12 * j;
    if (pj < -1 || pj >= j) {
      delete rb;
      return fail(PK_ERR_INVALID_ARG, "parent[%d] = %d must be in [-1, %d]", j, pj, j - 1);
    }
    if (tj != PK_JOINT_FIXED && tj != PK_JOINT_REVOLUTE && tj != PK_JOINT_PRISMATIC) {
      delete rb;
      return fail(PK_ERR_INVALID_ARG, "type[%d] = %d invalid", j, tj);
    }
    if (!finite_all(o, 12) || !rotation_ok(o)) {
      delete rb;
      return fail(PK_ERR_INVALID_ARG, "origin of joint %d is not a finite rigid transform", j);
    }
    rb->parent[j] = pj;
    rb->type[j] = tj;
    memcpy(&rb->origin[12 * j], o, 12 * sizeof(float));
    float a[3] = {0.f, 0.f, 1.f};
    float lo = 0.f, hi = 0.f;
    if (tj != PK_JOINT_FIXED) {
      if (!finite_all(axis + 3 * j, 3)) {
        delete rb;
        return fail(PK_ERR_INVALID_ARG, "axis of joint %d is not finite", j);
      }
      const double n = sqrt((double)axis[3 * j] * axis[3 * j] + (double)axis[3 * j + 1] * axis[3 * j + 1] +
                            (double)axis[3 * j + 2] * axis[3 * j + 2]);
      if (!(n > 1e-9)) {
        delete rb;
        return fail(PK_ERR_INVALID_ARG, "axis of movable joint %d is zero", j);
      }
      for (int i = 0; i < 3; ++i) a[i] = (float)(axis[3 * j + i] / n);
      lo = lower[j];
      hi = upper[j];
      if (!(lo <= hi) || !isfinite(lo) || !isfinite(hi)) {
        delete rb;
        return fail(PK_ERR_INVALID_ARG, "limits of joint %d invalid (need finite lower <= upper)", j);
      }
      rb->var[j] = nd++;
    } else {
      rb->var[j] = -1;
    }
    memcpy(&rb->axis[3 * j], a, sizeof a);
    rb->lower[j] = lo;
    rb->upper[j] = hi;
  }
  rb->n_dof = nd;
  rb->mimic.assign(total, -1);
  rb->mult.assign(total, 1.f);
  rb->offs.assign(total, 0.f);
  cudaGetDevice(&rb->device);
  cudaError_t e = cudaMalloc(&rb->d_blob, sizeof(pk::RobotDev));
  if (e != cudaSuccess) {
    delete rb;
    return cuda_fail(e, "cudaMalloc(robot)");
  }
  e = upload_robot(rb);
  if (e != cudaSuccess) {
    cudaFree(rb->d_blob);
    delete rb;
    return cuda_fail(e, "cudaMemcpy(robot)");
  }
  *out = rb;
  return PK_OK;
}

pk_status pk_robot_set_spheres(pk_robot* rb, int32_t n_spheres, const int32_t* joint, const float* centre,
                               const float* radius, int32_t n_pairs, const int32_t* pairs) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  if (n_spheres < 0 || n_spheres > pk::kMaxSpheres || n_pairs < 0 || n_pairs > pk::kMaxPairs)
    return fail(PK_ERR_INVALID_ARG, "need 0..%d spheres and 0..%d pairs", pk::kMaxSpheres, pk::kMaxPairs);
  if ((n_spheres > 0 && (!joint || !centre || !radius)) || (n_pairs > 0 && !pairs))
    return fail(PK_ERR_INVALID_ARG, "NULL sphere array");
  for (int i = 0; i < n_spheres; ++i)
    if (joint[i] < 0 || joint[i] >= rb->n_joints || !finite_all(centre + 3 * i, 3) || !(radius[i] >= 0.f) ||
        !isfinite(radius[i]))
      return fail(PK_ERR_INVALID_ARG, "sphere %d: bad joint, centre or radius", i);
  for (int i = 0; i < n_pairs; ++i)
    if (pairs[2 * i] < 0 || pairs[2 * i] >= n_spheres || pairs[2 * i + 1] < 0 || pairs[2 * i + 1] >= n_spheres ||
        pairs[2 * i] == pairs[2 * i + 1])
      return fail(PK_ERR_INVALID_ARG, "pair %d: sphere indices must be distinct and in range", i);
  rb->n_spheres = n_spheres;
  rb->n_pairs = n_pairs;
  rb->sph_joint.assign(joint, joint + n_spheres);
  rb->sph.resize(4 * (size_t)n_spheres);
  for (int i = 0; i < n_spheres; ++i) {
    for (int c = 0; c < 3; ++c) rb->sph[4 * i + c] = centre[3 * i + c];
    rb->sph[4 * i + 3] = radius[i];
  }
  rb->pairs.assign(pairs, pairs + 2 * (size_t)n_pairs);
  cudaError_t e = upload_robot(rb);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_robot_set_spheres");
}

pk_status pk_robot_set_mimic(pk_robot* rb, int32_t joint, int32_t source, float multiplier, float offset) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  if (joint < 0 || joint >= rb->n_joints || source < 0 || source >= rb->n_joints || joint == source)
    return fail(PK_ERR_INVALID_ARG, "joint and source must be distinct joints of the robot");
  if (rb->type[joint] == PK_JOINT_FIXED || rb->type[source] == PK_JOINT_FIXED)
    return fail(PK_ERR_INVALID_ARG, "mimic and source joints must be movable");
  if (rb->mimic[source] >= 0) return fail(PK_ERR_INVALID_ARG, "the source joint is itself a mimic joint");
  if (rb->mimic[joint] >= 0) return fail(PK_ERR_INVALID_ARG, "the joint is already a mimic joint");
  for (int j = 0; j < rb->n_joints; ++j)
    if (rb->mimic[j] == joint) return fail(PK_ERR_INVALID_ARG, "another joint mimics this joint");
  if (!isfinite(multiplier) || !isfinite(offset))
    return fail(PK_ERR_INVALID_ARG, "multiplier and offset must be finite");
  rb->mimic[joint] = source;
  rb->mult[joint] = multiplier;
  rb->offs[joint] = offset;
  rb->has_mimic = true;
  // renumber: variables belong to the movable joints that are not mimics
  int nd = 0;
  for (int j = 0; j < rb->n_joints; ++j)
    rb->var[j] = (rb->type[j] != PK_JOINT_FIXED && rb->mimic[j] < 0) ? nd++ : -1;
  for (int j = 0; j < rb->n_joints; ++j)
    if (rb->mimic[j] >= 0) rb->var[j] = rb->var[rb->mimic[j]];
  rb->n_dof = nd;
  cudaError_t e = upload_robot(rb);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_robot_set_mimic");
}

void pk_robot_destroy(pk_robot* rb) {
  if (!rb) return;
  if (rb->d_blob) cudaFree(rb->d_blob);
  delete rb;
}

int32_t pk_robot_n_joints(const pk_robot* rb) { return rb ? rb->n_joints : -1; }
int32_t pk_robot_n_dof(const pk_robot* rb) { return rb ? rb->n_dof : -1; }

pk_status pk_fk(const pk_robot* rb, int32_t batch, const float* d_q, float* d_T_out, void* stream) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  if (batch < 0) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  if (batch == 0) return PK_OK;
  if (!d_q || !d_T_out) return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  cudaError_t e = pk::launch_fk((const pk::RobotDev*)rb->d_blob, rb->n_joints, rb->n_dof, batch, d_q,
                                d_T_out, (cudaStream_t)stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_fk launch");
}

pk_status pk_ik_residual(const pk_robot* rb, const pk_ik_params* params, int32_t k,
                         const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                         const float* d_targets, const float* d_q, float* d_r_out, float* d_J_out,
                         void* stream) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  pk_status s = check_params(params);
  if (s != PK_OK) return s;
  bool pos_only = false;
  if ((s = check_targets(rb, k, target_links, target_kinds, &pos_only)) != PK_OK) return s;
  if (batch < 0) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  if (k != 1) return fail(PK_ERR_UNSUPPORTED, "pk_ik_residual takes one target (k = 1)");
  pk::ChainHost ch;
  if ((s = fold_chain(rb, target_links[0], &ch)) != PK_OK) return s;
  if (batch == 0) return PK_OK;
  if (!d_targets || !d_q || !d_r_out) return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  if (((uintptr_t)d_targets & 15) != 0) return fail(PK_ERR_INVALID_ARG, "d_targets must be 16-byte aligned");
  cudaError_t e = pk::launch_chain_residual(ch, lm_params(params, pos_only), d_targets, d_q, batch,
                                            d_r_out, d_J_out, (cudaStream_t)stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_ik_residual launch");
}

size_t pk_ik_workspace_bytes(const pk_robot* rb, int32_t batch, int32_t n_seeds) {
  if (!rb || batch < 0 || n_seeds < 1) return 0;
  return pk::ik_workspace_bytes(rb->n_dof, batch, n_seeds);
}

// Argument checks shared by the IK entry points; picks the chain or tree
// kernel.  *empty: batch == 0 (nothing to launch).
static pk_status ik_prepare(const pk_robot* rb, const pk_ik_params* params, int32_t k,
                            const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                            int32_t n_seeds, const float* d_targets, const float* d_seeds, float* d_q_out,
                            float* d_err_out, int32_t* d_iters_out, int32_t* d_status_out, bool* chain,
                            pk::ChainHost* ch, pk::TreeInfo* ti, bool* pos_only, bool* empty) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  pk_status s = check_params(params);
  if (s != PK_OK) return s;
  if ((s = check_targets(rb, k, target_links, target_kinds, pos_only)) != PK_OK) return s;
  if (batch < 0) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  if (n_seeds < 1) return fail(PK_ERR_INVALID_ARG, "n_seeds must be >= 1");
  if ((long long)batch * n_seeds > 0x7fffff00LL)
    return fail(PK_ERR_INVALID_ARG, "batch * n_seeds exceeds 2^31");
  *chain = chain_eligible(rb, k, target_links) && !self_collision(rb, params);
  if (*chain) {
    if ((s = fold_chain(rb, target_links[0], ch)) != PK_OK) return s;
  } else if (!pk::build_tree_info(rb, k, target_links, target_kinds, ti)) {
    return fail(PK_ERR_UNSUPPORTED, "IK supports up to %d movable joints, %d targets and %d joints",
                pk::kTreeMaxDof, pk::kTreeMaxTargets, pk::kMaxJoints);
  }
  *empty = batch == 0;
  if (*empty) return PK_OK;
  if (!d_targets || !d_seeds || !d_q_out || !d_err_out || !d_iters_out || !d_status_out)
    return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  if (((uintptr_t)d_targets & 15) != 0) return fail(PK_ERR_INVALID_ARG, "d_targets must be 16-byte aligned");
  return PK_OK;
}

}  // extern "C"

namespace pk {
pk_status ik_check_args(const pk_robot* rb, const pk_ik_params* params, int32_t k, const int32_t* target_links,
                        const int32_t* target_kinds, int32_t batch, int32_t n_seeds, const float* d_targets,
                        const float* d_seeds, float* d_q_out, float* d_err_out, int32_t* d_iters_out,
                        int32_t* d_status_out, bool* empty) {
  bool chain = false, pos_only = false;
  pk::ChainHost ch;
  pk::TreeInfo ti;
  return ik_prepare(rb, params, k, target_links, target_kinds, batch, n_seeds, d_targets, d_seeds, d_q_out,
                    d_err_out, d_iters_out, d_status_out, &chain, &ch, &ti, &pos_only, empty);
}
}  // namespace pk

extern "C" {

pk_status pk_ik_solve(const pk_robot* rb, const pk_ik_params* params, int32_t k,
                      const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                      int32_t n_seeds, const float* d_targets, const float* d_seeds,
                      float* d_q_out, float* d_err_out, int32_t* d_iters_out,
                      int32_t* d_status_out, void* d_workspace, size_t workspace_bytes,
                      void* stream) {
  bool chain = false, pos_only = false, empty = false;
  pk::ChainHost ch;
  pk::TreeInfo ti;
  pk_status s = ik_prepare(rb, params, k, target_links, target_kinds, batch, n_seeds, d_targets, d_seeds, d_q_out,
                           d_err_out, d_iters_out, d_status_out, &chain, &ch, &ti, &pos_only, &empty);
  if (s != PK_OK || empty) return s;
  const size_t need = pk::ik_workspace_bytes(rb->n_dof, batch, n_seeds);
  cudaStream_t st = (cudaStream_t)stream;
  void* ws_base = d_workspace;
  bool owned = false;
  if (ws_base) {
    if (workspace_bytes < need)
      return fail(PK_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    if (((uintptr_t)ws_base & 255) != 0) return fail(PK_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  } else {
    cudaError_t e = cudaMallocAsync(&ws_base, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(workspace)");
    owned = true;
  }
  pk::IkWorkspace ws;
  size_t zero_bytes = 0;
  pk::ik_workspace_carve(ws_base, rb->n_dof, batch, n_seeds, &ws, &zero_bytes);
  cudaError_t e = cudaMemsetAsync(ws_base, 0, zero_bytes, st);
  if (e == cudaSuccess) {
    if (chain) {
      e = pk::launch_chain_lm(ch, lm_params(params, pos_only), d_targets, d_seeds, batch, n_seeds, ws, d_q_out,
                              d_err_out, d_iters_out, d_status_out, st);
    } else {
      pk::LmParams lp = lm_params(params, false);
      lp.tol_rot = params->tol_rot;  // position targets report 0 rotation error
      e = pk::launch_tree_lm(rb, ti, lp, d_targets, d_seeds, batch, n_seeds, ws, d_q_out, d_err_out, d_iters_out,
                             d_status_out, st);
    }
  }
  if (owned) {
    cudaError_t e2 = cudaFreeAsync(ws_base, st);
    if (e == cudaSuccess) e = e2;
  }
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_ik_solve launch");
}

size_t pk_ik_split_workspace_bytes(const pk_robot* rb, int32_t batch, int32_t n_seeds) {
  if (!rb || batch < 0 || n_seeds < 1) return 0;
  return pk::ik_split_workspace_bytes(rb->n_dof, batch, n_seeds);
}

// One event per device and host thread orders the tail stream behind the
// first launch (recorded and waited on in the same call, so reuse is safe).
static cudaError_t split_event(cudaEvent_t* ev) {
  thread_local cudaEvent_t evs[pk::kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= pk::kMaxDevices) return cudaErrorInvalidDevice;
  if (!evs[dev] && (e = cudaEventCreateWithFlags(&evs[dev], cudaEventDisableTiming)) != cudaSuccess) return e;
  *ev = evs[dev];
  return cudaSuccess;
}

pk_status pk_ik_solve_split(const pk_robot* rb, const pk_ik_params* params, int32_t k,
                            const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                            int32_t n_seeds, const float* d_targets, const float* d_seeds, float* d_q_out,
                            float* d_err_out, int32_t* d_iters_out, int32_t* d_status_out, void* d_workspace,
                            size_t workspace_bytes, int32_t split_iters, int32_t tail_ctas, void* stream,
                            void* tail_stream) {
  bool chain = false, pos_only = false, empty = false;
  pk::ChainHost ch;
  pk::TreeInfo ti;
  pk_status s = ik_prepare(rb, params, k, target_links, target_kinds, batch, n_seeds, d_targets, d_seeds, d_q_out,
                           d_err_out, d_iters_out, d_status_out, &chain, &ch, &ti, &pos_only, &empty);
  if (s != PK_OK) return s;
  if (split_iters < 1) return fail(PK_ERR_INVALID_ARG, "split_iters must be >= 1");
  if (tail_ctas < 0) return fail(PK_ERR_INVALID_ARG, "tail_ctas must be >= 0");
  if (empty) return PK_OK;
  if (!d_workspace) return fail(PK_ERR_INVALID_ARG, "pk_ik_solve_split needs a caller workspace");
  const size_t need = pk::ik_split_workspace_bytes(rb->n_dof, batch, n_seeds);
  if (workspace_bytes < need)
    return fail(PK_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
  if (((uintptr_t)d_workspace & 255) != 0) return fail(PK_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream, tail = (cudaStream_t)tail_stream;
  cudaEvent_t ev = nullptr;
  cudaError_t e = split_event(&ev);
  if (e != cudaSuccess) return cuda_fail(e, "pk_ik_solve_split event");
  pk::IkWorkspace ws;
  size_t zero_bytes = 0;
  pk::ik_split_workspace_carve(d_workspace, rb->n_dof, batch, n_seeds, &ws, &zero_bytes);
  e = cudaMemsetAsync(d_workspace, 0, zero_bytes, st);
  if (e == cudaSuccess) {
    if (chain) {
      e = pk::launch_chain_lm_split(ch, lm_params(params, pos_only), d_targets, d_seeds, batch, n_seeds, ws,
                                    split_iters, tail_ctas, d_q_out, d_err_out, d_iters_out, d_status_out, st, tail,
                                    ev);
    } else {  // trees: one launch on `stream`, the tail stream waits for it
      pk::LmParams lp = lm_params(params, false);
      lp.tol_rot = params->tol_rot;
      e = pk::launch_tree_lm(rb, ti, lp, d_targets, d_seeds, batch, n_seeds, ws, d_q_out, d_err_out, d_iters_out,
                             d_status_out, st);
      if (e == cudaSuccess && tail != st) {
        e = cudaEventRecord(ev, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(tail, ev, 0);
      }
    }
  }
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_ik_solve_split launch");
}

void pk_ik_beam_params_default(pk_ik_beam_params* b) {
  if (!b) return;
  b->n_seeds = 64;
  b->steps1 = 6;
  b->keep = 4;
  b->steps2 = 10;
}

static bool beam_ok(const pk_ik_beam_params* b) {
  return b && b->keep >= 1 && b->keep <= 32 && b->n_seeds >= b->keep && b->n_seeds <= 1024 && b->steps1 >= 0 &&
         b->steps2 >= 0;
}

size_t pk_ik_beam_workspace_bytes(const pk_robot* rb, int32_t batch, const pk_ik_beam_params* beam) {
  if (!rb || batch < 0 || !beam_ok(beam)) return 0;
  pk::BeamWorkspace w;
  pk::beam_layout(rb->n_dof, batch, beam->n_seeds, beam->keep, &w, nullptr);
  return w.total;
}

pk_status pk_ik_beam_solve(const pk_robot* rb, const pk_ik_params* params, const pk_ik_beam_params* beam,
                           int32_t k, const int32_t* target_links, const int32_t* target_kinds, int32_t batch,
                           const float* d_targets, const float* d_seeds, float* d_q_out, float* d_err_out,
                           int32_t* d_iters_out, int32_t* d_status_out, int32_t* d_kept_out, void* d_workspace,
                           size_t workspace_bytes, void* stream) {
  if (!rb) return fail(PK_ERR_INVALID_ARG, "robot is NULL");
  pk_status s = check_params(params);
  if (s != PK_OK) return s;
  if (!beam_ok(beam))
    return fail(PK_ERR_INVALID_ARG, "beam: need 1 <= keep <= 32, keep <= n_seeds <= 1024, steps >= 0");
  bool pos_only = false;
  if ((s = check_targets(rb, k, target_links, target_kinds, &pos_only)) != PK_OK) return s;
  if (!chain_eligible(rb, k, target_links) || self_collision(rb, params))
    return fail(PK_ERR_UNSUPPORTED, "IK-Beam runs on serial chains with one target and no self-collision rows");
  pk::ChainHost ch;
  if ((s = fold_chain(rb, target_links[0], &ch)) != PK_OK) return s;
  if (batch < 0) return fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  if ((long long)batch * beam->n_seeds > 0x7fffff00LL)
    return fail(PK_ERR_INVALID_ARG, "batch * n_seeds exceeds 2^31");
  if (batch == 0) return PK_OK;
  if (!d_targets || !d_seeds || !d_q_out || !d_err_out || !d_iters_out || !d_status_out)
    return fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  if (((uintptr_t)d_targets & 15) != 0) return fail(PK_ERR_INVALID_ARG, "d_targets must be 16-byte aligned");
  pk::BeamWorkspace w;
  pk::beam_layout(rb->n_dof, batch, beam->n_seeds, beam->keep, &w, nullptr);
  cudaStream_t st = (cudaStream_t)stream;
  void* ws_base = d_workspace;
  bool owned = false;
  if (ws_base) {
    if (workspace_bytes < w.total)
      return fail(PK_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, w.total);
    if (((uintptr_t)ws_base & 255) != 0) return fail(PK_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  } else {
    cudaError_t e = cudaMallocAsync(&ws_base, w.total, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(workspace)");
    owned = true;
  }
  w.base = (char*)ws_base;
  cudaError_t e = pk::launch_beam(ch, lm_params(params, pos_only), beam->steps1, beam->steps2, d_targets, d_seeds,
                                  batch, beam->n_seeds, beam->keep, w, d_kept_out, d_q_out, d_err_out, d_iters_out,
                                  d_status_out, st);
  if (owned) {
    cudaError_t e2 = cudaFreeAsync(ws_base, st);
    if (e == cudaSuccess) e = e2;
  }
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "pk_ik_beam_solve launch");
}

}  // extern "C"
