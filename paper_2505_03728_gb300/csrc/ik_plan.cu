// ik_plan.cu -- plans for uneven batches: several (robot, target set, seeds)
// problem sets solved either by one persistent launch (ik_multi_kernel) or by
// one specialised launch per set (serial, or on forked streams so that their
// tails overlap), replayed as a CUDA graph, with a schedule picked by an
// autotuner.
//
// A plan fixes its buffers at creation, so the whole solve (workspace reset,
// the LM kernels, one best-seed reduction per set) is captured once into a
// graph and every pk_ik_plan_run is a single cudaGraphLaunch.  The autotuner
// times the candidate schedules -- kernel variant, block size, chain sets on
// the thread-per-problem or the warp-per-problem path, and the set order
// (largest estimated work first, or as given) -- with CUDA events and keeps the
// fastest; results are cached per device and plan signature.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ik_tree.cuh"
#include "pk_internal.h"

struct PlanSet {
  const pk_robot* robot;
  int k;
  std::vector<int32_t> links, kinds;
  int batch, n_seeds;
  const float* targets;
  const float* seeds;
  float* q_out;
  float* err_out;
  int32_t* iters_out;
  int32_t* status_out;
  bool chain_ok;  // eligible for the thread-per-problem chain path
  bool pos_only;
  pk::ChainHost ch;
  pk::TreeInfo ti;
  size_t flags_off, rec_off;
  double cost;  // estimated work
};

struct PlanConfig {
  int block = 128;
  int chains_as_trees = 0;
  int given_order = 0;
  // 0: one persistent launch, registers unconstrained; 1: the same, capped for
  // 3 blocks per SM; 2: one specialised launch per set, serial; 3: the same on
  // forked streams.
  int variant = 0;
};
constexpr int kPlanVariants = 4;

struct pk_ik_plan {
  pk_ik_params params;
  std::vector<PlanSet> sets;
  void* mp = nullptr;  // MultiParams (host copy)
  void* d_ws = nullptr;
  size_t ws_bytes = 0, zero_bytes = 0;
  PlanConfig cfg;
  int grid = 0;
  bool chain_path = false;  // some set runs on the thread-per-problem chain path
  std::vector<int> order;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t side[pk::kMaxSegs] = {};  // forked streams of variant 3
  cudaEvent_t fork = nullptr, join[pk::kMaxSegs] = {};
  int device = 0;
  std::string signature;
  float tuned_ms = -1.f;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, PlanConfig> g_tune_cache;

pk_status pfail(pk_status s, const char* msg) { return pk::set_error(s, msg); }
pk_status pcuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PK_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return pfail(e == cudaErrorMemoryAllocation ? PK_ERR_OOM : PK_ERR_CUDA, buf);
}

bool chain_like(const pk_robot* rb, int k, const int32_t* links) {
  if (k != 1 || (rb->n_dof != 6 && rb->n_dof != 7) || rb->has_mimic) return false;
  for (int j = 0; j < rb->n_joints; ++j)
    if (rb->parent[j] != j - 1) return false;
  for (int j = links[0] + 1; j < rb->n_joints; ++j)
    if (rb->type[j] != PK_JOINT_FIXED) return false;
  return true;
}

pk::LmParams plan_lm(const pk_ik_params* p) {
  pk::LmParams l;
  l.w_pos = p->w_pos; l.w_rot = p->w_rot; l.w_limit = p->w_limit; l.w_rest = p->w_rest;
  l.lambda0 = p->lambda0; l.lambda_min = p->lambda_min; l.lambda_max = p->lambda_max; l.nu = p->nu;
  l.tol_pos = p->tol_pos; l.tol_rot = p->tol_rot;
  l.max_iters = p->max_iters; l.early_exit = p->early_exit != 0; l.cancel = p->cancel_siblings != 0;
  l.pos_only = 0;
  l.w_self = p->w_self;
  l.eta_self = p->eta_self;
  return l;
}

// Fill the kernel parameters for configuration cfg.
void configure(pk_ik_plan* pl, const PlanConfig& cfg) {
  pl->cfg = cfg;
  const int n = (int)pl->sets.size();
  pl->order.resize(n);
  for (int i = 0; i < n; ++i) pl->order[i] = i;
  if (!cfg.given_order)
    std::stable_sort(pl->order.begin(), pl->order.end(),
                     [&](int a, int b) { return pl->sets[a].cost > pl->sets[b].cost; });
  char* ws = (char*)pl->d_ws;
  int c6 = 0, c7 = 0, tr = 0;
  pl->chain_path = false;
  for (int s = 0; s < n; ++s) {
    const PlanSet& ps = pl->sets[pl->order[s]];
    pk::MultiSeg g{};
    const bool chain = ps.chain_ok && !cfg.chains_as_trees;
    g.kind = chain ? 0 : 1;
    g.n = ps.robot->n_dof;
    g.pos_only = ps.pos_only;
    g.batch = ps.batch;
    g.n_seeds = ps.n_seeds;
    g.P = ps.batch * ps.n_seeds;
    g.targets = ps.targets;
    g.seeds = ps.seeds;
    g.head = (int32_t*)(ws + 64 + 4 * pl->order[s]);
    g.flags = (int32_t*)(ws + ps.flags_off);
    g.rec = (float*)(ws + ps.rec_off);
    g.rb = (const pk::RobotDev*)ps.robot->d_blob;
    if (chain) {
      pl->chain_path = true;
      g.slot = g.n == 6 ? c6++ : c7++;
      pk::ik_multi_set_chain(pl->mp, g.slot, ps.ch);
    } else {
      g.slot = tr++;
      pk::ik_multi_set_tree(pl->mp, g.slot, ps.ti);
    }
    pk::ik_multi_set_seg(pl->mp, s, g);
  }
  pk::ik_multi_set_common(pl->mp, n, plan_lm(&pl->params), (unsigned long long*)ws);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
  pl->grid = cfg.variant < 2
                 ? pk::ik_multi_max_blocks_per_sm(cfg.block, cfg.variant, pl->chain_path) * (sms > 0 ? sms : 1)
                 : 0;
  if (pl->exec) {
    cudaGraphExecDestroy(pl->exec);
    pl->exec = nullptr;
  }
  if (pl->graph) {
    cudaGraphDestroy(pl->graph);
    pl->graph = nullptr;
  }
}

// One specialised launch (LM kernel + best-seed reduction) for set i.
cudaError_t launch_set(pk_ik_plan* pl, int i, cudaStream_t st) {
  const PlanSet& ps = pl->sets[i];
  if (ps.batch == 0) return cudaSuccess;
  char* ws = (char*)pl->d_ws;
  pk::IkWorkspace w;
  w.stats = (unsigned long long*)ws;
  w.head = (int32_t*)(ws + 64 + 4 * i);
  w.flags = (int32_t*)(ws + ps.flags_off);
  w.rec = (float*)(ws + ps.rec_off);
  pk::LmParams lp = plan_lm(&pl->params);
  if (ps.chain_ok && !pl->cfg.chains_as_trees) {
    lp.pos_only = ps.pos_only;
    if (ps.pos_only) lp.tol_rot = INFINITY;
    return pk::launch_chain_lm(ps.ch, lp, ps.targets, ps.seeds, ps.batch, ps.n_seeds, w, ps.q_out, ps.err_out,
                               ps.iters_out, ps.status_out, st);
  }
  return pk::launch_tree_lm(ps.robot, ps.ti, lp, ps.targets, ps.seeds, ps.batch, ps.n_seeds, w, ps.q_out,
                            ps.err_out, ps.iters_out, ps.status_out, st);
}

cudaError_t ensure_side_streams(pk_ik_plan* pl) {
  if (pl->fork) return cudaSuccess;
  cudaError_t e = cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming);
  for (size_t i = 0; i < pl->sets.size() && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&pl->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->join[i], cudaEventDisableTiming);
  }
  return e;
}

cudaError_t enqueue(pk_ik_plan* pl, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(pl->d_ws, 0, pl->zero_bytes, st);
  if (e != cudaSuccess) return e;
  const int v = pl->cfg.variant;
  if (v == 2) {
    for (int i : pl->order)
      if ((e = launch_set(pl, i, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if (v == 3) {
    if ((e = ensure_side_streams(pl)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(pl->fork, st)) != cudaSuccess) return e;
    for (size_t s = 0; s < pl->order.size(); ++s) {
      cudaStream_t ss = pl->side[s];
      if ((e = cudaStreamWaitEvent(ss, pl->fork, 0)) != cudaSuccess) return e;
      if ((e = launch_set(pl, pl->order[s], ss)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(pl->join[s], ss)) != cudaSuccess) return e;
    }
    for (size_t s = 0; s < pl->order.size(); ++s)
      if ((e = cudaStreamWaitEvent(st, pl->join[s], 0)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  e = pk::launch_ik_multi(pl->mp, v, pl->chain_path, pl->cfg.block, pl->grid, st);
  if (e != cudaSuccess) return e;
  for (const PlanSet& ps : pl->sets) {
    if (ps.batch == 0) continue;
    e = pk::launch_ik_reduce((const float*)((char*)pl->d_ws + ps.rec_off), ps.robot->n_dof, ps.batch, ps.n_seeds,
                             ps.q_out, ps.err_out, ps.iters_out, ps.status_out, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

pk_status pk_ik_plan_create(const pk_ik_params* params, int32_t n_sets, const pk_ik_problem_set* sets,
                            pk_ik_plan** out) {
  if (!out) return pfail(PK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!params || !sets) return pfail(PK_ERR_INVALID_ARG, "params or sets is NULL");
  if (n_sets < 1 || n_sets > pk::kMaxSegs) return pfail(PK_ERR_INVALID_ARG, "n_sets must be in 1..8");
  if (!(params->nu > 1.f) || !(params->lambda0 > 0.f) || params->max_iters < 0 || params->reserved != 0)
    return pfail(PK_ERR_INVALID_ARG, "invalid LM parameters");
  pk_ik_plan* pl = new pk_ik_plan;
  pl->params = *params;
  cudaGetDevice(&pl->device);
  size_t off = 256;
  char sig[64];
  snprintf(sig, sizeof sig, "dev%d", pl->device);
  pl->signature = sig;
  for (int i = 0; i < n_sets; ++i) {
    const pk_ik_problem_set& s = sets[i];
    PlanSet ps{};
    ps.robot = s.robot;
    if (!s.robot || !s.target_links || s.k < 1 || s.k > pk::kTreeMaxTargets || s.batch < 0 || s.n_seeds < 1 ||
        (s.batch > 0 && (!s.d_targets || !s.d_seeds || !s.d_q_out || !s.d_err_out || !s.d_iters_out ||
                         !s.d_status_out))) {
      delete pl;
      return pfail(PK_ERR_INVALID_ARG, "malformed problem set");
    }
    for (int t = 0; t < s.k; ++t)
      if (s.target_links[t] < 0 || s.target_links[t] >= s.robot->n_joints ||
          (s.target_kinds && s.target_kinds[t] != PK_TARGET_POSE && s.target_kinds[t] != PK_TARGET_POSITION)) {
        delete pl;
        return pfail(PK_ERR_INVALID_ARG, "bad target link or kind");
      }
    if (((uintptr_t)s.d_targets & 15) != 0) {
      delete pl;
      return pfail(PK_ERR_INVALID_ARG, "d_targets must be 16-byte aligned");
    }
    ps.k = s.k;
    ps.links.assign(s.target_links, s.target_links + s.k);
    ps.kinds.assign(s.k, PK_TARGET_POSE);
    if (s.target_kinds) ps.kinds.assign(s.target_kinds, s.target_kinds + s.k);
    ps.batch = s.batch;
    ps.n_seeds = s.n_seeds;
    ps.targets = s.d_targets;
    ps.seeds = s.d_seeds;
    ps.q_out = s.d_q_out;
    ps.err_out = s.d_err_out;
    ps.iters_out = s.d_iters_out;
    ps.status_out = s.d_status_out;
    ps.chain_ok = chain_like(s.robot, s.k, s.target_links) && !(params->w_self > 0.f && s.robot->n_pairs > 0);
    ps.pos_only = ps.chain_ok && ps.kinds[0] == PK_TARGET_POSITION;
    if (ps.chain_ok) ps.chain_ok = pk::fold_chain_quiet(s.robot, s.target_links[0], &ps.ch);
    if (!pk::build_tree_info(s.robot, s.k, ps.links.data(), ps.kinds.data(), &ps.ti)) {
      delete pl;
      return pfail(PK_ERR_UNSUPPORTED, "robot too large for the warp-per-problem path");
    }
    const double n = s.robot->n_dof;
    ps.cost = (double)s.batch * s.n_seeds * n * n * (ps.chain_ok ? 1.0 : 32.0);
    ps.flags_off = off;
    off += (((size_t)s.batch * 4) + 255) & ~(size_t)255;
    pl->sets.push_back(ps);
    char part[96];
    const int bucket = s.batch > 0 ? (int)ceil(log2((double)s.batch)) : 0;
    snprintf(part, sizeof part, "|%d.%d.%d.%d.b%d.s%d", s.robot->n_joints, s.robot->n_dof, s.k,
             ps.chain_ok ? 1 : 0, bucket, s.n_seeds);
    pl->signature += part;
  }
  pl->zero_bytes = off;
  for (PlanSet& ps : pl->sets) {
    ps.rec_off = off;
    off += (((size_t)ps.batch * ps.n_seeds * pk::ik_rec_stride(ps.robot->n_dof) * 4) + 255) & ~(size_t)255;
  }
  pl->ws_bytes = off;
  cudaError_t e = cudaMalloc(&pl->d_ws, pl->ws_bytes);
  if (e != cudaSuccess) {
    delete pl;
    return pcuda(e, "pk_ik_plan_create");
  }
  pl->mp = pk::ik_multi_params_new();
  PlanConfig cfg;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(pl->signature);
    if (it != g_tune_cache.end()) cfg = it->second;
  }
  configure(pl, cfg);
  *out = pl;
  return PK_OK;
}

void pk_ik_plan_destroy(pk_ik_plan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->d_ws) cudaFree(pl->d_ws);
  if (pl->mp) pk::ik_multi_params_free(pl->mp);
  for (int i = 0; i < pk::kMaxSegs; ++i) {
    if (pl->side[i]) cudaStreamDestroy(pl->side[i]);
    if (pl->join[i]) cudaEventDestroy(pl->join[i]);
  }
  if (pl->fork) cudaEventDestroy(pl->fork);
  delete pl;
}

pk_status pk_ik_plan_run(pk_ik_plan* pl, void* stream) {
  if (!pl) return pfail(PK_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (!pl->exec) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return pcuda(e, "pk_ik_plan_run");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(pl, cs);
      e = cudaStreamEndCapture(cs, &pl->graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return pcuda(e, "pk_ik_plan_run (graph capture)");
  }
  return pcuda(cudaGraphLaunch(pl->exec, st), "pk_ik_plan_run");
}

pk_status pk_ik_plan_run_eager(pk_ik_plan* pl, void* stream) {
  if (!pl) return pfail(PK_ERR_INVALID_ARG, "plan is NULL");
  return pcuda(enqueue(pl, (cudaStream_t)stream), "pk_ik_plan_run_eager");
}

pk_status pk_ik_plan_autotune(pk_ik_plan* pl, int32_t reps, void* stream, float* best_ms) {
  if (!pl) return pfail(PK_ERR_INVALID_ARG, "plan is NULL");
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<PlanConfig> cands;
  bool any_chain = false;
  for (const PlanSet& ps : pl->sets) any_chain = any_chain || ps.chain_ok;
  for (int variant = 0; variant < kPlanVariants; ++variant)
    for (int block : {64, 128, 256}) {
      if (variant == 1 && block > 128) continue;
      if (variant >= 2 && block != 128) continue;  // the specialised kernels fix their own blocks
      for (int cat = 0; cat <= (any_chain ? 1 : 0); ++cat)
        for (int go = 0; go <= 1; ++go) cands.push_back(PlanConfig{block, cat, go, variant});
    }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = INFINITY;
  PlanConfig best_cfg = pl->cfg;
  cudaError_t e = cudaSuccess;
  for (const PlanConfig& c : cands) {
    configure(pl, c);
    e = enqueue(pl, st);  // warm-up
    if (e != cudaSuccess) break;
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue(pl, st);
    cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    ms /= reps;
    if (ms < best) {
      best = ms;
      best_cfg = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return pcuda(e, "pk_ik_plan_autotune");
  configure(pl, best_cfg);
  pl->tuned_ms = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[pl->signature] = best_cfg;
  }
  if (best_ms) *best_ms = best;
  return PK_OK;
}

pk_status pk_ik_plan_schedule(const pk_ik_plan* pl, int32_t* block, int32_t* grid, int32_t* chains_as_trees,
                              int32_t* given_order, int32_t* variant) {
  if (!pl) return pfail(PK_ERR_INVALID_ARG, "plan is NULL");
  if (variant) *variant = pl->cfg.variant;
  if (block) *block = pl->cfg.block;
  if (grid) *grid = pl->grid;
  if (chains_as_trees) *chains_as_trees = pl->cfg.chains_as_trees;
  if (given_order) *given_order = pl->cfg.given_order;
  return PK_OK;
}

pk_status pk_ik_plan_set_schedule(pk_ik_plan* pl, int32_t block, int32_t chains_as_trees, int32_t given_order,
                                  int32_t variant) {
  if (!pl) return pfail(PK_ERR_INVALID_ARG, "plan is NULL");
  if (block != 64 && block != 128 && block != 256) return pfail(PK_ERR_INVALID_ARG, "block must be 64, 128 or 256");
  if (variant < 0 || variant >= kPlanVariants) return pfail(PK_ERR_INVALID_ARG, "variant must be in 0..3");
  if (variant == 1 && block > 128) return pfail(PK_ERR_INVALID_ARG, "variant 1 takes blocks of at most 128");
  configure(pl, PlanConfig{block, chains_as_trees ? 1 : 0, given_order ? 1 : 0, variant});
  return PK_OK;
}

pk_status pk_ik_plan_stats(const pk_ik_plan* pl, int64_t* stats_out) {
  if (!pl || !stats_out) return pfail(PK_ERR_INVALID_ARG, "NULL argument");
  return pk_ik_workspace_stats(pl->d_ws, stats_out);
}

}  // extern "C"
