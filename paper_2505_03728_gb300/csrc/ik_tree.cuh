// ik_tree.cuh -- Levenberg-Marquardt IK for kinematic trees with several
// targets: one warp per (target set, seed) problem, lane i owning variable i.
//
// Per iteration (Sec. III-A, Sec. III-C): level-parallel FK over the tree
// (lanes take the joints of one depth level), per-target residuals on the
// target lanes (pose: log(T_target^-1 T_link) with the inverse left-Jacobian
// blocks; position: world-frame difference), joint-limit and rest rows on the
// variable lanes, warp-reduced cost and errors; accept/reject; on acceptance
// the Jacobian is formed one target at a time (lane i writes column i of the
// target's rows into shared memory) and lane i accumulates row i of J^T J and
// entry i of J^T r in registers; the damped system is factored by a
// right-looking Cholesky with the factor in shared memory (lane i updates row
// i) and solved by forward and backward substitution.
#pragma once
#include "pk_internal.h"
#include "pk_math.cuh"

namespace pk {

constexpr int kTreeMaxDof = 32;
constexpr int kTreeMaxTargets = 8;
constexpr int kTreeMaxMimic = 4;  // mimic joints per variable
constexpr unsigned kTreeFull = 0xffffffffu;

// Per-robot, per-target-set constants (global memory, built on the host).
struct TreeInfo {
  int32_t n_joints, n_dof, k;
  int32_t n_levels;
  int32_t level_start[kMaxJoints + 1];  // joints of depth level l: order[level_start[l] .. level_start[l+1])
  int32_t order[kMaxJoints];
  int32_t dof_joint[kTreeMaxDof];   // joint index of variable i
  uint32_t dof_targets[kTreeMaxDof];  // bit t: variable i moves target t's frame (any of its joints)
  uint32_t own_targets[kTreeMaxDof];  // bit t: variable i's own joint moves target t
  // mimic joints following variable i (Sec. III-B): joint, multiplier, targets moved
  int32_t n_mim[kTreeMaxDof];
  int32_t mim_joint[kTreeMaxDof][kTreeMaxMimic];
  float mim_mult[kTreeMaxDof][kTreeMaxMimic];
  uint32_t mim_targets[kTreeMaxDof][kTreeMaxMimic];
  int32_t links[kTreeMaxTargets];
  int32_t kinds[kTreeMaxTargets];
  float lo[kTreeMaxDof], hi[kTreeMaxDof];
};

// The per-variable and per-target fields of TreeInfo that one lane reads,
// loaded into registers once: indexed by lane in the parameter (constant)
// space, the lanes' distinct addresses would be served one after another at
// every use.
struct TreeLane {
  int32_t dof_joint = 0, n_mim = 0, link = 0, kind = 0;
  uint32_t dof_targets = 0u, own_targets = 0u;
  float lo = 0.f, hi = 0.f;
};
__device__ __forceinline__ TreeLane tree_lane(const TreeInfo& ti, int lane) {
  TreeLane t;
  if (lane < ti.n_dof) {
    t.dof_joint = ti.dof_joint[lane];
    t.n_mim = ti.n_mim[lane];
    t.dof_targets = ti.dof_targets[lane];
    t.own_targets = ti.own_targets[lane];
    t.lo = ti.lo[lane];
    t.hi = ti.hi[lane];
  }
  if (lane < ti.k) {
    t.link = ti.links[lane];
    t.kind = ti.kinds[lane];
  }
  return t;
}

// Shared memory of one warp.
struct TreeWarpSmem {
  float frames[kMaxJoints][12];
  float Jk[6][kTreeMaxDof];       // rows of the current target
  float Ti[kTreeMaxTargets][12];  // target inverses (pose) or -p (position)
  float xi[kTreeMaxTargets][6];   // unweighted residuals of the candidate
  float th[kTreeMaxTargets];
  float q[kTreeMaxDof];           // configuration being evaluated
  float L[kTreeMaxDof][kTreeMaxDof + 1];  // Cholesky factor, row i by lane i (padded rows)
  // self-collision pairs of the candidate: residual w f(d), slope w f'(d),
  // unit direction c_a - c_b and the two sphere centres (world)
  float pr[kMaxPairs], ps[kMaxPairs];
  float pn[kMaxPairs][3], pca[kMaxPairs][3], pcb[kMaxPairs][3];
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kTreeFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kTreeFull, v, o));
  return v;
}

// FK of sm.q into sm.frames, level by level.
__device__ __forceinline__ void tree_fk(const RobotDev* __restrict__ rb, const TreeInfo& ti, TreeWarpSmem& sm,
                                        int lane) {
  for (int l = 0; l < ti.n_levels; ++l) {
    for (int idx = ti.level_start[l] + lane; idx < ti.level_start[l + 1]; idx += 32) {
      const int j = ti.order[idx];
      if (!PK_IN_BOUNDS(j, kMaxJoints, kSiteTreeParent)) continue;
      Rt O, X, Lm;
      rt_load(rb->origin[j], O);
      rt_identity(X);
      const int t = rb->type[j];
      if (t != PK_JOINT_FIXED) {
        const int v = rb->var[j];
        const float qv = PK_IN_BOUNDS(v, kTreeMaxDof, kSiteTreeParent) ? fmaf(rb->mult[j], sm.q[v], rb->offs[j]) : 0.f;
        const float* a = rb->axis[j];
        if (t == PK_JOINT_REVOLUTE) {
          float u[3] = {a[0], a[1], a[2]}, s, c;
          sincos_rad(qv, &s, &c);
          rot_joint(X.r, u, a, s, c);
        } else {
          X.t[0] = a[0] * qv; X.t[1] = a[1] * qv; X.t[2] = a[2] * qv;
        }
      }
      rt_mul(O, X, Lm);
      const int p = rb->parent[j];
      if (p >= 0 && PK_IN_BOUNDS(p, kMaxJoints, kSiteTreeParent)) {
        Rt Tp;
        rt_load(sm.frames[p], Tp);
        rt_mul(Tp, Lm, Lm);
      }
      rt_store(sm.frames[j], Lm);
    }
    __syncwarp();
  }
}

// Evaluate sm.q: residual data into sm.xi / sm.th, returns the cost; the
// largest position and rotation errors over targets come back in pe / re.
__device__ __forceinline__ float tree_eval(const RobotDev* __restrict__ rb, const TreeInfo& ti, const TreeLane& tl,
                                           const LmParams& lp, TreeWarpSmem& sm, int lane, float& pe, float& re) {
  tree_fk(rb, ti, sm, lane);
  float acc = 0.f, mpe = 0.f, mre = 0.f;
  if (lane < ti.k && PK_IN_BOUNDS(tl.link, kMaxJoints, kSiteTreeLink)) {
    Rt Tl, Ti, E;
    rt_load(sm.frames[tl.link], Tl);
    rt_load(sm.Ti[lane], Ti);
    rt_mul(Ti, Tl, E);
    mpe = sqrtf(E.t[0] * E.t[0] + E.t[1] * E.t[1] + E.t[2] * E.t[2]);
    if (tl.kind == PK_TARGET_POSE) {
      float xi[6];
      const float th = se3_log(E, xi);
      mre = th;
#pragma unroll
      for (int i = 0; i < 6; ++i) sm.xi[lane][i] = xi[i];
      sm.th[lane] = th;
      acc = lp.w_pos * lp.w_pos * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]) +
            lp.w_rot * lp.w_rot * (xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        sm.xi[lane][i] = E.t[i];
        sm.xi[lane][3 + i] = 0.f;
      }
      sm.th[lane] = 0.f;
      acc = lp.w_pos * lp.w_pos * mpe * mpe;
    }
  }
  if (lane < ti.n_dof) {
    const float q = sm.q[lane];
    const float h = fmaxf(0.f, q - tl.hi) + fmaxf(0.f, tl.lo - q);
    const float d = q - 0.5f * (tl.lo + tl.hi);
    acc = fmaf(lp.w_limit * lp.w_limit, h * h, fmaf(lp.w_rest * lp.w_rest, d * d, acc));
  }
  if (lp.w_self > 0.f) {
    // self collision (Sec. III-C, Eq. 1): one row per sphere pair
    for (int p = lane; p < rb->n_pairs; p += 32) {
      const int sa = rb->pair[p][0], sb = rb->pair[p][1];
      float ca[3], cb[3];
      Rt Ta, Tb;
      rt_load(sm.frames[rb->sph_joint[sa]], Ta);
      rt_load(sm.frames[rb->sph_joint[sb]], Tb);
      mat_vec(Ta.r, rb->sph[sa], ca);
      mat_vec(Tb.r, rb->sph[sb], cb);
      float diff[3], dist2 = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ca[i] += Ta.t[i];
        cb[i] += Tb.t[i];
        diff[i] = ca[i] - cb[i];
        dist2 = fmaf(diff[i], diff[i], dist2);
      }
      const float dist = sqrtf(dist2);
      const float d = dist - rb->sph[sa][3] - rb->sph[sb][3];
      const float eta = lp.eta_self;
      float f, df;
      if (d <= 0.f) { f = 0.5f * eta - d; df = -1.f; }
      else if (d < eta) { f = 0.5f / eta * (eta - d) * (eta - d); df = -(eta - d) / eta; }
      else { f = 0.f; df = 0.f; }
      const float r = lp.w_self * f;
      sm.pr[p] = r;
      sm.ps[p] = dist > 1e-12f ? lp.w_self * df : 0.f;
      const float inv = dist > 1e-12f ? 1.f / dist : 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        sm.pn[p][i] = diff[i] * inv;
        sm.pca[p][i] = ca[i];
        sm.pcb[p][i] = cb[i];
      }
      acc = fmaf(r, r, acc);
    }
  }
  pe = warp_max(mpe);
  re = warp_max(mre);
  __syncwarp();
  return 0.5f * warp_sum(acc);
}

// Adds scale x the weighted Jacobian column of joint jj for target k (pose:
// Jl^-1 Ad(T_target^-1) xi_j; position: w x (p - p_j)) to col[6].
__device__ __forceinline__ void tree_joint_col(const RobotDev* __restrict__ rb, const TreeWarpSmem& sm, int k,
                                               bool pose, const LmParams& lp, int jj, float scale, float* col) {
  Rt Tj, Ti;
  rt_load(sm.frames[jj], Tj);
  rt_load(sm.Ti[k], Ti);
  float wj[3], pj[3] = {Tj.t[0], Tj.t[1], Tj.t[2]};
  mat_vec(Tj.r, rb->axis[jj], wj);
  const bool prism = rb->type[jj] == PK_JOINT_PRISMATIC;
  // joint axis and origin in the target frame
  float u[3], p[3];
  mat_vec(Ti.r, wj, u);
  mat_vec(Ti.r, pj, p);
  p[0] += Ti.t[0]; p[1] += Ti.t[1]; p[2] += Ti.t[2];
  if (pose) {
    float A[9], B[9];
    se3_jlinv_blocks(sm.xi[k], sm.xi[k] + 3, sm.th[k], A, B);
    float top[3], bot[3];
    if (prism) {
      mat_vec(A, u, top);
      bot[0] = bot[1] = bot[2] = 0.f;
    } else {
      float v[3], t1[3], t2[3];
      cross3(p, u, v);
      mat_vec(A, v, t1);
      mat_vec(B, u, t2);
      mat_vec(A, u, bot);
      top[0] = t1[0] + t2[0]; top[1] = t1[1] + t2[1]; top[2] = t1[2] + t2[2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      col[i] = fmaf(scale, lp.w_pos * top[i], col[i]);
      col[3 + i] = fmaf(scale, lp.w_rot * bot[i], col[3 + i]);
    }
  } else {
    float c[3];
    if (prism) {
      c[0] = u[0]; c[1] = u[1]; c[2] = u[2];
    } else {
      float d[3] = {sm.xi[k][0] - p[0], sm.xi[k][1] - p[1], sm.xi[k][2] - p[2]};
      cross3(u, d, c);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) col[i] = fmaf(scale, lp.w_pos * c[i], col[i]);
  }
}

// Row `lane` of J^T J (in Arow[0..N)) and entry g of J^T r at the configuration
// whose frames and residuals sm holds.
template <int N>
__device__ __forceinline__ void tree_normal(const RobotDev* __restrict__ rb, const TreeInfo& ti, const TreeLane& tl,
                                            const LmParams& lp, TreeWarpSmem& sm, int lane, float (&Arow)[N],
                                            float& g) {
#pragma unroll
  for (int j = 0; j < N; ++j) Arow[j] = 0.f;
  g = 0.f;
  const bool mine = lane < ti.n_dof;
  for (int k = 0; k < ti.k; ++k) {
    const bool pose = ti.kinds[k] == PK_TARGET_POSE;
    float col[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (mine && (tl.dof_targets >> k & 1u)) {
      if ((tl.own_targets >> k & 1u) && PK_IN_BOUNDS(tl.dof_joint, kMaxJoints, kSiteTreeLink))
        tree_joint_col(rb, sm, k, pose, lp, tl.dof_joint, 1.f, col);
      for (int m = 0; m < tl.n_mim; ++m)  // a mimic joint adds to its source's column
        if ((ti.mim_targets[lane][m] >> k & 1u) && PK_IN_BOUNDS(ti.mim_joint[lane][m], kMaxJoints, kSiteTreeLink))
          tree_joint_col(rb, sm, k, pose, lp, ti.mim_joint[lane][m], ti.mim_mult[lane][m], col);
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) sm.Jk[r][lane] = col[r];
    __syncwarp();
    const int rows = pose ? 6 : 3;
    for (int r = 0; r < rows; ++r) {
      const float wr = (r < 3 ? lp.w_pos : lp.w_rot) * sm.xi[k][r];
      g = fmaf(col[r], wr, g);
#pragma unroll
      for (int j = 0; j < N; ++j) Arow[j] = fmaf(col[r], sm.Jk[r][j], Arow[j]);
    }
    __syncwarp();
  }
  if (lp.w_self > 0.f) {
    // self-collision rows, six at a time through sm.Jk
    for (int p0 = 0; p0 < rb->n_pairs; p0 += 6) {
      const int rows = min(6, rb->n_pairs - p0);
      float col[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (mine) {
        for (int r = 0; r < rows; ++r) {
          const int p = p0 + r;
          if (sm.ps[p] == 0.f) continue;
          const int ja = rb->sph_joint[rb->pair[p][0]], jb = rb->sph_joint[rb->pair[p][1]];
          float v = 0.f;
          for (int m = -1; m < tl.n_mim; ++m) {  // the variable's own joint, then its mimics
            const int jj = m < 0 ? tl.dof_joint : ti.mim_joint[lane][m];
            const float scale = m < 0 ? 1.f : ti.mim_mult[lane][m];
            const bool ina = rb->subtree[jj] >> ja & 1ull, inb = rb->subtree[jj] >> jb & 1ull;
            if (!ina && !inb) continue;
            Rt Tj;
            rt_load(sm.frames[jj], Tj);
            float w[3];
            mat_vec(Tj.r, rb->axis[jj], w);
            // velocity of a point x moved by joint jj: revolute w x (x - p_j), prismatic w
            float va[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f};
            if (rb->type[jj] == PK_JOINT_REVOLUTE) {
              if (ina) {
                const float da[3] = {sm.pca[p][0] - Tj.t[0], sm.pca[p][1] - Tj.t[1], sm.pca[p][2] - Tj.t[2]};
                cross3(w, da, va);
              }
              if (inb) {
                const float db[3] = {sm.pcb[p][0] - Tj.t[0], sm.pcb[p][1] - Tj.t[1], sm.pcb[p][2] - Tj.t[2]};
                cross3(w, db, vb);
              }
            } else {
              if (ina) { va[0] = w[0]; va[1] = w[1]; va[2] = w[2]; }
              if (inb) { vb[0] = w[0]; vb[1] = w[1]; vb[2] = w[2]; }
            }
            const float dd = sm.pn[p][0] * (va[0] - vb[0]) + sm.pn[p][1] * (va[1] - vb[1]) +
                             sm.pn[p][2] * (va[2] - vb[2]);
            v = fmaf(scale, dd, v);
          }
          col[r] = sm.ps[p] * v;
        }
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) sm.Jk[r][lane] = col[r];
      __syncwarp();
      for (int r = 0; r < rows; ++r) {
        g = fmaf(col[r], sm.pr[p0 + r], g);
#pragma unroll
        for (int j = 0; j < N; ++j) Arow[j] = fmaf(col[r], sm.Jk[r][j], Arow[j]);
      }
      __syncwarp();
    }
  }
  if (mine) {
    const float q = sm.q[lane];
    float h = 0.f, d = 0.f;
    if (q > tl.hi) { h = q - tl.hi; d = 1.f; }
    if (q < tl.lo) { h = tl.lo - q; d = -1.f; }
    const float wl2 = lp.w_limit * lp.w_limit, wr2 = lp.w_rest * lp.w_rest;
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j == lane) Arow[j] += wl2 * d * d + wr2;
    g = fmaf(wl2 * d, h, fmaf(wr2, q - 0.5f * (tl.lo + tl.hi), g));
  }
}

// Solve (A + lam I) x = -g for the n x n system held row-per-lane (Arow on
// lane i is row i); returns false on a non-positive pivot.  The factor lives
// in shared memory so that every loop below stays rolled (small code).  The
// Cholesky runs left-looking (Crout order): step k forms column k, lane i its
// entry A_ik - sum_{j<k} L_ij L_kj from its own row and row k (broadcast),
// both already final, so the loop only loads and accumulates in a register
// (the same products in the same order as updating the trailing matrix after
// every column), and every lane runs the same k terms.  The substitutions
// broadcast one unknown per step.  x comes back on lane i.
template <int N>
__device__ __forceinline__ bool tree_solve(const float (&Arow)[N], float g, float lam, int n, int lane, float& x,
                                           TreeWarpSmem& sm) {
#pragma unroll
  for (int j = 0; j < N; ++j) sm.L[lane][j] = Arow[j] + ((j == lane) ? lam : 0.f);
  __syncwarp();
  // The forward substitution L y = -g runs inside the same loop: once column
  // k is formed, lane k's right-hand side is final, y_k is broadcast and the
  // lanes below take their term of it.
  bool ok = true;
  float b = -g, y = 0.f, dinv = 0.f;  // dinv: lane k's 1 / L_kk
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    float v = sm.L[lane][k];  // A_ik: entries k.. of row i are untouched so far
#pragma unroll 4
    for (int j = 0; j < k; ++j) v = fmaf(-sm.L[lane][j], sm.L[k][j], v);
    const float d = __shfl_sync(kTreeFull, v, k);
    ok = ok && (d > 0.f) && (d < INFINITY);
    const float inv = rsqrtf(d);
    const float lik = v * inv;
    if (lane == k) {
      sm.L[k][k] = d * inv;
      dinv = inv;
    } else if (lane > k && lane < n) {
      sm.L[lane][k] = lik;
    }
    const float yk = __shfl_sync(kTreeFull, b * inv, k);
    if (lane == k) y = yk;
    if (lane > k && lane < n) b = fmaf(-lik, yk, b);
    __syncwarp();
  }
  // backward: L^T x = y (row k of L, read by column, holds L[k][i] for lane i)
  float yr = y, xv = 0.f;
#pragma unroll 1
  for (int k = n - 1; k >= 0; --k) {
    const float xk = __shfl_sync(kTreeFull, yr * dinv, k);
    if (lane == k) xv = xk;
    if (lane < k) yr = fmaf(-sm.L[k][lane], xk, yr);
  }
  x = xv;
  __syncwarp();
  return ok;
}

}  // namespace pk

namespace pk {

#ifndef PK_CLAIM_ORDER
#define PK_CLAIM_ORDER 1
#endif
// Problem index -> (target, seed).  Without cancellation: target-major.  With
// it: seeds are claimed in waves (PK_CLAIM_ORDER 1: one seed per wave, i.e.
// seed-major; 2: waves of four seeds, target-major inside a wave; 0:
// target-major throughout).
__device__ __forceinline__ void claim_order(int prob, int batch, int n_seeds, bool cancel, int* tgt, int* sd) {
  const int W = (!cancel || PK_CLAIM_ORDER == 0) ? n_seeds : (PK_CLAIM_ORDER == 1 ? 1 : 4);
  const int wave_size = batch * W;
  const int wave = prob / wave_size, r = prob - wave * wave_size;
  const int w_here = min(W, n_seeds - wave * W);  // the last wave may be narrower
  *tgt = r / w_here;
  *sd = wave * W + r % w_here;
}

// Work counters kept per lane and flushed once per warp.
struct WorkCount {
  unsigned eval = 0, build = 0, solve = 0, done = 0;
};

// LM on problems of one (robot, target set, seeds) batch, one problem per warp
// at a time, problems claimed from *head until P are done.  Records as in the
// chain kernel: q[0..n), cost, pos_err, rot_err, (status << 24) | iters.
template <int N>
__device__ void tree_lm_run(const RobotDev* __restrict__ rb, const TreeInfo& ti, const LmParams& lp,
                            const float* __restrict__ targets, const float* __restrict__ seeds, int n_seeds, int P,
                            int32_t* head, int32_t* flags, float* rec, TreeWarpSmem& sm, WorkCount& wc) {
  const int lane = threadIdx.x & 31;
  const int n = ti.n_dof, k = ti.k;
  const int np = (n + 3) & ~3, stride = np + 4;
  const int batch = P / n_seeds;
  const TreeLane tl = tree_lane(ti, lane);
  for (;;) {
    int prob = 0;
    if (lane == 0) prob = atomicAdd(head, 1);
    prob = __shfl_sync(kTreeFull, prob, 0);
    if (prob >= P) break;
    // seed-major order and claim-time skipping under sibling cancellation
    int sd, tgt;
    claim_order(prob, batch, n_seeds, lp.cancel != 0, &tgt, &sd);
    const int pid = tgt * n_seeds + sd;
    if (!PK_IN_BOUNDS(pid, P, kSiteTreeClaimPid)) continue;
    if (lp.cancel) {
      int c = 0;
      if (lane == 0) c = __ldcg(flags + tgt);
      if (__shfl_sync(kTreeFull, c, 0)) {
        if (lane == 0) {
          float* r = rec + (size_t)pid * stride;
          r[np + 0] = INFINITY;
          r[np + 3] = __int_as_float(PK_P_CANCELLED << 24);
          ++wc.done;
        }
        continue;
      }
    }
    if (lane < k) {
      Rt T, Ti;
      rt_load(targets + ((size_t)tgt * k + lane) * 12, T);
      if (tl.kind == PK_TARGET_POSE) {
        rt_inv(T, Ti);
      } else {
        rt_identity(Ti);
        Ti.t[0] = -T.t[0]; Ti.t[1] = -T.t[1]; Ti.t[2] = -T.t[2];
      }
      rt_store(sm.Ti[lane], Ti);
    }
    float q = lane < n ? __ldg(seeds + (size_t)pid * n + lane) : 0.f;
    sm.q[lane] = q;
    __syncwarp();
    float pe, re;
    float f = tree_eval(rb, ti, tl, lp, sm, lane, pe, re);
    const unsigned one = lane == 0 ? 1u : 0u;  // warp-level work counted once
    wc.eval += one;
    float Arow[N], g = 0.f;
    float lam = lp.lambda0;
    int it = 0, status = PK_P_MAX_ITERS;
    bool conv = pe <= lp.tol_pos && re <= lp.tol_rot;
    bool done = false;
    if (!isfinite(f)) { done = true; status = PK_P_NONFINITE; }
    else if (lp.early_exit && conv) { done = true; status = PK_P_CONVERGED; }
    else if (lp.max_iters <= 0) { done = true; status = conv ? PK_P_CONVERGED : PK_P_MAX_ITERS; }
    else { tree_normal<N>(rb, ti, tl, lp, sm, lane, Arow, g); wc.build += one; }
    while (!done) {
      ++it;
      float dx;
      const bool ok = tree_solve<N>(Arow, g, lam, n, lane, dx, sm);
      wc.solve += one;
      const float qc = (ok && lane < n) ? q + dx : q;
      sm.q[lane] = qc;
      __syncwarp();
      float pe_c, re_c;
      const float fc = tree_eval(rb, ti, tl, lp, sm, lane, pe_c, re_c);
      wc.eval += one;
      if (fc < f) {
        q = qc;
        f = fc;
        pe = pe_c;
        re = re_c;
        lam = fmaxf(lam / lp.nu, lp.lambda_min);
        conv = pe <= lp.tol_pos && re <= lp.tol_rot;
        if (lp.early_exit && conv) {
          done = true;
          status = PK_P_CONVERGED;
        } else if (it < lp.max_iters) {
          tree_normal<N>(rb, ti, tl, lp, sm, lane, Arow, g);
          wc.build += one;
        }
      } else {
        lam = fminf(lam * lp.nu, lp.lambda_max);
      }
      if (!done && it >= lp.max_iters) {
        done = true;
        status = conv ? PK_P_CONVERGED : PK_P_MAX_ITERS;
      }
      if (!done && lp.cancel) {
        int c = 0;
        if (lane == 0) c = __ldcg(flags + tgt);
        if (__shfl_sync(kTreeFull, c, 0)) {
          done = true;
          status = PK_P_CANCELLED;
        }
      }
    }
    float* r = rec + (size_t)pid * stride;
    if (lane < n) r[lane] = q;
    if (lane == 0) {
      r[np + 0] = f;
      r[np + 1] = pe;
      r[np + 2] = re;
      r[np + 3] = __int_as_float((status << 24) | it);
      if (lp.cancel && status == PK_P_CONVERGED) __stcg(flags + tgt, 1);
      ++wc.done;
    }
    __syncwarp();
  }
}

}  // namespace pk

namespace pk {

// ---------------------------------------------------------------------------
// Per-warp problem queue for the thread-per-problem chain kernel.  The warp
// claims problems 32 at a time (one atomic) and copies their target poses,
// seeds and cancellation flags into shared memory with cp.async while it keeps
// iterating, double-buffered, so a lane that finishes a problem refills from
// shared memory instead of waiting on global memory.  The prefetched flag may
// be stale; it only lets a solved target's seed be skipped early, the loop's
// own flag poll is authoritative.
constexpr int kQ = 32;

template <int N>
struct ChainQueue {
  alignas(16) float tgt[2][kQ][12];
  float seed[2][kQ][N];
  int32_t flag[2][kQ];
  float lam[2][kQ];    // initial damping
  int32_t pid[2][kQ];  // record index, or -1 past the end
  int32_t tid[2][kQ];  // target index
  int32_t it0[2][kQ];  // resumed problems: their record's status word (iterations done in the low 24 bits)
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one_pending() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Claim the next 32 problems into buffer `buf` and start copying their inputs.
template <int N>
__device__ __forceinline__ void chain_chunk_claim(ChainQueue<N>& q, int buf, int32_t* head, int P, int batch,
                                                  int n_seeds, bool cancel, const float* __restrict__ targets,
                                                  const float* __restrict__ seeds, const int32_t* flags,
                                                  const LmParams& lp, int lane, const float* rec = nullptr) {
  int base = 0;
  if (lane == 0) base = atomicAdd(head, kQ);
  base = __shfl_sync(kTreeFull, base, 0);
  const int p = base + lane;
  int tgt = 0, pid = -1;
  if (p < P) {
    if (lp.resume_in) {  // a suspended problem: its record holds the configuration and iteration count
      pid = __ldcg(lp.resume_in + p);
      tgt = pid / n_seeds;
    } else {
      int sd;
      claim_order(p, batch, n_seeds, cancel, &tgt, &sd);
      pid = tgt * n_seeds + sd;
    }
    if (!PK_IN_BOUNDS(pid, (long long)batch * n_seeds, kSiteChainClaimPid) ||
        !PK_IN_BOUNDS(tgt, batch, kSiteChainClaimTgt))
      pid = -1;  // skipped like a claim past the end
  }
  if (pid >= 0) {
    q.pid[buf][lane] = pid;
    q.tid[buf][lane] = tgt;
    const float* tp = targets + (size_t)tgt * 12;
    if ((reinterpret_cast<uintptr_t>(targets) & 15) == 0) {
      cp_async16(&q.tgt[buf][lane][0], tp);
      cp_async16(&q.tgt[buf][lane][4], tp + 4);
      cp_async16(&q.tgt[buf][lane][8], tp + 8);
    } else {
#pragma unroll
      for (int j = 0; j < 12; ++j) cp_async4(&q.tgt[buf][lane][j], tp + j);
    }
    if (lp.resume_in) {
      constexpr int STRIDE = ((N + 3) & ~3) + 4;
      const float* r = rec + (size_t)pid * STRIDE;
#pragma unroll
      for (int j = 0; j < N; ++j) cp_async4(&q.seed[buf][lane][j], r + j);
      cp_async4(&q.it0[buf][lane], r + STRIDE - 1);
      cp_async4(&q.lam[buf][lane], lp.lam_sus + pid);
    } else {
      const float* sp = seeds + (size_t)pid * N;
#pragma unroll
      for (int j = 0; j < N; ++j) cp_async4(&q.seed[buf][lane][j], sp + j);
      q.it0[buf][lane] = 0;
      if (lp.lam_in)
        cp_async4(&q.lam[buf][lane], lp.lam_in + pid);
      else
        q.lam[buf][lane] = lp.lambda0;
    }
    if (cancel)
      cp_async4(&q.flag[buf][lane], flags + tgt);
    else
      q.flag[buf][lane] = 0;
  } else {
    q.pid[buf][lane] = -1;
  }
  cp_async_commit();
}

}  // namespace pk
