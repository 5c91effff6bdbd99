// ik_chain.cu -- fused Levenberg-Marquardt IK for serial chains, one thread per
// (target, seed) problem, persistent grid with a lane-refilling work queue.
//
// One LM iteration of one problem (Sec. III-A solver, Sec. III-C costs):
//   FK of the candidate q_c expressed in the target frame (T_target^-1 * FK),
//   pose residual log(E) (Sec. III-C joint pose cost), joint-limit hinge and
//   rest-pose rows, cost 1/2 sum r^2;  accept iff the cost strictly drops
//   (lambda /= nu) else reject (lambda *= nu);  on acceptance the analytic
//   Jacobian Jl^-1(log E) Ad(T_target^-1) xi_j and the packed normal matrix
//   J^T J and gradient J^T r are rebuilt;  (J^T J + lambda I) dq = -J^T r is
//   solved by a register-resident Cholesky and q_c = q + dq.
// A rejected step keeps J^T J and J^T r, so only the damping changes and no
// kinematics is redone.  Each lane owns one problem; when it finishes (tolerance
// met with early exit, iteration cap, or a converged sibling seed) it writes a
// result record and claims the next problem index from a warp-aggregated
// atomic queue, so early exits do not leave lanes idle.  A second kernel picks
// the best seed of every target.
#include "pk_internal.h"
#include "pk_math.cuh"
#include "pk_chain.cuh"
#include "ik_tree.cuh"

namespace pk {

constexpr int kLmThreads = 128;
constexpr unsigned kFull = 0xffffffffu;

template <int N>
struct Frames {
  float u[N][3];  // joint axis, target frame
  float p[N][3];  // joint origin, target frame
};

// FK of q expressed in the frame Ti (= T_target^-1, or a pure translation by
// -p_target for position targets), the target-frame residual xi (unweighted:
// log(E) for pose targets, E.t for position targets), the errors and the cost.
// F = kChainFast: all joints revolute, origins pure translations, a pure
// translation as tool, pose target -- the runtime feature tests compile away
// (smaller and denser code for the common arm); F = 0: general chain.
constexpr int kChainFast = 1;
#ifndef PK_CHAIN_FAST
#define PK_CHAIN_FAST 1
#endif

template <int N, int F = 0>
__device__ __forceinline__ void chain_eval(const ChainC<N>& rc, const LmParams& lp, const Rt& Ti,
                                           const float* q, Frames<N>& fr, float* xi, float& th,
                                           float& pe, float& f) {
  Rt T = Ti;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (F != kChainFast && (rc.orot & (1u << j))) {
      Rt O;
#pragma unroll
      for (int i = 0; i < 9; ++i) O.r[i] = rc.o_r[j][i];
#pragma unroll
      for (int i = 0; i < 3; ++i) O.t[i] = rc.o_t[j][i];
      rt_mul(T, O, T);
    } else {
      rt_translate(T, rc.o_t[j]);
    }
    mat_vec(T.r, rc.a[j], fr.u[j]);
    fr.p[j][0] = T.t[0];
    fr.p[j][1] = T.t[1];
    fr.p[j][2] = T.t[2];
    if (F != kChainFast && (rc.prism & (1u << j))) {
#pragma unroll
      for (int i = 0; i < 3; ++i) T.t[i] = fmaf(fr.u[j][i], q[j], T.t[i]);
    } else {
      float s, c;
      sincos_rad(q[j], &s, &c);
      rot_joint(T.r, fr.u[j], rc.a[j], s, c);
    }
  }
  if (F != kChainFast && rc.toolrot) {
    Rt O;
#pragma unroll
    for (int i = 0; i < 9; ++i) O.r[i] = rc.tool_r[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) O.t[i] = rc.tool_t[i];
    rt_mul(T, O, T);
  } else {
    rt_translate(T, rc.tool_t);
  }
  pe = sqrtf(fmaf(T.t[0], T.t[0], fmaf(T.t[1], T.t[1], T.t[2] * T.t[2])));
  float acc;
  if (F == kChainFast || !lp.pos_only) {
    th = se3_log(T, xi);
    const float a = lp.w_pos * lp.w_pos, b = lp.w_rot * lp.w_rot;
    acc = a * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]) +
          b * (xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
  } else {
    th = 0.f;
    xi[0] = T.t[0]; xi[1] = T.t[1]; xi[2] = T.t[2];
    xi[3] = xi[4] = xi[5] = 0.f;
    acc = lp.w_pos * lp.w_pos * (pe * pe);
  }
  const float wl2 = lp.w_limit * lp.w_limit, wr2 = lp.w_rest * lp.w_rest;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float h = fmaxf(0.f, q[j] - rc.hi[j]) + fmaxf(0.f, rc.lo[j] - q[j]);
    const float d = q[j] - rc.mid[j];
    acc = fmaf(wl2, h * h, fmaf(wr2, d * d, acc));
  }
  f = 0.5f * acc;
}

// Weighted pose (or position) rows of the Jacobian, J[6][N], and the weighted
// residual rw[6] (zero rows 3..5 for position targets).
template <int N, int F = 0>
__device__ __forceinline__ void chain_pose_jac(const ChainC<N>& rc, const LmParams& lp,
                                               const Frames<N>& fr, const float* xi, float th,
                                               float (&J)[6][N], float* rw) {
  if (F == kChainFast || !lp.pos_only) {
    float A[9], B[9];
    se3_jlinv_blocks(xi, xi + 3, th, A, B);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float top[3], bot[3];
      if (F != kChainFast && (rc.prism & (1u << j))) {
        mat_vec(A, fr.u[j], top);
        bot[0] = bot[1] = bot[2] = 0.f;
      } else {
        float v[3], t1[3], t2[3];
        cross3(fr.p[j], fr.u[j], v);  // revolute twist [p x w; w]
        mat_vec(A, v, t1);
        mat_vec(B, fr.u[j], t2);
        mat_vec(A, fr.u[j], bot);
        top[0] = t1[0] + t2[0];
        top[1] = t1[1] + t2[1];
        top[2] = t1[2] + t2[2];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        J[i][j] = lp.w_pos * top[i];
        J[3 + i][j] = lp.w_rot * bot[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      rw[i] = lp.w_pos * xi[i];
      rw[3 + i] = lp.w_rot * xi[3 + i];
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float col[3];
      if (rc.prism & (1u << j)) {
        col[0] = fr.u[j][0]; col[1] = fr.u[j][1]; col[2] = fr.u[j][2];
      } else {
        float d[3] = {xi[0] - fr.p[j][0], xi[1] - fr.p[j][1], xi[2] - fr.p[j][2]};
        cross3(fr.u[j], d, col);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        J[i][j] = lp.w_pos * col[i];
        J[3 + i][j] = 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      rw[i] = lp.w_pos * xi[i];
      rw[3 + i] = 0.f;
    }
  }
}

// Packed J^T J (lower) and J^T r including the limit and rest rows.
template <int N, int F = 0>
__device__ __forceinline__ void chain_normal(const ChainC<N>& rc, const LmParams& lp,
                                             const Frames<N>& fr, const float* xi, float th,
                                             const float* q, float* A, float* g) {
  float J[6][N], rw[6];
  chain_pose_jac<N, F>(rc, lp, fr, xi, th, J, rw);
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < 6; ++r) s = fmaf(J[r][i], J[r][j], s);
      A[tri(i, j)] = s;
    }
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 6; ++r) s = fmaf(J[r][i], rw[r], s);
    g[i] = s;
  }
  const float wl2 = lp.w_limit * lp.w_limit, wr2 = lp.w_rest * lp.w_rest;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float h = 0.f, d = 0.f;
    if (q[j] > rc.hi[j]) { h = q[j] - rc.hi[j]; d = 1.f; }
    if (q[j] < rc.lo[j]) { h = rc.lo[j] - q[j]; d = -1.f; }
    A[tri(j, j)] += wl2 * d * d + wr2;
    g[j] = fmaf(wl2 * d, h, fmaf(wr2, q[j] - rc.mid[j], g[j]));
  }
}

__device__ __forceinline__ void load_target_frame(const float* __restrict__ tp, bool pos_only,
                                                  Rt& Ti) {
  const float4* p4 = reinterpret_cast<const float4*>(tp);
  const float4 a = __ldg(p4), b = __ldg(p4 + 1), c = __ldg(p4 + 2);
  Rt Tt;
  Tt.r[0] = a.x; Tt.r[1] = a.y; Tt.r[2] = a.z; Tt.t[0] = a.w;
  Tt.r[3] = b.x; Tt.r[4] = b.y; Tt.r[5] = b.z; Tt.t[1] = b.w;
  Tt.r[6] = c.x; Tt.r[7] = c.y; Tt.r[8] = c.z; Tt.t[2] = c.w;
  if (pos_only) {
    rt_identity(Ti);
    Ti.t[0] = -Tt.t[0]; Ti.t[1] = -Tt.t[1]; Ti.t[2] = -Tt.t[2];
  } else {
    rt_inv(Tt, Ti);
  }
}

int ik_rec_stride(int n_dof) { return ((n_dof + 3) & ~3) + 4; }



// The lane-refilling LM loop over the P problems of one batch; problems are
// claimed from *head, results go to rec, converged flags to flags.
template <int N, int F = 0>
__device__ __forceinline__ void chain_lm_run(const ChainC<N>& rc, const LmParams& lp,
                                             const float* __restrict__ targets, const float* __restrict__ seeds,
                                             int n_seeds, int P, int32_t* head, int32_t* flags, float* rec,
                                             WorkCount& wc, ChainQueue<N>& qq, int batch_in = 0) {
  constexpr int NT = N * (N + 1) / 2;
  constexpr int NP = ((N + 3) & ~3);
  constexpr int STRIDE = NP + 4;
  const int lane = threadIdx.x & 31;
  bool need = true, exhausted = false, fresh = false;
  Rt Ti;
  float q[N], qc[N], A0[NT], g[N];
  float f = 0.f, lam = 0.f, pe_a = 0.f, re_a = 0.f;
  int it = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) { q[j] = qc[j] = g[j] = 0.f; }
#pragma unroll
  for (int j = 0; j < NT; ++j) A0[j] = 0.f;

  // Problems come from the warp's double-buffered queue (claim order: see
  // claim_order); a seed whose target is already solved is skipped.
  const int batch = batch_in > 0 ? batch_in : P / n_seeds;
  const bool cancel = lp.cancel != 0;
  int tgt = 0, pid = 0;  // target and record index of the lane's problem
  int qcur = 0, qpos = 0;
  chain_chunk_claim<N>(qq, 0, head, P, batch, n_seeds, cancel, targets, seeds, flags, lp, lane, rec);
  chain_chunk_claim<N>(qq, 1, head, P, batch, n_seeds, cancel, targets, seeds, flags, lp, lane, rec);
  cp_async_wait_one_pending();
  __syncwarp();
  for (;;) {
    // --- hand queued problems to the lanes that need one
    for (;;) {
      const bool want = need && !exhausted;
      const unsigned nm = __ballot_sync(kFull, want);
      if (!nm) break;
      if (qpos == kQ) {  // current chunk used up: switch and refill the other buffer
        cp_async_wait_all();
        __syncwarp();
        qcur ^= 1;
        qpos = 0;
        chain_chunk_claim<N>(qq, qcur ^ 1, head, P, batch, n_seeds, cancel, targets, seeds, flags, lp, lane, rec);
      }
      const int rank = __popc(nm & ((1u << lane) - 1u));
      const int avail = kQ - qpos;
      if (want && rank < avail) {
        const int e = qpos + rank;
        const int pe = qq.pid[qcur][e];
        if (pe < 0) {
          exhausted = true;
        } else {
          pid = pe;
          tgt = qq.tid[qcur][e];
          if (cancel && qq.flag[qcur][e]) {
            float* r = rec + (size_t)pid * STRIDE;
            r[NP + 0] = INFINITY;
            r[NP + 3] = __int_as_float(PK_P_CANCELLED << 24);
            ++wc.done;
          } else {
            Rt Tt;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
              for (int c = 0; c < 3; ++c) Tt.r[i * 3 + c] = qq.tgt[qcur][e][i * 4 + c];
              Tt.t[i] = qq.tgt[qcur][e][i * 4 + 3];
            }
            if (F != kChainFast && lp.pos_only) {
              rt_identity(Ti);
              Ti.t[0] = -Tt.t[0]; Ti.t[1] = -Tt.t[1]; Ti.t[2] = -Tt.t[2];
            } else {
              rt_inv(Tt, Ti);
            }
#pragma unroll
            for (int j = 0; j < N; ++j) qc[j] = qq.seed[qcur][e][j];
            fresh = true;
            it = qq.it0[qcur][e] & 0xffffff;  // 0, or the iterations a resumed problem has done
            lam = qq.lam[qcur][e];
            need = false;
          }
        }
      }
      qpos += min(__popc(nm), avail);
    }
    need = false;
    const bool active = !exhausted;
    if (!__any_sync(kFull, active)) break;
    if (!active) continue;

    int cancelled = 0;
    if (lp.cancel) cancelled = __ldcg(flags + tgt);

    // --- evaluate the candidate
    Frames<N> fr;
    float xi[6], th, pe, fc;
    chain_eval<N, F>(rc, lp, Ti, qc, fr, xi, th, pe, fc);
    ++wc.eval;

    bool acc, done = false;
    int status = PK_P_MAX_ITERS;
    if (fresh) {
      acc = true;
      if (!isfinite(fc)) { done = true; status = PK_P_NONFINITE; }
    } else {
      acc = fc < f;
      ++it;
    }
    if (acc) {
#pragma unroll
      for (int j = 0; j < N; ++j) q[j] = qc[j];
      f = fc;
      pe_a = pe;
      re_a = th;
      if (!fresh) lam = fmaxf(lam / lp.nu, lp.lambda_min);
    } else {
      lam = fminf(lam * lp.nu, lp.lambda_max);
    }
    const bool conv = pe_a <= lp.tol_pos && re_a <= lp.tol_rot;
    if (!done) {
      if (lp.early_exit && conv) { done = true; status = PK_P_CONVERGED; }
      else if (it >= lp.max_iters) { done = true; status = conv ? PK_P_CONVERGED : PK_P_MAX_ITERS; }
      else if (cancelled) { done = true; status = PK_P_CANCELLED; }
      else if (lp.suspend_at > 0 && it >= lp.suspend_at) { done = true; status = kStatusSuspended; }
    }
    fresh = false;

    if (!done) {
      // --- damped normal equations and the next candidate
      if (acc) {
        chain_normal<N, F>(rc, lp, fr, xi, th, q, A0, g);
        ++wc.build;
      }
      ++wc.solve;
      float L[NT], d[N];
#pragma unroll
      for (int j = 0; j < NT; ++j) L[j] = A0[j];
#pragma unroll
      for (int j = 0; j < N; ++j) { L[tri(j, j)] += lam; d[j] = -g[j]; }
      const bool ok = chol_packed<N>(L);
      chol_solve_packed<N>(L, d);
#pragma unroll
      for (int j = 0; j < N; ++j) qc[j] = ok ? q[j] + d[j] : q[j];
    } else {
      float* r = rec + (size_t)pid * STRIDE;
#pragma unroll
      for (int j = 0; j < N; ++j) r[j] = q[j];
      r[NP + 0] = f;
      r[NP + 1] = pe_a;
      r[NP + 2] = re_a;
      r[NP + 3] = __int_as_float((status << 24) | it);
      if (status == kStatusSuspended) {
        // the state a later launch continues from: q and the iteration count
        // (record), the damping, and the problem's place in the resume list
        lp.lam_sus[pid] = lam;
        lp.resume_ids[atomicAdd(lp.resume_n, 1)] = pid;
      } else {
        if (lp.lam_out) lp.lam_out[pid] = lam;
        if (lp.cancel && status == PK_P_CONVERGED) __stcg(flags + tgt, 1);
        ++wc.done;
      }
      need = true;
    }
  }
  cp_async_wait_all();
  __syncwarp();
}

// Per-lane work counters summed over the warp, one atomic per counter.
__device__ __forceinline__ void flush_counts(WorkCount wc, unsigned long long* stats) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wc.eval += __shfl_xor_sync(kFull, wc.eval, o);
    wc.build += __shfl_xor_sync(kFull, wc.build, o);
    wc.solve += __shfl_xor_sync(kFull, wc.solve, o);
    wc.done += __shfl_xor_sync(kFull, wc.done, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats + 0, (unsigned long long)wc.eval);
    atomicAdd(stats + 1, (unsigned long long)wc.build);
    atomicAdd(stats + 2, (unsigned long long)wc.solve);
    atomicAdd(stats + 3, (unsigned long long)wc.done);
  }
}

// Three 128-thread blocks per SM (the register budget that avoids spills);
// stating it lets the compiler schedule for that occupancy.
#ifndef PK_LM_MINB
#define PK_LM_MINB 3
#endif
template <int N, int F>
__global__ void __launch_bounds__(kLmThreads, PK_LM_MINB) chain_lm_kernel(
    const __grid_constant__ ChainC<N> rc, const __grid_constant__ LmParams lp,
    const float* __restrict__ targets, const float* __restrict__ seeds, int n_seeds, int P,
    IkWorkspace ws) {
  __shared__ ChainQueue<N> qq[kLmThreads / 32];
  WorkCount wc;
  if (lp.resume_in) {
    // the continuation of a split solve: the suspended problems, from their own queue head
    const int n = __ldcg(lp.resume_n);
    chain_lm_run<N, F>(rc, lp, targets, seeds, n_seeds, n, ws.head2, ws.flags, ws.rec, wc, qq[threadIdx.x >> 5],
                       P / n_seeds);
  } else {
    chain_lm_run<N, F>(rc, lp, targets, seeds, n_seeds, P, ws.head, ws.flags, ws.rec, wc, qq[threadIdx.x >> 5]);
  }
  flush_counts(wc, lp.resume_in ? ws.stats + 4 : ws.stats);  // a continuation counts apart
}

// Best seed per target: converged first, then lowest cost, then lowest index.
__global__ void ik_reduce_kernel(const float* __restrict__ rec, int n, int stride, int batch,
                                 int n_seeds, float* __restrict__ q_out, float* __restrict__ err_out,
                                 int32_t* __restrict__ iters_out, int32_t* __restrict__ status_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const int np = stride - 4;
  int best = 0, best_c = -1;
  float best_f = 0.f;
  for (int s = 0; s < n_seeds; ++s) {
    const float* r = rec + ((size_t)b * n_seeds + s) * stride;
    const int meta = __float_as_int(r[np + 3]);
    const int c = ((meta >> 24) == PK_P_CONVERGED) ? 1 : 0;
    float fv = r[np];
    if (!isfinite(fv)) fv = INFINITY;
    if (best_c < 0 || c > best_c || (c == best_c && fv < best_f)) {
      best = s;
      best_c = c;
      best_f = fv;
    }
  }
  if (!PK_IN_BOUNDS(best, n_seeds, kSiteReduceRec)) return;
  const float* r = rec + ((size_t)b * n_seeds + best) * stride;
  for (int j = 0; j < n; ++j) q_out[(size_t)b * n + j] = r[j];
  err_out[2 * (size_t)b] = r[np + 1];
  err_out[2 * (size_t)b + 1] = r[np + 2];
  const int meta = __float_as_int(r[np + 3]);
  iters_out[b] = meta & 0xffffff;
  status_out[b] = meta >> 24;
}

template <int N>
__global__ void chain_residual_kernel(const __grid_constant__ ChainC<N> rc,
                                      const __grid_constant__ LmParams lp,
                                      const float* __restrict__ targets,
                                      const float* __restrict__ qs, int batch,
                                      float* __restrict__ r_out, float* __restrict__ J_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  Rt Ti;
  load_target_frame(targets + (size_t)b * 12, lp.pos_only != 0, Ti);
  float q[N];
#pragma unroll
  for (int j = 0; j < N; ++j) q[j] = qs[(size_t)b * N + j];
  Frames<N> fr;
  float xi[6], th, pe, f;
  chain_eval<N>(rc, lp, Ti, q, fr, xi, th, pe, f);
  float J[6][N], rw[6];
  chain_pose_jac<N>(rc, lp, fr, xi, th, J, rw);
  const int rows = lp.pos_only ? 3 : 6;
  const int m = rows + 2 * N;
  float* r = r_out + (size_t)b * m;
  for (int i = 0; i < rows; ++i) r[i] = rw[i];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float h = fmaxf(0.f, q[j] - rc.hi[j]) + fmaxf(0.f, rc.lo[j] - q[j]);
    r[rows + j] = lp.w_limit * h;
    r[rows + N + j] = lp.w_rest * (q[j] - rc.mid[j]);
  }
  if (!J_out) return;
  float* Jo = J_out + (size_t)b * m * N;
  for (int i = 0; i < m * N; ++i) Jo[i] = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i)
    if (i < rows)
#pragma unroll
      for (int j = 0; j < N; ++j) Jo[i * N + j] = J[i][j];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float d = 0.f;
    if (q[j] > rc.hi[j]) d = 1.f;
    if (q[j] < rc.lo[j]) d = -1.f;
    Jo[(rows + j) * N + j] = lp.w_limit * d;
    Jo[(rows + N + j) * N + j] = lp.w_rest;
  }
}

// Generic tree FK, one thread per configuration; parents' frames are re-read
// from the output rows this thread already wrote.
__global__ void fk_kernel(const RobotDev* __restrict__ rb, int nj, int nd, int batch,
                          const float* __restrict__ qs, float* __restrict__ T_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  float* out = T_out + (size_t)b * nj * 12;
  for (int j = 0; j < nj; ++j) {
    Rt O, X, L;
    rt_load(rb->origin[j], O);
    rt_identity(X);
    const int t = rb->type[j];
    if (t != PK_JOINT_FIXED) {
      const float qv = fmaf(rb->mult[j], qs[(size_t)b * nd + rb->var[j]], rb->offs[j]);
      const float* a = rb->axis[j];
      if (t == PK_JOINT_REVOLUTE) {
        float u[3] = {a[0], a[1], a[2]}, s, c;
        sincos_rad(qv, &s, &c);
        rot_joint(X.r, u, a, s, c);
      } else {
        X.t[0] = a[0] * qv; X.t[1] = a[1] * qv; X.t[2] = a[2] * qv;
      }
    }
    rt_mul(O, X, L);
    const int p = rb->parent[j];
    if (p >= 0) {
      Rt Tp;
      rt_load(out + p * 12, Tp);
      rt_mul(Tp, L, L);
    }
    rt_store(out + j * 12, L);
  }
}

// ---------------------------------------------------------------------------
// Launchers

static int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int N>
static cudaError_t chain_lm_launch(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                   const float* d_seeds, int batch, int n_seeds, IkWorkspace ws,
                                   float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                                   cudaStream_t stream, int max_grid = 0) {
  // the fast variant when the chain has only revolute joints, translation-only
  // origins and tool, and a pose target (the common arm)
  const bool fast = PK_CHAIN_FAST && ch.prism == 0 && ch.orot == 0 && !ch.toolrot && !lp.pos_only;
  static int blocks_per_sm[2] = {0, 0};
  if (blocks_per_sm[fast] == 0) {
    int b = 0;
    cudaError_t e = fast ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, chain_lm_kernel<N, kChainFast>,
                                                                        kLmThreads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, chain_lm_kernel<N, 0>, kLmThreads, 0);
    if (e != cudaSuccess) return e;
    blocks_per_sm[fast] = b > 0 ? b : 1;
  }
  const long P = (long)batch * n_seeds;
  long grid = (long)blocks_per_sm[fast] * sm_count();
  const long need = (P + kLmThreads - 1) / kLmThreads;
  if (grid > need) grid = need;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  const ChainC<N> rc = chain_const<N>(ch);
  {
    TraceScope tr(lp.resume_in ? "ik_lm_tail" : "ik_lm", stream);
    if (fast)
      chain_lm_kernel<N, kChainFast><<<(unsigned)grid, kLmThreads, 0, stream>>>(rc, lp, d_targets, d_seeds,
                                                                                n_seeds, (int)P, ws);
    else
      chain_lm_kernel<N, 0><<<(unsigned)grid, kLmThreads, 0, stream>>>(rc, lp, d_targets, d_seeds, n_seeds,
                                                                       (int)P, ws);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !d_q) return e;
  return launch_ik_reduce(ws.rec, N, batch, n_seeds, d_q, d_err, d_iters, d_status, stream);
}

// Split solve: launch 1 (every problem, suspended after split_iters
// iterations) on `stream`, launch 2 (the suspended problems, resumed from
// their records) and the reduction on `tail`.  The problem count of launch 2
// is only known on the device, so its grid is fixed: tail_ctas blocks, or the
// full persistent grid.
template <int N>
static cudaError_t chain_lm_split_launch(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                         const float* d_seeds, int batch, int n_seeds, IkWorkspace ws,
                                         int split_iters, int tail_ctas, float* d_q, float* d_err,
                                         int32_t* d_iters, int32_t* d_status, cudaStream_t stream,
                                         cudaStream_t tail, cudaEvent_t ev) {
  LmParams l1 = lp;
  l1.suspend_at = split_iters;
  l1.resume_n = ws.resume_n;
  l1.resume_ids = ws.resume_ids;
  l1.lam_sus = ws.lam_sus;
  l1.lam_in = nullptr;
  l1.lam_out = nullptr;
  cudaError_t e = chain_lm_launch<N>(ch, l1, d_targets, d_seeds, batch, n_seeds, ws, nullptr, nullptr, nullptr,
                                     nullptr, stream);
  if (e != cudaSuccess) return e;
  if (tail != stream) {
    if ((e = cudaEventRecord(ev, stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(tail, ev, 0)) != cudaSuccess) return e;
  }
  LmParams l2 = l1;
  l2.suspend_at = 0;
  l2.resume_ids = nullptr;
  l2.resume_in = ws.resume_ids;
  e = chain_lm_launch<N>(ch, l2, d_targets, d_seeds, batch, n_seeds, ws, nullptr, nullptr, nullptr, nullptr, tail,
                         tail_ctas);
  if (e != cudaSuccess) return e;
  return launch_ik_reduce(ws.rec, N, batch, n_seeds, d_q, d_err, d_iters, d_status, tail);
}

template <int N>
static cudaError_t chain_res_launch(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                    const float* d_q, int batch, float* d_r, float* d_J,
                                    cudaStream_t stream) {
  const ChainC<N> rc = chain_const<N>(ch);
  chain_residual_kernel<N><<<(batch + 127) / 128, 128, 0, stream>>>(rc, lp, d_targets, d_q, batch, d_r, d_J);
  return cudaGetLastError();
}

#define PK_CHAIN_DISPATCH(FN, ...)         \
  switch (ch.n) {                          \
    case 1: return FN<1>(__VA_ARGS__);     \
    case 2: return FN<2>(__VA_ARGS__);     \
    case 3: return FN<3>(__VA_ARGS__);     \
    case 4: return FN<4>(__VA_ARGS__);     \
    case 5: return FN<5>(__VA_ARGS__);     \
    case 6: return FN<6>(__VA_ARGS__);     \
    case 7: return FN<7>(__VA_ARGS__);     \
    case 8: return FN<8>(__VA_ARGS__);     \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_ik_reduce(const float* rec, int n_dof, int batch, int n_seeds, float* d_q, float* d_err,
                             int32_t* d_iters, int32_t* d_status, cudaStream_t stream) {
  TraceScope tr("ik_reduce", stream);
  ik_reduce_kernel<<<(batch + 127) / 128, 128, 0, stream>>>(rec, n_dof, ik_rec_stride(n_dof), batch, n_seeds, d_q,
                                                            d_err, d_iters, d_status);
  return cudaGetLastError();
}

cudaError_t launch_chain_lm(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                            const float* d_seeds, int batch, int n_seeds, IkWorkspace ws,
                            float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                            cudaStream_t stream) {
  PK_CHAIN_DISPATCH(chain_lm_launch, ch, lp, d_targets, d_seeds, batch, n_seeds, ws, d_q, d_err,
                    d_iters, d_status, stream)
}

cudaError_t launch_chain_lm_split(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                  const float* d_seeds, int batch, int n_seeds, IkWorkspace ws, int split_iters,
                                  int tail_ctas, float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                                  cudaStream_t stream, cudaStream_t tail, cudaEvent_t ev) {
  PK_CHAIN_DISPATCH(chain_lm_split_launch, ch, lp, d_targets, d_seeds, batch, n_seeds, ws, split_iters, tail_ctas,
                    d_q, d_err, d_iters, d_status, stream, tail, ev)
}

cudaError_t launch_chain_residual(const ChainHost& ch, const LmParams& lp, const float* d_targets,
                                  const float* d_q, int batch, float* d_r, float* d_J,
                                  cudaStream_t stream) {
  PK_CHAIN_DISPATCH(chain_res_launch, ch, lp, d_targets, d_q, batch, d_r, d_J, stream)
}

cudaError_t launch_fk(const RobotDev* d_robot, int n_joints, int n_dof, int batch, const float* d_q,
                      float* d_T, cudaStream_t stream) {
  fk_kernel<<<(batch + 127) / 128, 128, 0, stream>>>(d_robot, n_joints, n_dof, batch, d_q, d_T);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Uneven batches: one persistent launch over several (robot, target set,
// seeds) segments.  Every warp walks the segments in the plan's order and
// drains each one (chains: lanes claim problems one by one; trees: the warp
// claims one problem at a time) before moving on, so warps that finish the
// expensive segments fall through to the cheap ones and the launch ends when
// the last problem of the last segment is done.

struct MultiParams {
  int32_t n_segs;
  LmParams lp;
  unsigned long long* stats;
  MultiSeg seg[kMaxSegs];
  ChainC<6> c6[kMaxSegs];
  ChainC<7> c7[kMaxSegs];
  TreeInfo tree[kMaxSegs];
};

// MINB = 1 lets the compiler keep every path in registers; MINB = 3 caps the
// registers for three 128-thread blocks per SM (the autotuner picks).
// CHAINS = false compiles the thread-per-problem chain path out, for plans
// whose sets all run on the warp path: the kernel then needs only the tree
// path's registers, and the capped variant takes four 128-thread blocks per
// SM (128 registers), as the specialised tree kernel does.
static_assert(sizeof(ChainQueue<7>) <= sizeof(TreeWarpSmem), "chain queue must fit the per-warp scratch");
static_assert(sizeof(TreeWarpSmem) % 16 == 0, "per-warp scratch must keep 16-byte alignment");

template <int MINB, bool CHAINS>
__global__ void __launch_bounds__(MINB == 1 ? 256 : 128, (MINB == 3 && !CHAINS) ? 4 : MINB)
    ik_multi_kernel(const __grid_constant__ MultiParams mp) {
  extern __shared__ TreeWarpSmem tsm[];
  TreeWarpSmem& sm = tsm[threadIdx.x >> 5];
  WorkCount wc;
  for (int s = 0; s < mp.n_segs; ++s) {
    const MultiSeg& g = mp.seg[s];
    if (CHAINS && g.kind == 0) {
      LmParams lp = mp.lp;
      lp.pos_only = g.pos_only;
      if (g.pos_only) lp.tol_rot = INFINITY;
      // the chain path's queue lives in this warp's tree scratch (one path at a time)
      if (g.n == 6)
        chain_lm_run<6>(mp.c6[g.slot], lp, g.targets, g.seeds, g.n_seeds, g.P, g.head, g.flags, g.rec, wc,
                        *reinterpret_cast<ChainQueue<6>*>(&sm));
      else
        chain_lm_run<7>(mp.c7[g.slot], lp, g.targets, g.seeds, g.n_seeds, g.P, g.head, g.flags, g.rec, wc,
                        *reinterpret_cast<ChainQueue<7>*>(&sm));
      __syncwarp();
    } else {
      tree_lm_run<kTreeMaxDof>(g.rb, mp.tree[g.slot], mp.lp, g.targets, g.seeds, g.n_seeds, g.P, g.head, g.flags,
                               g.rec, sm, wc);
    }
  }
  flush_counts(wc, mp.stats);
}

size_t ik_multi_params_size() { return sizeof(MultiParams); }
void* ik_multi_params_new() { return new MultiParams(); }
void ik_multi_params_free(void* p) { delete (MultiParams*)p; }

bool ik_multi_set_chain(void* p, int slot, const ChainHost& ch) {
  MultiParams* mp = (MultiParams*)p;
  if (ch.n == 6) mp->c6[slot] = chain_const<6>(ch);
  else if (ch.n == 7) mp->c7[slot] = chain_const<7>(ch);
  else return false;
  return true;
}
void ik_multi_set_tree(void* p, int slot, const TreeInfo& ti) { ((MultiParams*)p)->tree[slot] = ti; }
void ik_multi_set_seg(void* p, int s, const MultiSeg& seg) { ((MultiParams*)p)->seg[s] = seg; }
void ik_multi_set_common(void* p, int n_segs, const LmParams& lp, unsigned long long* stats) {
  MultiParams* mp = (MultiParams*)p;
  mp->n_segs = n_segs;
  mp->lp = lp;
  mp->stats = stats;
}

namespace {
template <int MINB, bool CHAINS>
int multi_blocks(int block, size_t smem) {
  int b = 0;
  cudaFuncSetAttribute(ik_multi_kernel<MINB, CHAINS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ik_multi_kernel<MINB, CHAINS>, block, smem) != cudaSuccess)
    return 1;
  return b > 0 ? b : 1;
}
}  // namespace

int ik_multi_max_blocks_per_sm(int block, int variant, bool chains) {
  const size_t smem = (size_t)(block / 32) * sizeof(TreeWarpSmem);
  if (variant == 1 && block > 128) return 0;
  if (variant == 1) return chains ? multi_blocks<3, true>(block, smem) : multi_blocks<3, false>(block, smem);
  return chains ? multi_blocks<1, true>(block, smem) : multi_blocks<1, false>(block, smem);
}

cudaError_t launch_ik_multi(const void* host_params, int variant, bool chains, int block, int grid,
                            cudaStream_t st) {
  const size_t smem = (size_t)(block / 32) * sizeof(TreeWarpSmem);
  TraceScope tr("ik_multi", st);
  const MultiParams& mp = *(const MultiParams*)host_params;
  if (variant == 1) {
    if (chains) ik_multi_kernel<3, true><<<grid, block, smem, st>>>(mp);
    else ik_multi_kernel<3, false><<<grid, block, smem, st>>>(mp);
  } else {
    if (chains) ik_multi_kernel<1, true><<<grid, block, smem, st>>>(mp);
    else ik_multi_kernel<1, false><<<grid, block, smem, st>>>(mp);
  }
  return cudaGetLastError();
}

}  // namespace pk
