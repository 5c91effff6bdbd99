// trajopt.cu -- collision-aware trajectory optimisation, one CTA per trajectory.
//
// Variables q_0 .. q_{T-1} of a serial chain (Sec. III-B).  Residuals (each
// weighted, Sec. III-C): start configuration, goal pose log(T_goal^-1
// FK(q_{T-1})), velocity q_t - q_{t-1} and acceleration q_{t+1} - 2 q_t + q_{t-1}
// (smoothness, finite differences), joint-limit hinges, and the world
// collision cost: for every link sphere and every obstacle sphere (and the
// ground plane), w_c f(d, eta) with f the activation of Eq. 1.  Link j carries
// S spheres centred at p_j + (s + 1/2)/S (p_{j+1} - p_j).  LM (Sec. III-A) with
// a fixed iteration count.
//
// The normal matrix is block banded in t with B = 2 block sub-diagonals
// (B = 4 with the five-point stencils): collision, limit, start and goal rows
// touch one timestep (full N x N diagonal blocks D_t), velocity-limit and swept
// rows add full blocks E_t at (t, t-1), and the smoothness rows add scalar
// multiples of I on the diagonal and every sub-diagonal.  Per LM iteration:
//   1. timestep threads run FK, limits, smoothness, start and goal terms;
//      warps then take timesteps and their lanes take link spheres, test them
//      against every obstacle and the plane, and reduce the active rows' rank-1
//      updates into D_t and J^T r;
//   2. accept/reject and the lambda update;
//   3. block-banded Cholesky, serial in t, each step a handful of N x N block
//      products spread over N*N threads (the inverse of each diagonal factor is
//      kept so that the off-diagonal factors are plain products);
//   4. block forward and backward substitution, then the next candidate.
#include <algorithm>

#include "pk_chain.cuh"
#include "pk_internal.h"
#include "pk_math.cuh"

namespace pk {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int N, int B, bool X>
struct TrajSmem {
  static constexpr int NT = N * (N + 1) / 2;
  float x[2][kTrajMaxT][8];    // current / candidate trajectories
  float D[2][kTrajMaxT][NT];   // diagonal blocks of J^T J without smoothness
  float E[X ? 2 : 1][X ? kTrajMaxT : 1][N][N];  // block (t, t-1) of J^T J beyond the smoothness
                                                // scalar (velocity limits, swept spheres; X only)
  float g[2][kTrajMaxT][8];    // J^T r
  float f[2], mind[2], gpe[2], gre[2];
  // The candidate's world frames live only through an evaluation and the
  // factor only through a solve, so they share space.
  union {
    struct {
      float p[kTrajMaxT][N + 1][3];  // joint origins and tool point (world), candidate
      float w[kTrajMaxT][N][3];      // joint axes (world), candidate
    };
    struct {
      float Linv[kTrajMaxT][NT];     // inverse of the diagonal Cholesky factor (lower)
      // L[k-1][t]: factor block (t, t-k).  Band 2 keeps only k = 1: the
      // two-ended solve forms the (t, t-2) block from Linv where it is used,
      // and the one-ended solve (T < 8) keeps it in L2s.
      float L[B == 2 ? 1 : B][kTrajMaxT][N][N];
    };
  };
  float L2s[B == 2 ? 8 : 1][N][N];
  // factor block (t, t-k) of the one-ended solve
  __device__ float (&Lb(int k, int t))[N][N] {
    if constexpr (B == 2) return k == 1 ? L[0][t] : L2s[t];
    else return L[k - 1][t];
  }
  float M[N][N];
  float Sch[NT];
  float tmp[8];
  float y[kTrajMaxT][8];
  // two-ended factorisation (B = 2): per-chain scratch and the four-row junction
  float cM[2][N][N];
  float cSch[2][NT];
  float cP[2][NT];     // the next row's A_tt + lambda I - L2 L2^T
  float ctmp[2][8];
  float JD[4][NT];      // junction diagonal blocks after both chains' updates
  float JE[2][N][N];    // blocks (m-1, m-2) and (m, m+1) after the chains' updates
  float JL1[4][N][N];   // junction factor blocks (j, j-1)
  float JL2[4][N][N];   // junction factor blocks (j, j-2)
  // two-ended factorisation with B = 4: junction factor blocks (a, a-k) of the
  // eight middle rows, [k-1][a]
  float JLb[B == 4 ? 4 : 1][B == 4 ? 8 : 1][N][N];
  float sbt[kTrajMaxT][B + 1];  // smoothness scalars of blocks (t, t-k) (two-ended solves)
  alignas(16) float obs[kTrajMaxObs][4];
  float rad[N][kTrajMaxS];
  float rmax[N];  // largest sphere radius of each link
  float qs[8];
  float Tgi[12];
  float red_f[kWarps], red_d[kWarps];
  int chol_fail;
};

struct Acc {
  float f, mind;
};

// Row and column (i >= j) of the packed lower-triangle index e: i counts the
// row starts at or below e (no data-dependent loop, so the lanes of a warp,
// each with its own e, stay together).  e < N(N+1)/2 for a valid pair.
template <int N>
__device__ __forceinline__ void tri_rc(int e, int& i, int& j) {
  i = 0;
#pragma unroll
  for (int r = 1; r < N; ++r) i += (e >= tri(r, 0)) ? 1 : 0;
  j = e - tri(i, 0);
}

// Element (a, b) of a packed lower-triangular N x N block, 0 above the
// diagonal.  tri(a, b) < N(N+1)/2 for every a, b < N, so the load is made
// unconditionally and lanes with different (a, b) do not branch apart.
template <int N>
__device__ __forceinline__ float ltri(const float* L, int a, int b) {
  const float v = L[tri(a, b)];
  return a >= b ? v : 0.f;
}

__device__ __forceinline__ float coll_act(float d, float eta, float* df) {
  if (d <= 0.f) {
    *df = -1.f;
    return -d + 0.5f * eta;
  }
  if (d < eta) {
    const float e = eta - d;
    *df = -e / eta;
    return 0.5f / eta * e * e;
  }
  *df = 0.f;
  return 0.f;
}

// Smoothness scalars of the normal matrix: diagonal s_t, first sub-diagonal
// b_t (block (t, t-1)), second sub-diagonal c_t (block (t, t-2)).
__device__ __forceinline__ void smooth_scalars(const TrajParamsDev& tp, int t, float* s, float* b, float* c) {
  const int T = tp.T;
  const float v2 = tp.w_vel * tp.w_vel, a2 = tp.w_acc * tp.w_acc;
  auto in = [&](int u) { return (u >= 1 && u <= T - 2) ? 1.f : 0.f; };  // acceleration residual u exists
  *s = v2 * ((t >= 1 ? 1.f : 0.f) + (t <= T - 2 ? 1.f : 0.f)) + a2 * (in(t + 1) + 4.f * in(t) + in(t - 1));
  *b = -v2 * (t >= 1 ? 1.f : 0.f) - 2.f * a2 * (in(t) + in(t - 1));
  *c = a2 * in(t - 1) * (t >= 2 ? 1.f : 0.f);
}

// Five-point stencils over q_{u-2} .. q_{u+2}, rows u = 2..T-3: acceleration
// (-1, 16, -30, 16, -1) / 12 and jerk (-1, 2, 0, -2, 1) / 2.
__device__ __forceinline__ float acc5_coef(int k) {
  return k == 2 ? -30.f / 12.f : (k == 1 || k == 3) ? 16.f / 12.f : -1.f / 12.f;
}
__device__ __forceinline__ float jerk_coef(int k) { return k == 2 ? 0.f : k == 1 ? 1.f : k == 3 ? -1.f : k == 0 ? -0.5f : 0.5f; }

// All smoothness scalars of block row t: sb[k] multiplies I in block (t, t-k),
// k = 0..B.
template <int B>
__device__ __forceinline__ void smooth_band(const TrajParamsDev& tp, int t, float* sb) {
  smooth_scalars(tp, t, &sb[0], &sb[1], &sb[2]);
  if constexpr (B == 4) {
    sb[3] = sb[4] = 0.f;
    const float wa2 = tp.w_acc5 * tp.w_acc5, wj2 = tp.w_jerk * tp.w_jerk;
#pragma unroll
    for (int du = -2; du <= 2; ++du) {  // row u = t + du holds q_t in slot o = 2 - du
      const int u = t + du, o = 2 - du;
      if (u < 2 || u > tp.T - 3) continue;
#pragma unroll
      for (int k = 0; k <= o; ++k)  // q_{t-k} sits in slot o - k
        sb[k] += wa2 * acc5_coef(o) * acc5_coef(o - k) + wj2 * jerk_coef(o) * jerk_coef(o - k);
    }
  }
}

// Per-timestep terms (thread t): FK, limits, smoothness, start and goal.
template <int N, int B, bool X>
__device__ void eval_timestep(const ChainC<N>& rc, const TrajParamsDev& tp, TrajSmem<N, B, X>& S, int buf, int t,
                              float& fpart) {
  constexpr int NT = N * (N + 1) / 2;
  const int T = tp.T;
  float q[N];
#pragma unroll
  for (int j = 0; j < N; ++j) q[j] = S.x[buf][t][j];
  float D[NT], g[N];
#pragma unroll
  for (int i = 0; i < NT; ++i) D[i] = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) g[j] = 0.f;
  float acc = 0.f;
  // FK in the world frame
  Rt Tw;
  rt_identity(Tw);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (rc.orot & (1u << j)) {
      Rt O;
#pragma unroll
      for (int i = 0; i < 9; ++i) O.r[i] = rc.o_r[j][i];
#pragma unroll
      for (int i = 0; i < 3; ++i) O.t[i] = rc.o_t[j][i];
      rt_mul(Tw, O, Tw);
    } else {
      rt_translate(Tw, rc.o_t[j]);
    }
    float u[3];
    mat_vec(Tw.r, rc.a[j], u);
    if (rc.prism & (1u << j)) {
#pragma unroll
      for (int i = 0; i < 3; ++i) Tw.t[i] = fmaf(u[i], q[j], Tw.t[i]);
    } else {
      float s, c;
      sincos_rad(q[j], &s, &c);
      rot_joint(Tw.r, u, rc.a[j], s, c);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S.w[t][j][i] = u[i];
      S.p[t][j][i] = Tw.t[i];
    }
  }
  if (rc.toolrot) {
    Rt O;
#pragma unroll
    for (int i = 0; i < 9; ++i) O.r[i] = rc.tool_r[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) O.t[i] = rc.tool_t[i];
    rt_mul(Tw, O, Tw);
  } else {
    rt_translate(Tw, rc.tool_t);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) S.p[t][N][i] = Tw.t[i];
  // joint limits
  const float wl2 = tp.w_limit * tp.w_limit;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float h = 0.f, d = 0.f;
    if (q[j] > rc.hi[j]) { h = q[j] - rc.hi[j]; d = 1.f; }
    if (q[j] < rc.lo[j]) { h = rc.lo[j] - q[j]; d = -1.f; }
    acc = fmaf(wl2, h * h, acc);
    D[tri(j, j)] += wl2 * d * d;
    g[j] = fmaf(wl2 * d, h, g[j]);
  }
  // smoothness (residuals owned by this t; gradient from every residual touching t)
  const float v2 = tp.w_vel * tp.w_vel, a2 = tp.w_acc * tp.w_acc;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float xm = t >= 1 ? S.x[buf][t - 1][j] : 0.f;
    const float xp = t + 1 < T ? S.x[buf][t + 1][j] : 0.f;
    const float xm2 = t >= 2 ? S.x[buf][t - 2][j] : 0.f;
    const float xp2 = t + 2 < T ? S.x[buf][t + 2][j] : 0.f;
    const float x0 = q[j];
    float gj = 0.f;
    if (t >= 1) {
      const float v = x0 - xm;
      acc = fmaf(v2, v * v, acc);
      gj = fmaf(v2, v, gj);
    }
    if (t + 1 < T) gj = fmaf(-v2, xp - x0, gj);
    if (t >= 1 && t <= T - 2) {
      const float a = xp - 2.f * x0 + xm;
      acc = fmaf(a2, a * a, acc);
      gj = fmaf(-2.f * a2, a, gj);
    }
    if (t - 1 >= 1 && t - 1 <= T - 2) gj = fmaf(a2, x0 - 2.f * xm + xm2, gj);
    if (t + 1 >= 1 && t + 1 <= T - 2) gj = fmaf(a2, xp2 - 2.f * xp + x0, gj);
    g[j] += gj;
  }
  if constexpr (B == 4) {
    // five-point rows u = t-2 .. t+2 that hold q_t; row t is owned by t
    const float wa2 = tp.w_acc5 * tp.w_acc5, wj2 = tp.w_jerk * tp.w_jerk;
#pragma unroll
    for (int du = -2; du <= 2; ++du) {
      const int u = t + du, o = 2 - du;
      if (u < 2 || u > T - 3) continue;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float ra = 0.f, rj = 0.f;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const float xv = S.x[buf][u - 2 + k][j];
          ra = fmaf(acc5_coef(k), xv, ra);
          rj = fmaf(jerk_coef(k), xv, rj);
        }
        g[j] = fmaf(wa2 * acc5_coef(o), ra, fmaf(wj2 * jerk_coef(o), rj, g[j]));
        if (du == 0) acc = fmaf(wa2, ra * ra, fmaf(wj2, rj * rj, acc));
      }
    }
  }
  // velocity-limit hinge (Sec. III-C, dt = 1): the row (t, t-1) is owned by t;
  // t also takes its part of the row (t+1, t).  E_t is written whole here.
  if constexpr (X) {
  float ed[N];
#pragma unroll
  for (int j = 0; j < N; ++j) ed[j] = 0.f;
  if (tp.w_vlimit > 0.f) {
    const float wv2 = tp.w_vlimit * tp.w_vlimit;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (t >= 1) {
        const float v = q[j] - S.x[buf][t - 1][j];
        const float h = fabsf(v) - tp.v_max;
        if (h > 0.f) {
          const float sg = v > 0.f ? 1.f : -1.f;
          acc = fmaf(wv2, h * h, acc);
          D[tri(j, j)] += wv2;
          ed[j] = -wv2;
          g[j] = fmaf(wv2 * sg, h, g[j]);
        }
      }
      if (t + 1 < T) {
        const float v = S.x[buf][t + 1][j] - q[j];
        const float h = fabsf(v) - tp.v_max;
        if (h > 0.f) {
          const float sg = v > 0.f ? 1.f : -1.f;
          D[tri(j, j)] += wv2;
          g[j] = fmaf(-wv2 * sg, h, g[j]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) S.E[buf][t][i][j] = (i == j) ? ed[i] : 0.f;
  }
  // start configuration
  if (t == 0) {
    const float s2 = tp.w_start * tp.w_start;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float r = q[j] - S.qs[j];
      acc = fmaf(s2, r * r, acc);
      D[tri(j, j)] += s2;
      g[j] = fmaf(s2, r, g[j]);
    }
  }
  // goal pose on the last timestep: r = w (.) log(T_goal^-1 T_ee)
  if (t == T - 1) {
    Rt Gi, E;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) Gi.r[i * 3 + k] = S.Tgi[i * 4 + k];
      Gi.t[i] = S.Tgi[i * 4 + 3];
    }
    rt_mul(Gi, Tw, E);
    float xi[6];
    const float th = se3_log(E, xi);
    S.gpe[buf] = sqrtf(E.t[0] * E.t[0] + E.t[1] * E.t[1] + E.t[2] * E.t[2]);
    S.gre[buf] = th;
    const float wv[6] = {tp.w_goal_pos, tp.w_goal_pos, tp.w_goal_pos, tp.w_goal_rot, tp.w_goal_rot, tp.w_goal_rot};
    float Ja[9], Jb[9];
    se3_jlinv_blocks(xi, xi + 3, th, Ja, Jb);
    float J[6][N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      // world twist of joint j expressed in the goal frame
      float pw[3] = {S.p[t][j][0], S.p[t][j][1], S.p[t][j][2]};
      float ww[3] = {S.w[t][j][0], S.w[t][j][1], S.w[t][j][2]};
      float pg[3], wg[3];
      mat_vec(Gi.r, pw, pg);
      pg[0] += Gi.t[0]; pg[1] += Gi.t[1]; pg[2] += Gi.t[2];
      mat_vec(Gi.r, ww, wg);
      float top[3], bot[3];
      if (rc.prism & (1u << j)) {
        mat_vec(Ja, wg, top);
        bot[0] = bot[1] = bot[2] = 0.f;
      } else {
        float v[3], t1[3], t2[3];
        cross3(pg, wg, v);
        mat_vec(Ja, v, t1);
        mat_vec(Jb, wg, t2);
        mat_vec(Ja, wg, bot);
        top[0] = t1[0] + t2[0]; top[1] = t1[1] + t2[1]; top[2] = t1[2] + t2[2];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        J[i][j] = wv[i] * top[i];
        J[3 + i][j] = wv[3 + i] * bot[i];
      }
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const float rr = wv[r] * xi[r];
      acc = fmaf(rr, rr, acc);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        g[i] = fmaf(J[r][i], rr, g[i]);
#pragma unroll
        for (int k = 0; k <= i; ++k) D[tri(i, k)] = fmaf(J[r][i], J[r][k], D[tri(i, k)]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < NT; ++i) S.D[buf][t][i] = D[i];
#pragma unroll
  for (int j = 0; j < N; ++j) S.g[buf][t][j] = g[j];
  fpart += acc;
}

// n . dc/dq_i for a point c carried by link l at timestep t (joints 0..l).
template <int N, int B, bool X>
__device__ __forceinline__ void coll_jrow(const ChainC<N>& rc, const TrajSmem<N, B, X>& S, int t, int l, const float* c,
                                          const float* nrm, float scale, float* jr) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float dc;
    if (i > l) {
      dc = 0.f;
    } else if (rc.prism & (1u << i)) {
      dc = S.w[t][i][0] * nrm[0] + S.w[t][i][1] * nrm[1] + S.w[t][i][2] * nrm[2];
    } else {
      // n . (w_i x (c - p_i)) = w_i . ((c - p_i) x n)
      const float e0 = c[0] - S.p[t][i][0], e1 = c[1] - S.p[t][i][1], e2 = c[2] - S.p[t][i][2];
      const float x0 = e1 * nrm[2] - e2 * nrm[1], x1 = e2 * nrm[0] - e0 * nrm[2], x2 = e0 * nrm[1] - e1 * nrm[0];
      dc = S.w[t][i][0] * x0 + S.w[t][i][1] * x1 + S.w[t][i][2] * x2;
    }
    jr[i] = scale * dc;
  }
}

// Collision terms of timestep t, one link sphere per lane (lanes >= N*S idle).
// Screening tests the (sphere, obstacle) pairs that pass a per-link broad
// phase on squared distances (no square root): |c - o|^2 < (r + r_o + eta)^2
// marks the pair active in a bit mask, and mind keeps a quantity with the
// sign of the smallest signed distance (|c - o|^2 - (r + r_o)^2 over the
// tested pairs, all others being farther than eta; the plane's distance
// itself), all the collision status needs.  Then the active pairs, lane by lane in lane order
// (a fixed summation order), are processed by the whole warp, which adds each
// row's cost, J^T r and J^T J contributions straight into timestep t's
// blocks.
template <int N, int B, bool X>
__device__ void eval_collisions(const ChainC<N>& rc, const TrajParamsDev& tp, TrajSmem<N, B, X>& S, int buf, int t,
                                int lane, float& fpart, float& mind) {
  const int nsph = N * tp.S;
  // active obstacles of this lane's sphere as two 32-bit halves (obstacles
  // 0-31 and 32-63): 32-bit mask arithmetic, and the upper half is empty for
  // scenes of up to 32 obstacles
  uint32_t am_lo = 0u, am_hi = 0u;
  bool aplane = false;
  float c[3] = {0.f, 0.f, 0.f}, rad = 0.f;
  int l = 0;
  if (lane < nsph) l = lane / tp.S;
  // broad phase: lane l < N forms link l's bounding sphere (its spheres'
  // centres lie on the segment p_l -> p_{l+1}: centre at the midpoint, radius
  // half the length plus the largest sphere radius), then lane o tests
  // obstacle o (and o + 32) against every link's bound.  A sphere can only
  // come within r + r_o + eta of an obstacle its link's bound comes within
  // r_o + eta of; the bound is widened by a relative 1e-5 so that rounding
  // cannot drop such a pair, and the exact test below decides every pair that
  // passes, so the active pairs are those of testing all of them.
  float bm[3] = {0.f, 0.f, 0.f}, bh = 0.f;
  if (lane < N) {
    float e2 = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float a = S.p[t][lane][i], b = S.p[t][lane + 1][i];
      bm[i] = 0.5f * (a + b);
      e2 = fmaf(b - a, b - a, e2);
    }
    bh = 0.5f * sqrtf(e2) + S.rmax[lane] + tp.eta;
  }
  const bool two = tp.n_obs > 32;
  float4 ob0 = make_float4(0.f, 0.f, 0.f, 0.f), ob1 = ob0;
  if (lane < tp.n_obs) ob0 = *reinterpret_cast<const float4*>(S.obs[lane]);
  if (two && lane + 32 < tp.n_obs) ob1 = *reinterpret_cast<const float4*>(S.obs[lane + 32]);
  uint32_t cand_lo = 0u, cand_hi = 0u;  // candidate obstacles of this lane's link
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const float mx = __shfl_sync(0xffffffffu, bm[0], k), my = __shfl_sync(0xffffffffu, bm[1], k),
                mz = __shfl_sync(0xffffffffu, bm[2], k), h = __shfl_sync(0xffffffffu, bh, k);
    float v0 = ob0.x - mx, v1 = ob0.y - my, v2 = ob0.z - mz;
    float th = fmaf(h + ob0.w, 1.00001f, 1e-6f);
    const unsigned lo = __ballot_sync(0xffffffffu, lane < tp.n_obs && fmaf(v0, v0, fmaf(v1, v1, v2 * v2)) < th * th);
    unsigned hi = 0u;
    if (two) {
      v0 = ob1.x - mx; v1 = ob1.y - my; v2 = ob1.z - mz;
      th = fmaf(h + ob1.w, 1.00001f, 1e-6f);
      hi = __ballot_sync(0xffffffffu, lane + 32 < tp.n_obs && fmaf(v0, v0, fmaf(v1, v1, v2 * v2)) < th * th);
    }
    if (l == k) {
      cand_lo = lo;
      cand_hi = hi;
    }
  }
  if (lane < nsph) {
    const int s = lane % tp.S;
    const float al = (s + 0.5f) / (float)tp.S;
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] = fmaf(al, S.p[t][l + 1][i] - S.p[t][l][i], S.p[t][l][i]);
    rad = S.rad[l][s];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      uint32_t cm = hf ? cand_hi : cand_lo;
      uint32_t am = 0u;
      while (cm) {
        const int ob_i = __ffs(cm) - 1;
        cm &= cm - 1;
        const int o = ob_i + 32 * hf;
        if (!PK_IN_BOUNDS(o, tp.n_obs, kSiteTrajSphere)) continue;
        const float4 ob = *reinterpret_cast<const float4*>(S.obs[o]);
        const float v0 = c[0] - ob.x, v1 = c[1] - ob.y, v2 = c[2] - ob.z;
        const float dd = fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
        const float R = rad + ob.w, Re = R + tp.eta;
        mind = fminf(mind, fmaf(-R, R, dd));
        if (dd < Re * Re) am |= 1u << ob_i;
      }
      if (hf) am_hi = am;
      else am_lo = am;
    }
    if (l != 0) {  // the first link is not tested against the plane
      const float d = tp.plane[0] * c[0] + tp.plane[1] * c[1] + tp.plane[2] * c[2] - tp.plane[3] - rad;
      mind = fminf(mind, d);
      aplane = d < tp.eta;
    }
  }
  // active pairs, lane by lane in lane order; every pair is processed by the
  // whole warp: lane i < N forms Jacobian entry i, lane e < N(N+1)/2 adds
  // J^T J entry e, lane i < N adds J^T r entry i
  constexpr int NT = N * (N + 1) / 2;
  int ei, ek;
  tri_rc<N>(lane, ei, ek);  // (ei, ek): this lane's J^T J entry when lane < NT
  unsigned lanes = __ballot_sync(0xffffffffu, (am_lo | am_hi) != 0u || aplane);
  // lane i < N keeps joint i's world origin and axis; without swept rows
  // (which other warps add into D_t and g_t) the timestep's J^T J entry and
  // J^T r entry stay in registers across the pairs (the same summation order
  // as adding each pair into shared memory)
  float pj[3] = {0.f, 0.f, 0.f}, wj[3] = {0.f, 0.f, 0.f};
  float dacc = 0.f, gacc = 0.f;
  if (lanes) {
    if (lane < N)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        pj[i] = S.p[t][lane][i];
        wj[i] = S.w[t][lane][i];
      }
    if constexpr (!X) {
      if (lane < NT) dacc = S.D[buf][t][lane];
      if (lane < N) gacc = S.g[buf][t][lane];
    }
  }
  while (lanes) {
    const int src = __ffs(lanes) - 1;
    lanes &= lanes - 1;
    uint32_t m_lo = __shfl_sync(0xffffffffu, am_lo, src), m_hi = __shfl_sync(0xffffffffu, am_hi, src);
    bool pl = __shfl_sync(0xffffffffu, aplane ? 1 : 0, src) != 0;
    const float cs[3] = {__shfl_sync(0xffffffffu, c[0], src), __shfl_sync(0xffffffffu, c[1], src),
                         __shfl_sync(0xffffffffu, c[2], src)};
    const float rs = __shfl_sync(0xffffffffu, rad, src);
    const int ls = __shfl_sync(0xffffffffu, l, src);
    for (;;) {
      int o;
      if (m_lo) {  // obstacles in increasing index, then the plane
        o = __ffs(m_lo) - 1;
        m_lo &= m_lo - 1;
      } else if (m_hi) {
        o = __ffs(m_hi) + 31;
        m_hi &= m_hi - 1;
      } else if (pl) {
        o = tp.n_obs;
        pl = false;
      } else {
        break;
      }
      // the pair's distance, normal and activation, the same on every lane
      float d, nrm[3];
      if (o < tp.n_obs) {
        const float4 ob = *reinterpret_cast<const float4*>(S.obs[o]);
        const float v0 = cs[0] - ob.x, v1 = cs[1] - ob.y, v2 = cs[2] - ob.z;
        const float len = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
        d = len - rs - ob.w;
        const float inv = 1.f / len;
        nrm[0] = v0 * inv; nrm[1] = v1 * inv; nrm[2] = v2 * inv;
      } else {
        nrm[0] = tp.plane[0]; nrm[1] = tp.plane[1]; nrm[2] = tp.plane[2];
        d = nrm[0] * cs[0] + nrm[1] * cs[1] + nrm[2] * cs[2] - tp.plane[3] - rs;
      }
      float df;
      const float fa = coll_act(d, tp.eta, &df);
      if (df == 0.f) continue;
      const float r = tp.w_coll * fa;
      if (lane == 0) fpart = fmaf(r, r, fpart);
      // Jacobian entry i = lane: d(c)/d(q_i) = w_i x (c - p_i) for the joints of links 0..ls
      float ji = 0.f;
      if (lane < N && lane <= ls) {
        float dc;
        if (rc.prism & (1u << lane)) {
          dc = wj[0] * nrm[0] + wj[1] * nrm[1] + wj[2] * nrm[2];
        } else {
          const float e0 = cs[0] - pj[0], e1 = cs[1] - pj[1], e2 = cs[2] - pj[2];
          const float x0 = e1 * nrm[2] - e2 * nrm[1], x1 = e2 * nrm[0] - e0 * nrm[2], x2 = e0 * nrm[1] - e1 * nrm[0];
          dc = wj[0] * x0 + wj[1] * x1 + wj[2] * x2;
        }
        ji = tp.w_coll * df * dc;
      }
      const float jei = __shfl_sync(0xffffffffu, ji, ei < N ? ei : 0);
      const float jek = __shfl_sync(0xffffffffu, ji, ek < N ? ek : 0);
      if constexpr (X) {
        if (lane < NT) atomicAdd(&S.D[buf][t][lane], jei * jek);
        if (lane < N) atomicAdd(&S.g[buf][t][lane], ji * r);
      } else {
        dacc = fmaf(jei, jek, dacc);
        gacc = fmaf(ji, r, gacc);
      }
    }
  }
  if constexpr (!X) {
    if (__any_sync(0xffffffffu, (am_lo | am_hi) != 0u || aplane)) {
      if (lane < NT) S.D[buf][t][lane] = dacc;
      if (lane < N) S.g[buf][t][lane] = gacc;
    }
  }
  // swept spheres (Sec. IV-A): the capsule of this lane's sphere from t to t+1
  // against every obstacle sphere; the row couples q_t and q_{t+1}
  if (X && tp.w_swept > 0.f && t + 1 < tp.T && lane < nsph) {
    const int l = lane / tp.S, s = lane % tp.S;
    const float al = (s + 0.5f) / (float)tp.S;
    float c0[3], c1[3], e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      c0[i] = fmaf(al, S.p[t][l + 1][i] - S.p[t][l][i], S.p[t][l][i]);
      c1[i] = fmaf(al, S.p[t + 1][l + 1][i] - S.p[t + 1][l][i], S.p[t + 1][l][i]);
      e[i] = c1[i] - c0[i];
    }
    const float ee = fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2]));
    const float rad = S.rad[l][s];
    for (int o = 0; o < tp.n_obs; ++o) {
      const float4 ob = *reinterpret_cast<const float4*>(S.obs[o]);
      float u = ee > 0.f ? ((ob.x - c0[0]) * e[0] + (ob.y - c0[1]) * e[1] + (ob.z - c0[2]) * e[2]) / ee : 0.f;
      u = fminf(fmaxf(u, 0.f), 1.f);
      const float v0 = fmaf(u, e[0], c0[0]) - ob.x, v1 = fmaf(u, e[1], c0[1]) - ob.y, v2 = fmaf(u, e[2], c0[2]) - ob.z;
      const float len = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
      const float d = len - rad - ob.w;
      float df;
      const float fa = coll_act(d, tp.eta, &df);
      if (df == 0.f || !(len > 0.f)) continue;
      const float r = tp.w_swept * fa;
      fpart = fmaf(r, r, fpart);
      const float inv = 1.f / len;
      const float nrm[3] = {v0 * inv, v1 * inv, v2 * inv};
      float a[N], bq[N];
      coll_jrow<N, B, X>(rc, S, t, l, c0, nrm, tp.w_swept * df * (1.f - u), a);
      coll_jrow<N, B, X>(rc, S, t + 1, l, c1, nrm, tp.w_swept * df * u, bq);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        atomicAdd(&S.g[buf][t][i], a[i] * r);
        atomicAdd(&S.g[buf][t + 1][i], bq[i] * r);
#pragma unroll
        for (int k = 0; k <= i; ++k) {
          atomicAdd(&S.D[buf][t][tri(i, k)], a[i] * a[k]);
          atomicAdd(&S.D[buf][t + 1][tri(i, k)], bq[i] * bq[k]);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) atomicAdd(&S.E[buf][t + 1][i][k], bq[i] * a[k]);
      }
    }
  }
}

// Cost, J^T J diagonal blocks and J^T r of trajectory buffer `buf`.
template <int N, int B, bool X>
__device__ void evaluate(const ChainC<N>& rc, const TrajParamsDev& tp, TrajSmem<N, B, X>& S, int buf) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float fpart = 0.f, mind = INFINITY;
  for (int t = tid; t < tp.T; t += kThreads) eval_timestep<N, B, X>(rc, tp, S, buf, t, fpart);
  __syncthreads();
  for (int t = warp; t < tp.T; t += kWarps) eval_collisions<N, B, X>(rc, tp, S, buf, t, lane, fpart, mind);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fpart += __shfl_xor_sync(0xffffffffu, fpart, o);
    mind = fminf(mind, __shfl_xor_sync(0xffffffffu, mind, o));
  }
  if (lane == 0) {
    S.red_f[warp] = fpart;
    S.red_d[warp] = mind;
  }
  __syncthreads();
  if (tid == 0) {
    float f = 0.f, m = INFINITY;
    for (int w = 0; w < kWarps; ++w) {
      f += S.red_f[w];
      m = fminf(m, S.red_d[w]);
    }
    S.f[buf] = 0.5f * f;
    S.mind[buf] = m;
  }
  __syncthreads();
}

// Block-banded Cholesky of D[buf] + smoothness + lambda I (B block
// sub-diagonals), then the two block substitutions for dq = -(A)^-1 g; the
// step lands in S.y.  Block row t of the factor:
//   L_{t,t-k} = (A_{t,t-k} - sum_{m=k+1..B} L_{t,t-m} L_{t-k,t-m}^T) Linv_{t-k}^T,
// k = B down to 1 (A_{t,t-B} is a scalar multiple of I, so the top block is a
// scaled transposed inverse), then the Schur complement
//   A_tt - sum_k L_{t,t-k} L_{t,t-k}^T
// is factored densely.  Returns false if a diagonal block was not positive
// definite.
template <int N, int B, bool X>
__device__ bool banded_solve(const TrajParamsDev& tp, TrajSmem<N, B, X>& S, int buf, float lam) {
  constexpr int NT = N * (N + 1) / 2;
  const int tid = threadIdx.x, T = tp.T;
  if (tid == 0) S.chol_fail = 0;
  for (int t = 0; t < T; ++t) {
    float sb[B + 1];
    smooth_band<B>(tp, t, sb);
    // (1) L_{t,t-B} = sb[B] Linv_{t-B}^T (kept inline) and M = A_{t,t-B+1} - L_{t,t-B} L_{t-B+1,t-B}^T
    if (tid < N * N && t >= B - 1) {
      const int i = tid / N, j = tid % N;
      const float cb = sb[B];
      float m = ((i == j) ? sb[B - 1] : 0.f);
      if constexpr (B == 2 && X) m += S.E[buf][t][i][j];
      if (t >= B) {
        S.Lb(B, t)[i][j] = (j >= i) ? cb * S.Linv[t - B][tri(j, i)] : 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k >= i) m = fmaf(-cb * S.Linv[t - B][tri(k, i)], S.Lb(1, t - B + 1)[j][k], m);
      }
      S.M[i][j] = m;
    }
    __syncthreads();
#pragma unroll
    for (int k = B - 1; k >= 1; --k) {
      if (k < B - 1) {
        // M = A_{t,t-k} - sum_{m > k} L_{t,t-m} L_{t-k,t-m}^T
        if (tid < N * N && t >= k) {
          const int i = tid / N, j = tid % N;
          float m = ((i == j) ? sb[k] : 0.f);
          if constexpr (X)
            if (k == 1) m += S.E[buf][t][i][j];
#pragma unroll
          for (int mm = k + 1; mm <= B; ++mm)
            if (t >= mm)
#pragma unroll
              for (int l = 0; l < N; ++l) m = fmaf(-S.Lb(mm, t)[i][l], S.Lb(mm - k, t - k)[j][l], m);
          S.M[i][j] = m;
        }
        __syncthreads();
      }
      // L_{t,t-k} = M Linv_{t-k}^T
      if (tid < N * N && t >= k) {
        const int i = tid / N, j = tid % N;
        float v = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l)
          v = fmaf(S.M[i][l], ltri<N>(S.Linv[t - k], j, l), v);
        S.Lb(k, t)[i][j] = v;
      }
      __syncthreads();
    }
    // Schur complement A_tt + lambda I - sum_k L_{t,t-k} L_{t,t-k}^T (lower)
    if (tid < NT) {
      int i, j;
      tri_rc<N>(tid, i, j);
      float v = S.D[buf][t][tid] + ((i == j) ? sb[0] + lam : 0.f);
#pragma unroll
      for (int k = 1; k <= B; ++k)
        if (t >= k)
#pragma unroll
          for (int l = 0; l < N; ++l) v = fmaf(-S.Lb(k, t)[i][l], S.Lb(k, t)[j][l], v);
      S.Sch[tid] = v;
    }
    __syncthreads();
    // dense Cholesky of the Schur complement (lane 0), then its inverse
    // (lane j computes column j)
    if (tid == 0) {
      float L[NT];
#pragma unroll
      for (int i = 0; i < NT; ++i) L[i] = S.Sch[i];
      const bool ok = chol_packed<N>(L);  // diagonal slots hold 1 / L_ii
      if (!ok) S.chol_fail = 1;
#pragma unroll
      for (int i = 0; i < NT; ++i) S.Sch[i] = L[i];
    }
    __syncwarp();
    if (tid < N) {
      const int j = tid;
      float col[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float v = (i == j) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < i) v = fmaf(-S.Sch[tri(i, k)], col[k], v);
        col[i] = (i >= j) ? v * S.Sch[tri(i, i)] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i >= j) S.Linv[t][tri(i, j)] = col[i];
    }
    __syncthreads();
  }
  const bool ok = S.chol_fail == 0;
  // forward substitution: y_t = Linv_t (-g_t - sum_k L_{t,t-k} y_{t-k})
  for (int t = 0; t < T; ++t) {
    if (tid < N) {
      float v = -S.g[buf][t][tid];
#pragma unroll
      for (int k = 1; k <= B; ++k)
        if (t >= k)
#pragma unroll
          for (int l = 0; l < N; ++l) v = fmaf(-S.Lb(k, t)[tid][l], S.y[t - k][l], v);
      S.tmp[tid] = v;
    }
    __syncthreads();
    if (tid < N) {
      float v = 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k)
        v = fmaf(ltri<N>(S.Linv[t], tid, k), S.tmp[k], v);
      S.y[t][tid] = v;
    }
    __syncthreads();
  }
  // backward substitution: dq_t = Linv_t^T (y_t - sum_k L_{t+k,t}^T dq_{t+k})
  for (int t = T - 1; t >= 0; --t) {
    if (tid < N) {
      float v = S.y[t][tid];
#pragma unroll
      for (int k = 1; k <= B; ++k)
        if (t + k < T)
#pragma unroll
          for (int l = 0; l < N; ++l) v = fmaf(-S.Lb(k, t + k)[l][tid], S.y[t + k][l], v);
      S.tmp[tid] = v;
    }
    __syncthreads();
    if (tid < N) {
      float v = 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k)
        v = fmaf(ltri<N>(S.Linv[t], k, tid), S.tmp[k], v);
      S.y[t][tid] = v;
    }
    __syncthreads();
  }
  return ok;
}

// Two-ended factorisation of the band-2 system (T >= 8): rows 0 .. m-3 are
// eliminated top-down by threads 0-63 while rows T-1 .. m+2 are eliminated
// bottom-up by threads 64-127 (the same recurrence on the reversed order, the
// (t, t+1) blocks being transposes of the stored (t+1, t) ones); the four rows
// m-2 .. m+1 between them (m = T / 2) take both sides' updates and are
// factored last.  The serial chain is half as long as banded_solve's and the
// solve is the same up to rounding order.  Factor blocks: L[0][t] is row t
// against its first predecessor in its chain's order; the block against the
// second is a scalar times the transposed inverse factor of that row and is
// never stored.
template <int N, bool X>
__device__ bool twisted_solve(const TrajParamsDev& tp, TrajSmem<N, 2, X>& S, int buf, float lam) {
  constexpr int NT = N * (N + 1) / 2, NN = N * N;
  const int tid = threadIdx.x, T = tp.T, m = T / 2;
  const int grp = (tid >> 6) & 1, gt = tid & 63;  // chain (0 top, 1 bottom) and thread within it
  auto gsync = [&] { asm volatile("bar.sync %0, 64;" ::"r"(1 + grp) : "memory"); };
  if (tid == 0) S.chol_fail = 0;
  for (int t = tid; t < T; t += kThreads) smooth_band<2>(tp, t, S.sbt[t]);
  __syncthreads();
  // smoothness scalar of block (t, u), 0 <= t - u <= 2
  auto sc = [&](int t, int u) { return S.sbt[t][t - u]; };
  // element (i, j) of the off-diagonal block (t, u) of A, |t - u| = 1
  auto a1 = [&](int t, int u, int i, int j) {
    const int hi = t > u ? t : u;
    const float sv = sc(hi, hi - 1);
    float v = (i == j) ? sv : 0.f;
    if constexpr (X) v += (t > u) ? S.E[buf][t][i][j] : S.E[buf][u][j][i];
    return v;
  };
  // dense factor of a Schur complement and its inverse into Linv[t]: each of
  // N threads factors the 7 x 7 block in its registers (the same arithmetic,
  // so no exchange or barrier is needed in between) and writes column lt of
  // the inverse
  auto factor_lane = [&](const float* sch, int t, int lt) {
    float L[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) L[i] = sch[i];
    const bool okf = chol_packed<N>(L);
    if (lt == 0 && !okf) S.chol_fail = 1;
    float col[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float v = (i == lt) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k < i) v = fmaf(-L[tri(i, k)], col[k], v);
      col[i] = (i >= lt) ? v * L[tri(i, i)] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i >= lt) S.Linv[t][tri(i, lt)] = col[i];
  };
  auto factor_diag = [&](const float* sch, int t, int lt, auto&& sync) {
    if (lt < N) factor_lane(sch, t, lt);
    sync();
  };
  // Chains.  Row t of a chain (direction d: +1 top-down, -1 bottom-up; k its
  // position; predecessors p1 = t - d, p2 = t - 2d):
  //   M_t  = A(t, p1) - L2_t L1_{p1}^T         (k >= 1)
  //   P_t  = A_tt + lambda I - L2_t L2_t^T     (lower, packed)
  //   L1_t = M_t Linv_{p1}^T,  Sch_t = P_t - L1_t L1_t^T,  factor Sch_t -> Linv_t
  // with L1 the stored block against p1 (S.L[0][t]) and L2_t = c2 Linv_{p2}^T
  // the block against p2 (A(t, p2) = c2 I, so it is formed where it is used).
  // M and P need nothing of row p1's factor, so they are prepared one row
  // ahead: each row takes two group barriers.  Phase 1: threads e < N(N+1)/2
  // form Sch_t entry e from rows i, j of L1_t (the diagonal threads store
  // them).  Phase 2: the group's first warp factors Sch_t while its second
  // warp prepares M, P of the next row and the forward-substitution row of
  // the previous one,
  //   y_p1 = Linv_p1 (-g_p1 - L1_p1 y_{p1-d} - L2_p1 y_{p1-2d}).
  // The chain's last two rows are not factored: the one before the last keeps
  // its Schur complement in JD, the last its M in JE and its P in JD (the
  // junction divides by their factors).
  const unsigned fullm = 0xffffffffu;
  auto c2_of = [&](int t, int d) { return d > 0 ? sc(t, t - 2) : sc(t + 2, t); };
  // entry e < N*N of M_t and entry e < N(N+1)/2 of P_t
  auto prep_m = [&](int t, int d, int k, int e, float* Mo) {
    const int p1 = t - d, p2 = t - 2 * d;
    const int i = e / N, j = e % N;
    float mm = a1(t, p1, i, j);
    if (k >= 2) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q) acc = fmaf(ltri<N>(S.Linv[p2], q, i), S.L[0][p1][j][q], acc);
      mm = fmaf(-c2_of(t, d), acc, mm);
    }
    Mo[e] = mm;
  };
  auto prep_p = [&](int t, int d, int k, int e, float* Po) {
    const int p2 = t - 2 * d;
    int i, j;
    tri_rc<N>(e, i, j);
    float v = S.D[buf][t][e] + ((i == j) ? sc(t, t) + lam : 0.f);
    if (k >= 2) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q) acc = fmaf(ltri<N>(S.Linv[p2], q, i), ltri<N>(S.Linv[p2], q, j), acc);
      const float c2 = c2_of(t, d);
      v = fmaf(-c2 * c2, acc, v);
    }
    Po[e] = v;
  };
  auto schur = [&](int t, int d, int k, float* out) {
    int i, j;
    tri_rc<N>(gt, i, j);
    float v = S.cP[grp][gt];
    if (k >= 1) {
      const float* Mi = &S.cM[grp][i][0];
      const float* Mj = &S.cM[grp][j][0];
      const float* Li = S.Linv[t - d];
      float ri[N], rj[N];
#pragma unroll
      for (int c = 0; c < N; ++c) {
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int q = 0; q <= c; ++q) {
          const float l = Li[tri(c, q)];
          a = fmaf(Mi[q], l, a);
          b = fmaf(Mj[q], l, b);
        }
        ri[c] = a;
        rj[c] = b;
      }
#pragma unroll
      for (int c = 0; c < N; ++c) v = fmaf(-ri[c], rj[c], v);
      if (i == j)
#pragma unroll
        for (int c = 0; c < N; ++c) S.L[0][t][i][c] = ri[c];
    }
    out[gt] = v;
  };
  // (L2_t y)_i for row t's block against p2: c2 sum_{q >= i} Linv_p2[q][i] y_q
  auto l2y = [&](int p2, float c2, int i, const float* y) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < N; ++q)
      acc = fmaf(ltri<N>(S.Linv[p2], q, i), y[q], acc);
    return c2 * acc;
  };
  auto fwd_row = [&](int s, int d, int ks, int lane) {
    const int li = lane < N ? lane : 0;
    float v = -S.g[buf][s][li];
    if (ks >= 1)
#pragma unroll
      for (int q = 0; q < N; ++q) v = fmaf(-S.L[0][s][li][q], S.y[s - d][q], v);
    if (ks >= 2) v -= l2y(s - 2 * d, c2_of(s, d), li, S.y[s - 2 * d]);
    float yv = 0.f;
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const float vq = __shfl_sync(fullm, v, q);
      yv = fmaf(ltri<N>(S.Linv[s], li, q), vq, yv);
    }
    if (lane < N) S.y[s][lane] = yv;
  };
  {
    // four warps per chain: the group's two warps (A: threads 0-31 of the
    // group, B: 32-63) and two of threads 128-255 (C, D); barrier 3 + grp
    // spans the 128 threads of a chain
    const int d = grp == 0 ? 1 : -1, t0 = grp == 0 ? 0 : T - 1;
    const int nf = grp == 0 ? m - 2 : T - m - 2;  // rows factored in the chain
    const int jd1 = grp == 0 ? 0 : 3, jd2 = grp == 0 ? 1 : 2;
    static_assert(kThreads == 256, "the two-ended solve runs each chain on four warps");
    const int lane = tid & 31, wsub = ((tid >> 7) << 1) | ((tid >> 5) & 1);
    auto csync = [&] { asm volatile("bar.sync %0, 128;" ::"r"(3 + grp) : "memory"); };
    if (wsub == 2 && lane < NT) prep_p(t0, d, 0, lane, S.cP[grp]);
    csync();
    for (int k = 0; k <= nf; ++k) {
      const int t = t0 + k * d;
      if (wsub == 0 && lane < NT) schur(t, d, k, k < nf ? S.cSch[grp] : S.JD[jd1]);
      csync();
      // A: factor row t; B, C: M and P of row t + d; D: forward row t - d
      float* Mo = k + 1 <= nf ? &S.cM[grp][0][0] : &S.JE[grp][0][0];
      float* Po = k + 1 <= nf ? S.cP[grp] : S.JD[jd2];
      if (wsub == 0) {
        if (k < nf && lane < N) factor_lane(S.cSch[grp], t, lane);
      } else if (wsub == 1) {
        prep_m(t + d, d, k + 1, lane, Mo);
      } else if (wsub == 2) {
        if (lane < NN - 32) prep_m(t + d, d, k + 1, 32 + lane, Mo);
        if (lane < NT) prep_p(t + d, d, k + 1, lane, Po);
      } else {
        if (k >= 1) fwd_row(t - d, d, k - 1, lane);
      }
      csync();
    }
  }
  __syncthreads();
  // junction rows m-2 .. m+1 (j = 0 .. 3) by threads 0-63
  if (tid < 64) {
    for (int j = 0; j < 4; ++j) {
      const int t = m - 2 + j;
      if (j >= 1) {
        const float c2 = j >= 2 ? sc(t, t - 2) : 0.f;
        for (int e = gt; e < NN; e += 64) {
          const int r = e / N, c = e % N;
          float mm = j == 1 ? S.JE[0][r][c] : j == 2 ? a1(m, m - 1, r, c) : S.JE[1][c][r];
          if (j >= 2) {
            S.JL2[j][r][c] = (c >= r) ? c2 * S.Linv[t - 2][tri(c, r)] : 0.f;
#pragma unroll
            for (int q = 0; q < N; ++q)
              mm = fmaf(-c2 * ltri<N>(S.Linv[t - 2], q, r), S.JL1[j - 1][c][q], mm);
          }
          S.cM[0][r][c] = mm;
        }
        gsync();
        for (int e = gt; e < NN; e += 64) {
          const int r = e / N, c = e % N;
          float v = 0.f;
#pragma unroll
          for (int q = 0; q < N; ++q)
            v = fmaf(S.cM[0][r][q], ltri<N>(S.Linv[t - 1], c, q), v);
          S.JL1[j][r][c] = v;
        }
        gsync();
      }
      if (gt < NT) {
        int r, c;
        tri_rc<N>(gt, r, c);
        float v = S.JD[j][gt];
        if (j >= 1)
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.JL1[j][r][q], S.JL1[j][c][q], v);
        if (j >= 2)
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.JL2[j][r][q], S.JL2[j][c][q], v);
        S.cSch[0][gt] = v;
      }
      gsync();
      factor_diag(S.cSch[0], t, gt, gsync);
    }
  }
  __syncthreads();
  const bool ok = S.chol_fail == 0;
  // junction: right-hand sides from both chains, forward, then backward
  if (tid < 64) {
    for (int j = 0; j < 4; ++j) {
      const int t = m - 2 + j;
      if (gt < N) {
        float v = -S.g[buf][t][gt];
        // blocks against the chains' rows: the stored (t, t -+ 1) ones of the
        // outer junction rows, and (t, t -+ 2) formed from the chains' Linv
        if (j == 0) v -= l2y(m - 4, c2_of(m - 2, 1), gt, S.y[m - 4]);
        if (j == 1) v -= l2y(m - 3, c2_of(m - 1, 1), gt, S.y[m - 3]);
        if (j == 2) v -= l2y(m + 2, c2_of(m, -1), gt, S.y[m + 2]);
        if (j == 3) v -= l2y(m + 3, c2_of(m + 1, -1), gt, S.y[m + 3]);
#pragma unroll
        for (int q = 0; q < N; ++q) {
          if (j == 0) v = fmaf(-S.L[0][t][gt][q], S.y[m - 3][q], v);
          if (j == 3) v = fmaf(-S.L[0][t][gt][q], S.y[m + 2][q], v);
          if (j >= 1) v = fmaf(-S.JL1[j][gt][q], S.y[t - 1][q], v);
          if (j >= 2) v = fmaf(-S.JL2[j][gt][q], S.y[t - 2][q], v);
        }
        S.ctmp[0][gt] = v;
      }
      gsync();
      if (gt < N) {
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < N; ++q)
          v = fmaf(ltri<N>(S.Linv[t], gt, q), S.ctmp[0][q], v);
        S.y[t][gt] = v;
      }
      gsync();
    }
    for (int j = 3; j >= 0; --j) {
      const int t = m - 2 + j;
      if (gt < N) {
        float v = S.y[t][gt];
#pragma unroll
        for (int q = 0; q < N; ++q) {
          if (j + 1 <= 3) v = fmaf(-S.JL1[j + 1][q][gt], S.y[t + 1][q], v);
          if (j + 2 <= 3) v = fmaf(-S.JL2[j + 2][q][gt], S.y[t + 2][q], v);
        }
        S.ctmp[0][gt] = v;
      }
      gsync();
      if (gt < N) {
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < N; ++q)
          v = fmaf(ltri<N>(S.Linv[t], q, gt), S.ctmp[0][q], v);
        S.y[t][gt] = v;
      }
      gsync();
    }
  }
  __syncthreads();
  // backward substitution in each chain, from the junction outwards,
  // x_t = Linv_t^T (y_t - L1_{t+d}^T x_{t+d} - L2_{t+2d}^T x_{t+2d}), by the
  // chain's first warp: lane i < N holds component i of the two later rows'
  // x in registers and the other components come by shuffle, so the rows
  // need no barrier
  if (tid < 128 && gt < 32) {
    const int d = grp == 0 ? 1 : -1;
    const int tb = grp == 0 ? m - 3 : m + 2, len = grp == 0 ? m - 2 : T - m - 2;
    const int li = gt < N ? gt : 0;
    float x1 = gt < N ? S.y[tb + d][li] : 0.f, x2 = gt < N ? S.y[tb + 2 * d][li] : 0.f;
    for (int k = 0; k < len; ++k) {
      const int t = tb - k * d;
      float v = gt < N ? S.y[t][li] : 0.f;
      // L2_{t+2d}^T x_{t+2d} = c2 Linv_t x_{t+2d}
      float w2 = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        const float a1v = __shfl_sync(fullm, x1, q), a2v = __shfl_sync(fullm, x2, q);
        v = fmaf(-S.L[0][t + d][q][li], a1v, v);
        w2 = fmaf(ltri<N>(S.Linv[t], li, q), a2v, w2);
      }
      v = fmaf(-c2_of(t + 2 * d, d), w2, v);
      float xv = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        const float vq = __shfl_sync(fullm, v, q);
        xv = fmaf(ltri<N>(S.Linv[t], q, li), vq, xv);
      }
      if (gt < N) S.y[t][gt] = xv;
      x2 = x1;
      x1 = xv;
    }
  }
  __syncthreads();
  return ok;
}

// Two-ended factorisation of a band of B block sub-diagonals (used for
// B = 4, T >= 16).  Threads 0-63 eliminate rows 0 .. m-B-1 top-down and
// threads 64-127 rows T-1 .. m+B bottom-up (m = T / 2), each row t against
// its chain's predecessors p_j = t - j d (d = +1 top, -1 bottom), j = 1 .. B:
//   L_j(t) = (A(t, p_j) - sum_{l > j} L_l(t) L_{l-j}(p_j)^T) Linv(p_j)^T,
//   stored in L[j-1][t], then the Schur complement of t is factored.
// The 2B middle rows take only the blocks against their chain's eliminated
// rows; their Schur complements (coupled within the band) form a small
// banded system factored last by threads 0-63, with the same recurrence in
// natural order.  Substitutions run down the chains, through the middle and
// back out.  Same result as the one-ended factorisation up to rounding order.
template <int N, int B, bool X>
__device__ bool twisted_solve_b(const TrajParamsDev& tp, TrajSmem<N, B, X>& S, int buf, float lam) {
  constexpr int NT = N * (N + 1) / 2, NN = N * N, J = 2 * B;
  const int tid = threadIdx.x, T = tp.T, m = T / 2, j0 = m - B;  // j0: first middle row
  const int grp = (tid >> 6) & 1, gt = tid & 63;
  auto gsync = [&] { asm volatile("bar.sync %0, 64;" ::"r"(1 + grp) : "memory"); };
  if (tid == 0) S.chol_fail = 0;
  for (int t = tid; t < T; t += kThreads) smooth_band<B>(tp, t, S.sbt[t]);
  __syncthreads();
  // smoothness scalar of block (t, u), 0 <= t - u <= B
  auto sc = [&](int t, int u) { return S.sbt[t][t - u]; };
  // element (i, j) of the off-diagonal block (t, u) of A, 1 <= |t - u| <= B
  auto aoff = [&](int t, int u, int i, int j) {
    const int hi = t > u ? t : u, lo = t + u - hi;
    float v = (i == j) ? sc(hi, lo) : 0.f;
    if constexpr (X)
      if (hi - lo == 1) v += (t > u) ? S.E[buf][t][i][j] : S.E[buf][u][j][i];
    return v;
  };
  // dense factor of a Schur complement (one thread), its inverse into Linv[t]
  auto factor_diag = [&](float* sch, int t) {
    if (gt == 0) {
      float L[NT];
#pragma unroll
      for (int i = 0; i < NT; ++i) L[i] = sch[i];
      if (!chol_packed<N>(L)) S.chol_fail = 1;
#pragma unroll
      for (int i = 0; i < NT; ++i) sch[i] = L[i];
    }
    gsync();
    if (gt < N) {
      const int j = gt;
      float col[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float v = (i == j) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < i) v = fmaf(-sch[tri(i, k)], col[k], v);
        col[i] = (i >= j) ? v * sch[tri(i, i)] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i >= j) S.Linv[t][tri(i, j)] = col[i];
    }
    gsync();
  };
  // factor blocks L_j(t), j = jhi down to jlo, against eliminated rows of t's chain
  auto row_blocks = [&](int t, int d, int jlo, int jhi) {
    for (int j = jhi; j >= jlo; --j) {
      const int pj = t - j * d;
      if (j == jhi && j >= 2) {  // A(t, p_j) = c I and nothing to subtract: c Linv(p_j)^T
        if (gt < NN) {
          const int r = gt / N, c = gt % N;
          const float cj = d > 0 ? sc(t, pj) : sc(pj, t);
          S.L[j - 1][t][r][c] = (c >= r) ? cj * S.Linv[pj][tri(c, r)] : 0.f;
        }
        gsync();
        continue;
      }
      if (gt < NN) {
        const int r = gt / N, c = gt % N;
        float mm = aoff(t, pj, r, c);
        for (int l = j + 1; l <= jhi; ++l)
#pragma unroll
          for (int q = 0; q < N; ++q) mm = fmaf(-S.L[l - 1][t][r][q], S.L[l - j - 1][pj][c][q], mm);
        S.cM[grp][r][c] = mm;
      }
      gsync();
      if (gt < NN) {
        const int r = gt / N, c = gt % N;
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < N; ++q)
          v = fmaf(S.cM[grp][r][q], ltri<N>(S.Linv[pj], c, q), v);
        S.L[j - 1][t][r][c] = v;
      }
      gsync();
    }
  };
  // a chain row: blocks, Schur complement, factor (k: rows of the chain before t)
  auto chain_row = [&](int t, int d, int k) {
    const int jhi = k < B ? k : B;
    if (jhi >= 1) row_blocks(t, d, 1, jhi);
    if (gt < NT) {
      int r, c;
      tri_rc<N>(gt, r, c);
      float v = S.D[buf][t][gt] + ((r == c) ? sc(t, t) + lam : 0.f);
      for (int j = 1; j <= jhi; ++j)
#pragma unroll
        for (int q = 0; q < N; ++q) v = fmaf(-S.L[j - 1][t][r][q], S.L[j - 1][t][c][q], v);
      S.cSch[grp][gt] = v;
    }
    gsync();
    factor_diag(S.cSch[grp], t);
  };
  if (tid < 128) {
    if (grp == 0) {
      for (int t = 0; t < j0; ++t) chain_row(t, 1, t);
      for (int a = 0; a < B; ++a) row_blocks(j0 + a, 1, a + 1, B);  // middle rows above m
    } else {
      for (int t = T - 1; t >= m + B; --t) chain_row(t, -1, T - 1 - t);
      for (int a = B; a < J; ++a) row_blocks(j0 + a, -1, J - a, B);  // middle rows from m
    }
  }
  __syncthreads();
  // element (r, c) of block (a, b), a >= b, of the middle rows' Schur
  // complement (b == a: the diagonal block without lambda on the diagonal)
  auto gblock = [&](int a, int b, int r, int c) {
    const int ia = j0 + a, ib = j0 + b, k = a - b;
    float v;
    if (a < B) {  // both above m: blocks against the top chain
      v = (k == 0) ? 0.f : aoff(ia, ib, r, c);
      for (int l = a + 1; l <= B; ++l)
#pragma unroll
        for (int q = 0; q < N; ++q) v = fmaf(-S.L[l - 1][ia][r][q], S.L[l - k - 1][ib][c][q], v);
    } else if (b >= B) {  // both from m: the transpose of block (b, a) against the bottom chain
      v = (k == 0) ? 0.f : aoff(ia, ib, r, c);
      for (int l = J - b; l <= B; ++l)
#pragma unroll
        for (int q = 0; q < N; ++q) v = fmaf(-S.L[l - 1][ib][c][q], S.L[l - k - 1][ia][r][q], v);
    } else {
      v = aoff(ia, ib, r, c);
    }
    return v;
  };
  if (tid < 64) {
    for (int a = 0; a < J; ++a) {
      const int ia = j0 + a, kmax = a < B ? a : B;
      for (int k = kmax; k >= 1; --k) {
        const int b = a - k;
        if (gt < NN) {
          const int r = gt / N, c = gt % N;
          float mm = gblock(a, b, r, c);
          for (int l = k + 1; l <= kmax; ++l)
#pragma unroll
            for (int q = 0; q < N; ++q) mm = fmaf(-S.JLb[l - 1][a][r][q], S.JLb[l - k - 1][b][c][q], mm);
          S.cM[0][r][c] = mm;
        }
        gsync();
        if (gt < NN) {
          const int r = gt / N, c = gt % N;
          float v = 0.f;
#pragma unroll
          for (int q = 0; q < N; ++q)
            v = fmaf(S.cM[0][r][q], ltri<N>(S.Linv[j0 + b], c, q), v);
          S.JLb[k - 1][a][r][c] = v;
        }
        gsync();
      }
      if (gt < NT) {
        int r, c;
        tri_rc<N>(gt, r, c);
        float v = S.D[buf][ia][gt] + ((r == c) ? sc(ia, ia) + lam : 0.f) + gblock(a, a, r, c);
        for (int k = 1; k <= kmax; ++k)
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.JLb[k - 1][a][r][q], S.JLb[k - 1][a][c][q], v);
        S.cSch[0][gt] = v;
      }
      gsync();
      factor_diag(S.cSch[0], ia);
    }
  }
  __syncthreads();
  const bool ok = S.chol_fail == 0;
  // y_t = Linv_t (rhs - sum of the given blocks times y), rhs built by `acc`
  auto solve_lower = [&](int t, auto&& acc) {
    if (gt < N) S.ctmp[grp][gt] = acc(gt);
    gsync();
    if (gt < N) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q)
        v = fmaf(ltri<N>(S.Linv[t], gt, q), S.ctmp[grp][q], v);
      S.y[t][gt] = v;
    }
    gsync();
  };
  auto solve_upper = [&](int t, auto&& acc) {
    if (gt < N) S.ctmp[grp][gt] = acc(gt);
    gsync();
    if (gt < N) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q)
        v = fmaf(ltri<N>(S.Linv[t], q, gt), S.ctmp[grp][q], v);
      S.y[t][gt] = v;
    }
    gsync();
  };
  // forward substitution down both chains
  if (tid < 128) {
    const int d = grp == 0 ? 1 : -1;
    // the top chain holds rows 0 .. m-B-1, the bottom one T-1 .. m+B (one
    // more row than the top for odd T)
    const int t0 = grp == 0 ? 0 : T - 1, len = grp == 0 ? j0 : T - m - B;
    for (int k = 0; k < len; ++k) {
      const int t = t0 + k * d, jhi = k < B ? k : B;
      solve_lower(t, [&](int i) {
        float v = -S.g[buf][t][i];
        for (int j = 1; j <= jhi; ++j)
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.L[j - 1][t][i][q], S.y[t - j * d][q], v);
        return v;
      });
    }
  }
  __syncthreads();
  // the middle rows: forward with the blocks against both chains, then back
  if (tid < 64) {
    for (int a = 0; a < J; ++a) {
      const int ia = j0 + a, kmax = a < B ? a : B;
      solve_lower(ia, [&](int i) {
        float v = -S.g[buf][ia][i];
        if (a < B) {
          for (int l = a + 1; l <= B; ++l)
#pragma unroll
            for (int q = 0; q < N; ++q) v = fmaf(-S.L[l - 1][ia][i][q], S.y[ia - l][q], v);
        } else {
          for (int l = J - a; l <= B; ++l)
#pragma unroll
            for (int q = 0; q < N; ++q) v = fmaf(-S.L[l - 1][ia][i][q], S.y[ia + l][q], v);
        }
        for (int k = 1; k <= kmax; ++k)
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.JLb[k - 1][a][i][q], S.y[ia - k][q], v);
        return v;
      });
    }
    for (int a = J - 1; a >= 0; --a) {
      const int ia = j0 + a;
      solve_upper(ia, [&](int i) {
        float v = S.y[ia][i];
        for (int k = 1; k <= B && a + k < J; ++k)
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.JLb[k - 1][a + k][q][i], S.y[ia + k][q], v);
        return v;
      });
    }
  }
  __syncthreads();
  // backward substitution up both chains, from the middle outwards
  if (tid < 128) {
    const int d = grp == 0 ? 1 : -1;
    const int tb = grp == 0 ? j0 - 1 : m + B, len = grp == 0 ? j0 : T - m - B;
    for (int k = 0; k < len; ++k) {
      const int t = tb - k * d;
      solve_upper(t, [&](int i) {
        float v = S.y[t][i];
        for (int j = 1; j <= B; ++j) {
          const int u = t + j * d;
#pragma unroll
          for (int q = 0; q < N; ++q) v = fmaf(-S.L[j - 1][u][q][i], S.y[u][q], v);
        }
        return v;
      });
    }
  }
  __syncthreads();
  return ok;
}

template <int N, int B, bool X>
__global__ void __launch_bounds__(kThreads, (B == 2 && !X) ? 3 : 2) trajopt_kernel(
    const __grid_constant__ ChainC<N> rc, const __grid_constant__ TrajParamsDev tp, const float* __restrict__ q_start,
    const float* __restrict__ goals, const float* __restrict__ q_init, const float* __restrict__ radii,
    const float* __restrict__ obs, float* __restrict__ q_out, float* __restrict__ cost_out,
    int32_t* __restrict__ status_out, float* __restrict__ D_out, float* __restrict__ E_out,
    float* __restrict__ g_out) {
  extern __shared__ float4 smem_f4[];
  TrajSmem<N, B, X>& S = *reinterpret_cast<TrajSmem<N, B, X>*>(smem_f4);
  const int b = blockIdx.x, tid = threadIdx.x, T = tp.T;
  // inputs
  for (int i = tid; i < T * N; i += kThreads) S.x[0][i / N][i % N] = q_init[(size_t)b * T * N + i];
  for (int i = tid; i < tp.n_obs * 4; i += kThreads) S.obs[i / 4][i % 4] = obs[i];
  for (int i = tid; i < N * tp.S; i += kThreads) S.rad[i / tp.S][i % tp.S] = radii[i];
  if (tid < N) {
    float r = 0.f;
    for (int k = 0; k < tp.S; ++k) r = fmaxf(r, radii[tid * tp.S + k]);
    S.rmax[tid] = r;
  }
  if (tid < N) S.qs[tid] = q_start[(size_t)b * N + tid];
  if (tid == 0) {
    Rt G, Gi;
    rt_load(goals + (size_t)b * 12, G);
    rt_inv(G, Gi);
    rt_store(S.Tgi, Gi);
  }
  __syncthreads();
  evaluate<N, B, X>(rc, tp, S, 0);
  if (D_out) {
    // normal equations only: full diagonal blocks (smoothness included) and J^T r
    for (int i = tid; i < T * N * N; i += kThreads) {
      const int t = i / (N * N), r = (i / N) % N, c = i % N;
      float sb[B + 1];
      smooth_band<B>(tp, t, sb);
      const float v = (r >= c) ? S.D[0][t][tri(r, c)] : S.D[0][t][tri(c, r)];
      D_out[(size_t)b * T * N * N + i] = v + ((r == c) ? sb[0] : 0.f);
    }
    if (E_out)
      for (int i = tid; i < T * N * N; i += kThreads) {
        const int t = i / (N * N), r = (i / N) % N, c = i % N;
        float sb[B + 1];
        smooth_band<B>(tp, t, sb);
        float e = 0.f;
        if constexpr (X) e = S.E[0][t][r][c];
        E_out[(size_t)b * T * N * N + i] = t >= 1 ? e + ((r == c) ? sb[1] : 0.f) : 0.f;
      }
    for (int i = tid; i < T * N; i += kThreads) g_out[(size_t)b * T * N + i] = S.g[0][i / N][i % N];
    if (tid == 0) cost_out[b] = S.f[0];
    return;
  }
  int u = 0;  // buffer of the accepted trajectory
  float lam = tp.lambda0;
  for (int it = 0; it < tp.iters; ++it) {
    bool ok;
    if constexpr (B == 2) {
      ok = T >= 8 ? twisted_solve<N, X>(tp, S, u, lam) : banded_solve<N, B, X>(tp, S, u, lam);
    } else {
      ok = T >= 4 * B ? twisted_solve_b<N, B, X>(tp, S, u, lam) : banded_solve<N, B, X>(tp, S, u, lam);
    }
    if (ok) {
      const int c = u ^ 1;
      for (int i = tid; i < T * N; i += kThreads) S.x[c][i / N][i % N] = S.x[u][i / N][i % N] + S.y[i / N][i % N];
      __syncthreads();
      evaluate<N, B, X>(rc, tp, S, c);
      if (S.f[c] < S.f[u]) {
        u = c;
        lam = fmaxf(lam / tp.nu, tp.lambda_min);
      } else {
        lam = fminf(lam * tp.nu, tp.lambda_max);
      }
    } else {
      lam = fminf(lam * tp.nu, tp.lambda_max);
    }
    __syncthreads();
  }
  for (int i = tid; i < T * N; i += kThreads) q_out[(size_t)b * T * N + i] = S.x[u][i / N][i % N];
  if (tid == 0) {
    cost_out[b] = S.f[u];
    int st = 0;
    if (!(S.gpe[u] <= tp.tol_pos && S.gre[u] <= tp.tol_rot)) st |= PK_T_GOAL_MISSED;
    if (!(S.mind[u] >= 0.f)) st |= PK_T_COLLISION;
    status_out[b] = st;
  }
}

template <int N, int B, bool X>
cudaError_t trajopt_launch(const ChainHost& ch, const TrajParamsDev& tp, int batch, const float* q_start,
                           const float* goals, const float* q_init, const float* radii, const float* obs,
                           float* q_out, float* cost_out, int32_t* status_out, float* D_out, float* E_out,
                           float* g_out, cudaStream_t st) {
  const size_t smem = sizeof(TrajSmem<N, B, X>);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(trajopt_kernel<N, B, X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const ChainC<N> rc = chain_const<N>(ch);
  TraceScope tr("trajopt", st);
  trajopt_kernel<N, B, X><<<batch, kThreads, smem, st>>>(rc, tp, q_start, goals, q_init, radii, obs, q_out, cost_out,
                                                   status_out, D_out, E_out, g_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trajopt(const ChainHost& ch, const TrajParamsDev& tp, int batch, const float* q_start,
                           const float* goals, const float* q_init, const float* radii, const float* obs,
                           float* q_out, float* cost_out, int32_t* status_out, float* D_out, float* E_out,
                           float* g_out, cudaStream_t st) {
  // four block sub-diagonals only when a five-point stencil is on, full
  // (t, t-1) blocks only with velocity-limit or swept rows: the smallest
  // shared-memory layout runs (three CTAs per SM without either)
  const bool b4 = tp.w_acc5 != 0.f || tp.w_jerk != 0.f;
  const bool x = tp.w_vlimit > 0.f || tp.w_swept > 0.f;
#define PK_TRAJ_ARGS ch, tp, batch, q_start, goals, q_init, radii, obs, q_out, cost_out, status_out, D_out, E_out, g_out, st
  switch ((ch.n == 7 ? 4 : 0) + (b4 ? 2 : 0) + (x ? 1 : 0) + (ch.n == 6 || ch.n == 7 ? 0 : 8)) {
    case 0: return trajopt_launch<6, 2, false>(PK_TRAJ_ARGS);
    case 1: return trajopt_launch<6, 2, true>(PK_TRAJ_ARGS);
    case 2: return trajopt_launch<6, 4, false>(PK_TRAJ_ARGS);
    case 3: return trajopt_launch<6, 4, true>(PK_TRAJ_ARGS);
    case 4: return trajopt_launch<7, 2, false>(PK_TRAJ_ARGS);
    case 5: return trajopt_launch<7, 2, true>(PK_TRAJ_ARGS);
    case 6: return trajopt_launch<7, 4, false>(PK_TRAJ_ARGS);
    case 7: return trajopt_launch<7, 4, true>(PK_TRAJ_ARGS);
    default: return cudaErrorInvalidValue;
  }
}

#undef PK_TRAJ_ARGS

namespace {

// Initial trajectory (Sec. IV-A): q_t = (1 - s_t) q_start + s_t q_goal with
// s_t = t / (T - 1), one thread per (trajectory, timestep, joint).
__global__ void interpolate_kernel(int batch, int T, int n, const float* __restrict__ q_start,
                                   const float* __restrict__ q_goal, float* __restrict__ q_out) {
  const long total = (long)batch * T * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int j = (int)(i % n);
    const int t = (int)((i / n) % T);
    const long b = i / ((long)n * T);
    const float s = T > 1 ? (float)t / (float)(T - 1) : 0.f;
    q_out[i] = (1.f - s) * q_start[b * n + j] + s * q_goal[b * n + j];
  }
}

}  // namespace

namespace {

// Joint origins p_0 .. p_{N-1} and the tool point p_N of a serial chain at q
// (the world-frame points the link spheres of the trajectory cost lie on).
template <int N>
__device__ void chain_points(const ChainC<N>& rc, const float* q, float (*p)[3]) {
  Rt Tw;
  rt_identity(Tw);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (rc.orot & (1u << j)) {
      Rt O;
#pragma unroll
      for (int i = 0; i < 9; ++i) O.r[i] = rc.o_r[j][i];
#pragma unroll
      for (int i = 0; i < 3; ++i) O.t[i] = rc.o_t[j][i];
      rt_mul(Tw, O, Tw);
    } else {
      rt_translate(Tw, rc.o_t[j]);
    }
    float u[3];
    mat_vec(Tw.r, rc.a[j], u);
    if (rc.prism & (1u << j)) {
#pragma unroll
      for (int i = 0; i < 3; ++i) Tw.t[i] = fmaf(u[i], q[j], Tw.t[i]);
    } else {
      float sn, cs;
      sincos_rad(q[j], &sn, &cs);
      rot_joint(Tw.r, u, rc.a[j], sn, cs);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) p[j][i] = Tw.t[i];
  }
  if (rc.toolrot) {
    Rt O;
#pragma unroll
    for (int i = 0; i < 9; ++i) O.r[i] = rc.tool_r[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) O.t[i] = rc.tool_t[i];
    rt_mul(Tw, O, Tw);
  } else {
    rt_translate(Tw, rc.tool_t);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) p[N][i] = Tw.t[i];
}

// Per target (one warp; lanes take the seeds): the seed of the multi-start
// solve whose records are in `rec` that is converged and whose link spheres
// clear every obstacle and the plane by `margin`, else converged, else any;
// within a class the lowest cost, then the lowest seed index.
template <int N>
__global__ void __launch_bounds__(128) select_clear_kernel(
    const __grid_constant__ ChainC<N> rc, const float* __restrict__ rec, int stride, int batch, int n_seeds, int S,
    const float* __restrict__ radii, int n_obs, const float* __restrict__ obs, float4 plane, float margin,
    float* __restrict__ q_out, float* __restrict__ err_out, int32_t* __restrict__ iters_out,
    int32_t* __restrict__ status_out) {
  const int b = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (b >= batch) return;  // uniform across the warp
  const int np = stride - 4;
  int bc = -1, bs = 0x7fffffff;
  float bf = INFINITY;
  for (int s = lane; s < n_seeds; s += 32) {
    const float* r = rec + ((size_t)b * n_seeds + s) * stride;
    const int meta = __float_as_int(r[np + 3]);
    const bool conv = (meta >> 24) == PK_P_CONVERGED;
    float fv = r[np];
    if (!isfinite(fv)) fv = INFINITY;
    int cls = conv ? 1 : 0;
    if (conv) {
      float q[N], p[N + 1][3];
#pragma unroll
      for (int j = 0; j < N; ++j) q[j] = r[j];
      chain_points<N>(rc, q, p);
      bool clear = true;
      for (int l = 0; l < N && clear; ++l) {
        for (int k = 0; k < S && clear; ++k) {
          const float al = (k + 0.5f) / (float)S, rad = __ldg(radii + l * S + k);
          float c[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) c[i] = fmaf(al, p[l + 1][i] - p[l][i], p[l][i]);
          for (int o = 0; o < n_obs; ++o) {
            const float4 ob = __ldg(reinterpret_cast<const float4*>(obs) + o);
            const float v0 = c[0] - ob.x, v1 = c[1] - ob.y, v2 = c[2] - ob.z;
            if (sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2))) - rad - ob.w < margin) {
              clear = false;
              break;
            }
          }
          // the first link's spheres are not tested against the plane
          if (clear && l >= 1 && fmaf(plane.x, c[0], fmaf(plane.y, c[1], plane.z * c[2])) - plane.w - rad < margin)
            clear = false;
        }
      }
      if (clear) cls = 2;
    }
    if (cls > bc || (cls == bc && (fv < bf || (fv == bf && s < bs)))) {
      bc = cls;
      bf = fv;
      bs = s;
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const int oc = __shfl_xor_sync(0xffffffffu, bc, off), os = __shfl_xor_sync(0xffffffffu, bs, off);
    const float of = __shfl_xor_sync(0xffffffffu, bf, off);
    if (oc > bc || (oc == bc && (of < bf || (of == bf && os < bs)))) {
      bc = oc;
      bf = of;
      bs = os;
    }
  }
  if (lane == 0 && PK_IN_BOUNDS(bs, n_seeds, kSiteSelectClear)) {
    const float* r = rec + ((size_t)b * n_seeds + bs) * stride;
#pragma unroll
    for (int j = 0; j < N; ++j) q_out[(size_t)b * N + j] = r[j];
    err_out[2 * (size_t)b] = r[np + 1];
    err_out[2 * (size_t)b + 1] = r[np + 2];
    const int meta = __float_as_int(r[np + 3]);
    iters_out[b] = meta & 0xffffff;
    status_out[b] = meta >> 24;
  }
}

}  // namespace

cudaError_t launch_select_clear(const ChainHost& ch, const float* rec, int batch, int n_seeds, int S,
                                const float* radii, int n_obs, const float* obs, const float* plane, float margin,
                                float* q_out, float* err_out, int32_t* iters_out, int32_t* status_out,
                                cudaStream_t st) {
  const float4 pl = make_float4(plane[0], plane[1], plane[2], plane[3]);
  const int grid = (int)(((long)batch * 32 + 127) / 128);
  if (ch.n == 7) {
    select_clear_kernel<7><<<grid, 128, 0, st>>>(chain_const<7>(ch), rec, ik_rec_stride(7), batch, n_seeds, S, radii,
                                                 n_obs, obs, pl, margin, q_out, err_out, iters_out, status_out);
  } else if (ch.n == 6) {
    select_clear_kernel<6><<<grid, 128, 0, st>>>(chain_const<6>(ch), rec, ik_rec_stride(6), batch, n_seeds, S, radii,
                                                 n_obs, obs, pl, margin, q_out, err_out, iters_out, status_out);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_interpolate(int batch, int T, int n, const float* q_start, const float* q_goal, float* q_out,
                               cudaStream_t st) {
  const long total = (long)batch * T * n;
  const int block = 256;
  const int grid = (int)std::min<long>((total + block - 1) / block, 152L * 8);
  interpolate_kernel<<<grid, block, 0, st>>>(batch, T, n, q_start, q_goal, q_out);
  return cudaGetLastError();
}

}  // namespace pk
