// seednet.cu -- the learned-seed network: a SiLU MLP that maps target poses to
// K joint-space proposals, trained and run on the tensor cores (tc_gemm.cuh).
//
// Features of one target pose (3x4 [R | t]): t (3) then the first two columns
// of R ([r00 r10 r20 r01 r11 r21]); k targets give 9k inputs, zero-padded to a
// multiple of 64.  Hidden layers: `depth` x `width` with SiLU; output layer
// K * n (padded to a multiple of 64); head q = mid + half * tanh(y) per joint.
// Loss per sample: min_k |q_k - q*|^2 + mu * mean_k |q_k - q*|^2.  AdamW with
// FP32 master weights; BF16 copies W [out][in] (forward) and W^T [in][out]
// (input gradients).  Training data: uniform random in-limit configurations
// drawn on the device with a counter-based SplitMix64 generator, their forward
// kinematics (the features) and themselves (the labels).
#include <cudaTypedefs.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <random>
#include <vector>

#include "pk_internal.h"
#include "pk_math.cuh"
#include "mlp_fused.cuh"
#include "tc_gemm.cuh"

using pk::tc::Epilogue;

struct pk_seednet {
  const pk::RobotDev* d_robot = nullptr;
  int n_dof = 0, n_joints = 0;
  int k = 0;                      // targets per sample
  int links[16] = {};
  int K = 0, width = 0, depth = 0;
  int in_dim = 0, in_pad = 0, out_dim = 0, out_pad = 0;
  int L = 0;                      // layers = depth + 1
  std::vector<int> din, dout;     // padded dims per layer
  std::vector<size_t> w_off, b_off;  // offsets into the FP32 parameter buffers
  size_t n_master = 0;            // padded parameter count
  float* master = nullptr;        // FP32 [n_master]
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  std::vector<__nv_bfloat16*> W, Wt;
  std::vector<float> lo, hi;      // joint limits per dof
  float* d_lohi = nullptr;        // [2][n]
  int* d_links = nullptr;
  int* d_err = nullptr;
  float* d_loss = nullptr;
  int64_t step = 0;
  uint64_t seed = 0;
  // activation buffers, sized for `cap_rows` rows
  int cap_rows = 0;
  __nv_bfloat16 *X = nullptr, *Xt = nullptr, *dY = nullptr, *dYt = nullptr;
  std::vector<__nv_bfloat16*> A, At;  // per hidden layer
  std::vector<float*> Z;
  __nv_bfloat16 *dZ[2] = {nullptr, nullptr}, *dZt[2] = {nullptr, nullptr};
  float* Y = nullptr;
  float* qstar = nullptr;
  // LM-refined label pool: (target poses [pool_n][k][12], labels [pool_n][n])
  const pk_robot* robot = nullptr;
  float* pool_T = nullptr;
  float* pool_q = nullptr;
  int pool_n = 0, pool_cap = 0;
  int64_t refine_round = 0;
  int* d_count = nullptr;
};

namespace {

std::mutex g_map_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

pk_status sn_fail(pk_status s, const char* msg) { return pk::set_error(s, msg); }

pk_status sn_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PK_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return sn_fail(e == cudaErrorMemoryAllocation ? PK_ERR_OOM : PK_ERR_CUDA, buf);
}

bool get_encode() {
  std::lock_guard<std::mutex> lk(g_map_mu);
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return true;
}

#ifndef PK_TMA_STORE
#define PK_TMA_STORE 1
#endif

// 2-D BF16 tensor map over a row-major [rows][cols] matrix, box 64 x box_rows,
// 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output map of the SiLU epilogue: BF16 [rows][cols] row-major, 32 x 32 boxes,
// no swizzle (the epilogue writes plain row-major tiles).
bool make_store_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols) {
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t gemm_launch(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc, int a_rows, int b_rows,
                        int K, int splits, const Epilogue& ep, int* d_err, cudaStream_t st) {
  using Lay = pk::tc::SmemLayout<BN>;
  static int sms = 0;
  if (!sms) {
    cudaError_t e = cudaFuncSetAttribute(pk::tc::gemm_bf16_tc_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kBytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int nkb = K / pk::tc::kBK;
  if (splits < 1) splits = 1;
  if (splits > nkb) splits = nkb;
  const int per = (nkb + splits - 1) / splits;
  splits = (nkb + per - 1) / per;
  const int m_tiles = a_rows / pk::tc::kBM, n_tiles = b_rows / BN;
  const int tiles = m_tiles * n_tiles * splits;
  const int grid = tiles < sms ? tiles : sms;
  pk::TraceScope tr(ep.mode == pk::tc::EPI_WGRAD_ADD ? "gemm_wgrad" : "gemm", st);
  pk::tc::gemm_bf16_tc_kernel<BN><<<grid, pk::tc::kThreads, Lay::kBytes, st>>>(ma, mb, mc, m_tiles, n_tiles,
                                                                              splits, K, per, ep, d_err);
  return cudaGetLastError();
}

// D[a_rows x b_rows] = A[a_rows x K] B[b_rows x K]^T with epilogue `ep`.
cudaError_t gemm(const __nv_bfloat16* A, int a_rows, const __nv_bfloat16* B, int b_rows, int K, int splits,
                 const Epilogue& ep, int* d_err, cudaStream_t st) {
  const int BN = (b_rows % 256 == 0) ? 256 : (b_rows % 128 == 0) ? 128 : 64;
  CUtensorMap ma, mb, mc;
  if (!make_map(&ma, A, a_rows, K, pk::tc::kBM) || !make_map(&mb, B, b_rows, K, BN))
    return cudaErrorInvalidValue;
  Epilogue e2 = ep;
  e2.tma_store = 0;
  mc = ma;  // unused unless the SiLU epilogue stores through it
  if (ep.mode == pk::tc::EPI_FWD_SILU && PK_TMA_STORE && ep.out_bf16 && ep.ld_bf16 == b_rows &&
      ep.m_valid == a_rows && (((uintptr_t)ep.out_bf16) & 15) == 0) {
    if (!make_store_map(&mc, ep.out_bf16, a_rows, b_rows)) return cudaErrorInvalidValue;
    e2.tma_store = 1;
  }
  if (BN == 256) return gemm_launch<256>(ma, mb, mc, a_rows, b_rows, K, splits, e2, d_err, st);
  if (BN == 128) return gemm_launch<128>(ma, mb, mc, a_rows, b_rows, K, splits, e2, d_err, st);
  return gemm_launch<64>(ma, mb, mc, a_rows, b_rows, K, splits, e2, d_err, st);
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Uniform in [0, 1) from the counter-based generator: the 24 high bits of
// SplitMix64(seed + counter * golden gamma).
__device__ __forceinline__ float uniform01(uint64_t seed, uint64_t counter) {
  const uint64_t r = splitmix64(seed + counter * 0x9e3779b97f4a7c15ull);
  return (float)(r >> 40) * (1.0f / 16777216.0f);
}

// Frame of joint `link` by generic tree FK (frames kept in local memory).
__device__ void tree_fk_link(const pk::RobotDev* __restrict__ rb, const float* q, int link, pk::Rt& out,
                             pk::Rt* frames) {
  for (int j = 0; j <= link; ++j) {
    pk::Rt O, X, Lm;
    pk::rt_load(rb->origin[j], O);
    pk::rt_identity(X);
    const int t = rb->type[j];
    if (t != PK_JOINT_FIXED) {
      const float qv = fmaf(rb->mult[j], q[rb->var[j]], rb->offs[j]);
      const float* a = rb->axis[j];
      if (t == PK_JOINT_REVOLUTE) {
        float u[3] = {a[0], a[1], a[2]}, s, c;
        pk::sincos_rad(qv, &s, &c);
        pk::rot_joint(X.r, u, a, s, c);
      } else {
        X.t[0] = a[0] * qv; X.t[1] = a[1] * qv; X.t[2] = a[2] * qv;
      }
    }
    pk::rt_mul(O, X, Lm);
    const int p = rb->parent[j];
    if (p >= 0) pk::rt_mul(frames[p], Lm, Lm);
    frames[j] = Lm;
  }
  out = frames[link];
}

__device__ __forceinline__ void pose_features(const pk::Rt& T, float* f) {
  f[0] = T.t[0]; f[1] = T.t[1]; f[2] = T.t[2];
  f[3] = T.r[0]; f[4] = T.r[3]; f[5] = T.r[6];
  f[6] = T.r[1]; f[7] = T.r[4]; f[8] = T.r[7];
}

// One row of features: 16-byte stores into X (8 BF16 at a time), scalar
// stores into the transposed copy used by the weight gradient.
__device__ __forceinline__ void store_features(const float* f, int in_dim, int in_pad, int row, int m_pad,
                                               __nv_bfloat16* X, __nv_bfloat16* Xt) {
  uint4* xr = reinterpret_cast<uint4*>(X + (size_t)row * in_pad);
  for (int c = 0; c < in_pad; c += 8) {
    uint4 pk4;
    uint32_t* w = reinterpret_cast<uint32_t*>(&pk4);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = c + 2 * i;
      __nv_bfloat162 h = __floats2bfloat162_rn(a < in_dim ? f[a] : 0.f, a + 1 < in_dim ? f[a + 1] : 0.f);
      w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    xr[c / 8] = pk4;
  }
  if (Xt)
    for (int i = 0; i < in_pad; ++i) Xt[(size_t)i * m_pad + row] = __float2bfloat16_rn(i < in_dim ? f[i] : 0.f);
}

// Features of given target poses [B][k][12]; rows >= B are zero.
__global__ void features_kernel(const float* __restrict__ targets, int B, int k, int in_pad, int m_pad,
                                __nv_bfloat16* X, __nv_bfloat16* Xt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m_pad) return;
  float f[9 * 16];
  const int in_dim = 9 * k;
  for (int t = 0; t < k; ++t) {
    pk::Rt T;
    if (b < B) {
      pk::rt_load(targets + ((size_t)b * k + t) * 12, T);
      pose_features(T, f + 9 * t);
    } else {
      for (int i = 0; i < 9; ++i) f[9 * t + i] = 0.f;
    }
  }
  store_features(f, in_dim, in_pad, b, m_pad, X, Xt);
}

// Training samples: q* uniform in the limits, features of FK(q*).
__global__ void datagen_kernel(const pk::RobotDev* __restrict__ rb, const int* __restrict__ links, int k,
                               const float* __restrict__ lohi, int n, uint64_t seed, int64_t step, int M,
                               int in_pad, int m_pad, __nv_bfloat16* X, __nv_bfloat16* Xt, float* qstar) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m_pad) return;
  float q[pk::kMaxJoints];
  float f[9 * 16];
  if (b < M) {
    const uint64_t base = ((uint64_t)step * (uint64_t)M + (uint64_t)b) * (uint64_t)n;
    for (int j = 0; j < n; ++j) {
      const float lo = lohi[j], hi = lohi[n + j];
      q[j] = lo + (hi - lo) * uniform01(seed, base + j);
      qstar[(size_t)b * n + j] = q[j];
    }
    pk::Rt frames[pk::kMaxJoints];
    for (int t = 0; t < k; ++t) {
      pk::Rt T;
      tree_fk_link(rb, q, links[t], T, frames);
      pose_features(T, f + 9 * t);
    }
  } else {
    for (int i = 0; i < 9 * k; ++i) f[i] = 0.f;
  }
  store_features(f, 9 * k, in_pad, b, m_pad, X, Xt);
}

// Fresh refinement targets: q uniform in the limits (generator keyed by the
// training seed and the refinement round, disjoint from the training draws)
// and the poses of the target frames, [M][k][12].
__global__ void refine_targets_kernel(const pk::RobotDev* __restrict__ rb, const int* __restrict__ links, int k,
                                      const float* __restrict__ lohi, int n, uint64_t key, int M, float* T_out,
                                      float* q_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= M) return;
  float q[pk::kMaxJoints];
  for (int j = 0; j < n; ++j) {
    const float lo = lohi[j], hi = lohi[n + j];
    q[j] = lo + (hi - lo) * uniform01(key, (uint64_t)b * n + j);
    q_out[(size_t)b * n + j] = q[j];
  }
  pk::Rt frames[pk::kMaxJoints];
  for (int t = 0; t < k; ++t) {
    pk::Rt T;
    tree_fk_link(rb, q, links[t], T, frames);
    float* o = T_out + ((size_t)b * k + t) * 12;
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) o[r * 4 + c] = T.r[r * 3 + c];
      o[r * 4 + 3] = T.t[r];
    }
  }
}

// Pool labels: the LM solution where the refinement converged (it becomes the
// label), else the drawn configuration (already in pool_q).
__global__ void refine_label_kernel(int M, int n, const int32_t* __restrict__ status, const float* __restrict__ q_lm,
                                    float* pool_q, int* count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= M || status[b] != PK_P_CONVERGED) return;
  for (int j = 0; j < n; ++j) pool_q[(size_t)b * n + j] = q_lm[(size_t)b * n + j];
  atomicAdd(count, 1);
}

// Rows [0, r0) of a training batch drawn from the label pool (row b takes pool
// entry hash(key, step, b) mod pool_n); datagen_kernel fills the others.
__global__ void pool_rows_kernel(const float* __restrict__ pool_T, const float* __restrict__ pool_q, int pool_n,
                                 int k, int n, uint64_t key, int64_t step, int r0, int in_pad, int m_pad,
                                 __nv_bfloat16* X, __nv_bfloat16* Xt, float* qstar) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= r0) return;
  const uint64_t h = splitmix64(key + ((uint64_t)step * (uint64_t)r0 + (uint64_t)b) * 0x9e3779b97f4a7c15ull);
  const int idx = (int)(h % (uint64_t)pool_n);
  float f[9 * 16];
  for (int t = 0; t < k; ++t) {
    pk::Rt T;
    pk::rt_load(pool_T + ((size_t)idx * k + t) * 12, T);
    pose_features(T, f + 9 * t);
  }
  store_features(f, 9 * k, in_pad, b, m_pad, X, Xt);
  for (int j = 0; j < n; ++j) qstar[(size_t)b * n + j] = pool_q[(size_t)idx * n + j];
}

// Head, min-over-K loss and dL/dy (scaled by 1/M) for M valid rows.
__global__ void head_loss_kernel(const float* __restrict__ Y, int ldy, int M, int m_pad, int K, int n,
                                 const float* __restrict__ lohi, const float* __restrict__ qstar, float mu,
                                 __nv_bfloat16* dY, int ld_dy, __nv_bfloat16* dYt, float* loss_sum) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m_pad) return;
  if (b >= M) {
    for (int i = 0; i < ld_dy; ++i) {
      dY[(size_t)b * ld_dy + i] = __float2bfloat16_rn(0.f);
      dYt[(size_t)i * m_pad + b] = __float2bfloat16_rn(0.f);
    }
    return;
  }
  const float* y = Y + (size_t)b * ldy;
  const float* qs = qstar + (size_t)b * n;
  float e[64];
  int best = 0;
  float mean = 0.f;
  for (int kk = 0; kk < K; ++kk) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) {
      const float lo = lohi[i], hi = lohi[n + i];
      const float q = 0.5f * (lo + hi) + 0.5f * (hi - lo) * tanhf(y[kk * n + i]);
      s = fmaf(q - qs[i], q - qs[i], s);
    }
    e[kk] = s;
    mean += s / K;
    if (s < e[best]) best = kk;
  }
  atomicAdd(loss_sum, e[best] + mu * mean);
  const float invM = 1.f / (float)M;
  for (int kk = 0; kk < K; ++kk) {
    const float w = (kk == best ? 1.f : 0.f) + mu / K;
    for (int i = 0; i < n; ++i) {
      const float lo = lohi[i], hi = lohi[n + i];
      const float t = tanhf(y[kk * n + i]);
      const float q = 0.5f * (lo + hi) + 0.5f * (hi - lo) * t;
      const float g = w * 2.f * (q - qs[i]) * 0.5f * (hi - lo) * (1.f - t * t) * invM;
      const __nv_bfloat16 h = __float2bfloat16_rn(g);
      dY[(size_t)b * ld_dy + kk * n + i] = h;
      dYt[(size_t)(kk * n + i) * m_pad + b] = h;
    }
  }
  for (int i = K * n; i < ld_dy; ++i) {
    dY[(size_t)b * ld_dy + i] = __float2bfloat16_rn(0.f);
    dYt[(size_t)i * m_pad + b] = __float2bfloat16_rn(0.f);
  }
}

// db[r] = sum over the m_pad columns of G^T row r (one warp per row).
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ Gt, int rows, int m_pad, float* db) {
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  float s = 0.f;
  for (int i = lane; i < m_pad; i += 32) s += __bfloat162float(Gt[(size_t)r * m_pad + i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) db[r] = s;
}

__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1,
                             float b2, float eps, float wd, float c1, float c2) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
}

// BF16 copies of one layer's weights: W [out][in] and W^T [in][out].
__global__ void cast_weights_kernel(const float* __restrict__ w, int out, int in, __nv_bfloat16* W,
                                    __nv_bfloat16* Wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= out * in) return;
  const int o = i / in, c = i % in;
  const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
  W[i] = h;
  Wt[(size_t)c * out + o] = h;
}

// ---------------------------------------------------------------- host helpers

void free_acts(pk_seednet* s) {
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(s->X); f(s->Xt); f(s->dY); f(s->dYt); f(s->Y); f(s->qstar);
  for (auto* p : s->A) f(p);
  for (auto* p : s->At) f(p);
  for (auto* p : s->Z) f(p);
  for (int i = 0; i < 2; ++i) { f(s->dZ[i]); f(s->dZt[i]); }
  s->X = s->Xt = s->dY = s->dYt = nullptr;
  s->Y = s->qstar = nullptr;
  s->A.assign(s->depth, nullptr);
  s->At.assign(s->depth, nullptr);
  s->Z.assign(s->depth, nullptr);
  s->dZ[0] = s->dZ[1] = s->dZt[0] = s->dZt[1] = nullptr;
  s->cap_rows = 0;
}

// Activation buffers for m_pad rows (training buffers included).
pk_status ensure_acts(pk_seednet* s, int m_pad) {
  if (s->cap_rows >= m_pad) return PK_OK;
  free_acts(s);
  const size_t H = s->width;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  al((void**)&s->X, (size_t)m_pad * s->in_pad * 2);
  al((void**)&s->Xt, (size_t)m_pad * s->in_pad * 2);
  al((void**)&s->dY, (size_t)m_pad * s->out_pad * 2);
  al((void**)&s->dYt, (size_t)m_pad * 128 * 2);
  al((void**)&s->Y, (size_t)m_pad * s->out_pad * 4);
  al((void**)&s->qstar, (size_t)m_pad * s->n_dof * 4);
  for (int l = 0; l < s->depth; ++l) {
    al((void**)&s->A[l], (size_t)m_pad * H * 2);
    al((void**)&s->At[l], (size_t)m_pad * H * 2);
    al((void**)&s->Z[l], (size_t)m_pad * H * 4);
  }
  for (int i = 0; i < 2; ++i) {
    al((void**)&s->dZ[i], (size_t)m_pad * H * 2);
    al((void**)&s->dZt[i], (size_t)m_pad * H * 2);
  }
  if (e == cudaSuccess) e = cudaMemset(s->dYt, 0, (size_t)m_pad * 128 * 2);
  if (e != cudaSuccess) {
    free_acts(s);
    return sn_cuda(e, "seednet activation buffers");
  }
  s->cap_rows = m_pad;
  return PK_OK;
}

cudaError_t cast_all(pk_seednet* s, cudaStream_t st) {
  for (int l = 0; l < s->L; ++l) {
    const int n = s->dout[l] * s->din[l];
    cast_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(s->master + s->w_off[l], s->dout[l], s->din[l], s->W[l],
                                                         s->Wt[l]);
  }
  return cudaGetLastError();
}

// Forward pass of m_pad rows whose features are in s->X (m_valid real rows).
// With `train`, pre-activations and transposed activations are kept.
cudaError_t forward(pk_seednet* s, int m_valid, int m_pad, bool train, cudaStream_t st,
                    float* seeds_out = nullptr) {
  const __nv_bfloat16* a = s->X;
  int K = s->in_pad;
  for (int l = 0; l < s->depth; ++l) {
    Epilogue ep{};
    ep.mode = pk::tc::EPI_FWD_SILU;
    ep.m_valid = m_pad;  // padded rows are zero features; keep them finite
    ep.bias = s->master + s->b_off[l];
    ep.out_f32 = train ? s->Z[l] : nullptr;
    ep.ld_f32 = s->width;
    ep.out_bf16 = s->A[l];
    ep.ld_bf16 = s->width;
    ep.out_t = train ? s->At[l] : nullptr;
    ep.ld_t = m_pad;
    cudaError_t e = gemm(a, m_pad, s->W[l], s->width, K, 1, ep, s->d_err, st);
    if (e != cudaSuccess) return e;
    a = s->A[l];
    K = s->width;
  }
  Epilogue ep{};
  ep.mode = seeds_out ? pk::tc::EPI_SEEDS : pk::tc::EPI_FWD_LINEAR;
  ep.m_valid = m_valid;
  ep.n_valid = seeds_out ? s->out_dim : s->out_pad;
  ep.bias = s->master + s->b_off[s->depth];
  ep.out_f32 = seeds_out ? seeds_out : s->Y;
  ep.ld_f32 = seeds_out ? s->out_dim : s->out_pad;
  ep.lohi = s->d_lohi;
  ep.n_dof = s->n_dof;
  return gemm(a, m_pad, s->W[s->depth], s->out_pad, K, 1, ep, s->d_err, st);
}

// Backward pass (gradients into s->grad) from dY / dYt; features in X / Xt.
cudaError_t backward(pk_seednet* s, int m_pad, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(s->grad, 0, s->n_master * sizeof(float), st);
  if (e != cudaSuccess) return e;
  const int splits = m_pad / 64 >= 16 ? 16 : 1;
  const int D = s->depth;
  // last layer: dW = dY^T A_{D-1}, db = column sums of dY
  {
    Epilogue ep{};
    ep.mode = pk::tc::EPI_WGRAD_ADD;
    ep.m_valid = s->out_pad;
    ep.out_f32 = s->grad + s->w_off[D];
    ep.ld_f32 = s->width;
    if ((e = gemm(s->dYt, 128, s->At[D - 1], s->width, m_pad, splits, ep, s->d_err, st)) != cudaSuccess) return e;
    bias_grad_kernel<<<(s->out_pad + 7) / 8, 256, 0, st>>>(s->dYt, s->out_pad, m_pad, s->grad + s->b_off[D]);
  }
  // dZ_{D-1} = (dY W_D) * silu'(Z_{D-1})
  const __nv_bfloat16* g = s->dY;
  int gk = s->out_pad;
  int cur = 0;
  for (int l = D - 1; l >= 0; --l) {
    Epilogue ep{};
    ep.mode = pk::tc::EPI_DGRAD_SILU;
    ep.m_valid = m_pad;
    ep.zprev = s->Z[l];
    ep.ld_zprev = s->width;
    ep.out_bf16 = s->dZ[cur];
    ep.ld_bf16 = s->width;
    ep.out_t = s->dZt[cur];
    ep.ld_t = m_pad;
    if ((e = gemm(g, m_pad, s->Wt[l + 1], s->width, gk, 1, ep, s->d_err, st)) != cudaSuccess) return e;
    // layer l weights: dW_l = dZ_l^T A_{l-1} (A_{-1} = X)
    Epilogue ew{};
    ew.mode = pk::tc::EPI_WGRAD_ADD;
    ew.m_valid = s->width;
    ew.out_f32 = s->grad + s->w_off[l];
    ew.ld_f32 = s->din[l];
    const __nv_bfloat16* prev_t = l > 0 ? s->At[l - 1] : s->Xt;
    if ((e = gemm(s->dZt[cur], s->width, prev_t, s->din[l], m_pad, splits, ew, s->d_err, st)) != cudaSuccess)
      return e;
    bias_grad_kernel<<<(s->width + 7) / 8, 256, 0, st>>>(s->dZt[cur], s->width, m_pad, s->grad + s->b_off[l]);
    g = s->dZ[cur];
    gk = s->width;
    cur ^= 1;
  }
  return cudaGetLastError();
}

cudaError_t loss_and_grad(pk_seednet* s, int M, int m_pad, float mu, cudaStream_t st) {
  cudaError_t e = forward(s, M, m_pad, true, st);
  if (e != cudaSuccess) return e;
  head_loss_kernel<<<(m_pad + 127) / 128, 128, 0, st>>>(s->Y, s->out_pad, M, m_pad, s->K, s->n_dof, s->d_lohi,
                                                        s->qstar, mu, s->dY, s->out_pad, s->dYt, s->d_loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return backward(s, m_pad, st);
}

cudaError_t adamw(pk_seednet* s, const pk_train_params* tp, float lr, cudaStream_t st) {
  s->step += 1;
  const float c1 = 1.f - powf(tp->beta1, (float)s->step), c2 = 1.f - powf(tp->beta2, (float)s->step);
  adamw_kernel<<<(unsigned)((s->n_master + 255) / 256), 256, 0, st>>>(s->master, s->grad, s->adam_m, s->adam_v,
                                                                     s->n_master, lr, tp->beta1, tp->beta2,
                                                                     tp->eps, tp->weight_decay, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cast_all(s, st);
}

pk_status check_err(pk_seednet* s, cudaStream_t st) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, s->d_err, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sn_cuda(e, "seednet");
  if (h != 0) {
    cudaMemsetAsync(s->d_err, 0, sizeof(int), st);
    char buf[128];
    snprintf(buf, sizeof buf, "tensor-core GEMM pipeline wait timed out (code %d)", h);
    return sn_fail(PK_ERR_TIMEOUT, buf);
  }
  return PK_OK;
}

// oracle-layout <-> padded-layout parameter copies
size_t oracle_count(const pk_seednet* s) {
  size_t n = 0;
  for (int l = 0; l < s->L; ++l) {
    const int i = l == 0 ? s->in_dim : s->width;
    const int o = l == s->L - 1 ? s->out_dim : s->width;
    n += (size_t)o * i + o;
  }
  return n;
}

// A padded FP32 device buffer of the parameter layout (master weights, AdamW
// moments) to and from the unpadded host order of pk_seednet_get_params: per
// layer W [out][in] row-major, then b [out].
pk_status device_to_layout(const pk_seednet* s, const float* dev, float* host, const char* what) {
  std::vector<float> h(s->n_master);
  cudaError_t e = cudaMemcpy(h.data(), dev, s->n_master * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sn_cuda(e, what);
  size_t o = 0;
  for (int l = 0; l < s->L; ++l) {
    const int fi = l == 0 ? s->in_dim : s->width;
    const int fo = l == s->L - 1 ? s->out_dim : s->width;
    for (int r = 0; r < fo; ++r)
      for (int c = 0; c < fi; ++c) host[o++] = h[s->w_off[l] + (size_t)r * s->din[l] + c];
    for (int r = 0; r < fo; ++r) host[o++] = h[s->b_off[l] + r];
  }
  return PK_OK;
}

cudaError_t layout_to_device(const pk_seednet* s, const float* host, float* dev) {
  std::vector<float> h(s->n_master, 0.f);
  size_t o = 0;
  for (int l = 0; l < s->L; ++l) {
    const int fi = l == 0 ? s->in_dim : s->width;
    const int fo = l == s->L - 1 ? s->out_dim : s->width;
    for (int r = 0; r < fo; ++r)
      for (int c = 0; c < fi; ++c) h[s->w_off[l] + (size_t)r * s->din[l] + c] = host[o++];
    for (int r = 0; r < fo; ++r) h[s->b_off[l] + r] = host[o++];
  }
  return cudaMemcpy(dev, h.data(), s->n_master * 4, cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

void pk_train_params_default(pk_train_params* p) {
  if (!p) return;
  p->epochs = 8;
  p->batch = 8192;
  p->steps_per_epoch = 1220;
  p->lr = 1e-3f;
  p->weight_decay = 1e-4f;
  p->beta1 = 0.9f;
  p->beta2 = 0.999f;
  p->eps = 1e-8f;
  p->mu = 0.01f;
  p->refine_every = 0;
  p->first_epoch = 0;
  p->last_epoch = 0;
  p->seed = 500;
  p->refine_n = 65536;
  p->refine_iters = 20;
  p->pool_frac = 0.5f;
}

pk_status pk_seednet_create(const pk_robot* rb, int32_t k, const int32_t* target_links, int32_t K,
                            int32_t width, int32_t depth, uint64_t seed, pk_seednet** out) {
  if (!out) return sn_fail(PK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!rb || !target_links) return sn_fail(PK_ERR_INVALID_ARG, "robot or target_links is NULL");
  if (k < 1 || k > 16) return sn_fail(PK_ERR_INVALID_ARG, "k must be in 1..16");
  for (int i = 0; i < k; ++i)
    if (target_links[i] < 0 || target_links[i] >= rb->n_joints)
      return sn_fail(PK_ERR_INVALID_ARG, "target link out of range");
  if (K < 1 || K > 64) return sn_fail(PK_ERR_INVALID_ARG, "K must be in 1..64");
  if (width < 64 || width % 256 != 0 || width > 2048)
    return sn_fail(PK_ERR_INVALID_ARG, "width must be a multiple of 256 in 256..2048");
  if (depth < 1 || depth > 8) return sn_fail(PK_ERR_INVALID_ARG, "depth must be in 1..8");
  if (K * rb->n_dof > 1024) return sn_fail(PK_ERR_INVALID_ARG, "K * n_dof must be <= 1024");
  if (!get_encode()) return sn_fail(PK_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  pk_seednet* s = new (std::nothrow) pk_seednet;
  if (!s) return sn_fail(PK_ERR_OOM, "host allocation failed");
  s->d_robot = (const pk::RobotDev*)rb->d_blob;
  s->robot = rb;
  s->n_dof = rb->n_dof;
  s->n_joints = rb->n_joints;
  s->k = k;
  memcpy(s->links, target_links, k * sizeof(int));
  s->K = K;
  s->width = width;
  s->depth = depth;
  s->L = depth + 1;
  s->in_dim = 9 * k;
  s->in_pad = round_up(s->in_dim, 64);
  s->out_dim = K * rb->n_dof;
  s->out_pad = round_up(s->out_dim, 64);
  s->seed = seed;
  for (int l = 0; l < s->L; ++l) {
    s->din.push_back(l == 0 ? s->in_pad : width);
    s->dout.push_back(l == s->L - 1 ? s->out_pad : width);
  }
  size_t off = 0;
  for (int l = 0; l < s->L; ++l) {
    s->w_off.push_back(off);
    off += (size_t)s->dout[l] * s->din[l];
    s->b_off.push_back(off);
    off += s->dout[l];
  }
  s->n_master = off;
  for (int j = 0; j < rb->n_joints; ++j)
    if (rb->var[j] >= 0 && rb->mimic[j] < 0) {  // the variables' own joints
      s->lo.push_back(rb->lower[j]);
      s->hi.push_back(rb->upper[j]);
    }
  // initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) on the real entries, zero padding
  std::vector<float> h(s->n_master, 0.f);
  std::mt19937_64 gen(seed);
  for (int l = 0; l < s->L; ++l) {
    const int fi = l == 0 ? s->in_dim : width;
    const int fo = l == s->L - 1 ? s->out_dim : width;
    const float bound = 1.f / sqrtf((float)fi);
    std::uniform_real_distribution<float> U(-bound, bound);
    for (int o = 0; o < fo; ++o) {
      for (int i = 0; i < fi; ++i) h[s->w_off[l] + (size_t)o * s->din[l] + i] = U(gen);
      h[s->b_off[l] + o] = U(gen);
    }
  }
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  al((void**)&s->master, s->n_master * 4);
  al((void**)&s->grad, s->n_master * 4);
  al((void**)&s->adam_m, s->n_master * 4);
  al((void**)&s->adam_v, s->n_master * 4);
  s->W.assign(s->L, nullptr);
  s->Wt.assign(s->L, nullptr);
  for (int l = 0; l < s->L; ++l) {
    al((void**)&s->W[l], (size_t)s->dout[l] * s->din[l] * 2);
    al((void**)&s->Wt[l], (size_t)s->dout[l] * s->din[l] * 2);
  }
  al((void**)&s->d_lohi, 2 * s->n_dof * 4);
  al((void**)&s->d_links, 16 * 4);
  al((void**)&s->d_err, 4);
  al((void**)&s->d_loss, 4);
  al((void**)&s->d_count, 4);
  s->A.assign(depth, nullptr);
  s->At.assign(depth, nullptr);
  s->Z.assign(depth, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(s->master, h.data(), s->n_master * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, s->n_master * 4);
  if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, s->n_master * 4);
  if (e == cudaSuccess) e = cudaMemset(s->d_err, 0, 4);
  std::vector<float> lohi(s->lo);
  lohi.insert(lohi.end(), s->hi.begin(), s->hi.end());
  if (e == cudaSuccess) e = cudaMemcpy(s->d_lohi, lohi.data(), lohi.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_links, s->links, 16 * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cast_all(s, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    pk_seednet_destroy(s);
    return sn_cuda(e, "pk_seednet_create");
  }
  *out = s;
  return PK_OK;
}

void pk_seednet_destroy(pk_seednet* s) {
  if (!s) return;
  free_acts(s);
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(s->master); f(s->grad); f(s->adam_m); f(s->adam_v); f(s->d_lohi); f(s->d_links); f(s->d_err); f(s->d_loss);
  f(s->d_count); f(s->pool_T); f(s->pool_q);
  for (auto* p : s->W) f(p);
  for (auto* p : s->Wt) f(p);
  delete s;
}

int64_t pk_seednet_n_params(const pk_seednet* s) { return s ? (int64_t)oracle_count(s) : -1; }

pk_status pk_seednet_get_params(const pk_seednet* s, float* host, int64_t n) {
  if (!s || !host) return sn_fail(PK_ERR_INVALID_ARG, "NULL argument");
  if ((size_t)n != oracle_count(s)) return sn_fail(PK_ERR_INVALID_ARG, "parameter count mismatch");
  return device_to_layout(s, s->master, host, "pk_seednet_get_params");
}

pk_status pk_seednet_set_params(pk_seednet* s, const float* host, int64_t n) {
  if (!s || !host) return sn_fail(PK_ERR_INVALID_ARG, "NULL argument");
  if ((size_t)n != oracle_count(s)) return sn_fail(PK_ERR_INVALID_ARG, "parameter count mismatch");
  cudaError_t e = layout_to_device(s, host, s->master);
  if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, s->n_master * 4);
  if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, s->n_master * 4);
  if (e == cudaSuccess) e = cast_all(s, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  s->step = 0;
  return sn_cuda(e, "pk_seednet_set_params");
}

// File layout of pk_seednet_save / pk_seednet_load (host byte order): the
// header below, the FP32 parameters (pk_seednet_get_params order), and from
// version 2 on the training state: step and refinement-round counters, the
// AdamW first and second moments (parameter order), the label pool's target
// poses [pool_n][k][12] and labels [pool_n][n_dof].
// Version 1 files (parameters only) still load.
namespace {
struct SeednetFileHeader {
  char magic[4];     // "PKSN"
  uint32_t version;  // 1 or 2
  int32_t k, K, n_dof, in_dim, out_dim, width, depth, reserved;
  int64_t n_params;
};
struct SeednetFileState {  // version 2, after the parameters
  int64_t step;            // AdamW step count, also the training data generator's counter
  int64_t refine_round;    // refinement rounds so far (keys the next round's targets)
  int32_t pool_n;          // label-pool rows
  int32_t reserved;
};

bool write_all(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, bytes, 1, f) == 1; }
bool read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, bytes, 1, f) == 1; }
}  // namespace

pk_status pk_seednet_save(const pk_seednet* s, const char* path) {
  if (!s || !path) return sn_fail(PK_ERR_INVALID_ARG, "NULL argument");
  const int64_t n = (int64_t)oracle_count(s);
  std::vector<float> h((size_t)n), m((size_t)n), v((size_t)n);
  pk_status st = device_to_layout(s, s->master, h.data(), "pk_seednet_save");
  if (st == PK_OK) st = device_to_layout(s, s->adam_m, m.data(), "pk_seednet_save");
  if (st == PK_OK) st = device_to_layout(s, s->adam_v, v.data(), "pk_seednet_save");
  if (st != PK_OK) return st;
  const size_t pT = (size_t)s->pool_n * s->k * 12, pq = (size_t)s->pool_n * s->n_dof;
  std::vector<float> poolT(pT), poolq(pq);
  cudaError_t e = cudaSuccess;
  if (s->pool_n > 0) {
    e = cudaMemcpy(poolT.data(), s->pool_T, pT * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(poolq.data(), s->pool_q, pq * 4, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_save");
  SeednetFileHeader hd{};
  memcpy(hd.magic, "PKSN", 4);
  hd.version = 2;
  hd.k = s->k;
  hd.K = s->K;
  hd.n_dof = s->n_dof;
  hd.in_dim = s->in_dim;
  hd.out_dim = s->out_dim;
  hd.width = s->width;
  hd.depth = s->depth;
  hd.n_params = n;
  SeednetFileState fs{};
  fs.step = s->step;
  fs.refine_round = s->refine_round;
  fs.pool_n = s->pool_n;
  FILE* f = fopen(path, "wb");
  if (!f) return sn_fail(PK_ERR_INVALID_ARG, "pk_seednet_save: cannot open the file for writing");
  const size_t nb = (size_t)n * 4;
  const bool ok = write_all(f, &hd, sizeof hd) && write_all(f, h.data(), nb) && write_all(f, &fs, sizeof fs) &&
                  write_all(f, m.data(), nb) && write_all(f, v.data(), nb) && write_all(f, poolT.data(), pT * 4) &&
                  write_all(f, poolq.data(), pq * 4);
  const bool closed = fclose(f) == 0;
  if (!ok || !closed) return sn_fail(PK_ERR_INVALID_ARG, "pk_seednet_save: write failed");
  return PK_OK;
}

pk_status pk_seednet_load(pk_seednet* s, const char* path) {
  if (!s || !path) return sn_fail(PK_ERR_INVALID_ARG, "NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return sn_fail(PK_ERR_INVALID_ARG, "pk_seednet_load: cannot open the file");
  SeednetFileHeader hd{};
  if (!read_all(f, &hd, sizeof hd) || memcmp(hd.magic, "PKSN", 4) != 0 || (hd.version != 1 && hd.version != 2)) {
    fclose(f);
    return sn_fail(PK_ERR_INVALID_ARG, "pk_seednet_load: not a seed-network file");
  }
  const int64_t n = (int64_t)oracle_count(s);
  if (hd.k != s->k || hd.K != s->K || hd.n_dof != s->n_dof || hd.in_dim != s->in_dim || hd.out_dim != s->out_dim ||
      hd.width != s->width || hd.depth != s->depth || hd.n_params != n) {
    fclose(f);
    return sn_fail(PK_ERR_INVALID_ARG, "pk_seednet_load: the file holds a network of another shape");
  }
  const size_t nb = (size_t)n * 4;
  std::vector<float> h((size_t)n), m, v, poolT, poolq;
  SeednetFileState fs{};
  bool ok = read_all(f, h.data(), nb);
  if (ok && hd.version == 2) {
    ok = read_all(f, &fs, sizeof fs) && fs.pool_n >= 0 && fs.step >= 0 && fs.refine_round >= 0;
    if (ok) {
      m.resize((size_t)n);
      v.resize((size_t)n);
      poolT.resize((size_t)fs.pool_n * s->k * 12);
      poolq.resize((size_t)fs.pool_n * s->n_dof);
      ok = read_all(f, m.data(), nb) && read_all(f, v.data(), nb) && read_all(f, poolT.data(), poolT.size() * 4) &&
           read_all(f, poolq.data(), poolq.size() * 4);
    }
  }
  fclose(f);
  if (!ok) return sn_fail(PK_ERR_INVALID_ARG, "pk_seednet_load: the file is truncated");
  pk_status st = pk_seednet_set_params(s, h.data(), n);  // weights (and their BF16 copies); AdamW state cleared
  if (st != PK_OK || hd.version == 1) return st;
  // the training state: moments, step (and generator position), label pool
  cudaError_t e = layout_to_device(s, m.data(), s->adam_m);
  if (e == cudaSuccess) e = layout_to_device(s, v.data(), s->adam_v);
  if (e == cudaSuccess && fs.pool_n > s->pool_cap) {
    if (s->pool_T) cudaFree(s->pool_T);
    if (s->pool_q) cudaFree(s->pool_q);
    s->pool_T = s->pool_q = nullptr;
    s->pool_cap = s->pool_n = 0;
    e = cudaMalloc(&s->pool_T, poolT.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->pool_q, poolq.size() * 4);
    if (e == cudaSuccess) s->pool_cap = fs.pool_n;
  }
  if (e == cudaSuccess && fs.pool_n > 0) {
    e = cudaMemcpy(s->pool_T, poolT.data(), poolT.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->pool_q, poolq.data(), poolq.size() * 4, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_load");
  s->pool_n = fs.pool_n;
  s->step = fs.step;
  s->refine_round = fs.refine_round;
  return PK_OK;
}

pk_status pk_seednet_forward(pk_seednet* s, int32_t batch, const float* d_targets, float* d_y_out,
                             void* stream) {
  if (!s) return sn_fail(PK_ERR_INVALID_ARG, "net is NULL");
  if (batch < 0) return sn_fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  if (batch == 0) return PK_OK;
  if (!d_targets || !d_y_out) return sn_fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const int m_pad = round_up(batch, 128);
  pk_status ps = ensure_acts(s, m_pad);
  if (ps != PK_OK) return ps;
  features_kernel<<<(m_pad + 127) / 128, 128, 0, st>>>(d_targets, batch, s->k, s->in_pad, m_pad, s->X, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = forward(s, batch, m_pad, false, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(d_y_out, s->out_dim * 4, s->Y, s->out_pad * 4, s->out_dim * 4, batch,
                          cudaMemcpyDeviceToDevice, st);
  return sn_cuda(e, "pk_seednet_forward");
}

namespace {

// The whole-network kernel takes widths 256 and 512 (the accumulator fits
// TMEM's 512 columns), inputs up to 256 and head outputs up to 256 wide.
// PK_SEEDNET_FUSED=0 selects the layer-by-layer GEMMs instead.
bool fused_ok(const pk_seednet* s) {
  const char* env = getenv("PK_SEEDNET_FUSED");
  if (env && env[0] == '0') return false;
  return (s->width == 256 || s->width == 512) && s->in_pad <= 256 && s->out_pad <= 256 &&
         s->L <= pk::tc::kMlpMaxLayers;
}

// 3-D view [din / 64][dout][64] of a BF16 weight matrix W[dout][din], boxes of
// 64 x box_rows x box_kb, 128-byte swizzle: one box is box_kb K-major tiles
// of box_rows x 64, 1024-byte aligned one after the other.
bool make_map_kblocks(CUtensorMap* m, const void* base, uint64_t dout, uint64_t din, uint32_t box_rows,
                      uint32_t box_kb) {
  cuuint64_t dims[3] = {64, dout, din / 64};
  cuuint64_t strides[2] = {din * 2, 128};
  cuuint32_t box[3] = {64, box_rows, box_kb};
  cuuint32_t estr[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// cudaErrorNotSupported: this network or batch does not fit the kernel's
// layout (the caller falls back to the layer-by-layer GEMMs).
cudaError_t infer_fused(pk_seednet* s, int batch, const float* d_targets, float* d_seeds_out, cudaStream_t st) {
  using namespace pk::tc;
  static int sms = 0, max_smem = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  MlpParams p{};
  p.n_layers = s->L;
  p.width = s->width;
  p.in_pad = s->in_pad;
  p.out_pad = s->out_pad;
  p.out_dim = s->out_dim;
  p.n_dof = s->n_dof;
  p.k = s->k;
  p.batch = batch;
  p.tiles = (batch + kBM - 1) / kBM;
  // weight stages: the largest divisor of the layer's K-blocks that keeps a
  // stage within kMlpStageBytes
  for (int l = 0; l < s->L; ++l) {
    const int rows = l == s->L - 1 ? s->out_pad : kMlpChunk, nkb = s->din[l] / 64;
    int kb = kMlpStageBytes / (rows * 128);
    if (kb > nkb) kb = nkb;
    while (nkb % kb) --kb;
    p.stage_kb[l] = kb;
  }
  // ring as deep as shared memory allows next to the keep area (one chunk of
  // BF16 results at width 512; PK_MLP_STAGES caps the ring, for tuning sweeps)
  int cap = kMlpMaxStages;
  if (const char* env = getenv("PK_MLP_STAGES")) cap = atoi(env) > 1 ? atoi(env) : 2;
  if (cap > kMlpMaxStages) cap = kMlpMaxStages;
  const int keep = s->width == 2 * kMlpChunk ? kMlpKeepBytes : 0;
  const int room = max_smem - MlpSmem::bytes(0, keep);
  p.vec4 = (s->out_dim % 4 == 0 && ((uintptr_t)d_seeds_out & 15) == 0) ? 1 : 0;
  p.area_bytes = keep;
  p.stages = room / kMlpStageBytes < cap ? room / kMlpStageBytes : cap;
  if (p.stages < 2) return cudaErrorNotSupported;
  MlpMaps maps;
  for (int l = 0; l < s->L; ++l) {
    const int rows = l == s->L - 1 ? s->out_pad : kMlpChunk;
    if (!make_map_kblocks(&maps.w[l], s->W[l], s->dout[l], s->din[l], rows, p.stage_kb[l])) return cudaErrorNotSupported;
    p.bias[l] = s->master + s->b_off[l];
  }
  p.lohi = s->d_lohi;
  p.targets = d_targets;
  p.seeds = d_seeds_out;
  // the fewest CTAs that keep the number of tile rounds (the busiest CTA sets
  // the launch time), so that the other SMs stay free for concurrent work
  const int rounds = (p.tiles + sms - 1) / sms;
  int grid = (p.tiles + rounds - 1) / rounds;
  if (const char* env = getenv("PK_MLP_GRID"))  // persistent grid size, for tuning sweeps
    if (atoi(env) > 0 && atoi(env) < grid) grid = atoi(env);
  const int smem = MlpSmem::bytes(p.stages, p.area_bytes);
  pk::TraceScope tr("seednet_mlp", st);
  mlp_fused_kernel<<<grid, kMlpThreads, smem, st>>>(maps, p, s->d_err);
  return cudaGetLastError();
}

}  // namespace

pk_status pk_seednet_infer(pk_seednet* s, int32_t batch, const float* d_targets, float* d_seeds_out,
                           void* stream) {
  if (!s) return sn_fail(PK_ERR_INVALID_ARG, "net is NULL");
  if (batch < 0) return sn_fail(PK_ERR_INVALID_ARG, "batch must be >= 0");
  if (batch == 0) return PK_OK;
  if (!d_targets || !d_seeds_out) return sn_fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  cudaStream_t st = (cudaStream_t)stream;
  if (fused_ok(s)) {
    const cudaError_t e = infer_fused(s, batch, d_targets, d_seeds_out, st);
    if (e != cudaErrorNotSupported) return sn_cuda(e, "pk_seednet_infer");
  }
  const int m_pad = round_up(batch, 128);
  pk_status ps = ensure_acts(s, m_pad);
  if (ps != PK_OK) return ps;
  {
    pk::TraceScope tr("features", st);
    features_kernel<<<(m_pad + 127) / 128, 128, 0, st>>>(d_targets, batch, s->k, s->in_pad, m_pad, s->X, nullptr);
  }
  cudaError_t e = cudaGetLastError();
  // the head q = mid + half tanh(y) runs in the output layer's epilogue
  if (e == cudaSuccess) e = forward(s, batch, m_pad, false, st, d_seeds_out);
  return sn_cuda(e, "pk_seednet_infer");
}

pk_status pk_seednet_check(pk_seednet* s, void* stream) {
  if (!s) return sn_fail(PK_ERR_INVALID_ARG, "net is NULL");
  return check_err(s, (cudaStream_t)stream);
}

pk_status pk_seednet_loss_grad(pk_seednet* s, int32_t batch, const float* d_targets, const float* d_qstar,
                               float* host_loss, float* host_grad, void* stream) {
  if (!s) return sn_fail(PK_ERR_INVALID_ARG, "net is NULL");
  if (batch < 1 || !d_targets || !d_qstar || !host_loss || !host_grad)
    return sn_fail(PK_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int m_pad = round_up(batch, 128);
  pk_status ps = ensure_acts(s, m_pad);
  if (ps != PK_OK) return ps;
  features_kernel<<<(m_pad + 127) / 128, 128, 0, st>>>(d_targets, batch, s->k, s->in_pad, m_pad, s->X, s->Xt);
  cudaError_t e = cudaMemcpyAsync(s->qstar, d_qstar, (size_t)batch * s->n_dof * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_loss, 0, 4, st);
  if (e == cudaSuccess) e = loss_and_grad(s, batch, m_pad, 0.01f, st);
  if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_loss_grad");
  if ((ps = check_err(s, st)) != PK_OK) return ps;
  float loss = 0.f;
  std::vector<float> g(s->n_master);
  e = cudaMemcpy(&loss, s->d_loss, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(g.data(), s->grad, s->n_master * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_loss_grad");
  *host_loss = loss / batch;
  size_t o = 0;
  for (int l = 0; l < s->L; ++l) {
    const int fi = l == 0 ? s->in_dim : s->width;
    const int fo = l == s->L - 1 ? s->out_dim : s->width;
    for (int r = 0; r < fo; ++r)
      for (int c = 0; c < fi; ++c) host_grad[o++] = g[s->w_off[l] + (size_t)r * s->din[l] + c];
    for (int r = 0; r < fo; ++r) host_grad[o++] = g[s->b_off[l] + r];
  }
  return PK_OK;
}

pk_status pk_seednet_refine(pk_seednet* s, int32_t n, int32_t max_iters, uint64_t seed, int32_t* n_converged,
                            void* stream) {
  if (!s) return sn_fail(PK_ERR_INVALID_ARG, "net is NULL");
  if (n < 1 || max_iters < 0) return sn_fail(PK_ERR_INVALID_ARG, "need n >= 1 and max_iters >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (n > s->pool_cap) {
    if (s->pool_T) cudaFree(s->pool_T);
    if (s->pool_q) cudaFree(s->pool_q);
    s->pool_T = s->pool_q = nullptr;
    s->pool_cap = s->pool_n = 0;
    e = cudaMalloc(&s->pool_T, (size_t)n * s->k * 12 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->pool_q, (size_t)n * s->n_dof * 4);
    if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_refine (pool)");
    s->pool_cap = n;
  }
  s->pool_n = 0;  // invalid until this round completes
  const int nd = s->n_dof, K = s->K;
  float *seeds = nullptr, *q_lm = nullptr, *err = nullptr;
  int32_t *iters = nullptr, *status = nullptr;
  e = cudaMallocAsync(&seeds, (size_t)n * K * nd * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&q_lm, (size_t)n * nd * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&err, (size_t)n * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&iters, (size_t)n * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&status, (size_t)n * 4, st);
  const uint64_t key = seed ^ (0x7265666eull + 0x9e3779b97f4a7c15ull * (uint64_t)(++s->refine_round));
  if (e == cudaSuccess) {
    refine_targets_kernel<<<(n + 127) / 128, 128, 0, st>>>(s->d_robot, s->d_links, s->k, s->d_lohi, nd, key, n,
                                                           s->pool_T, s->pool_q);
    e = cudaGetLastError();
  }
  pk_status ps = PK_OK;
  if (e == cudaSuccess) ps = pk_seednet_infer(s, n, s->pool_T, seeds, stream);
  if (e == cudaSuccess && ps == PK_OK) {
    pk_ik_params p;
    pk_ik_params_default(&p);
    p.max_iters = max_iters;
    p.early_exit = 1;
    p.cancel_siblings = 1;
    ps = pk_ik_solve(s->robot, &p, s->k, s->links, nullptr, n, K, s->pool_T, seeds, q_lm, err, iters, status,
                     nullptr, 0, stream);
  }
  if (e == cudaSuccess && ps == PK_OK) e = cudaMemsetAsync(s->d_count, 0, 4, st);
  if (e == cudaSuccess && ps == PK_OK) {
    refine_label_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, nd, status, q_lm, s->pool_q, s->d_count);
    e = cudaGetLastError();
  }
  int count = 0;
  if (e == cudaSuccess && ps == PK_OK) e = cudaMemcpyAsync(&count, s->d_count, 4, cudaMemcpyDeviceToHost, st);
  for (void* p : {(void*)seeds, (void*)q_lm, (void*)err, (void*)iters, (void*)status})
    if (p) cudaFreeAsync(p, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (ps != PK_OK) return ps;
  if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_refine");
  s->pool_n = n;
  if (n_converged) *n_converged = count;
  return PK_OK;
}

pk_status pk_seednet_pool(const pk_seednet* s, float* d_targets_out, float* d_labels_out, int32_t* n_out,
                          void* stream) {
  if (!s || !n_out) return sn_fail(PK_ERR_INVALID_ARG, "NULL argument");
  *n_out = s->pool_n;
  if (s->pool_n == 0 || (!d_targets_out && !d_labels_out)) return PK_OK;  // size query
  if (!d_targets_out || !d_labels_out) return sn_fail(PK_ERR_INVALID_ARG, "NULL device buffer");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(d_targets_out, s->pool_T, (size_t)s->pool_n * s->k * 48, cudaMemcpyDeviceToDevice,
                                  st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_labels_out, s->pool_q, (size_t)s->pool_n * s->n_dof * 4, cudaMemcpyDeviceToDevice, st);
  return sn_cuda(e, "pk_seednet_pool");
}

pk_status pk_seednet_train(pk_seednet* s, const pk_train_params* tp, float* host_loss, void* stream) {
  if (!s || !tp) return sn_fail(PK_ERR_INVALID_ARG, "NULL argument");
  if (tp->epochs < 0 || tp->batch < 128 || tp->steps_per_epoch < 1 || !(tp->lr > 0.f))
    return sn_fail(PK_ERR_INVALID_ARG, "invalid training parameters");
  if (tp->refine_every < 0 || (tp->refine_every > 0 && (tp->refine_n < 1 || tp->refine_iters < 0)) ||
      !(tp->pool_frac >= 0.f && tp->pool_frac <= 1.f))
    return sn_fail(PK_ERR_INVALID_ARG, "invalid refinement parameters");
  const int last = tp->last_epoch > 0 ? tp->last_epoch : tp->epochs;
  if (tp->first_epoch < 0 || tp->last_epoch < 0 || last > tp->epochs || tp->first_epoch > last)
    return sn_fail(PK_ERR_INVALID_ARG, "need 0 <= first_epoch <= last_epoch <= epochs");
  cudaStream_t st = (cudaStream_t)stream;
  const int M = tp->batch, m_pad = round_up(M, 128);
  pk_status ps = ensure_acts(s, m_pad);
  if (ps != PK_OK) return ps;
  const int64_t total = (int64_t)tp->epochs * tp->steps_per_epoch;
  int64_t t = (int64_t)tp->first_epoch * tp->steps_per_epoch;  // position in the cosine schedule
  for (int ep = tp->first_epoch; ep < last; ++ep) {
    cudaError_t e = cudaMemsetAsync(s->d_loss, 0, 4, st);
    for (int it = 0; it < tp->steps_per_epoch && e == cudaSuccess; ++it, ++t) {
      datagen_kernel<<<(m_pad + 127) / 128, 128, 0, st>>>(s->d_robot, s->d_links, s->k, s->d_lohi, s->n_dof,
                                                          tp->seed, s->step, M, s->in_pad, m_pad, s->X, s->Xt,
                                                          s->qstar);
      const int r0 = s->pool_n > 0 ? (int)(tp->pool_frac * (float)M) : 0;
      if (r0 > 0)
        pool_rows_kernel<<<(r0 + 127) / 128, 128, 0, st>>>(s->pool_T, s->pool_q, s->pool_n, s->k, s->n_dof,
                                                           tp->seed ^ 0x706f6f6cull, s->step, r0, s->in_pad, m_pad,
                                                           s->X, s->Xt, s->qstar);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = loss_and_grad(s, M, m_pad, tp->mu, st);
      const float lr = tp->lr * 0.5f * (1.f + cosf(3.14159265f * (float)t / (float)total));
      if (e == cudaSuccess) e = adamw(s, tp, lr, st);
    }
    if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_train");
    if ((ps = check_err(s, st)) != PK_OK) return ps;
    if (host_loss) {
      float l = 0.f;
      e = cudaMemcpy(&l, s->d_loss, 4, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_train");
      host_loss[ep - tp->first_epoch] = l / ((float)M * tp->steps_per_epoch);
    }
    if (tp->refine_every > 0 && (ep + 1) % tp->refine_every == 0 && ep + 1 < tp->epochs) {
      ps = pk_seednet_refine(s, tp->refine_n, tp->refine_iters, tp->seed, nullptr, stream);
      if (ps != PK_OK) return ps;
    }
  }
  return sn_cuda(cudaStreamSynchronize(st), "pk_seednet_train");
}

pk_status pk_seednet_train_step(pk_seednet* s, const pk_train_params* tp, int32_t batch,
                                const float* d_targets, const float* d_qstar, float lr, void* stream) {
  if (!s || !tp || batch < 1 || !d_targets || !d_qstar) return sn_fail(PK_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int m_pad = round_up(batch, 128);
  pk_status ps = ensure_acts(s, m_pad);
  if (ps != PK_OK) return ps;
  features_kernel<<<(m_pad + 127) / 128, 128, 0, st>>>(d_targets, batch, s->k, s->in_pad, m_pad, s->X, s->Xt);
  cudaError_t e = cudaMemcpyAsync(s->qstar, d_qstar, (size_t)batch * s->n_dof * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = loss_and_grad(s, batch, m_pad, tp->mu, st);
  if (e == cudaSuccess) e = adamw(s, tp, lr, st);
  if (e != cudaSuccess) return sn_cuda(e, "pk_seednet_train_step");
  return check_err(s, st);
}

}  // extern "C"
