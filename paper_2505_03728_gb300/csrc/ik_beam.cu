// ik_beam.cu -- IK-Beam (Sec. V-C): all seeds of every target take a first
// round of LM iterations, the lowest-cost seeds of each target continue from
// their LM state (configuration and damping) for a second round, and the best
// of those is returned.
//
// The two rounds are launches of the chain LM kernel (the second one seeded
// from the kept records, with their damping passed in); between them one warp
// per target ranks the first round's costs (`beam_select_kernel`), and after
// them one thread per target picks the result (`beam_final_kernel`).
#include <math.h>

#include "pk_internal.h"

namespace pk {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ float rank_cost(float f) { return isfinite(f) ? f : INFINITY; }

// Keep the `keep` lowest-cost seeds of target blockIdx.x * 4 + warp (ties:
// lower seed index), in ascending order, and gather their configuration,
// damping and iteration count for the second round.
__global__ void __launch_bounds__(128) beam_select_kernel(const float* __restrict__ rec1,
                                                           const float* __restrict__ lam1, int n_dof, int stride,
                                                           int np, int batch, int S1, int keep,
                                                           float* __restrict__ seeds2, float* __restrict__ lam2,
                                                           int32_t* __restrict__ it1, int32_t* __restrict__ kept) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= batch) return;  // whole warps leave together
  const float* rb = rec1 + (size_t)b * S1 * stride;
  uint32_t taken = 0;  // bit c: seed lane + 32 c already kept
  for (int r = 0; r < keep; ++r) {
    float bc = INFINITY;
    int bi = 0x7fffffff;
    for (int s = lane, c = 0; s < S1; s += 32, ++c) {
      if (taken & (1u << c)) continue;
      const float f = rank_cost(rb[(size_t)s * stride + np]);
      if (f < bc || (f == bc && s < bi)) {
        bc = f;
        bi = s;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oc = __shfl_xor_sync(kFullMask, bc, o);
      const int oi = __shfl_xor_sync(kFullMask, bi, o);
      if (oc < bc || (oc == bc && oi < bi)) {
        bc = oc;
        bi = oi;
      }
    }
    const int sel = bi;  // S1 >= keep, so some seed is always left
    if (!PK_IN_BOUNDS(sel, S1, kSiteBeamKeep)) continue;  // the same on every lane
    if ((sel & 31) == lane) taken |= 1u << (sel >> 5);
    const size_t dst = (size_t)b * keep + r;
    const float* src = rb + (size_t)sel * stride;
    if (lane < n_dof) seeds2[dst * n_dof + lane] = src[lane];
    if (lane == 0) {
      lam2[dst] = lam1[(size_t)b * S1 + sel];
      it1[dst] = __float_as_int(src[np + 3]) & 0xffffff;
      kept[dst] = sel;
    }
  }
}

// Best of the kept seeds: converged first, then lowest cost, then lowest
// original seed index; iterations = first round + second round.
__global__ void beam_final_kernel(const float* __restrict__ rec2, int n_dof, int stride, int np, int batch,
                                  int keep, const int32_t* __restrict__ it1, const int32_t* __restrict__ kept,
                                  float* __restrict__ q_out, float* __restrict__ err_out,
                                  int32_t* __restrict__ iters_out, int32_t* __restrict__ status_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  int best = 0, best_conv = -1, best_idx = 0x7fffffff;
  float best_f = INFINITY;
  for (int r = 0; r < keep; ++r) {
    const float* x = rec2 + ((size_t)b * keep + r) * stride;
    const int status = __float_as_int(x[np + 3]) >> 24;
    const int conv = status == PK_P_CONVERGED;
    const float f = rank_cost(x[np]);
    const int idx = kept[(size_t)b * keep + r];
    if (conv > best_conv || (conv == best_conv && (f < best_f || (f == best_f && idx < best_idx)))) {
      best = r;
      best_conv = conv;
      best_f = f;
      best_idx = idx;
    }
  }
  const size_t i = (size_t)b * keep + best;
  const float* x = rec2 + i * stride;
  for (int j = 0; j < n_dof; ++j) q_out[(size_t)b * n_dof + j] = x[j];
  err_out[2 * b] = x[np + 1];
  err_out[2 * b + 1] = x[np + 2];
  const int meta = __float_as_int(x[np + 3]);
  iters_out[b] = it1[i] + (meta & 0xffffff);
  status_out[b] = meta >> 24;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

void beam_layout(int n_dof, long batch, int S1, int keep, BeamWorkspace* w, char* base) {
  size_t off = 0;
  w->bytes1 = ik_workspace_bytes(n_dof, batch, S1);
  w->ws1_off = off;
  off += w->bytes1;
  w->lam1_off = off;
  off += round256((size_t)batch * S1 * 4);
  w->ws2_off = off;
  off += ik_workspace_bytes(n_dof, batch, keep);
  w->seeds2_off = off;
  off += round256((size_t)batch * keep * n_dof * 4);
  w->lam2_off = off;
  off += round256((size_t)batch * keep * 4);
  w->it1_off = off;
  off += round256((size_t)batch * keep * 4);
  w->kept_off = off;
  off += round256((size_t)batch * keep * 4);
  w->total = off;
  w->base = base;
}

cudaError_t launch_beam(const ChainHost& ch, const LmParams& lp, int steps1, int steps2, const float* d_targets,
                        const float* d_seeds, int batch, int S1, int keep, const BeamWorkspace& w,
                        int32_t* d_kept_out, float* d_q, float* d_err, int32_t* d_iters, int32_t* d_status,
                        cudaStream_t st) {
  const int n = ch.n;
  const int stride = ik_rec_stride(n);
  const int np = stride - 4;
  char* base = w.base;
  IkWorkspace ws1, ws2;
  size_t z1 = 0, z2 = 0;
  ik_workspace_carve(base + w.ws1_off, n, batch, S1, &ws1, &z1);
  ik_workspace_carve(base + w.ws2_off, n, batch, keep, &ws2, &z2);
  ws2.stats = ws1.stats;  // one set of work counters for both rounds
  float* lam1 = (float*)(base + w.lam1_off);
  float* seeds2 = (float*)(base + w.seeds2_off);
  float* lam2 = (float*)(base + w.lam2_off);
  int32_t* it1 = (int32_t*)(base + w.it1_off);
  int32_t* kept = d_kept_out ? d_kept_out : (int32_t*)(base + w.kept_off);
  cudaError_t e = cudaMemsetAsync(base + w.ws1_off, 0, z1, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + w.ws2_off, 0, z2, st);
  if (e != cudaSuccess) return e;
  LmParams p1 = lp;
  p1.max_iters = steps1;
  p1.cancel = 0;
  p1.lam_in = nullptr;
  p1.lam_out = lam1;
  e = launch_chain_lm(ch, p1, d_targets, d_seeds, batch, S1, ws1, nullptr, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  {
    TraceScope tr("beam_select", st);
    beam_select_kernel<<<(batch + 3) / 4, 128, 0, st>>>(ws1.rec, lam1, n, stride, np, batch, S1, keep, seeds2,
                                                        lam2, it1, kept);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  LmParams p2 = lp;
  p2.max_iters = steps2;
  p2.cancel = 0;
  p2.lam_in = lam2;
  p2.lam_out = nullptr;
  e = launch_chain_lm(ch, p2, d_targets, seeds2, batch, keep, ws2, nullptr, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  {
    TraceScope tr("beam_final", st);
    beam_final_kernel<<<(batch + 127) / 128, 128, 0, st>>>(ws2.rec, n, stride, np, batch, keep, it1, kept, d_q,
                                                           d_err, d_iters, d_status);
  }
  return cudaGetLastError();
}

}  // namespace pk
