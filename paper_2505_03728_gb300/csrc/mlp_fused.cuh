// mlp_fused.cuh -- seed-network inference (features, every hidden layer and
// the joint-limit head) in one persistent tcgen05 kernel.
//
// The layer-by-layer GEMMs write each 128 x width activation tile to global
// memory and read it back for the next layer; at the inference batch that
// round trip costs as much as the MMAs.  Here a CTA keeps its 128-row tile's
// activations in shared memory for the whole network:
//
//   ACT (shared)  [width / 64 K-blocks][128 rows][64 BF16], 128B-swizzled,
//                 exactly the K-major layout the MMA descriptor reads;
//   TMEM          the layer's FP32 accumulator, 128 lanes x width columns
//                 (two 256-column chunks at width 512);
//   ring          weight tiles [256 outputs][64 K] streamed by TMA from L2.
//
// Warp 0 / lane 0 streams the weights of every (tile, layer, chunk, K-block)
// in MMA order; warp 1 / lane 0 issues tcgen05.mma (M = 128, N = 256 or the
// head width, K = 16) chunk by chunk; eight epilogue warps read a finished
// chunk from TMEM, add the bias and apply SiLU, and write the BF16 result
// back into ACT as the next layer's A operand.  A chunk's results can only be
// written once every MMA of the layer has finished reading ACT, so the first
// chunk's results wait in registers while the MMAs of the second chunk run,
// and the next layer's MMAs over the first 256 inputs start while the
// epilogue still works on the second chunk.  The head writes
// q = mid + half tanh(y) straight to global memory; the next tile's features
// are computed in the same warps.
//
// Arithmetic per element is the layer-by-layer path's (same MMA shapes and
// K order, same SiLU and head formulas), so both give the same seeds.  Every
// mbarrier wait is bounded as in tc_gemm.cuh.
#pragma once
#include "tc_gemm.cuh"

namespace pk {
namespace tc {

constexpr int kMlpMaxLayers = 9;
constexpr int kMlpChunk = 256;                        // accumulator chunk = MMA N of hidden layers
constexpr int kMlpStageBytes = kMlpChunk * kBK * 2;   // one weight tile, 32 KB
constexpr int kMlpBlockBytes = kBM * kBK * 2;         // one ACT K-block, 16 KB
constexpr int kMlpEpiWarps = 8;
constexpr int kMlpThreads = 64 + 32 * kMlpEpiWarps;
constexpr int kMlpMaxStages = 6;
constexpr uint32_t kMlpTmemCols = 512;

struct MlpMaps {
  CUtensorMap w[kMlpMaxLayers];  // W_l [dout_l][din_l] BF16, boxes of 64 K x min(256, dout_l) rows
};

struct MlpParams {
  int n_layers;    // hidden layers + head
  int width;       // 256 or 512
  int in_pad;      // input features padded to a multiple of 64, <= width
  int out_pad;     // head outputs padded to a multiple of 64, <= 256
  int out_dim;     // K * n_dof real head outputs
  int n_dof;
  int k;           // target poses per row (9 features each)
  int batch;
  int tiles;       // ceil(batch / 128)
  int stages;      // weight ring depth
  const float* bias[kMlpMaxLayers];
  const float* lohi;     // joint limits [2][n_dof]
  const float* targets;  // [batch][k][12]
  float* seeds;          // [batch][out_dim]
};

struct MlpSmem {
  static constexpr int act_bytes(int width) { return width / kBK * kMlpBlockBytes; }
  static constexpr int bar_offset(int width, int stages) { return act_bytes(width) + stages * kMlpStageBytes; }
  static constexpr int bytes(int width, int stages) { return bar_offset(width, stages) + 256 + 1024; }
};

// BF16 SiLU of 32 accumulator columns; the arithmetic of epilogue_silu32.
__device__ __forceinline__ void silu_pack32(const float* bias, const uint32_t (&r)[32], uint32_t* packed) {
  const uint64_t half2 = f32x2(0.5f, 0.5f);
  const float2* b2 = reinterpret_cast<const float2*>(bias);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float2 b = __ldg(b2 + i);
    const uint64_t hb = fma_f32x2(f32x2(b.x, b.y), half2, f32x2(0.f, 0.f));
    const uint64_t h2 = fma_f32x2(f32x2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1])), half2, hb);
    const float2 h = f32x2_split(h2);
    const uint64_t s2 = fma_f32x2(h2, f32x2(tanh_fast(h.x), tanh_fast(h.y)), h2);
    const float2 sv = f32x2_split(s2);
    __nv_bfloat162 o = __floats2bfloat162_rn(sv.x, sv.y);
    packed[i] = *reinterpret_cast<uint32_t*>(&o);
  }
}

// 32 BF16 values (inputs n0 .. n0 + 31, n0 a multiple of 32) of tile row r
// into ACT: K-block n0 / 64, 16-byte chunks (n0 % 64) / 8 .. + 3, each at its
// 128B-swizzled position (chunk index XOR row % 8).
__device__ __forceinline__ void act_store32(uint8_t* act, int r, int n0, const uint32_t* packed) {
  uint8_t* row = act + (n0 >> 6) * kMlpBlockBytes + r * 128;
  const int c0 = (n0 & 63) >> 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<uint4*>(row + (((c0 + i) ^ (r & 7)) << 4)) =
        make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
}

// Pose features of one row (position, first two rotation columns per target;
// zero past 9 k and for rows past the batch) into ACT K-blocks 0 .. in_pad/64.
__device__ __forceinline__ void act_features(uint8_t* act, const MlpParams& p, int tile, int r) {
  const int row = tile * kBM + r;
  const bool ok = row < p.batch;
  const float* T = p.targets + (size_t)(ok ? row : 0) * p.k * 12;
  const int in_dim = 9 * p.k;
  // feature j of a target reads its 3 x 4 row-major pose at 3, 7, 11 (position),
  // 0, 4, 8 (rotation column 0), 1, 5, 9 (rotation column 1)
  auto off = [](int j) { return j < 3 ? 3 + 4 * j : j < 6 ? 4 * (j - 3) : 1 + 4 * (j - 6); };
  for (int n0 = 0; n0 < p.in_pad; n0 += 32) {
    uint32_t packed[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float v[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int a = n0 + 2 * i + e;
        v[e] = (ok && a < in_dim) ? __ldg(T + (a / 9) * 12 + off(a % 9)) : 0.f;
      }
      __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
      packed[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    act_store32(act, r, n0, packed);
  }
}

__global__ void __launch_bounds__(kMlpThreads, 1)
    mlp_fused_kernel(const __grid_constant__ MlpMaps maps, const __grid_constant__ MlpParams p, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* act = smem;
  uint8_t* ring = smem + MlpSmem::act_bytes(p.width);
  uint64_t* full = (uint64_t*)(smem + MlpSmem::bar_offset(p.width, p.stages));
  uint64_t* empty = full + p.stages;
  uint64_t* tfull = empty + p.stages;  // [2] accumulator chunk ready (MMA -> epilogue)
  uint64_t* tfree = tfull + 2;         // [2] accumulator chunk read out (epilogue -> MMA)
  uint64_t* actb = tfree + 2;          // [4] ACT inputs 128 b .. 128 b + 127 written (epilogue -> MMA)
  uint64_t* stg = actb + 4;            // [2] head staging written / read out (epilogue warps)
  uint64_t* drain = stg + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = p.n_layers, nch = p.width / kMlpChunk, S = p.stages;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(&tfull[c], 1);
      mbar_init(&tfree[c], kMlpEpiWarps);
      mbar_init(&stg[c], kMlpEpiWarps);
    }
    for (int b = 0; b < 4; ++b) mbar_init(&actb[b], kMlpEpiWarps);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, kMlpTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- weight producer, in the MMA's order
      uint32_t it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < p.tiles && ok; t += gridDim.x)
        for (int l = 0; l < L && ok; ++l) {
          const bool head = l == L - 1;
          const int nc_n = head ? 1 : nch, kb_n = (l == 0 ? p.in_pad : p.width) / kBK;
          const uint32_t bytes = (uint32_t)(head ? p.out_pad : kMlpChunk) * kBK * 2;
          for (int nc = 0; nc < nc_n && ok; ++nc)
            for (int kb = 0; kb < kb_n; ++kb, ++it) {
              const int s = it % S;
              const uint32_t round = it / S;
              if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, err, 11)) {
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&full[s], bytes);
              tma_load_2d(ring + s * kMlpStageBytes, &maps.w[l], &full[s], kb * kBK, nc * kMlpChunk);
              ++issued;
            }
        }
      if (!ok)  // let the loads already issued land before teardown
        for (uint32_t i = (issued > (uint32_t)S ? issued - S : 0); i < issued; ++i)
          mbar_drain(&full[i % S], (i / S) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      uint32_t it = 0, uses0 = 0, uses1 = 0, acts = 0;  // completions consumed per barrier (acts: 8 bits each)
      bool ok = true;
      for (int t = blockIdx.x; t < p.tiles && ok; t += gridDim.x)
        for (int l = 0; l < L && ok; ++l) {
          const bool head = l == L - 1;
          // the head accumulates in chunk 1's columns, so that the next tile's
          // first chunk can start while the head is read out
          const int nc0 = head ? 1 : 0, nc1 = head ? 2 : nch, kb_n = (l == 0 ? p.in_pad : p.width) / kBK;
          const uint32_t idesc = idesc_bf16(head ? p.out_pad : kMlpChunk);
          for (int nc = nc0; nc < nc1 && ok; ++nc) {
            const uint32_t used = nc ? uses1 : uses0;
            if (used > 0 && !mbar_wait(&tfree[nc], (used - 1) & 1, err, 14)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(nc * kMlpChunk);
            for (int kb = 0; kb < kb_n; ++kb, ++it) {
              if (nc == nc0 && (kb & 1) == 0) {  // first read of ACT inputs 64 kb .. 64 kb + 127 in this layer
                const int b = kb >> 1;
                if (!mbar_wait(&actb[b], (acts >> (8 * b)) & 1, err, 15)) {
                  ok = false;
                  break;
                }
                acts ^= 1u << (8 * b);
                tc_fence_after();
              }
              const int s = it % S;
              if (!mbar_wait(&full[s], (it / S) & 1, err, 12)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t ad = smem_desc(smem_u32(act + kb * kMlpBlockBytes));
              const uint64_t bd = smem_desc(smem_u32(ring + s * kMlpStageBytes));
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k) mma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
              mma_commit(&empty[s]);
            }
            if (!ok) break;
            mma_commit(&tfull[nc]);
            if (nc) ++uses1; else ++uses0;
          }
        }
      mma_commit(drain);  // completes once every MMA issued above has finished
      mbar_drain(drain, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile
    //      rows) and half h = (w - 2) / 4 of each chunk's columns
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int r = q * 32 + lane, te = threadIdx.x - 64;  // te: 0 .. 255 over the epilogue warps
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    const int in_blocks = p.in_pad / kBK;
    // the head's outputs are staged in ACT blocks past the inputs (free once
    // the head's MMAs are done) and written out row-contiguously; pitch odd
    // for conflict-free column writes
    const bool staged = (p.out_dim & 3) == 0 && ((uintptr_t)p.seeds & 15) == 0 &&
                        (p.width / kBK - in_blocks) * kMlpBlockBytes >= kBM * p.out_dim * 4;
    float* stage = reinterpret_cast<float*>(act + in_blocks * kMlpBlockBytes);
    uint32_t tf[2] = {0, 0};
    bool ok = true;
    auto wait_chunk = [&](int c) -> bool {
      uint32_t ready = 0;
      if (lane == 0) ready = mbar_wait(&tfull[c], tf[c] & 1, err, 13) ? 1u : 0u;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      ++tf[c];
      if (ready) tc_fence_after();
      return ready != 0;
    };
    auto signal = [&](uint64_t* bar) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar);
    };
    // bounded rendezvous of the epilogue warps on stg[i] (one phase per tile)
    uint32_t sg[2] = {0, 0};
    auto epi_sync = [&](int i) -> bool {
      signal(&stg[i]);
      uint32_t ready = 0;
      if (lane == 0) ready = mbar_wait(&stg[i], sg[i] & 1, err, 16) ? 1u : 0u;
      ++sg[i];
      return __shfl_sync(0xffffffffu, ready, 0) != 0;
    };
    // column of piece i (0..3) of chunk c for this warp: both warps of a lane
    // quarter finish the chunk's lower 128 columns (pieces 0, 1) before the
    // upper ones, so that the next layer's MMAs can read them early
    auto pcol = [&](int c, int i) { return c * kMlpChunk + (i >> 1) * 128 + h * 64 + (i & 1) * 32; };
    // the warp's four pieces of chunk c, TMEM loads one piece ahead of the
    // SiLU; `sink(i, packed)` takes piece i's 16 BF16 pairs
    auto chunk_silu = [&](int c, const float* bias, auto&& sink) {
      uint32_t ra[32], rb[32], pk[16];
      tmem_ld32_issue(lane_base + (uint32_t)pcol(c, 0), ra);
      tmem_ld_wait(ra);
      tmem_ld32_issue(lane_base + (uint32_t)pcol(c, 1), rb);
      silu_pack32(bias + pcol(c, 0), ra, pk);
      sink(0, pk);
      tmem_ld_wait(rb);
      tmem_ld32_issue(lane_base + (uint32_t)pcol(c, 2), ra);
      silu_pack32(bias + pcol(c, 1), rb, pk);
      sink(1, pk);
      tmem_ld_wait(ra);
      tmem_ld32_issue(lane_base + (uint32_t)pcol(c, 3), rb);
      silu_pack32(bias + pcol(c, 2), ra, pk);
      sink(2, pk);
      tmem_ld_wait(rb);
      silu_pack32(bias + pcol(c, 3), rb, pk);
      sink(3, pk);
    };
    // ACT pieces written to shared memory -> visible to the MMA, then signal
    auto publish = [&](uint64_t* bar) {
      fence_proxy_async_smem();
      signal(bar);
    };
    auto features = [&](int t) {
      if (h == 0) act_features(act, p, t, r);
      fence_proxy_async_smem();
      for (int b = 0; b < (in_blocks + 1) / 2; ++b) signal(&actb[b]);
    };
    auto prefetch_targets = [&](int t) {  // next tile's target poses into L2
      if (te != 0 || t >= p.tiles) return;
      const int rows = min(kBM, p.batch - t * kBM);
      const float* src = p.targets + (size_t)t * kBM * p.k * 12;
      if (((uintptr_t)src & 15) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((uint32_t)(rows * p.k * 48))
                     : "memory");
    };
    if (blockIdx.x < p.tiles) features(blockIdx.x);
    for (int t = blockIdx.x; t < p.tiles && ok; t += gridDim.x) {
      const int tn = t + gridDim.x;
      prefetch_targets(tn);
      for (int l = 0; l + 1 < L && ok; ++l) {
        const float* bias = p.bias[l];
        // ACT inputs 128 b .. 128 b + 127 are published on actb[b] once both
        // warps of every lane quarter have written their pieces
        auto to_act = [&](int c) {
          return [&, c](int i, const uint32_t* pk) {
            act_store32(act, r, pcol(c, i), pk);
            if (i & 1) publish(&actb[2 * c + (i >> 1)]);
          };
        };
        if (nch == 2) {
          // chunk 0 waits in registers until the layer's last MMA has read ACT
          uint32_t keep[64];
          if (!(ok = wait_chunk(0))) break;
          chunk_silu(0, bias, [&](int i, const uint32_t* pk) {
#pragma unroll
            for (int j = 0; j < 16; ++j) keep[16 * i + j] = pk[j];
          });
          tc_fence_before();
          signal(&tfree[0]);
          if (!(ok = wait_chunk(1))) break;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            act_store32(act, r, pcol(0, i), keep + 16 * i);
            if (i & 1) publish(&actb[i >> 1]);
          }
          chunk_silu(1, bias, to_act(1));
          tc_fence_before();
          signal(&tfree[1]);
        } else {
          if (!(ok = wait_chunk(0))) break;
          chunk_silu(0, bias, to_act(0));
          tc_fence_before();
          signal(&tfree[0]);
        }
      }
      if (!ok) break;
      // head (chunk 1's columns): its last MMA has read ACT, so the next
      // tile's features go in first and its first chunk starts at once
      if (!(ok = wait_chunk(1))) break;
      if (tn < p.tiles) features(tn);
      const int row0 = t * kBM, row = row0 + r;
      const bool row_ok = row < p.batch;
      const float* bias = p.bias[L - 1];
      const int half = p.out_pad >> 1;
#pragma unroll 1
      for (int c0 = h * half; c0 < (h + 1) * half; c0 += 32) {
        uint32_t rr[32];
        tmem_ld32_issue(lane_base + (uint32_t)(kMlpChunk + c0), rr);
        tmem_ld_wait(rr);
        if (c0 >= p.out_dim) continue;
        float v[32];
        int j = c0 % p.n_dof;  // joint of column c0 + i, advanced incrementally
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int c = c0 + i;
          v[i] = 0.f;
          if (c < p.out_dim) {
            const float lo = __ldg(p.lohi + j), hi = __ldg(p.lohi + p.n_dof + j);
            v[i] = 0.5f * (lo + hi) + 0.5f * (hi - lo) * tanhf(__uint_as_float(rr[i]) + __ldg(bias + c));
            if (!staged && row_ok) p.seeds[(size_t)row * p.out_dim + c] = v[i];
          }
          if (++j == p.n_dof) j = 0;
        }
        if (staged)  // out_dim % 4 == 0: a group of four is all in or all out
#pragma unroll
          for (int g = 0; g < 8; ++g)
            if (c0 + 4 * g < p.out_dim)
              *reinterpret_cast<float4*>(stage + r * p.out_dim + c0 + 4 * g) =
                  make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
      }
      tc_fence_before();
      signal(&tfree[1]);
      if (staged) {
        // every epilogue warp's head columns are staged; copy the tile's rows
        // out contiguously, then release the staging area
        if (!(ok = epi_sync(0))) break;
        // staging holds the tile's rows in their global layout: a flat copy
        const int n4 = min(kBM, p.batch - row0) * p.out_dim / 4;
        float4* dst = reinterpret_cast<float4*>(p.seeds + (size_t)row0 * p.out_dim);
        const float4* src = reinterpret_cast<const float4*>(stage);
        for (int i = te; i < n4; i += 32 * kMlpEpiWarps) dst[i] = src[i];
        if (!(ok = epi_sync(1))) break;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kMlpTmemCols);
}

}  // namespace tc
}  // namespace pk
