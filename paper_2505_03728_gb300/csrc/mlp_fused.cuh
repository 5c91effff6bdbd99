// mlp_fused.cuh -- seed-network inference (features, every hidden layer and
// the joint-limit head) in one persistent tcgen05 kernel.
//
// The layer-by-layer GEMMs write each 128 x width activation tile to global
// memory and read it back for the next layer.  Here a CTA keeps its 128-row
// tile's activations in tensor memory for the whole network and feeds them
// to the MMA as the A operand straight from TMEM:
//
//   TMEM columns [256, 512)  ACT: row r in lane r, inputs 2c, 2c+1 packed in
//                            column 256 + c (BF16 pairs; up to 512 inputs);
//   TMEM columns [0, 256)    the FP32 accumulator of one output chunk (256
//                            features, or the head);
//   shared memory            a ring of 64 KB weight stages (one 3-D TMA box:
//                            [K-blocks][256 outputs][64 K], 128B-swizzled)
//                            and the first chunk's BF16 results while the
//                            second is computed.
//
// Measured on sm_103a (M = 128, K = 16, BF16): an MMA instruction costs a
// fixed ~116 cycles up to N = 128; at N = 256 it takes ~138 cycles with A in
// TMEM and ~171 with A in shared memory, so N = 256 with A in TMEM is the
// only shape near the tensor peak.  A TMA request likewise costs a roughly
// fixed few hundred cycles, hence the large boxes.
//
// Warp 0 / lane 0 streams the weights of every (tile, layer, chunk, stage) in
// MMA order; warp 1 / lane 0 issues tcgen05.mma; sixteen epilogue warps (four
// per TMEM lane quarter) drain the accumulator into registers (after which
// the MMA may overwrite it), add the bias and apply SiLU.  Each warp owns 16
// columns of every 64-column quarter of a chunk, so all sixteen warps finish
// each 128 ACT inputs together (the MUFU tanh throughput bounds this work).
// A layer's outputs can only replace ACT once every MMA of the layer has
// read it, so the first chunk's results wait in shared memory; when the
// second chunk is drained they are stored to ACT and published per 128
// inputs, and the next layer's MMAs start on them while the second chunk is
// finished, again 128 inputs at a time.  The head releases the accumulator
// as soon as it is in registers and stores q = mid + half tanh(y) straight to
// global memory; the next tile's features go into ACT right after the head's
// last MMA.
//
// Arithmetic per element is the layer-by-layer path's (same MMA K order,
// same SiLU and head formulas).  Every mbarrier wait is bounded as in
// tc_gemm.cuh.
#pragma once
#include "tc_gemm.cuh"

namespace pk {
namespace tc {

constexpr int kMlpMaxLayers = 9;
constexpr int kMlpChunk = 256;                    // output features per accumulator chunk (MMA N)
constexpr int kMlpStageBytes = 65536;             // largest weight stage
constexpr int kMlpKeepBytes = kBM * kMlpChunk * 2;  // one chunk of BF16 results
constexpr int kMlpEpiWarps = 16;
constexpr int kMlpThreads = 64 + 32 * kMlpEpiWarps;
constexpr int kMlpMaxStages = 3;
constexpr uint32_t kMlpTmemCols = 512;
constexpr uint32_t kMlpActCol = 256;              // first TMEM column of ACT

struct MlpMaps {
  // W_l viewed as [din_l / 64][dout_l][64] BF16: 3-D boxes of 64 x rows x stage_kb[l]
  CUtensorMap w[kMlpMaxLayers];
};

struct MlpParams {
  int n_layers;    // hidden layers + head
  int width;       // 256 or 512
  int in_pad;      // input features padded to a multiple of 64, <= 256
  int out_pad;     // head outputs padded to a multiple of 64, <= 256
  int out_dim;     // K * n_dof real head outputs
  int n_dof;
  int k;           // target poses per row (9 features each)
  int batch;
  int tiles;       // ceil(batch / 128)
  int stages;      // weight ring depth (slots of kMlpStageBytes)
  int area_bytes;  // keep / staging area after the ring
  int vec4;        // head outputs as float4 stores (out_dim % 4 == 0, 16-byte aligned output)
  int stage_kb[kMlpMaxLayers];  // K-blocks of 64 per weight stage of layer l
  const float* bias[kMlpMaxLayers];
  const float* lohi;     // joint limits [2][n_dof]
  const float* targets;  // [batch][k][12]
  float* seeds;          // [batch][out_dim]
};

struct MlpSmem {
  static constexpr int bar_offset(int stages, int area) { return stages * kMlpStageBytes + ((area + 1023) & ~1023); }
  static constexpr int bytes(int stages, int area) { return bar_offset(stages, area) + 256 + 1024; }
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// D (TMEM) (+)= A (TMEM) * B (shared memory descriptor)^T
__device__ __forceinline__ void mma_bf16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 32 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint4& a, const uint4& b, const uint4& c,
                                          const uint4& d) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w), "r"(c.x), "r"(c.y),
      "r"(c.z), "r"(c.w), "r"(d.x), "r"(d.y), "r"(d.z), "r"(d.w)
      : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane into r[O .. O + 15]
// (completed by tmem_ld_wait on r).
template <int O>
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[O + 0]), "=r"(r[O + 1]), "=r"(r[O + 2]), "=r"(r[O + 3]), "=r"(r[O + 4]), "=r"(r[O + 5]),
        "=r"(r[O + 6]), "=r"(r[O + 7]), "=r"(r[O + 8]), "=r"(r[O + 9]), "=r"(r[O + 10]), "=r"(r[O + 11]),
        "=r"(r[O + 12]), "=r"(r[O + 13]), "=r"(r[O + 14]), "=r"(r[O + 15])
      : "r"(taddr));
}

// 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint4& a, const uint4& b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

// BF16 SiLU of the 16 accumulator columns r[O .. O + 15] (bias of their
// first feature at `bias`); per element the arithmetic of silu_pack32.
template <int O>
__device__ __forceinline__ void silu_pack16(const float* bias, const uint32_t (&r)[32], uint32_t (&packed)[8]) {
  const uint64_t half2 = f32x2(0.5f, 0.5f);
  const float2* b2 = reinterpret_cast<const float2*>(bias);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 b = __ldg(b2 + i);
    const uint64_t hb = fma_f32x2(f32x2(b.x, b.y), half2, f32x2(0.f, 0.f));
    const uint64_t h2 =
        fma_f32x2(f32x2(__uint_as_float(r[O + 2 * i]), __uint_as_float(r[O + 2 * i + 1])), half2, hb);
    const float2 h = f32x2_split(h2);
    const uint64_t s2 = fma_f32x2(h2, f32x2(tanh_fast(h.x), tanh_fast(h.y)), h2);
    const float2 sv = f32x2_split(s2);
    __nv_bfloat162 o = __floats2bfloat162_rn(sv.x, sv.y);
    packed[i] = *reinterpret_cast<uint32_t*>(&o);
  }
}

// BF16 SiLU of 32 accumulator columns; the arithmetic of epilogue_silu32.
__device__ __forceinline__ void silu_pack32(const float* bias, const uint32_t (&r)[32], uint32_t (&packed)[16]) {
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

// Pose features of tile row r (position, first two rotation columns per
// target; zero past 9 k and for rows past the batch), packed BF16 pairs,
// into ACT columns 0 .. in_pad / 2 of this thread's lane.
__device__ __forceinline__ void act_features(uint32_t act_lane, const MlpParams& p, int tile, int r) {
  const int row = tile * kBM + r;
  const bool ok = row < p.batch;
  const float* T = p.targets + (size_t)(ok ? row : 0) * p.k * 12;
  const int in_dim = 9 * p.k;
  if (p.k == 1 && p.in_pad == 64 && ((uintptr_t)p.targets & 15) == 0) {
    // one pose per row: three 16-byte loads instead of nine scattered ones
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
    if (ok) {
      const float4* T4 = reinterpret_cast<const float4*>(T);
      a = __ldg(T4);
      b = __ldg(T4 + 1);
      c = __ldg(T4 + 2);
    }
    const float f[10] = {a.w, b.w, c.w, a.x, b.x, c.x, a.y, b.y, c.y, 0.f};
    uint32_t packed[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      __nv_bfloat162 hv = __floats2bfloat162_rn(i < 5 ? f[2 * i] : 0.f, i < 5 ? f[2 * i + 1] : 0.f);
      packed[i] = *reinterpret_cast<uint32_t*>(&hv);
    }
    tmem_st32(act_lane, packed);
    return;
  }
  // feature j of a target reads its 3 x 4 row-major pose at 3, 7, 11 (position),
  // 0, 4, 8 (rotation column 0), 1, 5, 9 (rotation column 1)
  auto off = [](int j) { return j < 3 ? 3 + 4 * j : j < 6 ? 4 * (j - 3) : 1 + 4 * (j - 6); };
  for (int n0 = 0; n0 < p.in_pad; n0 += 64) {
    uint32_t packed[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float v[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int a = n0 + 2 * i + e;
        v[e] = (ok && a < in_dim) ? __ldg(T + (a / 9) * 12 + off(a % 9)) : 0.f;
      }
      __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
      packed[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    tmem_st32(act_lane + (uint32_t)(n0 >> 1), packed);
  }
}

__global__ void __launch_bounds__(kMlpThreads, 1)
    mlp_fused_kernel(const __grid_constant__ MlpMaps maps, const __grid_constant__ MlpParams p, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  uint8_t* ring = smem;
  uint8_t* area = smem + S * kMlpStageBytes;  // first chunk's results, then the head's staging
  float* stage = reinterpret_cast<float*>(area);
  uint64_t* full = (uint64_t*)(smem + MlpSmem::bar_offset(S, p.area_bytes));
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;   // accumulator ready (MMA -> epilogue)
  uint64_t* tfree = tfull + 1;   // accumulator drained (epilogue -> MMA)
  uint64_t* actb = tfree + 1;    // [4] ACT inputs 128 b .. 128 b + 127 written (epilogue -> MMA)
  uint64_t* drain = actb + 4;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = p.n_layers;
  const int hidden_chunks = p.width / kMlpChunk;  // 1 or 2

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tfree, kMlpEpiWarps);
    for (int b = 0; b < 4; ++b) mbar_init(&actb[b], kMlpEpiWarps);  // every epilogue warp writes a part
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, kMlpTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // per layer: K-blocks of 64 inputs, output chunks and rows (outputs) per chunk
  auto kblocks = [&](int l) { return (l == 0 ? p.in_pad : p.width) / kBK; };
  auto chunks = [&](int l) { return l == L - 1 ? 1 : hidden_chunks; };
  auto rows = [&](int l) { return l == L - 1 ? p.out_pad : kMlpChunk; };

  if (warp == 0) {
    if (lane == 0) {
      // ---- weight producer, in the MMA's order
      uint32_t it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < p.tiles && ok; t += gridDim.x)
        for (int l = 0; l < L && ok; ++l) {
          const int nkb = kblocks(l), nc = chunks(l), nr = rows(l), kbs = p.stage_kb[l];
          for (int c = 0; c < nc && ok; ++c)
            for (int kb0 = 0; kb0 < nkb; kb0 += kbs, ++it) {
              const int s = it % S;
              const uint32_t round = it / S;
              if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, err, 11)) {
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&full[s], (uint32_t)(nr * kbs * kBK * 2));
              tma_load_3d(ring + s * kMlpStageBytes, &maps.w[l], &full[s], 0, c * nr, kb0);
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
      // ---- MMA issuer: one accumulator, chunks in turn
      uint32_t it = 0, used = 0, acts = 0;  // acts: parity bit 8 b of ACT barrier b
      bool ok = true;
      for (int t = blockIdx.x; t < p.tiles && ok; t += gridDim.x)
        for (int l = 0; l < L && ok; ++l) {
          const int nkb = kblocks(l), nc = chunks(l), nr = rows(l), kbs = p.stage_kb[l];
          const uint32_t idesc = idesc_bf16(nr);
          for (int c = 0; c < nc && ok; ++c) {
            if (used > 0 && !mbar_wait(tfree, (used - 1) & 1, err, 14)) {
              ok = false;
              break;
            }
            tc_fence_after();
            for (int kb0 = 0; kb0 < nkb && ok; kb0 += kbs, ++it) {
              if (c == 0)  // first read of ACT inputs 64 kb0 .. 64 (kb0 + kbs) in this layer
                for (int pc = kb0 >> 1; pc < (kb0 + kbs + 1) >> 1 && ok; ++pc) {
                  ok = mbar_wait(&actb[pc], (acts >> (8 * pc)) & 1, err, 15);
                  acts ^= 1u << (8 * pc);
                }
              const int s = it % S;
              if (!ok || !mbar_wait(&full[s], (it / S) & 1, err, 12)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sb = smem_u32(ring + s * kMlpStageBytes);
              for (int j = 0; j < kbs; ++j) {
                const uint64_t bd = smem_desc(sb + (uint32_t)(j * nr * 128));
                const uint32_t a = tmem + kMlpActCol + (uint32_t)((kb0 + j) * (kBK / 2));
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                  mma_bf16_tmem_a(tmem, a + (uint32_t)(k * 8), bd + 2 * k, idesc, (kb0 + j > 0 || k > 0) ? 1u : 0u);
              }
              mma_commit(&empty[s]);
            }
            if (!ok) break;
            mma_commit(tfull);
            ++used;
          }
        }
      mma_commit(drain);  // completes once every MMA issued above has finished
      mbar_drain(drain, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile
    //      rows) and, of every 64-column quarter m of a chunk, the columns
    //      64 m + 16 h .. 64 m + 16 h + 15, h = (w - 2) / 4
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int r = q * 32 + lane, te = threadIdx.x - 64;  // te: 0 .. 511 over the epilogue warps
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t act_lane = lane_base + kMlpActCol;
    uint32_t tf = 0;
    bool ok = true;
    // this thread's 32 words of a kept chunk (its row, its 64 features), in
    // 16-byte pieces rotated by the row so that a warp's accesses spread over
    // all banks
    uint8_t* keep_row = area + (size_t)(r * 4 + h) * 128;
    auto keep_at = [&](int i) { return reinterpret_cast<uint4*>(keep_row + ((i ^ (r & 7)) << 4)); };
    auto signal = [&](uint64_t* bar) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar);
    };
    auto wait_acc = [&]() -> bool {
      uint32_t ready = 0;
      if (lane == 0) ready = mbar_wait(tfull, tf & 1, err, 13) ? 1u : 0u;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      ++tf;
      if (ready) tc_fence_after();
      return ready != 0;
    };
    // this warp's TMEM stores into ACT are complete and ordered before the
    // MMA's reads; then signal
    auto publish = [&](uint64_t* bar) {
      tmem_st_wait();
      tc_fence_before();
      signal(bar);
    };
    // this warp's 64 accumulator columns into registers (quarters 0, 1 in v0,
    // 2, 3 in v1; one wait for all four loads), then release the accumulator
    auto drain = [&](uint32_t (&v0)[32], uint32_t (&v1)[32]) {
      tmem_ld16_issue<0>(lane_base + (uint32_t)(16 * h), v0);
      tmem_ld16_issue<16>(lane_base + (uint32_t)(64 + 16 * h), v0);
      tmem_ld16_issue<0>(lane_base + (uint32_t)(128 + 16 * h), v1);
      tmem_ld16_issue<16>(lane_base + (uint32_t)(192 + 16 * h), v1);
      tmem_ld_wait(v0);
      tmem_ld_wait(v1);
      tc_fence_before();
      signal(tfree);
    };
    // SiLU of this warp's 16 columns of quarter m of a chunk whose first
    // feature is f0: 8 packed BF16 pairs (ACT columns f0 / 2 + 32 m + 8 h ..)
    auto silu_q = [&](const float* bias, int f0, int m, const uint32_t (&v0)[32], const uint32_t (&v1)[32],
                      uint32_t (&pk)[8]) {
      const float* b = bias + f0 + 64 * m + 16 * h;
      if (m == 0)
        silu_pack16<0>(b, v0, pk);
      else if (m == 1)
        silu_pack16<16>(b, v0, pk);
      else if (m == 2)
        silu_pack16<0>(b, v1, pk);
      else
        silu_pack16<16>(b, v1, pk);
    };
    auto features = [&](int t) {  // written by the h = 0 warps, published by all
      if (h == 0) act_features(act_lane, p, t, r);
      for (int b = 0; b < (p.in_pad + 127) / 128; ++b) publish(&actb[b]);
    };
    auto prefetch_targets = [&](int t) {  // next tile's target poses into L2
      if (te != 0 || t >= p.tiles) return;
      const int nrow = min(kBM, p.batch - t * kBM);
      const float* src = p.targets + (size_t)t * kBM * p.k * 12;
      if (((uintptr_t)src & 15) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((uint32_t)(nrow * p.k * 48))
                     : "memory");
    };
    if (blockIdx.x < p.tiles) features(blockIdx.x);
    for (int t = blockIdx.x; t < p.tiles && ok; t += gridDim.x) {
      const int tn = t + gridDim.x;
      prefetch_targets(tn);
      for (int l = 0; l + 1 < L && ok; ++l) {
        const float* bias = p.bias[l];
        uint32_t v0[32], v1[32];
        if (!(ok = wait_acc())) break;
        drain(v0, v1);
        if (hidden_chunks == 2) {
          // chunk 0 waits in shared memory until the layer's last MMA has read ACT
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            uint32_t pk[8];
            silu_q(bias, 0, m, v0, v1, pk);
            *keep_at(2 * m) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *keep_at(2 * m + 1) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          }
          if (!(ok = wait_acc())) break;
          drain(v0, v1);
          // every MMA of the layer is done: chunk 0 into ACT, each 128 inputs
          // published at once (the next layer starts on them), then chunk 1
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            tmem_st8(act_lane + (uint32_t)(32 * m + 8 * h), *keep_at(2 * m), *keep_at(2 * m + 1));
            if (m & 1) publish(&actb[m >> 1]);
          }
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            uint32_t pk[8];
            silu_q(bias, kMlpChunk, m, v0, v1, pk);
            tmem_st8(act_lane + (uint32_t)(kMlpChunk / 2 + 32 * m + 8 * h), make_uint4(pk[0], pk[1], pk[2], pk[3]),
                     make_uint4(pk[4], pk[5], pk[6], pk[7]));
            if (m & 1) publish(&actb[2 + (m >> 1)]);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            uint32_t pk[8];
            silu_q(bias, 0, m, v0, v1, pk);
            tmem_st8(act_lane + (uint32_t)(32 * m + 8 * h), make_uint4(pk[0], pk[1], pk[2], pk[3]),
                     make_uint4(pk[4], pk[5], pk[6], pk[7]));
            if (m & 1) publish(&actb[m >> 1]);
          }
        }
      }
      if (!ok) break;
      // head: q = mid + half tanh(y + b); its last MMA has read ACT, so the next
      // tile's features go in first
      if (!(ok = wait_acc())) break;
      if (tn < p.tiles) features(tn);
      const int row = t * kBM + r;
      const bool row_ok = row < p.batch;
      const float* bias = p.bias[L - 1];
      const int wc = p.out_pad / 4;  // this warp's columns of the head: 16 .. 64
      // 16 columns c0 .. c0 + 15 of this row, in groups of four
      auto head16 = [&](int c0, const float (&v)[16]) {
        if (c0 >= p.out_dim || !row_ok) return;
        float* dst = p.seeds + (size_t)row * p.out_dim + c0;
        int j = c0 % p.n_dof;  // joint of the current column, advanced incrementally
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          float o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = c0 + 4 * g + e;
            o[e] = 0.f;
            if (c < p.out_dim) {
              const float lo = __ldg(p.lohi + j), hi = __ldg(p.lohi + p.n_dof + j);
              o[e] = 0.5f * (lo + hi) + 0.5f * (hi - lo) * tanhf(v[4 * g + e] + __ldg(bias + c));
              if (!p.vec4) dst[4 * g + e] = o[e];
            }
            if (++j == p.n_dof) j = 0;
          }
          if (p.vec4 && c0 + 4 * g < p.out_dim)
            *reinterpret_cast<float4*>(dst + 4 * g) = make_float4(o[0], o[1], o[2], o[3]);
        }
      };
      float v[16];
      if (wc == 16) {
        // one 16-column piece per warp: release the accumulator before the
        // arithmetic, so the next tile's first MMAs overlap it
        tmem_ld16(lane_base + (uint32_t)(h * 16), v);
        tc_fence_before();
        signal(tfree);
        head16(h * 16, v);
      } else {
        // wider heads 16 columns at a time (few registers; the accumulator
        // is released at the end)
#pragma unroll 1
        for (int c0 = h * wc; c0 < (h + 1) * wc; c0 += 16) {
          tmem_ld16(lane_base + (uint32_t)c0, v);
          head16(c0, v);
        }
        tc_fence_before();
        signal(tfree);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kMlpTmemCols);
}

}  // namespace tc
}  // namespace pk
