// tc_gemm.cuh -- BF16 tensor-core GEMM for sm_103a with tcgen05 (TMEM
// accumulators), TMA tile loads and mbarrier pipelines, and fused epilogues
// for the seed network's forward and backward passes.
//
//   D[M x N] (FP32, in TMEM) = A[M x K] * B[N x K]^T      A, B: BF16, K-major
//
// Persistent kernel, one CTA per SM striding over the (m, n, k-split) output
// tiles of 128 x BN (BN = 64, 128 or 256; split-K over grid tiles for the
// weight gradients).  Warp 0 / lane 0 issues the TMA loads of a 4-stage ring
// (128B-swizzled 64-wide K blocks), warp 1 / lane 0 issues tcgen05.mma (M = 128,
// N = BN, K = 16, four per K block) into one of two TMEM accumulators and
// commits each stage back to the producer; eight epilogue warps (two per TMEM
// lane quarter, each taking half of the columns) read the other accumulator
// with tcgen05.ld 32x32b and run the fused epilogue, so the epilogue of one
// tile overlaps the MMAs of the next.
//
// Every mbarrier wait is bounded (1 s of %globaltimer); on timeout the kernel
// records an error code in *err, skips the rest of its work, frees its TMEM
// and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pk {
namespace tc {

constexpr int kBM = 128;
constexpr int kBK = 64;  // one 128-byte swizzle atom of BF16
constexpr int kStages = 4;
constexpr uint64_t kWaitNs = 1000000000ull;

enum EpiMode : int {
  EPI_FWD_SILU = 0,    // z = acc + b; Z(f32) optional; A = silu(z) (bf16, row-major + transposed)
  EPI_FWD_LINEAR = 1,  // y = acc + b -> f32 [M][n_valid]
  EPI_DGRAD_SILU = 2,  // d = acc * silu'(Zprev) -> bf16 row-major + transposed
  EPI_WGRAD_ADD = 3,   // atomically add acc into f32 [M][N] (split-K partial sums)
  EPI_SEEDS = 4,       // q = mid + half tanh(acc + b) -> f32 [M][n_valid] (seed-network head)
};

struct Epilogue {
  int mode;
  int m_valid;             // rows < m_valid are stored
  int n_valid;             // columns < n_valid are stored (FWD_LINEAR)
  const float* bias;       // [N]
  float* out_f32;          // Z (FWD_SILU, optional), Y (FWD_LINEAR) or dW (WGRAD_ADD)
  int ld_f32;
  __nv_bfloat16* out_bf16;  // row-major [M][ld_bf16]
  int ld_bf16;
  __nv_bfloat16* out_t;     // transposed [N][ld_t] (optional)
  int ld_t;
  const float* zprev;       // DGRAD_SILU: pre-activation [M][ld_zprev]
  int ld_zprev;
  const float* lohi;        // SEEDS: joint limits [2][n_dof]
  int n_dof;
  int tma_store;            // FWD_SILU: out_bf16 is written through the output tensor map
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and *err set) after kWaitNs, or as soon as another
// thread of the grid has reported an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int*)err != 0) return false;
    if (globaltimer() - t0 > kWaitNs) {
      atomicCAS(err, 0, code);
      return false;
    }
  }
}

// Bounded wait that does not give up early on other threads' errors: used to
// let this CTA's own in-flight copies and MMAs finish before teardown.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Bulk tensor store shared -> global (one bulk group per call site's commit).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one group still reading shared memory
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the bulk-copy engine
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows, 128B swizzle,
// 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
// SiLU through one MUFU tanh: z sigmoid(z) = z (1 + tanh(z / 2)) / 2.  The
// hardware tanh approximation (relative error ~2^-11) is below the BF16
// rounding the output receives.
__device__ __forceinline__ float silu_fast(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return 0.5f * z * (1.f + t);
}
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Split form of the 32-column TMEM load: issue, then wait with the registers
// bound to the wait so that no use can be scheduled before the data arrives.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Packed FP32 pairs (two lanes of work per instruction on sm_100-class SMs).
__device__ __forceinline__ uint64_t f32x2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f32x2_split(uint64_t r) {
  float2 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}
__device__ __forceinline__ uint64_t fma_f32x2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t add_f32x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float tanh_fast(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}

// SiLU epilogue of 32 accumulator columns: h = acc/2 + b/2 = z/2,
// silu(z) = h + h tanh(h), in packed pairs; z = 2h goes to Z when kept
// (training), the BF16 transposed copy too.  The BF16 row-major output goes
// either straight to global memory or, with `stage` set, into this lane's
// 64-byte row of a 32 x 32 shared-memory tile (16-byte chunks written in a
// lane-rotated order: conflict-free) for a bulk tensor store.
__device__ __forceinline__ void epilogue_silu32(const Epilogue& ep, int row, bool row_ok, int col0,
                                                const uint32_t (&r)[32], uint8_t* stage, int lane) {
  const uint64_t half2 = f32x2(0.5f, 0.5f);
  uint32_t packed[16];
  float z[32];
  const float2* b2 = reinterpret_cast<const float2*>(ep.bias + col0);
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
    z[2 * i] = h.x + h.x;
    z[2 * i + 1] = h.y + h.y;
  }
  if (ep.out_t) {  // transposed copy for the weight gradients; padded rows stay zero
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint32_t w = row_ok ? packed[i] : 0u;
      ep.out_t[(size_t)(col0 + 2 * i) * ep.ld_t + row] = __ushort_as_bfloat16((unsigned short)(w & 0xffffu));
      ep.out_t[(size_t)(col0 + 2 * i + 1) * ep.ld_t + row] = __ushort_as_bfloat16((unsigned short)(w >> 16));
    }
  }
  if (row_ok && ep.out_f32) {
    float4* o = (float4*)(ep.out_f32 + (size_t)row * ep.ld_f32 + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = make_float4(z[4 * i], z[4 * i + 1], z[4 * i + 2], z[4 * i + 3]);
  }
  if (stage) {
    uint4* rowp = reinterpret_cast<uint4*>(stage + lane * 64);
    const int rot = (lane >> 1) & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = (i + rot) & 3;
      uint4 w;
      w.x = k == 0 ? packed[0] : k == 1 ? packed[4] : k == 2 ? packed[8] : packed[12];
      w.y = k == 0 ? packed[1] : k == 1 ? packed[5] : k == 2 ? packed[9] : packed[13];
      w.z = k == 0 ? packed[2] : k == 1 ? packed[6] : k == 2 ? packed[10] : packed[14];
      w.w = k == 0 ? packed[3] : k == 1 ? packed[7] : k == 2 ? packed[11] : packed[15];
      rowp[k] = w;
    }
    return;
  }
  if (!row_ok) return;
  uint4* o = (uint4*)(ep.out_bf16 + (size_t)row * ep.ld_bf16 + col0);
#pragma unroll
  for (int i = 0; i < 4; ++i) o[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
}

#ifndef PK_EPI_WARPS
#define PK_EPI_WARPS 8
#endif
// Epilogue warps: two per TMEM lane quarter, each taking half of the columns
// (or one per quarter with 4).
constexpr int kEpiWarps = PK_EPI_WARPS;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // warp 0: TMA, warp 1: MMA, then the epilogue warps

template <int BN>
struct SmemLayout {
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kBarOffset = kStages * kStageBytes;
  // output staging of the SiLU epilogue: two 32 x 32 BF16 tiles per epilogue warp
  static constexpr int kStoreOffset = (kBarOffset + 256 + 1023) & ~1023;
  static constexpr int kStoreTile = 32 * 32 * 2;
  static constexpr int kBytes = kStoreOffset + kEpiWarps * 2 * kStoreTile + 1024;  // + alignment slack
  static constexpr uint32_t kTmemCols = 2 * BN;           // two accumulator buffers
};


// Epilogue of 32 columns [col0, col0 + 32) of one accumulator row.
__device__ __forceinline__ void epilogue32(const Epilogue& ep, int row, bool row_ok, int col0, float* v) {
  if (ep.mode == EPI_WGRAD_ADD) {
    if (row_ok) {
      float* o = ep.out_f32 + (size_t)row * ep.ld_f32 + col0;
#pragma unroll
      for (int i = 0; i < 32; i += 4) atomicAdd((float4*)(o + i), make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
    }
    return;
  }
  if (ep.mode == EPI_FWD_LINEAR) {
    if (row_ok) {
      float* o = ep.out_f32 + (size_t)row * ep.ld_f32;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (col0 + i < ep.n_valid) o[col0 + i] = v[i] + __ldg(ep.bias + col0 + i);
    }
    return;
  }
  if (ep.mode == EPI_SEEDS) {
    if (row_ok) {
      float* o = ep.out_f32 + (size_t)row * ep.ld_f32;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int c = col0 + i;
        if (c < ep.n_valid) {
          const int j = c % ep.n_dof;
          const float lo = __ldg(ep.lohi + j), hi = __ldg(ep.lohi + ep.n_dof + j);
          o[c] = 0.5f * (lo + hi) + 0.5f * (hi - lo) * tanhf(v[i] + __ldg(ep.bias + c));
        }
      }
    }
    return;
  }
  float a[32];
  if (ep.mode == EPI_FWD_SILU) {
    const float4* b4 = (const float4*)(ep.bias + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 b = __ldg(b4 + i);
      v[4 * i + 0] += b.x; v[4 * i + 1] += b.y; v[4 * i + 2] += b.z; v[4 * i + 3] += b.w;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = silu_fast(v[i]);
    if (ep.out_f32 && row_ok) {
      float4* o = (float4*)(ep.out_f32 + (size_t)row * ep.ld_f32 + col0);
#pragma unroll
      for (int i = 0; i < 8; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
  } else {  // EPI_DGRAD_SILU
    const float4* zp = (const float4*)(ep.zprev + (size_t)(row_ok ? row : 0) * ep.ld_zprev + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 z = row_ok ? zp[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      a[4 * i + 0] = v[4 * i + 0] * dsilu_f(z.x);
      a[4 * i + 1] = v[4 * i + 1] * dsilu_f(z.y);
      a[4 * i + 2] = v[4 * i + 2] * dsilu_f(z.z);
      a[4 * i + 3] = v[4 * i + 3] * dsilu_f(z.w);
    }
  }
  if (row_ok) {
    uint4 pk4[4];
    uint32_t* w = (uint32_t*)pk4;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      __nv_bfloat162 h = __floats2bfloat162_rn(a[2 * i], a[2 * i + 1]);
      w[i] = *(uint32_t*)&h;
    }
    uint4* o = (uint4*)(ep.out_bf16 + (size_t)row * ep.ld_bf16 + col0);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = pk4[i];
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = 0.f;  // padded rows stay zero in the transposed copy
  }
  if (ep.out_t) {
#pragma unroll
    for (int i = 0; i < 32; ++i) ep.out_t[(size_t)(col0 + i) * ep.ld_t + row] = __float2bfloat16_rn(a[i]);
  }
}

// Persistent GEMM: CTAs stride over the (m, n, k-split) tiles; the MMA warp
// fills one TMEM accumulator while the epilogue warps drain the other.
template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, int m_tiles, int n_tiles, int splits, int K,
                        int kb_per_split, Epilogue ep, int* err) {
  using L = SmemLayout<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + L::kBarOffset);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;  // [2] accumulator ready (MMA -> epilogue)
  uint64_t* tempty = tfull + 2;       // [2] accumulator drained (epilogue -> MMA)
  uint64_t* drain = tempty + 2;       // teardown: all MMAs of this CTA done
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb_total = K / kBK;
  const int n_tiles_total = m_tiles * n_tiles * splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  const bool silu_fwd = ep.mode == EPI_FWD_SILU;
  if (warp == 0) tmem_alloc(tmem_slot, L::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      uint32_t it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x) {
        const int z = t / (m_tiles * n_tiles), r = t % (m_tiles * n_tiles);
        const int m0 = (r / n_tiles) * kBM, n0 = (r % n_tiles) * BN;
        const int kb0 = z * kb_per_split;
        const int kb1 = min(kb0 + kb_per_split, nkb_total);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % kStages;
          const uint32_t round = it / kStages;
          if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, err, 1)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * L::kStageBytes;
          mbar_arrive_expect_tx(&full[s], L::kStageBytes);
          tma_load_2d(sa, &tmA, &full[s], kb * kBK, m0);
          tma_load_2d(sa + L::kABytes, &tmB, &full[s], kb * kBK, n0);
          ++issued;
        }
      }
      if (!ok)  // let the loads already issued land before teardown
        for (uint32_t i = (issued > (uint32_t)kStages ? issued - kStages : 0); i < issued; ++i)
          mbar_drain(&full[i % kStages], (i / kStages) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BN);
      uint32_t it = 0, tc = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x, ++tc) {
        const int z = t / (m_tiles * n_tiles);
        const int kb0 = z * kb_per_split;
        const int kb1 = min(kb0 + kb_per_split, nkb_total);
        const uint32_t acc = tc & 1, use = tc >> 1;
        if (use > 0 && !mbar_wait(&tempty[acc], (use - 1) & 1, err, 4)) break;
        tc_fence_after();
        const uint32_t d = tmem + acc * BN;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % kStages;
          if (!mbar_wait(&full[s], (it / kStages) & 1, err, 2)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * L::kStageBytes);
          const uint64_t ad = smem_desc(sa), bd = smem_desc(sa + L::kABytes);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            mma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&tfull[acc]);
      }
      mma_commit(drain);  // completes once every MMA issued above has finished
      mbar_drain(drain, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31,
    //      columns [h BN / H, (h + 1) BN / H) with h = (w - 2) / 4, H = kEpiWarps / 4
    const int q = warp & 3;
    constexpr int H = kEpiWarps / 4;
    const int h = (warp - 2) / 4;
    uint8_t* stage_base = smem + L::kStoreOffset + (warp - 2) * 2 * L::kStoreTile;
    int sbuf = 0;
    uint32_t tc = 0;
    for (int t = blockIdx.x; t < n_tiles_total; t += gridDim.x, ++tc) {
      const int r = t % (m_tiles * n_tiles);
      const int m0 = (r / n_tiles) * kBM, n0 = (r % n_tiles) * BN;
      const uint32_t acc = tc & 1;
      // lane 0 waits, the warp follows (keeps the collective TMEM loads uniform)
      uint32_t ready = 0;
      if (lane == 0) ready = mbar_wait(&tfull[acc], (tc >> 1) & 1, err, 3) ? 1u : 0u;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) break;
      tc_fence_after();
      const int row = m0 + q * 32 + lane;
      const bool row_ok = row < ep.m_valid;
      const uint32_t base = tmem + acc * BN + ((uint32_t)(q * 32) << 16);
      const int cbeg = h * (BN / H), cend = (h + 1) * (BN / H);
      if (silu_fwd) {
        // TMEM loads one chunk ahead of the arithmetic; with the tensor-map
        // store, each 32 x 32 output block goes through a double-buffered
        // shared-memory tile (the store issued two blocks earlier must have
        // finished reading a buffer before it is rewritten)
        uint32_t ra[32], rb[32];
        const int y0 = m0 + q * 32;
        auto chunk = [&](int c, const uint32_t(&rr)[32]) {
          uint8_t* buf = nullptr;
          if (ep.tma_store) {
            buf = stage_base + sbuf * L::kStoreTile;
            if (lane == 0) bulk_wait_read_1();
            __syncwarp();
          }
          epilogue_silu32(ep, row, row_ok, n0 + c, rr, buf, lane);
          if (ep.tma_store) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(&tmC, buf, n0 + c, y0);
              bulk_commit();
            }
            sbuf ^= 1;
          }
        };
        tmem_ld32_issue(base + (uint32_t)cbeg, ra);
        tmem_ld_wait(ra);
#pragma unroll 1
        for (int c0 = cbeg; c0 < cend; c0 += 64) {
          const bool more = c0 + 32 < cend;
          if (more) tmem_ld32_issue(base + (uint32_t)(c0 + 32), rb);
          chunk(c0, ra);
          if (!more) break;
          tmem_ld_wait(rb);
          const bool more2 = c0 + 64 < cend;
          if (more2) tmem_ld32_issue(base + (uint32_t)(c0 + 64), ra);
          chunk(c0 + 32, rb);
          if (more2) tmem_ld_wait(ra);
        }
      } else {
#pragma unroll 1
        for (int c0 = cbeg; c0 < cend; c0 += 32) {
          float v[32];
          tmem_ld32(base + (uint32_t)c0, v);
          epilogue32(ep, row, row_ok, n0 + c0, v);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
    if (lane == 0) bulk_wait_all();  // the output stores are complete before the CTA exits
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, L::kTmemCols);
}

}  // namespace tc
}  // namespace pk
