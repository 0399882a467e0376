// Blackwell tensor-core GEMM of the learned coarse basis's network:
// C (M x N) = A (M x K) B (N x K)^T with bfloat16 operands, both K-major
// (k contiguous), rows padded to a multiple of 8 entries (16 bytes, the TMA
// stride rule), FP32 accumulation in tensor memory, and the network's fused
// epilogues (bias; ReLU to bfloat16; ReLU-mask to bfloat16; FP32).
//
// One CTA of four warps per 128 x BN tile of C (BN = 64 or 128):
//   warp 0, lane 0: TMA producer -- 2-D tiled copies (cp.async.bulk.tensor)
//     of a 128 x 64 tile of A and a BN x 64 tile of B per stage into a
//     four-stage ring, 128-byte swizzle, completion counted on the stage's
//     "full" mbarrier;
//   warp 1, lane 0: MMA issuer -- four tcgen05.mma (M 128, N BN, K 16) per
//     stage from shared-memory descriptors into one TMEM accumulator, then
//     tcgen05.commit to the stage's "empty" mbarrier (the producer reuses the
//     stage) and, after the last stage, to "done";
//   all four warps: epilogue -- each warp reads its 32 TMEM lanes (rows) with
//     tcgen05.ld and writes its rows of C.
// Warp 1 allocates and frees the 128 TMEM columns.  Every mbarrier wait is
// bounded; on expiry the kernel raises g_gemm_timeout, skips the rest of its
// work (the waits that follow are bounded too), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "../../include/tgms.h"
#include "common.cuh"

namespace tg {

__device__ int g_gemm_timeout;   // raised by an expired wait of k_gemm_tc (read and cleared by the host)

namespace {

constexpr int kTcM = 128;                 // rows of a CTA tile (the tcgen05.mma M)
constexpr int kTcBK = 64;                 // K per stage: 64 bfloat16 = one 128-byte swizzle row
constexpr int kTcStages = 4;
constexpr int kTcMaxBN = 128;
constexpr unsigned kTcBytesA = kTcM * kTcBK * 2;        // 16 KB
constexpr unsigned kTcBytesB = kTcMaxBN * kTcBK * 2;    // 16 KB (BN = 64 uses half)
constexpr unsigned kTcStage = kTcBytesA + kTcBytesB;
constexpr unsigned kTcTmemCols = 128;
constexpr long long kTcWaitLimit = 1LL << 24;

struct TcArgs {
  int M, N, K, bn;
  const float* bias;   // [N] or NULL
  int epi;             // kEpi* (common.cuh)
  float* outf;
  __nv_bfloat16* outh;
  long long som;
  const __nv_bfloat16* mask;
};

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(unsigned bar, unsigned parity) {
  for (long long i = 0; i < kTcWaitLimit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// 2-D tiled TMA load: box at (c0 = k, c1 = row) of the tensor map into dst
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int c0, int c1, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused for this layout, the fixed 0b001 at bits 46-48,
// swizzle mode 2 (128 B) at bits 61-63.
__device__ __forceinline__ unsigned long long desc_k128(unsigned addr) {
  unsigned long long d = (unsigned long long)((addr & 0x3FFFFu) >> 4);
  d |= 1ull << 16;
  d |= (unsigned long long)(1024u >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}
// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr unsigned idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                    const __grid_constant__ CUtensorMap tb, TcArgs g) {
  extern __shared__ unsigned char dyn[];
  __shared__ __align__(8) unsigned long long full_bar[kTcStages], empty_bar[kTcStages], done_bar;
  __shared__ unsigned tmem_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the stage ring, 1024-byte aligned (the swizzle pattern repeats every 1024 bytes)
  const unsigned raw = saddr(dyn);
  const unsigned ring = raw + ((1024u - (raw & 1023u)) & 1023u);
  const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * g.bn;
  const int nk = (g.K + kTcBK - 1) / kTcBK;
  const unsigned bytes_stage = kTcBytesA + (unsigned)g.bn * kTcBK * 2;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      bar_init(saddr(&full_bar[s]), 1);
      bar_init(saddr(&empty_bar[s]), 1);
    }
    bar_init(saddr(&done_bar), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_sh)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_sh;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kTcStages;
      if (kb >= kTcStages && !bar_wait(saddr(&empty_bar[s]), (unsigned)((kb / kTcStages - 1) & 1))) {
        atomicExch(&abort_sh, 1);
        break;
      }
      if (*(volatile int*)&abort_sh) break;
      const unsigned a = ring + (unsigned)s * kTcStage;
      bar_expect_tx(saddr(&full_bar[s]), bytes_stage);
      tma_load_2d(a, &ta, kb * kTcBK, m0, saddr(&full_bar[s]));
      tma_load_2d(a + kTcBytesA, &tb, kb * kTcBK, n0, saddr(&full_bar[s]));
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const unsigned idesc = idesc_bf16(kTcM, g.bn);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kTcStages;
      if (!bar_wait(saddr(&full_bar[s]), (unsigned)((kb / kTcStages) & 1))) {
        atomicExch(&abort_sh, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a = ring + (unsigned)s * kTcStage, b = a + kTcBytesA;
#pragma unroll
      for (int k = 0; k < kTcBK / 16; ++k) {
        const unsigned long long ad = desc_k128(a + 32u * k), bd = desc_k128(b + 32u * k);
        const unsigned acc = (kb > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       saddr(&empty_bar[s]))
                   : "memory");
    }
    // the accumulator is complete once every MMA issued above has finished
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     saddr(&done_bar))
                 : "memory");
  }
  __syncwarp();
  // epilogue: warp w owns TMEM lanes (rows of the tile) 32 w .. 32 w + 31
  if (!bar_wait(saddr(&done_bar), 0u)) atomicExch(&abort_sh, 1);
  __syncthreads();   // every role has finished: the abort flag is final and the same for all threads
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool run_epilogue = (*(volatile int*)&abort_sh) == 0;
  if (run_epilogue) {   // uniform over the CTA, so every warp runs its tcgen05.ld converged
    const int row = m0 + 32 * warp + lane;
    for (int c0 = 0; c0 < g.bn; c0 += 32) {
      unsigned r[32];
      const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < g.M) {
        const int col0 = n0 + c0;
        const long long o0 = (long long)row * g.som + col0;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          v[j] = __uint_as_float(r[j]);
          if (g.bias && col0 + j < g.N) v[j] += g.bias[col0 + j];
        }
        // a row's 32 columns as 16-byte vectors where the tile is whole and aligned
        const bool whole = col0 + 32 <= g.N;
        if (g.epi == kEpiF32) {
          if (whole && (o0 & 3) == 0) {
            float4* dst = reinterpret_cast<float4*>(g.outf + o0);
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col0 + j < g.N) g.outf[o0 + j] = v[j];
          }
        } else {
          if (g.epi == kEpiMaskBf16) {
            if (whole && (o0 & 7) == 0) {
              const uint4* mk = reinterpret_cast<const uint4*>(g.mask + o0);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const uint4 m = mk[q];
                const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&m);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  const float2 f = __bfloat1622float2(h[t]);
                  if (!(f.x > 0.0f)) v[8 * q + 2 * t] = 0.0f;
                  if (!(f.y > 0.0f)) v[8 * q + 2 * t + 1] = 0.0f;
                }
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (col0 + j < g.N && !(__bfloat162float(g.mask[o0 + j]) > 0.0f)) v[j] = 0.0f;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.0f);
          }
          if (whole && (o0 & 7) == 0) {
            uint4* dst = reinterpret_cast<uint4*>(g.outh + o0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint4 w;
              __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
              for (int t = 0; t < 4; ++t) h[t] = __floats2bfloat162_rn(v[8 * q + 2 * t], v[8 * q + 2 * t + 1]);
              dst[q] = w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col0 + j < g.N) g.outh[o0 + j] = __float2bfloat16_rn(v[j]);
          }
        }
      }
    }
  }
  if (threadIdx.x == 0 && !run_epilogue) atomicOr(&g_gemm_timeout, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

// Operand packing: dst[r * ld + k] = src[(rmap ? rmap[r] : r) * s_row +
// (kmap ? kmap[k] : k) * s_k] for k < K, zero for K <= k < ld.  Gathers the
// training batch's rows, transposes the backward pass's operands to K-major
// and pads rows to the 16-byte TMA stride.
__global__ void k_pack_kmajor(const __nv_bfloat16* __restrict__ src, long long s_row, long long s_k,
                              const int* __restrict__ rmap, const int* __restrict__ kmap, int R, int K, int ld,
                              __nv_bfloat16* __restrict__ dst) {
  const long long tot = (long long)R * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / ld), k = (int)(t % ld);
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    if (k < K) {
      const long long rr = rmap ? (long long)rmap[r] : (long long)r;
      const long long kk = kmap ? (long long)kmap[k] : (long long)k;
      v = src[rr * s_row + kk * s_k];
    }
    dst[t] = v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// tensor map of a K-major bfloat16 operand: rows x K (row stride ld entries),
// boxes of 64 (k) x box_rows, 128-byte swizzle, zero fill outside
int encode_operand(CUtensorMap* map, const __nv_bfloat16* ptr, int rows, int K, int ld, int box_rows) {
  auto fn = tensor_map_encoder();
  if (!fn) return TG_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TG_OK : TG_ERR_CUDA;
}

}  // namespace

size_t gemm_tc_smem() { return (size_t)kTcStages * kTcStage + 1024; }

int gemm_tc(const TcOperand& a, const TcOperand& b, int M, int N, int K, const float* bias, int epi, float* outf,
            __nv_bfloat16* outh, long long som, const __nv_bfloat16* mask, cudaStream_t s) {
  if (M <= 0 || N <= 0) return TG_OK;
  // the TMA rules: 16-byte aligned base, row stride a multiple of 16 bytes
  auto ok = [](const TcOperand& o) {
    return (reinterpret_cast<uintptr_t>(o.p) & 15u) == 0 && o.ld % 8 == 0 && o.ld >= o.K;
  };
  if (!ok(a) || !ok(b) || a.K < K || b.K < K || a.rows < M || b.rows < N) return TG_ERR_INVALID_ARG;
  const int bn = (N <= 64) ? 64 : kTcMaxBN;
  CUtensorMap ta, tb;
  int rc = encode_operand(&ta, a.p, a.rows, K, a.ld, kTcM);
  if (!rc) rc = encode_operand(&tb, b.p, b.rows, K, b.ld, bn);
  if (rc) return rc;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem());
  });
  TcArgs g{M, N, K, bn, bias, epi, outf, outh, som, mask};
  dim3 grid((N + bn - 1) / bn, (M + kTcM - 1) / kTcM);
  TG_COUNT(1);
  k_gemm_tc<<<grid, 128, gemm_tc_smem(), s>>>(ta, tb, g);
  return TG_OK;
}

void pack_kmajor(const __nv_bfloat16* src, long long s_row, long long s_k, const int* rmap, const int* kmap, int R,
                 int K, int ld, __nv_bfloat16* dst, cudaStream_t s) {
  const long long tot = (long long)R * ld;
  if (tot <= 0) return;
  TG_COUNT(1);
  k_pack_kmajor<<<(int)std::min<long long>((tot + 255) / 256, 4096), 256, 0, s>>>(src, s_row, s_k, rmap, kmap, R,
                                                                                  K, ld, dst);
}

int read_and_clear_gemm_timeout() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_gemm_timeout, sizeof(int)) != cudaSuccess) return 1;
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_gemm_timeout, &zero, sizeof(int));
  }
  return v;
}

}  // namespace tg
