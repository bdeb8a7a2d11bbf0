// BF16 tensor-core GEMM on tcgen05 (sm_103a) and the small kernels around
// it that the learned proposal's MLP needs (forward, backward, Adam).
//
// gemm_bf16_tn: D[M x N] = epilogue(alpha * A[M x K] * B[N x K]^T), A and B
// bf16 row-major with K contiguous ("TN"), accumulation in fp32 in TMEM.
// One CTA of 4 warps computes a 128 x BN tile (BN <= 256): K is staged in
// chunks of 64 into shared memory in the canonical K-major layout, one
// thread issues the MMAs and commits them to an mbarrier, all threads wait
// (bounded), and the four warps read their 32 TMEM lanes for the epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pb_internal.h"
#include "tc_gemm.cuh"

namespace pb {

enum : int {
  kEpiRelu = 1,     // max(x, 0)
  kEpiOutBf16 = 2,  // store bf16 (else fp32)
  kEpiAccum = 4,    // fp32 output: D += x
  kEpiMask = 8,     // x *= (mask[row, col] > 0)   (ReLU derivative)
};

struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  void* D;
  const float* bias;  // per output column, may be null
  const __nv_bfloat16* mask;
  int lda, ldb, ldd, ldm;
  int M, N, K;
  int flags;
  float alpha;
  uint32_t* status;  // set to PB_ETIMEOUT when a bounded wait expires
};

__host__ __device__ inline int gemm_tile_n(int N) {
  int bn = ((N + 15) / 16) * 16;
  return bn > 256 ? 256 : bn;
}
__host__ __device__ inline uint32_t tmem_cols(int bn) {
  uint32_t c = 32;
  while ((int)c < bn) c <<= 1;
  return c;
}

__global__ void __launch_bounds__(128) gemm_bf16_tn_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int BN = gemm_tile_n(g.N);
  uint8_t* sA = sm;            // 128 x 64 bf16 (16 KiB)
  uint8_t* sB = sm + 16384;    // BN x 64 bf16 (<= 32 KiB)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  const uint32_t ncols = tmem_cols(BN);

  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = tc::idesc_bf16_f32(128, BN);
  uint32_t phase = 0;
  bool ok = true;

  for (int k0 = 0; k0 < g.K; k0 += tc::kChunkK) {
    // stage A (128 x 64) and B (BN x 64): one 16-byte vector = 8 K-elements
    for (int v = tid; v < 128 * 8; v += 128) {
      const int r = v >> 3, c = v & 7, k = k0 + c * 8, row = m0 + r;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (row < g.M && k < g.K)
        val = *reinterpret_cast<const uint4*>(g.A + (size_t)row * g.lda + k);
      *reinterpret_cast<uint4*>(sA + tc::chunk_offset(r, c * 8)) = val;
    }
    for (int v = tid; v < BN * 8; v += 128) {
      const int r = v >> 3, c = v & 7, k = k0 + c * 8, row = n0 + r;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (row < g.N && k < g.K)
        val = *reinterpret_cast<const uint4*>(g.B + (size_t)row * g.ldb + k);
      *reinterpret_cast<uint4*>(sB + tc::chunk_offset(r, c * 8)) = val;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
      for (int s = 0; s < tc::kChunkK / 16; ++s) {
        if (k0 + 16 * s >= g.K) break;
        // K-step s covers the K-chunks 2s, 2s+1 (LBO apart)
        const uint64_t ad = tc::smem_desc(a0 + s * 2 * tc::kLBO, tc::kLBO, tc::kSBO);
        const uint64_t bd = tc::smem_desc(b0 + s * 2 * tc::kLBO, tc::kLBO, tc::kSBO);
        tc::mma_bf16(tbase, ad, bd, idesc, (k0 > 0) || (s > 0));
      }
      tc::mma_commit(&mbar);
    }
    ok = tc::mbar_wait(&mbar, phase);
    phase ^= 1u;
    if (!ok) {
      if (g.status) atomicCAS(g.status, 0u, (uint32_t)PB_ETIMEOUT);
      break;
    }
    tc::fence_after_sync();
    __syncthreads();  // shared operands may be overwritten now
  }

  if (ok) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row >= g.M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = n0 + c0 + i;
        if (col >= g.N) continue;
        float x = g.alpha * v[i];
        if (g.bias) x += g.bias[col];
        if (g.flags & kEpiRelu) x = fmaxf(x, 0.f);
        if (g.flags & kEpiMask)
          x = (__bfloat162float(g.mask[(size_t)row * g.ldm + col]) > 0.f) ? x : 0.f;
        if (g.flags & kEpiOutBf16) {
          reinterpret_cast<__nv_bfloat16*>(g.D)[(size_t)row * g.ldd + col] = __float2bfloat16(x);
        } else {
          float* d = reinterpret_cast<float*>(g.D) + (size_t)row * g.ldd + col;
          *d = (g.flags & kEpiAccum) ? *d + x : x;
        }
      }
    }
  }
  if (!ok) tc::mbar_wait(&mbar, phase ^ 1u);  // let MMAs in flight drain (bounded)
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tn_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int BN = gemm_tile_n(g.N);
  dim3 grid((g.M + 127) / 128, (g.N + BN - 1) / BN);
  gemm_bf16_tn_kernel<<<grid, 128, 16384 + BN * 64 * 2, st>>>(g);
  return cudaGetLastError();
}

}  // namespace pb

using namespace pb;

extern "C" PB_API int pb_gemm_bf16(const void* dA, int lda, const void* dB, int ldb, void* dD,
                                   int ldd, const float* dbias, const void* dmask, int ldm, int M,
                                   int N, int K, int flags, float alpha, uintptr_t stream) {
  if (!dA || !dB || !dD || M <= 0 || N <= 0 || K <= 0) return PB_EINVAL;
  if ((K % 8) || (lda % 8) || (ldb % 8) || lda < K || ldb < K || ldd < N) return PB_EINVAL;
  if (((uintptr_t)dA & 15) || ((uintptr_t)dB & 15)) return PB_EINVAL;
  if ((flags & kEpiMask) && (!dmask || ldm < N)) return PB_EINVAL;
  GemmArgs g{};
  g.A = static_cast<const __nv_bfloat16*>(dA);
  g.B = static_cast<const __nv_bfloat16*>(dB);
  g.D = dD;
  g.bias = dbias;
  g.mask = static_cast<const __nv_bfloat16*>(dmask);
  g.lda = lda;
  g.ldb = ldb;
  g.ldd = ldd;
  g.ldm = ldm;
  g.M = M;
  g.N = N;
  g.K = K;
  g.flags = flags;
  g.alpha = alpha;
  g.status = nullptr;
  return launch_gemm_bf16(g, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? PB_OK
                                                                                   : PB_ECUDA;
}
