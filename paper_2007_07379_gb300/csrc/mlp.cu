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
#include "philox.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

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

// Tile width: N rounded up to 16, at most 256, narrowed to 128 or 64 when
// the row tiles alone would leave most of the 152 SMs idle.
__host__ __device__ inline int gemm_tile_n(int M, int N) {
  int bn = ((N + 15) / 16) * 16;
  if (bn > 256) bn = 256;
  const int mt = (M + 127) / 128;
  if (bn > 128 && mt * ((N + bn - 1) / bn) < 120) bn = 128;
  if (bn > 64 && mt * ((N + bn - 1) / bn) < 120) bn = 64;
  return bn;
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
  const int BN = gemm_tile_n(g.M, g.N);
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
      const bool in = row < g.M && k < g.K;
      tc::cp_async16(sA + tc::chunk_offset(r, c * 8),
                     in ? (const void*)(g.A + (size_t)row * g.lda + k) : (const void*)g.A, in ? 16u : 0u);
    }
    for (int v = tid; v < BN * 8; v += 128) {
      const int r = v >> 3, c = v & 7, k = k0 + c * 8, row = n0 + r;
      const bool in = row < g.N && k < g.K;
      tc::cp_async16(sB + tc::chunk_offset(r, c * 8),
                     in ? (const void*)(g.B + (size_t)row * g.ldb + k) : (const void*)g.B, in ? 16u : 0u);
    }
    tc::cp_async_wait_all();
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
    // one decision for the whole CTA: a thread that gave up and one that saw
    // the commit must take the same branch (the loop has barriers)
    ok = __syncthreads_and(tc::mbar_wait(&mbar, phase)) != 0;
    phase ^= 1u;
    if (!ok) {
      if (tid == 0 && g.status) atomicCAS(g.status, 0u, (uint32_t)PB_ETIMEOUT);
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
  if (!ok && tid == 0) tc::mbar_wait(&mbar, phase ^ 1u);  // let MMAs in flight drain (bounded)
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// One-time set-up outside any stream capture (shared-memory opt-in).
cudaError_t mlp_fused_prepare();
cudaError_t mlp_prepare() {
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tn_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
  return e == cudaSuccess ? mlp_fused_prepare() : e;
}

cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t st) {
  const int BN = gemm_tile_n(g.M, g.N);
  dim3 grid((g.M + 127) / 128, (g.N + BN - 1) / BN);
  gemm_bf16_tn_kernel<<<grid, 128, 16384 + BN * 64 * 2, st>>>(g);
  return cudaGetLastError();
}

}  // namespace pb

namespace pb {

// Self-test of the bounded wait every tensor-core kernel here uses: one
// thread initialises a one-arrival mbarrier, arrives on it or not, and
// waits for its first phase with tc::mbar_wait(max_iters).  A wait that runs
// out records PB_ETIMEOUT in the status word the way the GEMM and fused
// kernels do; nothing else (no MMA, no copy, no tensor memory) is in flight.
__device__ uint32_t g_selftest_status;

__global__ void selftest_wait_kernel(int arrive, uint32_t max_iters) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&mbar, 1u);
  if (arrive) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&mbar)) : "memory");
  }
  const bool ok = tc::mbar_wait(&mbar, 0u, max_iters);
  if (!ok) atomicCAS(&g_selftest_status, 0u, (uint32_t)PB_ETIMEOUT);
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(&mbar)) : "memory");
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
  if (mlp_prepare() != cudaSuccess) return PB_ECUDA;
  return launch_gemm_bf16(g, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? PB_OK
                                                                                   : PB_ECUDA;
}

// ===========================================================================
// The proposal network q(s_j | s_{j-1}, j): K_in -> H -> H -> n, ReLU, BF16
// tensor-core GEMMs with fp32 accumulation, fp32 master weights and Adam.
// ===========================================================================
namespace pb {

// Parameter block (fp32, flat): W1 [H x kin], b1 [H], W2 [H x H], b2 [H],
// W3 [npad x H] (rows >= n stay zero), b3 [npad].
struct MlpOffsets {
  size_t W1, b1, W2, b2, W3, b3, total;
};
inline MlpOffsets mlp_offsets(int kin, int H, int npad) {
  MlpOffsets o;
  size_t p = 0;
  o.W1 = p; p += (size_t)H * kin;
  o.b1 = p; p += H;
  o.W2 = p; p += (size_t)H * H;
  o.b2 = p; p += H;
  o.W3 = p; p += (size_t)npad * H;
  o.b3 = p; p += npad;
  o.total = p;
  return o;
}

__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ src, int R, int C,
                                      __nv_bfloat16* __restrict__ dst) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C) tile[i][threadIdx.x] = src[(size_t)r * C + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < C) dst[(size_t)c * R + r] = tile[threadIdx.x][i];
  }
}

cudaError_t transpose_bf16(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst,
                           cudaStream_t st) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  transpose_bf16_kernel<<<grid, block, 0, st>>>(src, R, C, dst);
  return cudaGetLastError();
}

// fp32 [R x C] -> bf16 [R x C] and, when dst_t is given, bf16 [C x R].
__global__ void to_bf16_kernel(const float* __restrict__ src, int R, int C,
                               __nv_bfloat16* __restrict__ dst, __nv_bfloat16* __restrict__ dst_t) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)R * C) return;
  const __nv_bfloat16 v = __float2bfloat16(src[i]);
  dst[i] = v;
  if (dst_t) {
    const size_t r = i / C, c = i % C;
    dst_t[c * R + r] = v;
  }
}

// Columns [k0, k0 + K) of a row-major bf16 [R x ld] matrix into the canonical
// K-major image the tensor cores read from shared memory: core matrices of
// 8 rows x 8 elements (128 bytes), K-adjacent ones 128 bytes apart, 8-row
// groups K * 16 bytes apart.
__global__ void pack_canonical_kernel(const __nv_bfloat16* __restrict__ src, int R, int ld, int k0,
                                      int K, __nv_bfloat16* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one 8-element vector
  const int vecs = K / 8;
  if (i >= R * vecs) return;
  const int r = i / vecs, c = i % vecs;
  const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)r * ld + k0 + c * 8);
  *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(dst) + (size_t)(r >> 3) * (K * 16) + c * 128 +
                            (r & 7) * 16) = v;
}

// dY = (sigmoid(l) - t) / B for the first n columns (0 beyond), bf16, both
// layouts.
__device__ __forceinline__ float bce_grad(float l, float t, int B) {
  return (1.f / (1.f + __expf(-l)) - t) / (float)B;
}
__global__ void bce_grad_kernel(const float* __restrict__ logits, const float* __restrict__ target,
                                int B, int n, int npad, __nv_bfloat16* __restrict__ dY,
                                __nv_bfloat16* __restrict__ dYt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * npad) return;
  const int r = i / npad, c = i % npad;
  const float g = c < n ? bce_grad(logits[(size_t)r * npad + c], target[(size_t)r * n + c], B) : 0.f;
  const __nv_bfloat16 gb = __float2bfloat16(g);
  dY[(size_t)r * npad + c] = gb;
  dYt[(size_t)c * B + r] = gb;
}

// Block c < n: db3[c] = sum over the rows of the fp32 gradient of column c;
// block n: loss = the mean BCE, -[t log s(l) + (1-t) log s(-l)] =
// softplus(l) - t l, computed stably.  Each sum is taken in a fixed order
// (per-thread strided partial sums, then a tree), so that a training run is
// reproducible bit for bit.
__global__ void __launch_bounds__(256) bce_sums_kernel(const float* __restrict__ logits,
                                                       const float* __restrict__ target, int B,
                                                       int n, int npad, float* __restrict__ db3,
                                                       float* __restrict__ loss) {
  __shared__ float part[256];
  const int c = blockIdx.x, tid = threadIdx.x;
  float acc = 0.f;
  if (c < n) {
    for (int r = tid; r < B; r += 256)
      acc += bce_grad(logits[(size_t)r * npad + c], target[(size_t)r * n + c], B);
  } else {
    for (int i = tid; i < B * n; i += 256) {
      const int r = i / n, q = i % n;
      const float l = logits[(size_t)r * npad + q], t = target[(size_t)r * n + q];
      acc += (fmaxf(l, 0.f) + log1pf(__expf(-fabsf(l))) - t * l) / (float)B;
    }
  }
  part[tid] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) part[tid] += part[tid + s];
    __syncthreads();
  }
  if (tid == 0) {
    if (c < n) db3[c] = part[0];
    else if (loss) *loss = part[0];
  }
}

// out[j] = sum_b M[j][b] (bf16 rows, fp32 sums), one warp per row.
__global__ void rowsum_bf16_kernel(const __nv_bfloat16* __restrict__ Mt, int R, int C,
                                   float* __restrict__ out) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= R) return;
  float s = 0.f;
  for (int c = lane; c < C; c += 32) s += __bfloat162float(Mt[(size_t)row * C + c]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[row] = s;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace pb

namespace {

struct MlpLayout {
  size_t w, m, v, g, W1, W2, W3, W2t, W3t, W1p, W2p, W3p, X, Xt, H1, H1t, H2, H2t, dY, dYt, dZ2,
      dZ2t, dZ1, dZ1t, logits, target, loss, status, total;
};

MlpLayout mlp_layout(int kin, int H, int npad, int B) {
  const pb::MlpOffsets o = pb::mlp_offsets(kin, H, npad);
  MlpLayout L{};
  size_t p = 0;
  auto take = [&](size_t bytes) {
    p = (p + 255) & ~(size_t)255;
    size_t at = p;
    p += bytes;
    return at;
  };
  L.w = take(o.total * 4);
  L.m = take(o.total * 4);
  L.v = take(o.total * 4);
  L.g = take(o.total * 4);
  L.W1 = take((size_t)H * kin * 2);
  L.W2 = take((size_t)H * H * 2);
  L.W3 = take((size_t)npad * H * 2);
  L.W2t = take((size_t)H * H * 2);
  L.W3t = take((size_t)H * npad * 2);
  L.W1p = take((size_t)H * kin * 2);
  L.W2p = take((size_t)H * H * 2);
  L.W3p = take((size_t)npad * H * 2);
  L.X = take((size_t)B * kin * 2);
  L.Xt = take((size_t)B * kin * 2);
  L.H1 = take((size_t)B * H * 2);
  L.H1t = take((size_t)B * H * 2);
  L.H2 = take((size_t)B * H * 2);
  L.H2t = take((size_t)B * H * 2);
  L.dY = take((size_t)B * npad * 2);
  L.dYt = take((size_t)B * npad * 2);
  L.dZ2 = take((size_t)B * H * 2);
  L.dZ2t = take((size_t)B * H * 2);
  L.dZ1 = take((size_t)B * H * 2);
  L.dZ1t = take((size_t)B * H * 2);
  L.logits = take((size_t)B * npad * 4);
  L.target = take((size_t)B * npad * 4);
  L.loss = take(256);
  L.status = take(16);
  L.total = (p + 255) & ~(size_t)255;
  return L;
}

int mlp_dims(int n, int d, int hidden, int batch, int* kin, int* npad) {
  if (n < 1 || n > 32 || d < 1 || d > 64) return PB_ERANGE;
  if (hidden < 16 || hidden > 256 || hidden % 16) return PB_ERANGE;
  if (batch < 128 || batch % 128) return PB_ERANGE;
  *kin = ((n + d + 15) / 16) * 16;
  *npad = ((n + 15) / 16) * 16;
  return PB_OK;
}

// GEMM helper: D = epi(A[M x K] B[N x K]^T)
cudaError_t mm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, void* D, int ldd,
               int M, int N, int K, int flags, const float* bias, const __nv_bfloat16* mask,
               int ldm, cudaStream_t st, uint32_t* status) {
  pb::GemmArgs g{};
  g.A = A;
  g.B = B;
  g.D = D;
  g.bias = bias;
  g.mask = mask;
  g.lda = lda;
  g.ldb = ldb;
  g.ldd = ldd;
  g.ldm = ldm;
  g.M = M;
  g.N = N;
  g.K = K;
  g.flags = flags;
  g.alpha = 1.f;
  g.status = status;
  return pb::launch_gemm_bf16(g, st);
}

// bf16 copies of the fp32 master weights (W2t, W3t transposed for the backward).
cudaError_t refresh_bf16(pb_mlp* p) {
  const int T = 256;
  const float* w = p->w;
  size_t c = (size_t)p->H * p->kin;
  pb::to_bf16_kernel<<<(unsigned)((c + T - 1) / T), T, 0, p->st>>>(w + p->off_W1, p->H, p->kin, p->W1, nullptr);
  c = (size_t)p->H * p->H;
  pb::to_bf16_kernel<<<(unsigned)((c + T - 1) / T), T, 0, p->st>>>(w + p->off_W2, p->H, p->H, p->W2, p->W2t);
  c = (size_t)p->npad * p->H;
  pb::to_bf16_kernel<<<(unsigned)((c + T - 1) / T), T, 0, p->st>>>(w + p->off_W3, p->npad, p->H, p->W3, p->W3t);
  // canonical images for the fused kernel (W2 in K-chunks of 64)
  auto pack = [&](const __nv_bfloat16* src, int R, int ld, int k0, int K, __nv_bfloat16* dst) {
    const int v = R * (K / 8);
    pb::pack_canonical_kernel<<<(v + T - 1) / T, T, 0, p->st>>>(src, R, ld, k0, K, dst);
  };
  pack(p->W1, p->H, p->kin, 0, p->kin, p->W1p);
  for (int k0 = 0; k0 < p->H; k0 += 64)
    pack(p->W2, p->H, p->H, k0, std::min(64, p->H - k0), p->W2p + (size_t)p->H * k0);
  pack(p->W3, p->npad, p->H, 0, p->H, p->W3p);
  return cudaGetLastError();
}

// Forward of `rows` inputs already in p->X: H1, H2 (bf16), logits (fp32).
cudaError_t mlp_fwd(pb_mlp* p, int rows) {
  cudaError_t e;
  const int flags = pb::kEpiRelu | pb::kEpiOutBf16;
  if ((e = mm(p->X, p->kin, p->W1, p->kin, p->H1, p->H, rows, p->H, p->kin, flags,
              p->w + p->off_b1, nullptr, 0, p->st, p->status)) != cudaSuccess)
    return e;
  if ((e = mm(p->H1, p->H, p->W2, p->H, p->H2, p->H, rows, p->H, p->H, flags, p->w + p->off_b2,
              nullptr, 0, p->st, p->status)) != cudaSuccess)
    return e;
  return mm(p->H2, p->H, p->W3, p->H, p->logits, p->npad, rows, p->npad, p->H, 0,
            p->w + p->off_b3, nullptr, 0, p->st, p->status);
}

// Backward of the mean BCE over `rows` (targets in p->target): gradients
// into p->g, loss into p->loss[0].
cudaError_t mlp_bwd(pb_mlp* p, int rows) {
  cudaError_t e;
  const int B = rows, H = p->H, T = 256;
  cudaMemsetAsync(p->g, 0, p->n_params * 4, p->st);
  cudaMemsetAsync(p->loss, 0, 4, p->st);
  pb::bce_grad_kernel<<<(B * p->npad + T - 1) / T, T, 0, p->st>>>(p->logits, p->target, B, p->n,
                                                                   p->npad, p->dY, p->dYt);
  pb::bce_sums_kernel<<<p->n + 1, 256, 0, p->st>>>(p->logits, p->target, B, p->n, p->npad,
                                                   p->g + p->off_b3, p->loss);
  if ((e = pb::transpose_bf16(p->H2, B, H, p->H2t, p->st)) != cudaSuccess) return e;
  if ((e = pb::transpose_bf16(p->H1, B, H, p->H1t, p->st)) != cudaSuccess) return e;
  if ((e = pb::transpose_bf16(p->X, B, p->kin, p->Xt, p->st)) != cudaSuccess) return e;
  // gW3 = dY^T H2
  if ((e = mm(p->dYt, B, p->H2t, B, p->g + p->off_W3, H, p->npad, H, B, 0, nullptr, nullptr, 0,
              p->st, p->status)) != cudaSuccess)
    return e;
  // dZ2 = (dY W3) * [H2 > 0]
  if ((e = mm(p->dY, p->npad, p->W3t, p->npad, p->dZ2, H, B, H, p->npad,
              pb::kEpiMask | pb::kEpiOutBf16, nullptr, p->H2, H, p->st, p->status)) != cudaSuccess)
    return e;
  if ((e = pb::transpose_bf16(p->dZ2, B, H, p->dZ2t, p->st)) != cudaSuccess) return e;
  // gW2 = dZ2^T H1, gb2 = column sums of dZ2
  if ((e = mm(p->dZ2t, B, p->H1t, B, p->g + p->off_W2, H, H, H, B, 0, nullptr, nullptr, 0,
              p->st, p->status)) != cudaSuccess)
    return e;
  pb::rowsum_bf16_kernel<<<(H + 7) / 8, 256, 0, p->st>>>(p->dZ2t, H, B, p->g + p->off_b2);
  // dZ1 = (dZ2 W2) * [H1 > 0]
  if ((e = mm(p->dZ2, H, p->W2t, H, p->dZ1, H, B, H, H, pb::kEpiMask | pb::kEpiOutBf16, nullptr,
              p->H1, H, p->st, p->status)) != cudaSuccess)
    return e;
  if ((e = pb::transpose_bf16(p->dZ1, B, H, p->dZ1t, p->st)) != cudaSuccess) return e;
  // gW1 = dZ1^T X, gb1 = column sums of dZ1
  if ((e = mm(p->dZ1t, B, p->Xt, B, p->g + p->off_W1, p->kin, H, p->kin, B, 0, nullptr, nullptr,
              0, p->st, p->status)) != cudaSuccess)
    return e;
  pb::rowsum_bf16_kernel<<<(H + 7) / 8, 256, 0, p->st>>>(p->dZ1t, H, B, p->g + p->off_b1);
  return cudaGetLastError();
}

}  // namespace

namespace pb {
cudaError_t mlp_forward_rows(pb_mlp* p, int rows) { return mlp_fwd(p, rows); }
cudaError_t mlp_backward_rows(pb_mlp* p, int rows) { return mlp_bwd(p, rows); }
cudaError_t mlp_adam_step(pb_mlp* p, float lr) {
  p->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
  const size_t c = p->n_params;
  adam_kernel<<<(unsigned)((c + 255) / 256), 256, 0, p->st>>>(p->w, p->g, p->m, p->v, c, lr, b1, b2,
                                                             1e-8f, c1, c2);
  // keep the padded rows of W3 / b3 at zero
  if (p->npad > p->n) {
    cudaMemsetAsync(p->w + p->off_W3 + (size_t)p->n * p->H, 0, (size_t)(p->npad - p->n) * p->H * 4, p->st);
    cudaMemsetAsync(p->w + p->off_b3 + p->n, 0, (size_t)(p->npad - p->n) * 4, p->st);
  }
  return refresh_bf16(p);
}
}  // namespace pb

extern "C" {

PB_API int pb_mlp_workspace_bytes(int n, int d, int hidden, int batch, size_t* bytes) {
  if (!bytes) return PB_EINVAL;
  int kin, npad;
  int rc = mlp_dims(n, d, hidden, batch, &kin, &npad);
  if (rc != PB_OK) return rc;
  *bytes = mlp_layout(kin, hidden, npad, batch).total;
  return PB_OK;
}

PB_API int pb_mlp_create(int n, int d, int hidden, int batch, uint64_t seed, void* d_ws,
                         size_t ws_bytes, uintptr_t stream, pb_mlp** out) {
  if (!out) return PB_EINVAL;
  *out = nullptr;
  int kin, npad;
  int rc = mlp_dims(n, d, hidden, batch, &kin, &npad);
  if (rc != PB_OK) return rc;
  if (!d_ws || ((uintptr_t)d_ws & 255)) return PB_EINVAL;
  const MlpLayout L = mlp_layout(kin, hidden, npad, batch);
  if (ws_bytes < L.total) return PB_ERANGE;
  pb_mlp* p = new (std::nothrow) pb_mlp;
  if (!p) return PB_ENOMEM;
  p->n = n; p->d = d; p->H = hidden; p->kin = kin; p->npad = npad; p->batch = batch;
  p->st = reinterpret_cast<cudaStream_t>(stream);
  p->ws = static_cast<char*>(d_ws);
  p->ws_bytes = ws_bytes;
  {
    const pb::MlpOffsets o = pb::mlp_offsets(kin, hidden, npad);
    p->off_W1 = o.W1; p->off_b1 = o.b1; p->off_W2 = o.W2; p->off_b2 = o.b2;
    p->off_W3 = o.W3; p->off_b3 = o.b3; p->n_params = o.total;
  }
  char* b = p->ws;
  p->w = (float*)(b + L.w); p->m = (float*)(b + L.m); p->v = (float*)(b + L.v); p->g = (float*)(b + L.g);
  p->W1 = (__nv_bfloat16*)(b + L.W1); p->W2 = (__nv_bfloat16*)(b + L.W2); p->W3 = (__nv_bfloat16*)(b + L.W3);
  p->W2t = (__nv_bfloat16*)(b + L.W2t); p->W3t = (__nv_bfloat16*)(b + L.W3t);
  p->W1p = (__nv_bfloat16*)(b + L.W1p); p->W2p = (__nv_bfloat16*)(b + L.W2p);
  p->W3p = (__nv_bfloat16*)(b + L.W3p);
  p->X = (__nv_bfloat16*)(b + L.X); p->Xt = (__nv_bfloat16*)(b + L.Xt);
  p->H1 = (__nv_bfloat16*)(b + L.H1); p->H1t = (__nv_bfloat16*)(b + L.H1t);
  p->H2 = (__nv_bfloat16*)(b + L.H2); p->H2t = (__nv_bfloat16*)(b + L.H2t);
  p->dY = (__nv_bfloat16*)(b + L.dY); p->dYt = (__nv_bfloat16*)(b + L.dYt);
  p->dZ2 = (__nv_bfloat16*)(b + L.dZ2); p->dZ2t = (__nv_bfloat16*)(b + L.dZ2t);
  p->dZ1 = (__nv_bfloat16*)(b + L.dZ1); p->dZ1t = (__nv_bfloat16*)(b + L.dZ1t);
  p->logits = (float*)(b + L.logits); p->target = (float*)(b + L.target); p->loss = (float*)(b + L.loss);
  p->status = (uint32_t*)(b + L.status);
  // Initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64(seed), biases 0.
  std::vector<float> w(p->n_params, 0.f);
  uint64_t s = seed;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto fill = [&](size_t o, int rows, int cols, int fan_in, int live_rows, int live_cols) {
    const float a = 1.f / std::sqrt((float)fan_in);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        const float u = (float)((next() >> 11) * (1.0 / 9007199254740992.0));
        w[o + (size_t)r * cols + c] = (r < live_rows && c < live_cols) ? (2.f * u - 1.f) * a : 0.f;
      }
  };
  fill(p->off_W1, hidden, kin, n + d, hidden, n + d);
  fill(p->off_W2, hidden, hidden, hidden, hidden, hidden);
  fill(p->off_W3, npad, hidden, hidden, n, hidden);
  if (pb::mlp_prepare() != cudaSuccess || cudaMemsetAsync(p->ws, 0, L.total, p->st) != cudaSuccess ||
      cudaMemcpyAsync(p->w, w.data(), w.size() * 4, cudaMemcpyHostToDevice, p->st) != cudaSuccess ||
      refresh_bf16(p) != cudaSuccess || cudaStreamSynchronize(p->st) != cudaSuccess) {
    delete p;
    return PB_ECUDA;
  }
  *out = p;
  return PB_OK;
}

PB_API int pb_selftest_wait(int arrive, uint32_t max_iters, int* status) {
  if (!status || max_iters == 0u || max_iters > (1u << 20)) return PB_EINVAL;
  const uint32_t zero = 0u;
  uint32_t v = 0u;
  if (cudaMemcpyToSymbol(pb::g_selftest_status, &zero, 4) != cudaSuccess) return PB_ECUDA;
  pb::selftest_wait_kernel<<<1, 32>>>(arrive ? 1 : 0, max_iters);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(&v, pb::g_selftest_status, 4) != cudaSuccess)
    return PB_ECUDA;
  *status = (int)v;
  return PB_OK;
}

PB_API int pb_mlp_status(pb_mlp* p, int clear, int* status) {
  if (!p || !status) return PB_EINVAL;
  uint32_t v = 0u;
  if (cudaStreamSynchronize(p->st) != cudaSuccess ||
      cudaMemcpy(&v, p->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PB_ECUDA;
  *status = (int)v;
  if (clear && v != 0u && cudaMemset(p->status, 0, 4) != cudaSuccess) return PB_ECUDA;
  return PB_OK;
}

PB_API int pb_mlp_info(const pb_mlp* p, int* dims /* n, d, hidden, k_in, batch, n_params */) {
  if (!p || !dims) return PB_EINVAL;
  dims[0] = p->n; dims[1] = p->d; dims[2] = p->H; dims[3] = p->kin; dims[4] = p->batch;
  dims[5] = (int)p->n_params;
  return PB_OK;
}

// get != 0: copy the fp32 master parameters to host (flat W1, b1, W2, b2,
// W3 [npad x H], b3 [npad]); get == 0: load them from host and refresh the
// bf16 copies.  Synchronous.
PB_API int pb_mlp_params(pb_mlp* p, float* host, int get) {
  if (!p || !host) return PB_EINVAL;
  if (cudaStreamSynchronize(p->st) != cudaSuccess) return PB_ECUDA;
  if (get) return cudaMemcpy(host, p->w, p->n_params * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? PB_OK : PB_ECUDA;
  if (cudaMemcpy(p->w, host, p->n_params * 4, cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
  if (refresh_bf16(p) != cudaSuccess) return PB_ECUDA;
  return cudaStreamSynchronize(p->st) == cudaSuccess ? PB_OK : PB_ECUDA;
}

PB_API int pb_mlp_grads(pb_mlp* p, float* host) {
  if (!p || !host) return PB_EINVAL;
  if (cudaStreamSynchronize(p->st) != cudaSuccess) return PB_ECUDA;
  return cudaMemcpy(host, p->g, p->n_params * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? PB_OK : PB_ECUDA;
}

// Forward of rows inputs (device bf16 [rows x k_in]) into device fp32
// logits [rows x n] (rows <= batch).
PB_API int pb_mlp_forward(pb_mlp* p, const void* d_x, int rows, float* d_logits) {
  if (!p || !d_x || !d_logits || rows <= 0 || rows > p->batch) return PB_EINVAL;
  if (cudaMemcpyAsync(p->X, d_x, (size_t)rows * p->kin * 2, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess)
    return PB_ECUDA;
  if (mlp_fwd(p, rows) != cudaSuccess) return PB_ECUDA;
  if (cudaMemcpy2DAsync(d_logits, (size_t)p->n * 4, p->logits, (size_t)p->npad * 4, (size_t)p->n * 4,
                        rows, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess)
    return PB_ECUDA;
  return PB_OK;
}

// Gradients of the mean BCE of rows (inputs bf16 [rows x k_in], targets fp32
// 0/1 [rows x n]) into the internal gradient block (pb_mlp_grads reads it);
// d_loss (device fp32, may be NULL) receives the loss.  rows: multiple of
// 8, <= batch.
PB_API int pb_mlp_backward(pb_mlp* p, const void* d_x, const float* d_target, int rows, float* d_loss) {
  if (!p || !d_x || !d_target || rows <= 0 || rows > p->batch || rows % 8) return PB_EINVAL;
  if (cudaMemcpyAsync(p->X, d_x, (size_t)rows * p->kin * 2, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess ||
      cudaMemcpy2DAsync(p->target, (size_t)p->n * 4, d_target, (size_t)p->n * 4, (size_t)p->n * 4, rows,
                        cudaMemcpyDeviceToDevice, p->st) != cudaSuccess)
    return PB_ECUDA;
  if (mlp_fwd(p, rows) != cudaSuccess || mlp_bwd(p, rows) != cudaSuccess) return PB_ECUDA;
  if (d_loss && cudaMemcpyAsync(d_loss, p->loss, 4, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess)
    return PB_ECUDA;
  return PB_OK;
}

// One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the current gradients.
PB_API int pb_mlp_adam(pb_mlp* p, float lr) {
  if (!p || !(lr > 0.f)) return PB_EINVAL;
  return pb::mlp_adam_step(p, lr) == cudaSuccess ? PB_OK : PB_ECUDA;
}

PB_API void pb_mlp_free(pb_mlp* p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  delete p;
}

}  // extern "C"

// ===========================================================================
// Fused forward of the whole network for inference: one CTA of 4 warps per
// 128 rows; x, the hidden activations and the weights (W2 streamed in
// K-chunks of 64, double-buffered) stay in shared memory, the accumulators in
// TMEM (256 columns, reused by the three layers).
// ===========================================================================
namespace pb {

// Modes of the fused kernel:
//   kFusedLogits  rows of x from global memory -> logits to global memory;
//   kFusedLogQ    rows (chain c, layer j = k + blockIdx.y) built from the
//                 per-chain words P -> lq[c d + j-1] = log q(P[c][j-1] | x);
//   kFusedSample  rows (chain c, layer j) built from P (j == k) or Pn (j > k)
//                 -> s'_j drawn from q into Pn[c][j-1], lqf[c] += log q(s'_j | x).
enum : int { kFusedLogits = 0, kFusedLogQ = 1, kFusedSample = 2 };

struct FusedArgs {
  const __nv_bfloat16* X;  // [rows x kin] (kFusedLogits)
  const __nv_bfloat16 *W1p, *W2p, *W3p;  // canonical images (W2 in K-chunks of 64)
  const float *b1, *b2, *b3;
  float* logits;  // [rows x npad] (kFusedLogits)
  int rows, kin, H, npad;
  uint32_t* status;
  // per-chain modes
  const uint32_t* P;
  uint32_t* Pn;
  float* lq;
  float* lqf;
  const uint32_t* move_dev;
  const int* k_dev;  // per-chain modes: when set, the suffix start k is read here
                     // (kFusedLogQ: layers k + blockIdx.y; kFusedSample: j = k,
                     // jlast = d) and CTAs past layer d leave at once
  uint32_t beta, k0, k1, group0;
  int n, d, k, j, jlast;  // kFusedSample: layers j .. jlast, one after the other
  // shared-memory layout (byte offsets; fused_layout) and W2 chunk buffers
  uint32_t offH, offW1, offW3, offB, offWb, chunk_bytes;
  int nb;
};

// Dynamic shared memory of the fused kernel, sized per network: the x tile
// (128 x kin), the h tile (128 x H), W1, W3 and the biases resident for the
// whole launch, and nb buffers for the K-chunks of W2 (64 columns each)
// streamed in by bulk copies; nb is as large as the space allows.
constexpr size_t kFusedSmemMax = 222 * 1024;  // with the kernel's static shared memory (< 5 KB)

inline size_t round_kb(size_t b) { return (b + 1023) & ~(size_t)1023; }

// Fills the layout fields of `a`; returns the dynamic shared-memory size (0
// when not even two chunk buffers fit).
inline size_t fused_layout(FusedArgs& a) {
  const size_t X = round_kb((size_t)128 * a.kin * 2), Hs = round_kb((size_t)128 * a.H * 2);
  const size_t W1 = round_kb((size_t)a.H * a.kin * 2), W3 = round_kb((size_t)a.npad * a.H * 2);
  const size_t B = round_kb((size_t)(2 * a.H + a.npad) * 4);
  const int nchunks = (a.H + 63) / 64;
  const size_t chunk = round_kb((size_t)a.H * std::min(64, a.H) * 2);
  a.offH = (uint32_t)X;
  a.offW1 = (uint32_t)(X + Hs);
  a.offW3 = (uint32_t)(X + Hs + W1);
  a.offB = (uint32_t)(X + Hs + W1 + W3);
  a.offWb = (uint32_t)(X + Hs + W1 + W3 + B);
  a.chunk_bytes = (uint32_t)chunk;
  const size_t fixed = a.offWb;
  if (fixed + std::min(2, nchunks) * chunk > kFusedSmemMax) return 0;
  a.nb = (int)std::min<size_t>((size_t)nchunks, (kFusedSmemMax - fixed) / chunk);
  return fixed + (size_t)a.nb * chunk;
}

// Rows [r0, r0+nrows) x K of a row-major bf16 matrix into the canonical
// K-major layout at `dst` (8-row groups SBO = K * 16 bytes apart).
// The copies are asynchronous (cp.async, zero-filled past rmax); the caller
// waits with tc::cp_async_wait_all() before the data is used.
__device__ __forceinline__ void stage_rows(uint8_t* dst, const __nv_bfloat16* src, int ld, int r0,
                                           int nrows, int rmax, int k0, int K, int tid, int nthr) {
  const int vecs = K / 8;
  for (int v = tid; v < nrows * vecs; v += nthr) {
    const int r = v / vecs, c = v % vecs, row = r0 + r;
    const bool in = row < rmax;
    tc::cp_async16(dst + (r >> 3) * (K * 16) + c * 128 + (r & 7) * 16,
                   in ? (const void*)(src + (size_t)row * ld + k0 + c * 8) : (const void*)src,
                   in ? 16u : 0u);
  }
}

// Elements [8 c_lo, 8 c_hi) of row r of the x tile (canonical layout, SBO =
// kin * 16): x = [2 prev - 1 (n), onehot(j-1) (d), 0...], written as bf16
// bit patterns (1.0 = 0x3F80, -1.0 = 0xBF80).
__device__ __forceinline__ void build_x_part(uint8_t* sX, int kin, int n, int r, uint32_t prev,
                                             int j, int c_lo, int c_hi) {
  uint8_t* base = sX + (r >> 3) * (kin * 16) + (r & 7) * 16;
  auto elem = [&](int i) -> uint32_t {
    if (i < n) return ((prev >> i) & 1u) ? 0x3F80u : 0xBF80u;
    return i == n + j - 1 ? 0x3F80u : 0u;
  };
  for (int c = c_lo; c < c_hi; ++c) {
    uint4 w;
    w.x = elem(8 * c) | (elem(8 * c + 1) << 16);
    w.y = elem(8 * c + 2) | (elem(8 * c + 3) << 16);
    w.z = elem(8 * c + 4) | (elem(8 * c + 5) << 16);
    w.w = elem(8 * c + 6) | (elem(8 * c + 7) << 16);
    *reinterpret_cast<uint4*>(base + c * 128) = w;
  }
}

// log(1 + e^{-|l|}), the shared part of log sigma(l) and log sigma(-l):
// log sigma(+-l) = -(max(-+l, 0) + softplus_tail(l)).  Both fused modes that
// evaluate log q use this one expression, so a proposal's log q computed
// while it is drawn equals the one computed later for the same path.
__device__ __forceinline__ float softplus_tail(float l) { return __logf(1.f + __expf(-fabsf(l))); }

// Threads per row of the fused kernel: warps w, w + 4, ... share TMEM lane
// quadrant w % 4 (rows 32 (w % 4) ..) and split each row's work.
constexpr int kFusedParts = 4;
constexpr int kFusedThreads = 128 * kFusedParts;

template <int MODE>
__global__ void __launch_bounds__(kFusedThreads) mlp_fused_kernel(FusedArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  // mbarriers: wbar = W1 and W3 delivered; lbar[b] = the W2 chunk in buffer
  // b delivered; cbar[b] = the MMAs reading buffer b done (committed only
  // when the buffer is refilled within the same GEMM); done = all MMAs of
  // the current GEMM done (every thread waits once per GEMM); drain = all
  // MMAs done (after a failed wait only)
  constexpr int kMaxNb = 4;
  __shared__ uint64_t bars[2 + 2 * kMaxNb + 1];
  __shared__ uint32_t tmem_base;
  // the parts of a row exchange their bits and log q terms here
  __shared__ uint32_t xw[kFusedParts][128];
  __shared__ float xq[kFusedParts][128];
  uint64_t* wbar = &bars[0];
  uint64_t* done = &bars[1];
  uint64_t* drain = &bars[2];
  uint64_t* lbar = &bars[3];
  uint64_t* cbar = &bars[3 + kMaxNb];
  uint8_t* sX = sm;
  uint8_t* sH = sm + a.offH;
  uint8_t* sW1 = sm + a.offW1;
  uint8_t* sW3 = sm + a.offW3;
  float* sB = reinterpret_cast<float*>(sm + a.offB);  // b1 [H], b2 [H], b3 [npad]
  uint8_t* sWb = sm + a.offWb;                           // nb chunk buffers
  // warp w reads TMEM lanes 32 (w & 3) .. +31 (its rows) and handles part
  // w >> 2 (of kFusedParts) of the columns, x elements and bits of those rows
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;
  const int rl = quad * 32 + lane;  // row within the tile
  const int r0 = blockIdx.x * 128;
  const int H = a.H, kin = a.kin, npad = a.npad, nb = min(a.nb, kMaxNb);
  const int nchunks = (H + 63) / 64;
  auto chunk_k = [&](int c) { return (c == nchunks - 1 && (H % 64)) ? (H % 64) : 64; };
  const int kk = (MODE != kFusedLogits && a.k_dev) ? *a.k_dev : a.k;
  const int jfirst = MODE == kFusedLogQ ? kk + (int)blockIdx.y : (a.k_dev ? kk : a.j);
  const int jend = MODE == kFusedSample ? (a.k_dev ? a.d : a.jlast) : jfirst;
  if (MODE != kFusedLogits && (jfirst < 1 || jfirst > a.d)) return;  // whole CTA: no layer here

  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    for (int i = 0; i < 2 + 2 * kMaxNb + 1; ++i) tc::mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < H; i += kFusedThreads) {
    sB[i] = a.b1[i];
    sB[H + i] = a.b2[i];
  }
  for (int i = tid; i < npad; i += kFusedThreads) sB[2 * H + i] = a.b3[i];
  __syncthreads();  // TMEM address, barriers and biases visible
  const uint32_t tb = tmem_base;
  bool ok = true;
  uint32_t dph = 0u;  // parity of `done` (every thread)
  // thread 0: parities and the copies still to be waited for
  uint32_t wph = 0u, lph[kMaxNb] = {0u, 0u, 0u, 0u}, cph[kMaxNb] = {0u, 0u, 0u, 0u};
  bool lpend[kMaxNb] = {false, false, false, false};
  // After a failed wait the thread skips further waits and work but keeps
  // the same sequence of CTA barriers as the others.
  auto wait_on = [&](uint64_t* bar, uint32_t& ph) {
    if (!ok) return;
    ok = tc::mbar_wait(bar, ph);
    if (ok) ph ^= 1u;
  };
  // K-chunk c of W2 into buffer b (thread 0; the buffer is free)
  auto load_chunk = [&](int c, int b) {
    const uint32_t bytes = (uint32_t)(H * chunk_k(c) * 2);
    tc::mbar_expect_tx(&lbar[b], bytes);
    tc::bulk_load(sWb + (size_t)b * a.chunk_bytes, a.W2p + (size_t)H * c * 64, bytes, &lbar[b]);
    lpend[b] = true;
  };
  // the first min(nb, nchunks) chunks of the next GEMM over W2
  auto prefetch_w2 = [&]() {
    for (int c = 0; c < nb && c < nchunks; ++c) load_chunk(c, c);
  };
  if (tid == 0) {
    const uint32_t w1 = (uint32_t)(H * kin * 2), w3 = (uint32_t)(npad * H * 2);
    tc::mbar_expect_tx(wbar, w1 + w3);
    tc::bulk_load(sW1, a.W1p, w1, wbar);
    tc::bulk_load(sW3, a.W3p, w3, wbar);
    prefetch_w2();
  }
  const uint32_t taddr_row = tb + ((uint32_t)(quad * 32) << 16);
  const int row = r0 + rl;
  // generic-proxy shared writes of all threads visible to the tensor core
  auto publish = [&]() {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  auto wait_done = [&]() {
    wait_on(done, dph);
    tc::fence_after_sync();
  };
  // h = relu(D + b) in bf16, into sH (canonical, K = H): this thread's row,
  // the part's share of the 8-column groups; one 64-column TMEM read covers
  // it (a share is at most 64 columns and starts at most at column 192)
  const int ngrp = H / 8;
  const int hc_lo = 8 * (part * ngrp / kFusedParts), hc_hi = 8 * ((part + 1) * ngrp / kFusedParts);
  auto epilogue_to_h = [&](const float* bias) {
    uint8_t* base = sH + (rl >> 3) * (H * 16) + (rl & 7) * 16;
    for (int c0 = hc_lo; c0 < hc_hi; c0 += 64) {
      float v[64];
      tc::tmem_ld64(taddr_row + (uint32_t)c0, v);
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        if (c0 + 8 * g < hc_hi) {
          const float4 bl = *reinterpret_cast<const float4*>(bias + c0 + 8 * g);
          const float4 bh = *reinterpret_cast<const float4*>(bias + c0 + 8 * g + 4);
          const float bv[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
          __align__(16) __nv_bfloat162 hb[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            hb[i] = __floats2bfloat162_rn(fmaxf(v[8 * g + 2 * i] + bv[2 * i], 0.f),
                                          fmaxf(v[8 * g + 2 * i + 1] + bv[2 * i + 1], 0.f));
          *reinterpret_cast<uint4*>(base + ((c0 >> 3) + g) * 128) = *reinterpret_cast<uint4*>(hb);
        }
      }
    }
  };

  // per-chain modes: this thread's chain, its previous layer word and the
  // running log q of the proposal
  const int chain = row;
  uint32_t prev = a.beta;
  if (MODE != kFusedLogits && chain < a.rows && jfirst > 1)
    prev = a.P[(size_t)chain * a.d + (jfirst - 2)];
  float lq_acc = 0.f;

  for (int jl = jfirst; jl <= jend; ++jl) {
    // ---- x tile (row = chain r0 + r at layer jl, or a staged input row)
    if (MODE == kFusedLogits) {
      stage_rows(sX, a.X, kin, r0, 128, a.rows, 0, kin, tid, kFusedThreads);
      tc::cp_async_wait_all();
    } else {
      build_x_part(sX, kin, a.n, rl, prev, jl, part * (kin / 8) / kFusedParts,
                   (part + 1) * (kin / 8) / kFusedParts);
    }
    publish();

    // ---- layer 1: D = x W1^T
    if (tid == 0) {
      if (jl == jfirst) wait_on(wbar, wph);
      if (ok) {
        const uint32_t ax = tc::smem_u32(sX), bw = tc::smem_u32(sW1);
        const uint32_t idesc = tc::idesc_bf16_f32(128, H);
        for (int s = 0; s < kin / 16; ++s)
          tc::mma_bf16(tb, tc::smem_desc(ax + s * 256, 128, kin * 16),
                       tc::smem_desc(bw + s * 256, 128, kin * 16), idesc, s > 0);
      }
      tc::mma_commit(done);
    }
    wait_done();
    if (ok) epilogue_to_h(sB);
    publish();

    // ---- layer 2: D = h W2^T over the K-chunks of W2 (chunk c in buffer
    // c % nb); chunk c + nb - 1 is fetched once the MMAs of chunk c - 1 are done
    if (tid == 0) {
      for (int c = 0; c < nchunks; ++c) {
        const int b = c % nb;
        wait_on(&lbar[b], lph[b]);
        if (!ok) continue;
        lpend[b] = false;
        const int kc = chunk_k(c);
        const uint32_t ah = tc::smem_u32(sH) + c * 8 * 128;
        const uint32_t bw = tc::smem_u32(sWb + (size_t)b * a.chunk_bytes);
        const uint32_t idesc = tc::idesc_bf16_f32(128, H);
        for (int s = 0; s < kc / 16; ++s)
          tc::mma_bf16(tb, tc::smem_desc(ah + s * 256, 128, H * 16),
                       tc::smem_desc(bw + s * 256, 128, kc * 16), idesc, (c > 0) || (s > 0));
        if (c + nb < nchunks) tc::mma_commit(&cbar[b]);  // buffer b is refilled below
        if (c >= 1 && c - 1 + nb < nchunks) {
          const int bp = (c - 1) % nb;
          wait_on(&cbar[bp], cph[bp]);
          if (ok) load_chunk(c - 1 + nb, bp);
        }
      }
      tc::mma_commit(done);
    }
    wait_done();
    // every W2 buffer is free: thread 0 fetches the next layer's first chunks
    if (tid == 0 && ok && jl < jend) prefetch_w2();
    if (ok) epilogue_to_h(sB + H);
    publish();

    // ---- layer 3: D = h W3^T
    if (tid == 0) {
      if (ok) {
        const uint32_t ah = tc::smem_u32(sH), bw = tc::smem_u32(sW3);
        const uint32_t idesc = tc::idesc_bf16_f32(128, npad);
        for (int s = 0; s < H / 16; ++s)
          tc::mma_bf16(tb, tc::smem_desc(ah + s * 256, 128, H * 16),
                       tc::smem_desc(bw + s * 256, 128, H * 16), idesc, s > 0);
      }
      tc::mma_commit(done);
    }
    wait_done();
    // logits of this thread's row (npad is 16 or 32); the row's bits are
    // split between the two halves by Philox output (4 bits each):
    // part p takes bits 4 g .. 4 g + 3 for the g with g % kFusedParts == p
    uint32_t word = 0u;
    float sq = 0.f;
    if (ok) {
      float l[32];
      if (npad > 16) {
        tc::tmem_ld32(taddr_row, l);
      } else {
        float v[16];
        tc::tmem_ld16(taddr_row, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) l[i] = v[i];
#pragma unroll
        for (int i = 16; i < 32; ++i) l[i] = 0.f;
      }
      const float* b3 = sB + 2 * H;
#pragma unroll
      for (int i = 0; i < 32; ++i) l[i] += i < npad ? b3[i] : 0.f;
      if (row < a.rows) {
        if (MODE == kFusedLogits) {
          if (part == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < npad) a.logits[(size_t)row * npad + i] = l[i];
          }
        } else if (MODE == kFusedLogQ) {
          // log q of the current layer word: sum_q log sigma(+-l_q)
          const uint32_t bits = a.P[(size_t)row * a.d + (jl - 1)];
#pragma unroll
          for (int qb = 0; qb < 32; ++qb) {
            if (qb < a.n && (qb >> 2) % kFusedParts == part) {
              const float z = ((bits >> qb) & 1u) ? -l[qb] : l[qb];
              sq -= fmaxf(z, 0.f) + softplus_tail(l[qb]);
            }
          }
        } else {
          // draw s'_j bit by bit: u < sigmoid(l_q), u from Philox (chain,
          // move, (j-1) | tag 2 << 16, q/4)
          const uint32_t move = *a.move_dev;
          const uint32_t gc = a.group0 * 32u + (uint32_t)row;
          uint4 u4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (int qb = 0; qb < 32; ++qb) {
            if (qb < a.n && (qb >> 2) % kFusedParts == part) {
              if ((qb & 3) == 0)
                u4 = philox4x32_10(make_uint4(gc, move, (uint32_t)(jl - 1) | (kTagMH << 16),
                                              (uint32_t)(qb >> 2)), a.k0, a.k1);
              const uint32_t u = (qb & 3) == 0 ? u4.x : (qb & 3) == 1 ? u4.y : (qb & 3) == 2 ? u4.z : u4.w;
              const float e = __expf(-fabsf(l[qb]));
              const float r = __fdividef(1.f, 1.f + e);
              const float p1 = l[qb] >= 0.f ? r : e * r;  // sigma(l)
              const float uf = ((float)(u >> 8) + 0.5f) * (1.f / 16777216.f);
              const uint32_t bit = uf < p1 ? 1u : 0u;
              word |= bit << qb;
              const float z = bit ? -l[qb] : l[qb];
              sq -= fmaxf(z, 0.f) + softplus_tail(l[qb]);
            }
          }
        }
      }
    }
    if (MODE != kFusedLogits) {
      xw[part][rl] = word;
      xq[part][rl] = sq;
    }
    // the TMEM reads of this layer are complete before the next layer's
    // MMAs, and the halves' bits are exchanged
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (MODE != kFusedLogits && ok && row < a.rows) {
      float sql = 0.f;
      uint32_t wrd = 0u;
#pragma unroll
      for (int q = 0; q < kFusedParts; ++q) {
        sql += xq[q][rl];
        wrd |= xw[q][rl];
      }
      if (MODE == kFusedLogQ) {
        if (part == 0) a.lq[(size_t)row * a.d + (jl - 1)] = sql;
      } else {
        prev = wrd;
        if (part == 0) a.Pn[(size_t)row * a.d + (jl - 1)] = prev;
        lq_acc += sql;
      }
    }
  }  // layers
  if (MODE == kFusedSample && ok && row < a.rows && part == 0) a.lqf[row] += lq_acc;
  if (!__syncthreads_and(ok)) {
    if (tid == 0) {
      if (a.status) atomicCAS(a.status, 0u, (uint32_t)PB_ETIMEOUT);
      // let MMAs and copies still in flight drain (bounded waits) before the
      // accumulator and the shared memory are given up
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0u);
      for (int b = 0; b < kMaxNb; ++b)
        if (lpend[b]) tc::mbar_wait(&lbar[b], lph[b]);
      if (wph == 0u) tc::mbar_wait(wbar, wph);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 256);
}

template __global__ void mlp_fused_kernel<kFusedLogits>(FusedArgs);
template __global__ void mlp_fused_kernel<kFusedLogQ>(FusedArgs);
template __global__ void mlp_fused_kernel<kFusedSample>(FusedArgs);

// ===========================================================================
// The per-chain modes with 64-row tiles: twice the CTAs of the 128-row
// kernel, and with half the rows the x and h tiles shrink enough that W1,
// W2 and W3 all stay in shared memory for the whole launch (one bulk copy
// each at the start; no W2 chunks streamed per layer).  MMAs are M = 64
// (idesc M field 4): row r of an accumulator sits in TMEM lane
// 32 (r / 16) + r % 16, so warp w (lane quadrant q = w % 4) holds rows
// 16 q .. 16 q + 15; its epilogue reads them with the 16x256b shape (thread
// t: rows t / 4 and 8 + t / 4 of the 16, columns 2 (t % 4) and the next, of
// each 8-column block), and the four warps of a quadrant split the hidden
// columns.  The logits of row 16 q + i are read by lane i < 16 of warp q
// (32x32b shape), which draws or scores the row's bits as the 128-row
// kernel does.  Same modes, arguments and results (the accumulation order
// of the tensor cores may differ in the last bit).
// ===========================================================================
constexpr int kTile64 = 64;

// Dynamic shared memory of the 64-row kernel: x (64 x kin), h (64 x H),
// W1, the whole W2 image, W3 and the biases; 0 when they do not fit.
inline size_t fused64_layout(FusedArgs& a) {
  const size_t X = round_kb((size_t)kTile64 * a.kin * 2), Hs = round_kb((size_t)kTile64 * a.H * 2);
  const size_t W1 = round_kb((size_t)a.H * a.kin * 2), W2 = round_kb((size_t)a.H * a.H * 2);
  const size_t W3 = round_kb((size_t)a.npad * a.H * 2);
  const size_t B = round_kb((size_t)(2 * a.H + a.npad) * 4);
  a.offH = (uint32_t)X;
  a.offW1 = (uint32_t)(X + Hs);
  a.offWb = (uint32_t)(X + Hs + W1);  // W2, chunk c at + c * H * 64 * 2
  a.offW3 = (uint32_t)(X + Hs + W1 + W2);
  a.offB = (uint32_t)(X + Hs + W1 + W2 + W3);
  a.chunk_bytes = (uint32_t)(a.H * 64 * 2);
  a.nb = 0;
  const size_t total = X + Hs + W1 + W2 + W3 + B;
  if (a.H % 64 != 0 || total > kFusedSmemMax) return 0;
  return total;
}

// 16 lanes x 256 bits (8 fp32 columns) of the warp's TMEM lane quadrant, 8
// blocks of 8 columns (addresses taddr + 8 j), one completion wait: v[4 j +
// 0, 1] = rows t / 4, columns 8 j + 2 (t % 4) + {0, 1}; v[4 j + 2, 3] = row
// 8 + t / 4, the same columns.
__device__ __forceinline__ void tmem_ld_16x256b_x8(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[4 * j]), "=r"(r[4 * j + 1]), "=r"(r[4 * j + 2]), "=r"(r[4 * j + 3])
                 : "r"(taddr + 8u * (uint32_t)j)
                 : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int MODE>
__global__ void __launch_bounds__(kFusedThreads) mlp_move64_kernel(FusedArgs a) {
  static_assert(MODE == kFusedLogQ || MODE == kFusedSample, "per-chain modes only");
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t bars[3];  // weights delivered, MMAs of a GEMM done, drain
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t wrd[kTile64];  // drawn words of the layer, by row
  // the four parts of a row exchange their bits and log q terms here
  __shared__ uint32_t xw[kFusedParts][kTile64];
  __shared__ float xq[kFusedParts][kTile64];
  uint64_t* wbar = &bars[0];
  uint64_t* done = &bars[1];
  uint64_t* drain = &bars[2];
  uint8_t* sX = sm;
  uint8_t* sH = sm + a.offH;
  uint8_t* sW1 = sm + a.offW1;
  uint8_t* sW2 = sm + a.offWb;
  uint8_t* sW3 = sm + a.offW3;
  float* sB = reinterpret_cast<float*>(sm + a.offB);  // b1 [H], b2 [H], b3 [npad]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;
  const int H = a.H, kin = a.kin, npad = a.npad;
  const int r0 = blockIdx.x * kTile64;
  const int kk = a.k_dev ? *a.k_dev : a.k;
  // kFusedLogQ: layers kk + y L .. kk + y L + L - 1 (L = a.jlast layers per
  // CTA, so the weights are loaded once for several layers); kFusedSample:
  // the suffix, layer after layer
  const int jfirst = MODE == kFusedLogQ ? kk + (int)blockIdx.y * a.jlast : (a.k_dev ? kk : a.j);
  const int jend = MODE == kFusedSample ? (a.k_dev ? a.d : a.jlast) : min(jfirst + a.jlast - 1, a.d);
  if (jfirst < 1 || jfirst > a.d) return;  // whole CTA: no layer here

  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < H; i += kFusedThreads) {
    sB[i] = a.b1[i];
    sB[H + i] = a.b2[i];
  }
  for (int i = tid; i < npad; i += kFusedThreads) sB[2 * H + i] = a.b3[i];
  __syncthreads();  // TMEM address, barriers and biases visible
  const uint32_t tb = tmem_base;
  if (tid == 0) {
    const uint32_t w1 = (uint32_t)(H * kin * 2), w2 = (uint32_t)(H * H * 2), w3 = (uint32_t)(npad * H * 2);
    tc::mbar_expect_tx(wbar, w1 + w2 + w3);
    tc::bulk_load(sW1, a.W1p, w1, wbar);
    tc::bulk_load(sW2, a.W2p, w2, wbar);
    tc::bulk_load(sW3, a.W3p, w3, wbar);
  }
  bool ok = true, weights = false;
  uint32_t dph = 0u;
  // A wait whose outcome the whole CTA shares (every thread takes the same
  // branches and barriers after it).
  auto wait_all = [&](uint64_t* bar, uint32_t ph) {
    const bool w = ok && tc::mbar_wait(bar, ph);
    ok = __syncthreads_and(w) != 0;
    tc::fence_after_sync();
  };
  auto publish = [&]() {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  // h = relu(D + bias) in bf16 into sH (canonical, K = H): warp (quad,
  // part) converts rows 16 quad .. + 15, columns 64 part .. + 63
  const uint32_t tq = tb + ((uint32_t)(quad * 32) << 16);
  auto epilogue = [&](const float* bias) {
    const int ra = 16 * quad + (lane >> 2), rb = ra + 8;
    uint8_t* ha = sH + (ra >> 3) * (H * 16) + (ra & 7) * 16;
    uint8_t* hb = sH + (rb >> 3) * (H * 16) + (rb & 7) * 16;
    for (int c0 = 64 * part; c0 < H; c0 += 256) {
      float v[32];
      tmem_ld_16x256b_x8(tq + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + 8 * j + 2 * (lane & 3);
        const float b0 = bias[c], b1 = bias[c + 1];
        const __nv_bfloat162 xa = __floats2bfloat162_rn(fmaxf(v[4 * j] + b0, 0.f), fmaxf(v[4 * j + 1] + b1, 0.f));
        const __nv_bfloat162 xb = __floats2bfloat162_rn(fmaxf(v[4 * j + 2] + b0, 0.f), fmaxf(v[4 * j + 3] + b1, 0.f));
        const int off = (c >> 3) * 128 + (c & 7) * 2;
        *reinterpret_cast<__nv_bfloat162*>(ha + off) = xa;
        *reinterpret_cast<__nv_bfloat162*>(hb + off) = xb;
      }
    }
  };

  // this thread's row for the logits: lanes < 16 of every warp
  const int srow = 16 * quad + lane;  // row within the tile (lanes < 16)
  const int chain = r0 + srow;
  const bool live = lane < 16 && chain < a.rows;
  float lq_acc = 0.f;
  const int groups = (a.n + 3) / 4;  // 4-bit groups of a layer's bits (n <= 32: at most 8)
  const uint32_t move = MODE == kFusedSample ? *a.move_dev : 0u;
  const uint32_t gc = a.group0 * 32u + (uint32_t)chain;
  // the previous-layer word of every row of the tile, for the x builders
  for (int r = tid; r < kTile64; r += kFusedThreads) {
    const int c = r0 + r;
    wrd[r] = (c < a.rows && jfirst > 1) ? a.P[(size_t)c * a.d + (jfirst - 2)] : a.beta;
  }
  __syncthreads();

  for (int jl = jfirst; jl <= jend; ++jl) {
    // ---- x tile: 64 rows x kin, 16-byte pieces of 8 elements
    const int pieces = kin / 8;
    for (int v = tid; v < kTile64 * pieces; v += kFusedThreads) {
      const int r = v / pieces, c = v % pieces;
      build_x_part(sX, kin, a.n, r, wrd[r], jl, c, c + 1);
    }
    publish();
    // ---- layer 1: D = x W1^T
    if (tid == 0 && ok) {
      if (!weights) {
        weights = tc::mbar_wait(wbar, 0u);
        if (!weights) ok = false;
      }
      if (ok) {
        const uint32_t ax = tc::smem_u32(sX), bw = tc::smem_u32(sW1);
        const uint32_t idesc = tc::idesc_bf16_f32(kTile64, H);
        for (int s = 0; s < kin / 16; ++s)
          tc::mma_bf16(tb, tc::smem_desc(ax + s * 256, 128, kin * 16),
                       tc::smem_desc(bw + s * 256, 128, kin * 16), idesc, s > 0);
        tc::mma_commit(done);
      }
    }
    ok = __syncthreads_and(ok) != 0;  // thread 0's weight wait, shared
    wait_all(done, dph);
    dph ^= 1u;
    if (ok) epilogue(sB);
    publish();
    // ---- layer 2: D = h W2^T, W2 resident (K-chunk c of 64 at c H 128 bytes)
    if (tid == 0 && ok) {
      const uint32_t idesc = tc::idesc_bf16_f32(kTile64, H);
      const uint32_t ah = tc::smem_u32(sH), bw = tc::smem_u32(sW2);
      for (int c = 0; c < H / 64; ++c)
        for (int s = 0; s < 4; ++s)
          tc::mma_bf16(tb, tc::smem_desc(ah + c * 8 * 128 + s * 256, 128, H * 16),
                       tc::smem_desc(bw + c * a.chunk_bytes + s * 256, 128, 64 * 16), idesc,
                       (c > 0) || (s > 0));
      tc::mma_commit(done);
    }
    // while the tensor cores run layer 2: this thread's inputs to the logits
    // step (the draw's Philox outputs for groups part and part + 4, or the
    // current word), which depend on nothing the MMAs produce
    uint4 upre[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
    uint32_t bits = 0u;
    if (live) {
      if (MODE == kFusedSample) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int g = part + kFusedParts * t;
          if (g < groups)
            upre[t] = philox4x32_10(make_uint4(gc, move, (uint32_t)(jl - 1) | (kTagMH << 16), (uint32_t)g),
                                    a.k0, a.k1);
        }
      } else {
        bits = a.P[(size_t)chain * a.d + (jl - 1)];
      }
    }
    wait_all(done, dph);
    dph ^= 1u;
    if (ok) epilogue(sB + H);
    publish();
    // ---- layer 3: D = h W3^T
    if (tid == 0 && ok) {
      const uint32_t ah = tc::smem_u32(sH), bw = tc::smem_u32(sW3);
      const uint32_t idesc = tc::idesc_bf16_f32(kTile64, npad);
      for (int s = 0; s < H / 16; ++s)
        tc::mma_bf16(tb, tc::smem_desc(ah + s * 256, 128, H * 16),
                     tc::smem_desc(bw + s * 256, 128, H * 16), idesc, s > 0);
      tc::mma_commit(done);
    }
    wait_all(done, dph);
    dph ^= 1u;
    // ---- logits: the four parts of a quadrant split each row's bits by
    // Philox output (part p takes the 4-bit groups g = p, p + 4, ...): lane
    // i < 16 of warp (quad, part) scores row 16 quad + i, logit columns
    // 4 g .. 4 g + 3; log q of the current word, or the draw
    uint32_t wpart = 0u;
    float qpart = 0.f;
    if (ok) {
      const float* b3 = sB + 2 * H;
#pragma unroll
      for (int t = 0; t < 2; ++t) {  // groups part, part + 4 (warp-uniform)
        const int g = part + kFusedParts * t;
        if (g >= groups) break;
        float la[4];
        tc::tmem_ld4(tq + 4u * (uint32_t)g, la);
        if (!live) continue;
        const uint4 u4 = upre[t];
        const uint32_t U[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int qb = 4 * g + i;
          if (qb >= a.n) break;
          const float l = la[i] + b3[qb];
          uint32_t bit;
          if (MODE == kFusedLogQ) {
            bit = (bits >> qb) & 1u;
          } else {
            const float e = __expf(-fabsf(l));
            const float r = __fdividef(1.f, 1.f + e);
            const float p1 = l >= 0.f ? r : e * r;  // sigma(l)
            const float uf = ((float)(U[i] >> 8) + 0.5f) * (1.f / 16777216.f);
            bit = uf < p1 ? 1u : 0u;
          }
          wpart |= bit << qb;
          const float z = bit ? -l : l;
          qpart -= fmaxf(z, 0.f) + softplus_tail(l);
        }
      }
    }
    if (live) {
      xw[part][srow] = wpart;
      xq[part][srow] = qpart;
    }
    // the TMEM reads of this layer are complete before the next layer's
    // MMAs; the parts' bits and log q terms are exchanged
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (ok && live && part == 0) {
      uint32_t word = 0u;
      float sq = 0.f;
#pragma unroll
      for (int q = 0; q < kFusedParts; ++q) {
        word |= xw[q][srow];
        sq += xq[q][srow];
      }
      if (MODE == kFusedLogQ) {
        a.lq[(size_t)chain * a.d + (jl - 1)] = sq;
        wrd[srow] = word;  // the current word: the next layer's input
      } else {
        wrd[srow] = word;
        a.Pn[(size_t)chain * a.d + (jl - 1)] = word;
        lq_acc += sq;
      }
    }
    __syncthreads();  // the drawn words are visible to the next x tile
  }  // layers
  if (MODE == kFusedSample && ok && live && part == 0) a.lqf[chain] += lq_acc;
  if (!ok && tid == 0) {
    if (a.status) atomicCAS(a.status, 0u, (uint32_t)PB_ETIMEOUT);
    // let MMAs and copies in flight drain (bounded) before TMEM and shared
    // memory are given up
    tc::mma_commit(drain);
    tc::mbar_wait(drain, 0u);
    if (!weights) tc::mbar_wait(wbar, 0u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 256);
}

template __global__ void mlp_move64_kernel<kFusedLogQ>(FusedArgs);
template __global__ void mlp_move64_kernel<kFusedSample>(FusedArgs);

static FusedArgs fused_args(pb_mlp* p, int rows) {
  FusedArgs a{};
  a.jlast = 0;
  a.W1p = p->W1p;
  a.W2p = p->W2p;
  a.W3p = p->W3p;
  a.b1 = p->w + p->off_b1;
  a.b2 = p->w + p->off_b2;
  a.b3 = p->w + p->off_b3;
  a.rows = rows;
  a.kin = p->kin;
  a.H = p->H;
  a.npad = p->npad;
  a.n = p->n;
  a.d = p->d;
  a.status = p->status;
  return a;
}

// log q of the current suffix layers k..d of all chains (one launch).
cudaError_t mlp_fused_logq(pb_mlp* p, const uint32_t* P, uint32_t beta, int chains, int k, float* lq,
                           cudaStream_t st) {
  FusedArgs a = fused_args(p, chains);
  a.P = P;
  a.beta = beta;
  a.k = k;
  a.lq = lq;
  dim3 grid((chains + 127) / 128, p->d - k + 1);
  const size_t smem = fused_layout(a);
  if (smem == 0) return cudaErrorInvalidValue;
  mlp_fused_kernel<kFusedLogQ><<<grid, kFusedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// The same with the suffix start read from k_dev on the device (a grid over
// all d layers; the CTAs of layers before k leave at once), so that one
// captured graph serves every k.
cudaError_t mlp_fused_logq_dev(pb_mlp* p, const uint32_t* P, uint32_t beta, int chains,
                               const int* k_dev, float* lq, cudaStream_t st) {
  FusedArgs a = fused_args(p, chains);
  a.P = P;
  a.beta = beta;
  a.k = 1;
  a.k_dev = k_dev;
  a.lq = lq;
  if (const size_t smem64 = fused64_layout(a)) {  // 64-row tiles, weights resident
    // layers per CTA: one while the (tile, layer) pairs are few, more as the
    // chains grow, so that the weights are loaded once for several layers
    const int tiles = (chains + kTile64 - 1) / kTile64;
    a.jlast = std::max(1, std::min(p->d, tiles * p->d / 4096));
    dim3 grid(tiles, (p->d + a.jlast - 1) / a.jlast);
    mlp_move64_kernel<kFusedLogQ><<<grid, kFusedThreads, smem64, st>>>(a);
    return cudaGetLastError();
  }
  dim3 grid((chains + 127) / 128, p->d);
  const size_t smem = fused_layout(a);
  if (smem == 0) return cudaErrorInvalidValue;
  mlp_fused_kernel<kFusedLogQ><<<grid, kFusedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// Layers j .. jlast of the proposal for all chains (one launch; each CTA
// carries its 128 chains through the layers in turn).
cudaError_t mlp_fused_sample(pb_mlp* p, const uint32_t* P, uint32_t* Pn, uint32_t beta, int chains,
                             int k, int j, int jlast, float* lqf, uint32_t k0, uint32_t k1,
                             const uint32_t* move_dev, uint32_t group0, cudaStream_t st) {
  FusedArgs a = fused_args(p, chains);
  a.P = P;
  a.Pn = Pn;
  a.beta = beta;
  a.k = k;
  a.j = j;
  a.jlast = jlast;
  a.lqf = lqf;
  a.k0 = k0;
  a.k1 = k1;
  a.move_dev = move_dev;
  a.group0 = group0;
  const size_t smem = fused_layout(a);
  if (smem == 0) return cudaErrorInvalidValue;
  mlp_fused_kernel<kFusedSample><<<(chains + 127) / 128, kFusedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// Layers k .. d of the proposal, k read from k_dev on the device.
cudaError_t mlp_fused_sample_dev(pb_mlp* p, const uint32_t* P, uint32_t* Pn, uint32_t beta,
                                 int chains, const int* k_dev, float* lqf, uint32_t k0, uint32_t k1,
                                 const uint32_t* move_dev, uint32_t group0, cudaStream_t st) {
  FusedArgs a = fused_args(p, chains);
  a.P = P;
  a.Pn = Pn;
  a.beta = beta;
  a.k = 1;
  a.j = 1;
  a.jlast = p->d;
  a.k_dev = k_dev;
  a.lqf = lqf;
  a.k0 = k0;
  a.k1 = k1;
  a.move_dev = move_dev;
  a.group0 = group0;
  if (const size_t smem64 = fused64_layout(a)) {  // 64-row tiles, weights resident
    mlp_move64_kernel<kFusedSample><<<(chains + kTile64 - 1) / kTile64, kFusedThreads, smem64, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = fused_layout(a);
  if (smem == 0) return cudaErrorInvalidValue;
  mlp_fused_kernel<kFusedSample><<<(chains + 127) / 128, kFusedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t mlp_forward_fused(pb_mlp* p, int rows) {
  FusedArgs a{};
  a.X = p->X;
  a.W1p = p->W1p;
  a.W2p = p->W2p;
  a.W3p = p->W3p;
  a.b1 = p->w + p->off_b1;
  a.b2 = p->w + p->off_b2;
  a.b3 = p->w + p->off_b3;
  a.logits = p->logits;
  a.rows = rows;
  a.kin = p->kin;
  a.H = p->H;
  a.npad = p->npad;
  a.status = p->status;
  a.n = p->n;
  const size_t smem = fused_layout(a);
  if (smem == 0) return cudaErrorInvalidValue;
  mlp_fused_kernel<kFusedLogits><<<(rows + 127) / 128, kFusedThreads, smem, p->st>>>(a);
  return cudaGetLastError();
}

cudaError_t mlp_fused_prepare() {
  cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel<kFusedLogits>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_fused_kernel<kFusedLogQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFusedSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_fused_kernel<kFusedSample>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_move64_kernel<kFusedLogQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFusedSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_move64_kernel<kFusedSample>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax);
  return e;
}

}  // namespace pb

extern "C" PB_API int pb_mlp_forward_fused(pb_mlp* p, const void* d_x, int rows, float* d_logits) {
  if (!p || !d_x || !d_logits || rows <= 0 || rows > p->batch) return PB_EINVAL;
  if (p->kin > 96 || p->npad > 32) return PB_ERANGE;
  if (cudaMemcpyAsync(p->X, d_x, (size_t)rows * p->kin * 2, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess)
    return PB_ECUDA;
  if (pb::mlp_forward_fused(p, rows) != cudaSuccess) return PB_ECUDA;
  if (cudaMemcpy2DAsync(d_logits, (size_t)p->n * 4, p->logits, (size_t)p->npad * 4, (size_t)p->n * 4,
                        rows, cudaMemcpyDeviceToDevice, p->st) != cudaSuccess)
    return PB_ECUDA;
  return PB_OK;
}
