// Column sampling of the period-finding circuit (sm_103a): Sec. 5.2 and its
// column-sampling figure.
//
// Sample i draws a column x_i of the inverse QFT on n bits; its entries
// 2^{-n/2} e^{2 pi i k x_i / 2^n} are added to column y_i = a^{x_i} mod N of
// psi, and P[k] = sum_y |psi[k, y]|^2.  Instead of the 2^n x 2^n table (or the
// paper's 3 x 2^n) the samples are sorted by (y, x) on the device, so each
// y's samples are contiguous, and a thread that owns 32 consecutive k walks
// the sorted list: per sample an exact anchor e^{2 pi i k0 x / 2^n} (integer
// phase k0 x mod 2^n, FP32 sincospif) times the sample's table
// e^{2 pi i j x / 2^n}, j = 0..31 (shared by every thread, read from shared
// memory), one complex multiply-add per k into the group's 32 complex sums;
// at a group's end the squared moduli go into P.  Memory: 2^n doubles of output
// plus O(T).  The only contention is the FP64 atomic add of a block's P into
// the output when the samples are split over several blocks (at group
// boundaries, so that every |sum|^2 is complete in one block).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "pb_internal.h"

namespace pb {
namespace {

constexpr int kShorK = 32;          // k values per thread
constexpr int kShorThreads = 256;   // threads per block
constexpr int kShorChunk = 128;     // samples staged in shared memory per pass

// Sort key of sample i: y << 32 | x (T <= i < Tpad: all ones, sorted last).
__global__ void shor_modexp_kernel(const uint32_t* __restrict__ x, uint32_t T, uint32_t Tpad,
                                   uint64_t N, uint64_t a, unsigned long long* __restrict__ keys,
                                   unsigned long long* __restrict__ ys) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Tpad) return;
  if (i >= T) {
    keys[i] = ~0ull;
    return;
  }
  // binary exponentiation; N < 2^32, so every product fits in 64 bits
  uint64_t r = 1u % N, b = a % N, e = x[i];
  while (e) {
    if (e & 1u) r = r * b % N;
    b = b * b % N;
    e >>= 1;
  }
  keys[i] = (r << 32) | x[i];
  ys[i] = r;
}

// One compare-exchange stage (j, k) of a bitonic sort of Tpad keys (ascending).
__global__ void bitonic_step_kernel(unsigned long long* __restrict__ keys, uint32_t Tpad, uint32_t j,
                                    uint32_t k) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Tpad) return;
  const uint32_t l = i ^ j;
  if (l <= i) return;
  const unsigned long long u = keys[i], v = keys[l];
  const bool ascending = (i & k) == 0u;
  if ((u > v) == ascending) {
    keys[i] = v;
    keys[l] = u;
  }
}

// Sorted keys -> x, the group-end flag (the next sample has another y) and
// the sample's table e^{2 pi i j x / 2^n}, j = 0 .. kShorK - 1 (exact integer
// phase j x mod 2^n, FP64 sincospi, rounded to FP32); one thread per (i, j).
__global__ void shor_prep_kernel(const unsigned long long* __restrict__ keys, uint32_t T, int n,
                                 uint32_t* __restrict__ xs, float2* __restrict__ tab,
                                 uint8_t* __restrict__ gend) {
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned long long)T * kShorK) return;
  const uint32_t i = (uint32_t)(t / kShorK), j = (uint32_t)(t % kShorK);
  const unsigned long long key = keys[i];
  const uint32_t x = (uint32_t)key;
  if (j == 0) {
    xs[i] = x;
    gend[i] = (i + 1 == T || (keys[i + 1] >> 32) != (key >> 32)) ? 1 : 0;
  }
  const unsigned long long mask = (n == 64) ? ~0ull : ((1ull << n) - 1ull);
  const unsigned long long ph = ((unsigned long long)j * x) & mask;
  double s, c;
  sincospi(ldexp((double)ph, 1 - n), &s, &c);  // angle 2 pi j x / 2^n
  tab[t] = make_float2((float)c, (float)s);
}

// Slice s of the sorted samples starts at the first group start at or after
// s T / S (bounds[S] = T).
__global__ void shor_bounds_kernel(const uint8_t* __restrict__ gend, uint32_t T, uint32_t S,
                                   uint32_t* __restrict__ bounds) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > S) return;
  uint32_t i = (uint32_t)(((unsigned long long)T * s) / S);
  while (i > 0 && i < T && !gend[i - 1]) ++i;
  bounds[s] = s == S ? T : i;
}

// P for k = k0 .. k0 + 31 of this thread over the samples of slice
// blockIdx.y, added (times `scale`) into prob.
__global__ void __launch_bounds__(kShorThreads) shor_columns_kernel(
    const uint32_t* __restrict__ xs, const float2* __restrict__ tab,
    const uint8_t* __restrict__ gend, const uint32_t* __restrict__ bounds, int n, double scale,
    double* __restrict__ prob) {
  __shared__ uint32_t sx[kShorChunk];
  __shared__ __align__(16) float2 sr[kShorChunk * kShorK];
  __shared__ uint8_t sg[kShorChunk];
  const unsigned long long Ktot = 1ull << n;
  const unsigned long long k0 =
      ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * (unsigned long long)kShorK;
  const uint32_t lo = bounds[blockIdx.y], hi = bounds[blockIdx.y + 1];
  const int sh = 32 - n;                        // phase bits live in the low n bits
  const float to_half_turns = ldexpf(1.0f, 1 - n);  // phase units -> sincospif argument
  float ar[kShorK], ai[kShorK], P[kShorK];
#pragma unroll
  for (int j = 0; j < kShorK; ++j) ar[j] = ai[j] = P[j] = 0.0f;
  const uint32_t k0w = (uint32_t)k0;  // k x mod 2^n needs the low 32 bits only
#pragma unroll 1
  for (uint32_t c0 = lo; c0 < hi; c0 += kShorChunk) {
    const uint32_t cn = min((uint32_t)kShorChunk, hi - c0);
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < cn; t += blockDim.x) {
      sx[t] = xs[c0 + t];
      sg[t] = gend[c0 + t];
    }
    {  // the chunk's tables, 16 bytes at a time
      const float4* src = reinterpret_cast<const float4*>(tab + (size_t)c0 * kShorK);
      float4* dst = reinterpret_cast<float4*>(sr);
      for (uint32_t t = threadIdx.x; t < cn * (kShorK / 2); t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();
#pragma unroll 1
    for (uint32_t t = 0; t < cn; ++t) {
      const uint32_t x = sx[t];
      // exact integer phase k0 x mod 2^n, centred to [-2^{n-1}, 2^{n-1})
      const int32_t ph = (int32_t)((k0w * x) << sh) >> sh;
      float pr, pi;
      sincospif((float)ph * to_half_turns, &pi, &pr);
      const float4* w4 = reinterpret_cast<const float4*>(sr + t * kShorK);
#pragma unroll
      for (int j2 = 0; j2 < kShorK / 2; ++j2) {
        const float4 w = w4[j2];  // e^{i 2 pi (2 j2) x / 2^n}, e^{i 2 pi (2 j2 + 1) x / 2^n}
        const int j = 2 * j2;
        ar[j] = fmaf(pr, w.x, fmaf(-pi, w.y, ar[j]));
        ai[j] = fmaf(pr, w.y, fmaf(pi, w.x, ai[j]));
        ar[j + 1] = fmaf(pr, w.z, fmaf(-pi, w.w, ar[j + 1]));
        ai[j + 1] = fmaf(pr, w.w, fmaf(pi, w.z, ai[j + 1]));
      }
      if (sg[t]) {  // end of this y's samples: |sum|^2 into P
#pragma unroll
        for (int j = 0; j < kShorK; ++j) {
          P[j] = fmaf(ar[j], ar[j], fmaf(ai[j], ai[j], P[j]));
          ar[j] = ai[j] = 0.0f;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kShorK; ++j)
    if (k0 + (unsigned long long)j < Ktot && P[j] != 0.0f)
      atomicAdd(&prob[k0 + j], (double)P[j] * scale);
}

// The largest probability (positive doubles order like their bit patterns).
__global__ void max_kernel(const double* __restrict__ prob, unsigned long long n,
                           unsigned long long* __restrict__ out) {
  unsigned long long best = 0ull;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fmax(prob[i], 0.0));
    best = b > best ? b : best;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// Peaks: local maxima (cyclic in k; >= the left neighbour, > the right one)
// at or above `thr`.  Their count, and the first max_pos positions found.
__global__ void peaks_kernel(const double* __restrict__ prob, unsigned long long n, double thr,
                             unsigned int* __restrict__ count, unsigned long long* __restrict__ pos,
                             uint32_t max_pos) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double v = prob[i];
    if (v < thr) continue;
    const double l = prob[i == 0 ? n - 1 : i - 1], r = prob[i + 1 == n ? 0 : i + 1];
    if (v >= l && v > r) {
      const unsigned int c = atomicAdd(count, 1u);
      if (c < max_pos) pos[c] = i;
    }
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ShorLayout {
  size_t x, keys, ys, xs, tab, gend, bounds, misc, total;
  uint32_t Tpad, S;
};

// Blocks over k, then slices of the samples so that the launch fills the GPU.
ShorLayout shor_layout(int n, uint32_t T) {
  ShorLayout L{};
  uint32_t Tpad = 1;
  while (Tpad < T) Tpad <<= 1;
  L.Tpad = Tpad;
  const unsigned long long kthreads = ((1ull << n) + kShorK - 1) / kShorK;
  const unsigned long long kblocks = (kthreads + kShorThreads - 1) / kShorThreads;
  const unsigned long long want = 152ull * 8;  // eight blocks per SM
  unsigned long long S = kblocks >= want ? 1 : (want + kblocks - 1) / kblocks;
  S = std::min<unsigned long long>(S, std::max<uint32_t>(1u, T / 64));  // at least ~64 samples a slice
  L.S = (uint32_t)std::max<unsigned long long>(1, std::min<unsigned long long>(S, 65535));
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t at = off;
    off = align256(off + std::max<size_t>(b, 1));
    return at;
  };
  L.x = take((size_t)T * 4);
  L.keys = take((size_t)Tpad * 8);
  L.ys = take((size_t)T * 8);
  L.xs = take((size_t)T * 4);
  L.tab = take((size_t)T * kShorK * 8);
  L.gend = take((size_t)T);
  L.bounds = take((size_t)(L.S + 1) * 4);
  L.misc = take(64);
  L.total = off;
  return L;
}

int check_shor(uint64_t N, int n, uint32_t T) {
  if (n < 1 || n > 32) return PB_ERANGE;
  if (N < 2 || N > 0xFFFFFFFFull) return PB_ERANGE;
  if (T == 0 || T > (1u << 26)) return PB_ERANGE;
  return PB_OK;
}

}  // namespace
}  // namespace pb

using namespace pb;

extern "C" {

PB_API int pb_shor_workspace_bytes(int n, uint32_t T, size_t* bytes) {
  if (!bytes) return PB_EINVAL;
  if (n < 1 || n > 32 || T == 0 || T > (1u << 26)) return PB_ERANGE;
  *bytes = shor_layout(n, T).total;
  return PB_OK;
}

PB_API int pb_shor_columns(uint64_t N, uint64_t a, int n, const uint32_t* x, uint32_t T,
                           void* d_workspace, size_t workspace_bytes, double* d_prob,
                           uint64_t* y_out, uintptr_t stream) {
  if (!x || !d_workspace || !d_prob) return PB_EINVAL;
  int rc = check_shor(N, n, T);
  if (rc != PB_OK) return rc;
  if (((uintptr_t)d_workspace & 255u) != 0 || ((uintptr_t)d_prob & 7u) != 0) return PB_EINVAL;
  for (uint32_t i = 0; i < T; ++i)
    if (n < 32 && (x[i] >> n) != 0) return PB_EINVAL;
  const ShorLayout L = shor_layout(n, T);
  if (workspace_bytes < L.total) return PB_ERANGE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_workspace);
  uint32_t* dx = reinterpret_cast<uint32_t*>(ws + L.x);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  unsigned long long* ys = reinterpret_cast<unsigned long long*>(ws + L.ys);
  uint32_t* xs = reinterpret_cast<uint32_t*>(ws + L.xs);
  float2* tab = reinterpret_cast<float2*>(ws + L.tab);
  uint8_t* gend = reinterpret_cast<uint8_t*>(ws + L.gend);
  uint32_t* bounds = reinterpret_cast<uint32_t*>(ws + L.bounds);
  const unsigned long long K = 1ull << n;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dx, x, (size_t)T * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_prob, 0, K * 8, st)) != cudaSuccess)
    return PB_ECUDA;
  const int tpb = 256;
  shor_modexp_kernel<<<(L.Tpad + tpb - 1) / tpb, tpb, 0, st>>>(dx, T, L.Tpad, N, a, keys, ys);
  for (uint32_t k = 2; k <= L.Tpad; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1)
      bitonic_step_kernel<<<(L.Tpad + tpb - 1) / tpb, tpb, 0, st>>>(keys, L.Tpad, j, k);
  shor_prep_kernel<<<(unsigned)(((unsigned long long)T * kShorK + tpb - 1) / tpb), tpb, 0, st>>>(
      keys, T, n, xs, tab, gend);
  shor_bounds_kernel<<<(L.S + 1 + tpb - 1) / tpb, tpb, 0, st>>>(gend, T, L.S, bounds);
  const unsigned long long kthreads = (K + kShorK - 1) / kShorK;
  const unsigned long long kblocks = (kthreads + kShorThreads - 1) / kShorThreads;
  if (kblocks > 0x7FFFFFFFull) return PB_ERANGE;
  // prob[k] = P[k] / T with the IQFT's 2^{-n} folded in
  const double scale = std::ldexp(1.0, -n) / (double)T;
  shor_columns_kernel<<<dim3((unsigned)kblocks, L.S), kShorThreads, 0, st>>>(xs, tab, gend, bounds,
                                                                            n, scale, d_prob);
  if ((e = cudaGetLastError()) != cudaSuccess) return PB_ECUDA;
  if (y_out) {
    std::vector<unsigned long long> h(T);
    if ((e = cudaMemcpyAsync(h.data(), ys, (size_t)T * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return PB_ECUDA;
    for (uint32_t i = 0; i < T; ++i) y_out[i] = h[i];
  }
  return PB_OK;
}

PB_API int pb_shor_peaks(const double* d_prob, int n, double threshold, void* d_workspace,
                         size_t workspace_bytes, uint64_t* positions, uint32_t max_positions,
                         uint32_t* count, double* max_prob, uintptr_t stream) {
  if (!d_prob || !d_workspace || !count) return PB_EINVAL;
  if (n < 1 || n > 32) return PB_ERANGE;
  if (workspace_bytes < 256 + (size_t)max_positions * 8) return PB_ERANGE;
  if (((uintptr_t)d_workspace & 255u) != 0) return PB_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_workspace);
  unsigned long long* dmax = reinterpret_cast<unsigned long long*>(ws);
  unsigned int* dcount = reinterpret_cast<unsigned int*>(ws + 8);
  unsigned long long* dpos = reinterpret_cast<unsigned long long*>(ws + 256);
  const unsigned long long K = 1ull << n;
  if (cudaMemsetAsync(ws, 0, 256, st) != cudaSuccess) return PB_ECUDA;
  const int tpb = 256;
  const unsigned blocks = (unsigned)std::min<unsigned long long>((K + tpb - 1) / tpb, 152ull * 16);
  max_kernel<<<blocks, tpb, 0, st>>>(d_prob, K, dmax);
  peaks_kernel<<<blocks, tpb, 0, st>>>(d_prob, K, threshold, dcount, dpos, max_positions);
  if (cudaGetLastError() != cudaSuccess) return PB_ECUDA;
  unsigned long long hm = 0;
  unsigned int hc = 0;
  if (cudaMemcpyAsync(&hm, dmax, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&hc, dcount, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PB_ECUDA;
  *count = hc;
  if (max_prob) std::memcpy(max_prob, &hm, 8);
  if (positions && max_positions) {
    std::vector<unsigned long long> h(std::min(hc, max_positions));
    if (!h.empty()) {
      if (cudaMemcpy(h.data(), dpos, h.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PB_ECUDA;
      std::sort(h.begin(), h.end());
      for (size_t i = 0; i < h.size(); ++i) positions[i] = h[i];
    }
  }
  return PB_OK;
}

}  // extern "C"
