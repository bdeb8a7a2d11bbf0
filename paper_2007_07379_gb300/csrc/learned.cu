// Learned proposal for the Gibbs sampler: a Metropolis-Hastings suffix move
// whose proposal is the network q(s_j | s_{j-1}, j) (Fig. 2 Steps 1-2 with
// "Metropolis-Hastings" acceptance), path collection for training, and the
// training loop on collected paths.
//
// Move (all chains of one model, a layer k* in 1..d drawn per move from the
// seed and the move index):
//   1. the chain words are unsliced into one n-bit word per chain and layer;
//   2. log q of the current suffix s_{k*}..s_d given s_{k*-1} (rows batched
//      through the network);
//   3. a proposal s'_{k*}..s'_d is drawn layer by layer from q;
//   4. the violation counts v, v' of the links of layers k*..d give the
//      target ratio e^{-J (v' - v)} (Re E = J v, Appendix J-penalty);
//   5. accept with min(1, e^{-J (v'-v)} q(s | .) / q(s' | .)); accepted
//      suffixes replace the current ones and the words are sliced back.
// Random numbers: Philox4x32-10, key = run seed, counters (chain, move,
// (j-1) | 2 << 16, q/4) for proposal bits, (chain, move, 0xFFFF | 2 << 16, 0)
// for the acceptance uniform.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pb_internal.h"
#include "philox.cuh"

namespace pb {

// Gate layer L (s_L -> s_{L+1}) in per-chain form: H outputs, X (NOT)
// bits and CNOT pairs.
struct LayerTab {
  uint32_t hmask;
  uint32_t xmask;
  uint32_t ncnot;
  uint8_t c[16], t[16];
};

// Deterministic map of a non-H layer: X bits flip, CNOT targets take
// control XOR target.
__device__ __forceinline__ uint32_t layer_map(const LayerTab& L, uint32_t x) {
  uint32_t y = x ^ L.xmask;
  for (uint32_t i = 0; i < L.ncnot; ++i) y ^= ((x >> L.c[i]) & 1u) << L.t[i];
  return y;
}

__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = 16 >> k;
    const uint32_t M = masks[k];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~M) | ((y & ~M) >> j)) : ((x & M) | ((y & M) << j));
  }
  return x;
}

// Bit-sliced words [g][j-1][q] -> per-chain words P[32 g + c][j-1]; one warp
// per (group, layer).
__global__ void unslice_kernel(const uint32_t* __restrict__ state, int n, int d, uint32_t groups,
                               uint32_t* __restrict__ P) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= groups * (uint32_t)d) return;
  const uint32_t g = w / d, j = w % d;
  const uint32_t x = lane < n ? state[((size_t)g * d + j) * n + lane] : 0u;
  const uint32_t y = warp_transpose(x, lane);
  P[(size_t)(g * 32 + lane) * d + j] = y;
}

// SplitMix64 (Steele, Lea, Flood 2014): the suffix start of a move.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__host__ __device__ inline int suffix_start(uint64_t seed, uint32_t move, int d) {
  return 1 + (int)(splitmix64(seed ^ (0xA5A5ull << 40) ^ move) % (uint64_t)d);
}

// The start of a move: unslice as above, and (thread 0) the suffix start k*
// from the seed and the move count (SplitMix64, so that one captured graph
// serves every move), and the proposal's log q sums cleared.
__global__ void move_begin_kernel(const uint32_t* __restrict__ state, int n, int d, uint32_t groups,
                                  uint32_t* __restrict__ P, MhCounters* __restrict__ ctr, uint64_t seed,
                                  float* __restrict__ lqf, uint32_t chains) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) ctr->k = suffix_start(seed, ctr->moves, d);
  if (i < chains) lqf[i] = 0.f;
  const uint32_t w = i >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= groups * (uint32_t)d) return;
  const uint32_t g = w / d, j = w % d;
  const uint32_t x = lane < n ? state[((size_t)g * d + j) * n + lane] : 0u;
  const uint32_t y = warp_transpose(x, lane);
  P[(size_t)(g * 32 + lane) * d + j] = y;
}

// Per-chain words -> bit-sliced words for layers k..d (1-based), k read from
// k_dev; one warp per (group, layer) over all d layers, the warps of layers
// before k leave at once.
__global__ void slice_kernel(const uint32_t* __restrict__ P, int n, int d, MhCounters* __restrict__ ctr,
                             uint32_t groups, uint32_t* __restrict__ state) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int* k_dev = &ctr->k;
  // the end of the move: its count (read by no kernel of this move after
  // the acceptance, which ran before)
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr->moves += 1u;
  if (w >= groups * (uint32_t)d) return;
  const uint32_t g = w / d, j = w % d;
  if ((int)j + 1 < *k_dev) return;  // the whole warp: layer j+1 is before the suffix
  const uint32_t x = P[(size_t)(g * 32 + lane) * d + j];
  const uint32_t y = warp_transpose(x, lane);
  if (lane < n) state[((size_t)g * d + j) * n + lane] = y;
}

// Row x = [2 s_{j-1} - 1 (n), onehot(j-1) (d), 0...] in bf16, written in
// 16-byte pieces (k_in is a multiple of 16).
__device__ __forceinline__ void write_row(__nv_bfloat16* X, int kin, int n, int d, int row,
                                          uint32_t prev, int j) {
  uint4* x = reinterpret_cast<uint4*>(X + (size_t)row * kin);
  const __nv_bfloat16 one = __float2bfloat16(1.f), mone = __float2bfloat16(-1.f),
                      zero = __float2bfloat16(0.f);
  for (int i0 = 0; i0 < kin; i0 += 8) {
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = i0 + t;
      v[t] = i < n ? (((prev >> i) & 1u) ? one : mone) : (i == n + j - 1 ? one : zero);
    }
    x[i0 / 8] = *reinterpret_cast<const uint4*>(v);
  }
}

// Rows (chain c, layer j = k + r % L) of the current suffix, r from r0.
__global__ void rows_current_kernel(const uint32_t* __restrict__ P, uint32_t beta, int n, int d,
                                    int kin, int k, uint64_t r0, int rows, __nv_bfloat16* X) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int L = d - k + 1;
  const uint64_t rr = r0 + (uint64_t)r;
  const uint32_t c = (uint32_t)(rr / L);
  const int j = k + (int)(rr % L);
  const uint32_t prev = j == 1 ? beta : P[(size_t)c * d + (j - 2)];
  write_row(X, kin, n, d, r, prev, j);
}

// log q of the current suffix rows: lq[c * d + (j-1)] (fixed order, summed later).
__global__ void logq_current_kernel(const float* __restrict__ logits, int npad, const uint32_t* P,
                                    int n, int d, int k, uint64_t r0, int rows,
                                    float* __restrict__ lq) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int L = d - k + 1;
  const uint64_t rr = r0 + (uint64_t)r;
  const uint32_t c = (uint32_t)(rr / L);
  const int j = k + (int)(rr % L);
  const uint32_t bits = P[(size_t)c * d + (j - 1)];
  float s = 0.f;
  for (int q = 0; q < n; ++q) {
    const float l = logits[(size_t)r * npad + q];
    // log sigma(+-l) = -softplus(-+l)
    const float z = ((bits >> q) & 1u) ? -l : l;
    s -= fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z)));
  }
  lq[(size_t)c * d + (j - 1)] = s;
}

// Rows (chain c0 + r, layer j) of the proposal: s'_{j-1} from Pn (j > k) or
// P (j == k).
__global__ void rows_proposal_kernel(const uint32_t* __restrict__ P, const uint32_t* __restrict__ Pn,
                                     uint32_t beta, int n, int d, int kin, int k, int j, uint32_t c0,
                                     int rows, __nv_bfloat16* X) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const uint32_t c = c0 + (uint32_t)r;
  uint32_t prev = beta;
  if (j > 1) prev = (j == k ? P : Pn)[(size_t)c * d + (j - 2)];
  write_row(X, kin, n, d, r, prev, j);
}

// Draw s'_j of each row from sigmoid(logits); accumulate log q'.
__global__ void sample_kernel(const float* __restrict__ logits, int npad, int n, int d, int j,
                              uint32_t c0, int rows, uint32_t k0, uint32_t k1,
                              const uint32_t* __restrict__ move_dev, uint32_t group0,
                              uint32_t* __restrict__ Pn, float* __restrict__ lqf) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const uint32_t move = *move_dev;
  const uint32_t c = c0 + (uint32_t)r;
  const uint32_t gc = group0 * 32u + c;  // global chain id
  uint32_t word = 0u;
  float s = 0.f;
  uint4 u4 = make_uint4(0, 0, 0, 0);
  for (int q = 0; q < n; ++q) {
    if ((q & 3) == 0)
      u4 = philox4x32_10(make_uint4(gc, move, (uint32_t)(j - 1) | (kTagMH << 16), (uint32_t)(q >> 2)),
                         k0, k1);
    const uint32_t u = (q & 3) == 0 ? u4.x : (q & 3) == 1 ? u4.y : (q & 3) == 2 ? u4.z : u4.w;
    const float l = logits[(size_t)r * npad + q];
    const float p1 = 1.f / (1.f + __expf(-l));
    const float uf = ((float)(u >> 8) + 0.5f) * (1.f / 16777216.f);
    const uint32_t b = uf < p1 ? 1u : 0u;
    word |= b << q;
    const float z = b ? -l : l;
    s -= fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z)));
  }
  Pn[(size_t)c * d + (j - 1)] = word;
  lqf[c] += s;
}

// Violation counts of layers k..d for the current and proposed suffix, the
// Metropolis-Hastings decision, and the accepted suffix copied into P.  One
// warp per chain: lane l takes layers k + l, k + l + 32, ...; the warp sums
// the counts and the log q terms (a fixed tree), lane 0 decides.
__global__ void accept_kernel(uint32_t* __restrict__ P, const uint32_t* __restrict__ Pn,
                              const LayerTab* __restrict__ tab, uint32_t beta, uint32_t nmask,
                              int d, float J, const float* __restrict__ lq,
                              const float* __restrict__ lqf, uint32_t chains, uint32_t k0,
                              uint32_t k1, MhCounters* __restrict__ ctr, uint32_t group0) {
  __shared__ uint32_t n_acc;
  if (threadIdx.x == 0) n_acc = 0u;
  __syncthreads();
  const uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const bool in = c < chains;  // warp-uniform
  const uint32_t move = ctr->moves;
  const int k = ctr->k;
  bool acc = false;
  if (in) {
    const uint32_t* cur = P + (size_t)c * d;
    const uint32_t* prop = Pn + (size_t)c * d;
    int v = 0, vn = 0;
    float lrev = 0.f;
    for (int j = k + lane; j <= d; j += 32) {
      const LayerTab& L = tab[j - 1];
      const uint32_t link = ~L.hmask & nmask;
      const uint32_t pc = j == 1 ? beta : cur[j - 2];   // s_{j-1}
      const uint32_t pn = j == k ? pc : prop[j - 2];    // s'_{j-1}, s'_{k-1} = s_{k-1}
      v += __popc((cur[j - 1] ^ layer_map(L, pc)) & link);
      vn += __popc((prop[j - 1] ^ layer_map(L, pn)) & link);
      lrev += lq[(size_t)c * d + (j - 1)];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, off);
      vn += __shfl_xor_sync(0xffffffffu, vn, off);
      lrev += __shfl_xor_sync(0xffffffffu, lrev, off);
    }
    if (lane == 0) {
      const float logA = -J * (float)(vn - v) + lrev - lqf[c];
      const uint32_t gc = group0 * 32u + c;
      const uint32_t u = philox4x32_10(make_uint4(gc, move, 0xFFFFu | (kTagMH << 16), 0u), k0, k1).x;
      const float uf = ((float)(u >> 8) + 0.5f) * (1.f / 16777216.f);
      acc = logf(uf) < logA;
      if (acc) atomicAdd(&n_acc, 1u);
    }
    acc = __shfl_sync(0xffffffffu, acc, 0);
    if (acc)
      for (int j = k + lane; j <= d; j += 32) P[(size_t)c * d + (j - 1)] = prop[j - 1];
  }
  __syncthreads();
  if (threadIdx.x == 0 && n_acc) atomicAdd(&ctr->accepted, (unsigned long long)n_acc);
}

// A host-drawn k* (networks that do not fit the fused kernel).
__global__ void set_k_kernel(MhCounters* ctr, int k) { ctr->k = k; }

__global__ void zero_f32_kernel(float* __restrict__ x, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.f;
}

// Valid paths (no violated link) appended to out[count][d] while room is
// left, in chain order: one CTA walks the chains in tiles of its threads; a
// tile's valid chains take consecutive slots by a warp ballot and the
// warps' counts (an exclusive prefix sum), so the collected data, and a
// training run on it, are the same on every run.  *count grows by the
// number of valid chains (also past the capacity).
__global__ void __launch_bounds__(1024) collect_kernel(const uint32_t* __restrict__ P,
                                                       const LayerTab* __restrict__ tab,
                                                       uint32_t beta, uint32_t nmask, int d,
                                                       uint32_t chains, uint32_t* __restrict__ out,
                                                       unsigned long long capacity,
                                                       unsigned long long* __restrict__ count) {
  __shared__ unsigned long long base;
  __shared__ uint32_t wcount[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid == 0) base = *count;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < chains; c0 += blockDim.x) {
    const uint32_t c = c0 + (uint32_t)tid;
    bool valid = false;
    if (c < chains) {
      const uint32_t* s = P + (size_t)c * d;
      uint32_t prev = beta;
      int v = 0;
      for (int j = 1; j <= d; ++j) {
        const LayerTab& L = tab[j - 1];
        v += __popc((s[j - 1] ^ layer_map(L, prev)) & ~L.hmask & nmask);
        prev = s[j - 1];
      }
      valid = v == 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) wcount[warp] = (uint32_t)__popc(bal);
    __syncthreads();
    uint32_t off = 0, total = 0;
    for (int w = 0; w < nwarps; ++w) {
      if (w < warp) off += wcount[w];
      total += wcount[w];
    }
    const unsigned long long slot = base + off + (uint32_t)__popc(bal & ((1u << lane) - 1u));
    if (valid && slot < capacity) {
      const uint32_t* s = P + (size_t)c * d;
      for (int j = 0; j < d; ++j) out[slot * d + j] = s[j];
    }
    __syncthreads();  // every thread has read base and wcount
    if (tid == 0) base += total;
    __syncthreads();
  }
  if (tid == 0) *count = base;
}

// Training rows from collected paths: row r takes path i and layer j drawn
// from Philox (key = seed, counter (r, step, 3 << 16, 0)); input s_{j-1},
// target bits s_j.
__global__ void train_rows_kernel(const uint32_t* __restrict__ paths, unsigned long long n_paths,
                                  uint32_t beta, int n, int d, int kin, int rows, uint32_t k0,
                                  uint32_t k1, uint32_t step, __nv_bfloat16* X, float* target) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const uint4 u = philox4x32_10(make_uint4((uint32_t)r, step, 3u << 16, 0u), k0, k1);
  const unsigned long long i =
      ((((unsigned long long)u.x << 32) | u.y) % n_paths);  // < n_paths
  const int j = 1 + (int)(((unsigned long long)u.z * (unsigned long long)d) >> 32);
  const uint32_t* p = paths + i * d;
  const uint32_t prev = j == 1 ? beta : p[j - 2];
  write_row(X, kin, n, d, r, prev, j);
  const uint32_t nxt = p[j - 1];
  for (int q = 0; q < n; ++q) target[(size_t)r * n + q] = (float)((nxt >> q) & 1u);
}

}  // namespace pb

using namespace pb;

namespace {

std::vector<LayerTab> layer_table(const pb_model& m) {
  std::vector<LayerTab> t(m.d);
  for (auto& L : t) std::memset(&L, 0, sizeof L);
  for (const pb_gate& g : m.gates) {
    LayerTab& L = t[g.layer];
    if (g.op == PB_H) L.hmask |= 1u << g.q0;
    if (g.op == PB_X) L.xmask |= 1u << g.q0;
    if (g.op == PB_CNOT && L.ncnot < 16) {
      L.c[L.ncnot] = (uint8_t)g.q0;
      L.t[L.ncnot] = (uint8_t)g.q1;
      ++L.ncnot;
    }
  }
  return t;
}

struct MhLayout {
  size_t ctr, tab, P, Pn, lq, lqf, total;
};

MhLayout mh_layout(int d, uint32_t groups) {
  MhLayout L{};
  size_t p = 0;
  auto take = [&](size_t b) {
    p = (p + 255) & ~(size_t)255;
    size_t at = p;
    p += b;
    return at;
  };
  const size_t C = (size_t)groups * 32;
  L.ctr = take(sizeof(MhCounters));  // offset 0
  L.tab = take(sizeof(LayerTab) * 64);
  L.P = take(C * d * 4);
  L.Pn = take(C * d * 4);
  L.lq = take(C * d * 4);
  L.lqf = take(C * 4);
  L.total = (p + 255) & ~(size_t)255;
  return L;
}

// The pieces of a move region.
struct MhPtrs {
  MhCounters* ctr;
  const LayerTab* tab;
  uint32_t *P, *Pn;
  float *lq, *lqf;
};
MhPtrs mh_ptrs(const MhCtx& c) {
  const MhLayout L = mh_layout(c.model->d, c.groups);
  MhPtrs q;
  q.ctr = reinterpret_cast<MhCounters*>(c.ws + L.ctr);
  q.tab = reinterpret_cast<const LayerTab*>(c.ws + L.tab);
  q.P = reinterpret_cast<uint32_t*>(c.ws + L.P);
  q.Pn = reinterpret_cast<uint32_t*>(c.ws + L.Pn);
  q.lq = reinterpret_cast<float*>(c.ws + L.lq);
  q.lqf = reinterpret_cast<float*>(c.ws + L.lqf);
  return q;
}

// Acceptance, slicing back and the move counter: the end of every move.
cudaError_t finish_move(const MhCtx& c, const MhPtrs& q, cudaStream_t st) {
  const pb_model& m = *c.model;
  const int n = m.n, d = m.d, T = 256;
  const uint32_t nmask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
  accept_kernel<<<(c.chains * 32 + T - 1) / T, T, 0, st>>>(q.P, q.Pn, q.tab, m.beta, nmask, d, (float)m.J,
                                                           q.lq, q.lqf, c.chains, k0, k1, q.ctr, c.group0);
  // slicing back also counts the move
  const uint32_t sw = c.groups * (uint32_t)d;
  slice_kernel<<<(sw * 32 + T - 1) / T, T, 0, st>>>(q.P, n, d, q.ctr, c.groups, c.state);
  return cudaGetLastError();
}

// The kernels of one move with a host-drawn suffix start k (networks that
// do not fit the fused kernel: rows batched through the layer-by-layer GEMMs).
cudaError_t enqueue_move_host_k(const MhCtx& c, int k, cudaStream_t st) {
  const pb_model& m = *c.model;
  pb_mlp* mlp = c.mlp;
  const MhPtrs q = mh_ptrs(c);
  const int n = m.n, d = m.d, kin = mlp->kin, npad = mlp->npad, B = mlp->batch;
  const uint32_t C = c.chains;
  const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
  const int T = 256;
  const int Ls = d - k + 1;
  cudaStream_t mst = mlp->st;
  mlp->st = st;
  cudaError_t e = cudaSuccess;
  const uint32_t warps = c.groups * (uint32_t)d;
  unslice_kernel<<<(warps * 32 + T - 1) / T, T, 0, st>>>(c.state, n, d, c.groups, q.P);
  set_k_kernel<<<1, 1, 0, st>>>(q.ctr, k);
  const uint64_t rows_total = (uint64_t)C * Ls;
  for (uint64_t r0 = 0; r0 < rows_total && e == cudaSuccess; r0 += B) {
    const int rows = (int)std::min<uint64_t>(B, rows_total - r0);
    rows_current_kernel<<<(rows + T - 1) / T, T, 0, st>>>(q.P, m.beta, n, d, kin, k, r0, rows, mlp->X);
    if ((e = mlp_forward_rows(mlp, rows)) != cudaSuccess) break;
    logq_current_kernel<<<(rows + T - 1) / T, T, 0, st>>>(mlp->logits, npad, q.P, n, d, k, r0, rows, q.lq);
  }
  zero_f32_kernel<<<(C + T - 1) / T, T, 0, st>>>(q.lqf, C);
  for (int j = k; j <= d && e == cudaSuccess; ++j) {
    for (uint32_t c0 = 0; c0 < C && e == cudaSuccess; c0 += (uint32_t)B) {
      const int rows = (int)std::min<uint32_t>((uint32_t)B, C - c0);
      rows_proposal_kernel<<<(rows + T - 1) / T, T, 0, st>>>(q.P, q.Pn, m.beta, n, d, kin, k, j, c0,
                                                             rows, mlp->X);
      if ((e = mlp_forward_rows(mlp, rows)) != cudaSuccess) break;
      sample_kernel<<<(rows + T - 1) / T, T, 0, st>>>(mlp->logits, npad, n, d, j, c0, rows, k0, k1,
                                                      &q.ctr->moves, c.group0, q.Pn, q.lqf);
    }
  }
  if (e == cudaSuccess) e = finish_move(c, q, st);
  mlp->st = mst;
  return e;
}

}  // namespace

namespace pb {

size_t mh_region_bytes(int d, uint32_t groups) { return mh_layout(d, groups).total; }

bool mh_fused(const pb_mlp* mlp) { return mlp->kin <= 96 && mlp->npad <= 32; }

cudaError_t mh_region_init(const MhCtx& c, cudaStream_t st) {
  const MhLayout L = mh_layout(c.model->d, c.groups);
  const std::vector<LayerTab> tab = layer_table(*c.model);
  cudaError_t e = cudaMemsetAsync(c.ws, 0, L.total, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.ws + L.tab, tab.data(), sizeof(LayerTab) * c.model->d, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host table is a local
  return e;
}

// One move (fused networks): unslice, draw k*, log q of the current suffix,
// the proposal layer by layer, acceptance, slice back; no host value depends
// on k*, so the sequence is captured once.
cudaError_t mh_enqueue_move_dev(const MhCtx& c, cudaStream_t st) {
  const pb_model& m = *c.model;
  const MhPtrs q = mh_ptrs(c);
  const int n = m.n, d = m.d, T = 256;
  const uint32_t C = c.chains;
  const uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
  const uint32_t warps = c.groups * (uint32_t)d;
  move_begin_kernel<<<(warps * 32 + T - 1) / T, T, 0, st>>>(c.state, n, d, c.groups, q.P, q.ctr, c.seed,
                                                            q.lqf, C);
  // the proposal (sequential over the suffix layers, one CTA per 128
  // chains) first on st; log q of the current suffix (one CTA per tile and
  // layer) beside it on the side stream; both read P and k only
  cudaError_t e = cudaSuccess;
  if (c.side) {
    if ((e = cudaEventRecord(c.fork, st)) != cudaSuccess || (e = cudaStreamWaitEvent(c.side, c.fork, 0)) != cudaSuccess)
      return e;
  }
  e = mlp_fused_sample_dev(c.mlp, q.P, q.Pn, m.beta, (int)C, &q.ctr->k, q.lqf, k0, k1, &q.ctr->moves,
                           c.group0, st);
  if (e != cudaSuccess) return e;
  e = mlp_fused_logq_dev(c.mlp, q.P, m.beta, (int)C, &q.ctr->k, q.lq, c.side ? c.side : st);
  if (e != cudaSuccess) return e;
  if (c.side) {
    if ((e = cudaEventRecord(c.join, c.side)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c.join, 0)) != cudaSuccess)
      return e;
  }
  return finish_move(c, q, st);
}

cudaError_t mh_ctx_open(MhCtx& c) {
  cudaError_t e = cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming);
  return e;
}

void mh_ctx_close(MhCtx& c) {
  if (c.fork) cudaEventDestroy(c.fork);
  if (c.join) cudaEventDestroy(c.join);
  if (c.side) cudaStreamDestroy(c.side);
  c.fork = c.join = nullptr;
  c.side = nullptr;
}

}  // namespace pb

namespace {

MhCtx mh_ctx(const RunView& v, pb_mlp* mlp, char* ws) {
  MhCtx c;
  c.model = v.model;
  c.mlp = mlp;
  c.state = v.state;
  c.chains = v.chains;
  c.groups = v.groups;
  c.group0 = v.group0;
  c.seed = v.seed;
  c.ws = ws;
  return c;
}

}  // namespace

extern "C" {

PB_API int pb_mh_workspace_bytes(const pb_run* run, int model, size_t* bytes) {
  RunView v;
  if (!bytes) return PB_EINVAL;
  int rc = run_view(run, model, &v);
  if (rc != PB_OK) return rc;
  *bytes = mh_layout(v.model->d, v.groups).total;
  return PB_OK;
}

}  // extern "C"

struct pb_mh {
  pb_run* run = nullptr;
  RunView v{};
  MhCtx c{};
  uint32_t moves = 0;
  cudaStream_t cap_st = nullptr;
  cudaGraphExec_t graph = nullptr;      // fused networks: one graph, k* drawn on the device
  std::vector<cudaGraphExec_t> graphs;  // otherwise one per k* (1..d), built on first use
};

extern "C" {

PB_API int pb_mh_create(pb_run* run, int model, pb_mlp* mlp, void* d_ws, size_t ws_bytes,
                        pb_mh** out) {
  if (!out) return PB_EINVAL;
  *out = nullptr;
  RunView v;
  int rc = run_view(run, model, &v);
  if (rc != PB_OK) return rc;
  if (!mlp || !d_ws || ((uintptr_t)d_ws & 255)) return PB_EINVAL;
  const pb_model& m = *v.model;
  if (mlp->n != m.n || mlp->d != m.d) return PB_EINVAL;
  if (ws_bytes < mh_layout(m.d, v.groups).total) return PB_ERANGE;
  pb_mh* h = new (std::nothrow) pb_mh;
  if (!h) return PB_ENOMEM;
  h->run = run;
  h->v = v;
  h->c = mh_ctx(v, mlp, static_cast<char*>(d_ws));
  h->graphs.assign(m.d + 1, nullptr);
  cudaError_t e = mh_ctx_open(h->c);
  if (e == cudaSuccess) e = mh_region_init(h->c, v.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mlp->st);
  if (e == cudaSuccess) e = mlp_prepare();
  if (e != cudaSuccess) {
    mh_ctx_close(h->c);
    delete h;
    return PB_ECUDA;
  }
  *out = h;
  return PB_OK;
}

// n_moves further moves, each a replay of a captured graph (asynchronous on
// the run's stream).
PB_API int pb_mh_moves(pb_mh* h, uint32_t n_moves) {
  if (!h) return PB_EINVAL;
  const int d = h->v.model->d;
  const bool fused = mh_fused(h->c.mlp);
  for (uint32_t i = 0; i < n_moves; ++i) {
    const int k = suffix_start(h->v.seed, h->moves, d);
    cudaGraphExec_t& ex = fused ? h->graph : h->graphs[k];
    if (!ex) {
      if (!h->cap_st && cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking) != cudaSuccess)
        return PB_ECUDA;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PB_ECUDA;
      cudaError_t e = fused ? mh_enqueue_move_dev(h->c, h->cap_st) : enqueue_move_host_k(h->c, k, h->cap_st);
      cudaError_t e2 = cudaStreamEndCapture(h->cap_st, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return PB_ECUDA;
      }
      e = cudaGraphInstantiate(&ex, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) { ex = nullptr; return PB_ECUDA; }
    }
    if (cudaGraphLaunch(ex, h->v.st) != cudaSuccess) return PB_ECUDA;
    h->moves += 1;
  }
  return PB_OK;
}

// Moves done and proposals accepted so far (synchronous).
PB_API int pb_mh_stats(pb_mh* h, uint64_t* moves, uint64_t* accepted) {
  if (!h) return PB_EINVAL;
  MhCounters ctr{};
  uint32_t st = 0u;
  if (cudaMemcpyAsync(&ctr, h->c.ws, sizeof ctr, cudaMemcpyDeviceToHost, h->v.st) != cudaSuccess ||
      cudaMemcpyAsync(&st, h->c.mlp->status, 4, cudaMemcpyDeviceToHost, h->v.st) != cudaSuccess ||
      cudaStreamSynchronize(h->v.st) != cudaSuccess)
    return PB_ECUDA;
  if (moves) *moves = h->moves;
  if (accepted) *accepted = ctr.accepted;
  // a bounded wait of the network's kernels ran out: the moves since are not valid
  return st != 0u ? (int)st : PB_OK;
}

PB_API void pb_mh_free(pb_mh* h) {
  if (!h) return;
  cudaStreamSynchronize(h->v.st);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (auto& g : h->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  mh_ctx_close(h->c);
  delete h;
}

PB_API int pb_run_collect_paths(pb_run* run, int model, void* d_ws, size_t ws_bytes,
                                uint32_t* d_paths, uint64_t capacity, uint64_t* d_count) {
  RunView v;
  int rc = run_view(run, model, &v);
  if (rc != PB_OK) return rc;
  if (!d_ws || !d_paths || !d_count || ((uintptr_t)d_ws & 255)) return PB_EINVAL;
  const pb_model& m = *v.model;
  const MhLayout L = mh_layout(m.d, v.groups);
  if (ws_bytes < L.total) return PB_ERANGE;
  char* ws = static_cast<char*>(d_ws);
  uint32_t* P = reinterpret_cast<uint32_t*>(ws + L.P);
  const std::vector<LayerTab> tab = layer_table(m);
  cudaError_t e = cudaMemcpyAsync(ws + L.tab, tab.data(), sizeof(LayerTab) * m.d,
                                  cudaMemcpyHostToDevice, v.st);
  const int T = 256;
  const uint32_t warps = v.groups * (uint32_t)m.d;
  unslice_kernel<<<(warps * 32 + T - 1) / T, T, 0, v.st>>>(v.state, m.n, m.d, v.groups, P);
  const uint32_t nmask = m.n == 32 ? 0xFFFFFFFFu : ((1u << m.n) - 1u);
  collect_kernel<<<1, 1024, 0, v.st>>>(P, reinterpret_cast<const LayerTab*>(ws + L.tab), m.beta, nmask,
                                       m.d, v.chains, d_paths, capacity,
                                       reinterpret_cast<unsigned long long*>(d_count));
  if (e == cudaSuccess) e = cudaGetLastError();
  // host layer table must outlive the staged copy
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.st);
  return e == cudaSuccess ? PB_OK : PB_ECUDA;
}

PB_API int pb_mlp_train_paths(pb_mlp* mlp, const uint32_t* d_paths, uint64_t n_paths, uint32_t beta,
                              int steps, int rows, float lr, uint64_t seed, float* d_losses) {
  if (!mlp || !d_paths || n_paths == 0 || steps <= 0) return PB_EINVAL;
  if (rows <= 0 || rows > mlp->batch || rows % 8) return PB_EINVAL;
  const int T = 256;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < steps && e == cudaSuccess; ++s) {
    train_rows_kernel<<<(rows + T - 1) / T, T, 0, mlp->st>>>(d_paths, n_paths, beta, mlp->n, mlp->d,
                                                             mlp->kin, rows, k0, k1, (uint32_t)s,
                                                             mlp->X, mlp->target);
    if ((e = mlp_forward_rows(mlp, rows)) != cudaSuccess) break;
    if ((e = mlp_backward_rows(mlp, rows)) != cudaSuccess) break;
    if (d_losses) cudaMemcpyAsync(d_losses + s, mlp->loss, 4, cudaMemcpyDeviceToDevice, mlp->st);
    e = mlp_adam_step(mlp, lr);
  }
  return e == cudaSuccess ? PB_OK : PB_ECUDA;
}

}  // extern "C"
