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

// Per-chain words -> bit-sliced words for layers k0..d (1-based).
__global__ void slice_kernel(const uint32_t* __restrict__ P, int n, int d, int k0, uint32_t groups,
                             uint32_t* __restrict__ state) {
  const int L = d - k0 + 1;
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= groups * (uint32_t)L) return;
  const uint32_t g = w / L, j = (k0 - 1) + w % L;
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
// Metropolis-Hastings decision, and the accepted suffix copied into P.
__global__ void accept_kernel(uint32_t* __restrict__ P, const uint32_t* __restrict__ Pn,
                              const LayerTab* __restrict__ tab, uint32_t beta, uint32_t nmask,
                              int d, int k, float J, const float* __restrict__ lq,
                              const float* __restrict__ lqf, uint32_t chains, uint32_t k0,
                              uint32_t k1, const uint32_t* __restrict__ move_dev, uint32_t group0,
                              unsigned long long* __restrict__ n_accept) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= chains) return;
  const uint32_t move = *move_dev;
  const uint32_t* cur = P + (size_t)c * d;
  const uint32_t* prop = Pn + (size_t)c * d;
  const uint32_t base = k == 1 ? beta : cur[k - 2];
  int v = 0, vn = 0;
  uint32_t pc = base, pn = base;
  float lrev = 0.f;
  for (int j = k; j <= d; ++j) {
    const LayerTab& L = tab[j - 1];
    const uint32_t link = ~L.hmask & nmask;
    v += __popc((cur[j - 1] ^ layer_map(L, pc)) & link);
    vn += __popc((prop[j - 1] ^ layer_map(L, pn)) & link);
    pc = cur[j - 1];
    pn = prop[j - 1];
    lrev += lq[(size_t)c * d + (j - 1)];
  }
  const float logA = -J * (float)(vn - v) + lrev - lqf[c];
  const uint32_t gc = group0 * 32u + c;
  const uint32_t u = philox4x32_10(make_uint4(gc, move, 0xFFFFu | (kTagMH << 16), 0u), k0, k1).x;
  const float uf = ((float)(u >> 8) + 0.5f) * (1.f / 16777216.f);
  const bool acc = logf(uf) < logA;
  // one counter update per warp (the accepted lanes' count)
  const unsigned act = __activemask();
  const unsigned accm = __ballot_sync(act, acc);
  if (accm != 0u && (int)(threadIdx.x & 31u) == __ffs((int)act) - 1)
    atomicAdd(n_accept, (unsigned long long)__popc(accm));
  if (acc)
    for (int j = k; j <= d; ++j) P[(size_t)c * d + (j - 1)] = prop[j - 1];
}

__global__ void mh_advance_kernel(uint32_t* move_dev) { *move_dev += 1u; }

// Valid paths (no violated link) appended to out[count][d] while room is left.
__global__ void collect_kernel(const uint32_t* __restrict__ P, const LayerTab* __restrict__ tab,
                               uint32_t beta, uint32_t nmask, int d, uint32_t chains,
                               uint32_t* __restrict__ out, unsigned long long capacity,
                               unsigned long long* __restrict__ count) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= chains) return;
  const uint32_t* s = P + (size_t)c * d;
  uint32_t prev = beta;
  int v = 0;
  for (int j = 1; j <= d; ++j) {
    const LayerTab& L = tab[j - 1];
    v += __popc((s[j - 1] ^ layer_map(L, prev)) & ~L.hmask & nmask);
    prev = s[j - 1];
  }
  if (v != 0) return;
  const unsigned long long slot = atomicAdd(count, 1ull);
  if (slot >= capacity) return;
  for (int j = 0; j < d; ++j) out[slot * d + j] = s[j];
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
  size_t tab, P, Pn, lq, lqf, cnt, move, total;
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
  L.tab = take(sizeof(LayerTab) * 64);
  L.P = take(C * d * 4);
  L.Pn = take(C * d * 4);
  L.lq = take(C * d * 4);
  L.lqf = take(C * 4);
  L.cnt = take(16);
  L.move = take(16);
  L.total = (p + 255) & ~(size_t)255;
  return L;
}

uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
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
  pb_mlp* mlp = nullptr;
  int model = 0;
  RunView v{};
  char* ws = nullptr;
  size_t ws_bytes = 0;
  MhLayout L{};
  uint32_t moves = 0;
  cudaStream_t cap_st = nullptr;
  std::vector<cudaGraphExec_t> graphs;  // one per k* (1..d), built on first use
};

namespace {

// The kernels of one move with suffix start k, in stream order.
cudaError_t enqueue_move(pb_mh* h, int k, cudaStream_t st) {
  const pb_model& m = *h->v.model;
  pb_mlp* mlp = h->mlp;
  char* ws = h->ws;
  const MhLayout& L = h->L;
  uint32_t* P = reinterpret_cast<uint32_t*>(ws + L.P);
  uint32_t* Pn = reinterpret_cast<uint32_t*>(ws + L.Pn);
  float* lq = reinterpret_cast<float*>(ws + L.lq);
  float* lqf = reinterpret_cast<float*>(ws + L.lqf);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ws + L.cnt);
  uint32_t* move_dev = reinterpret_cast<uint32_t*>(ws + L.move);
  const LayerTab* dtab = reinterpret_cast<const LayerTab*>(ws + L.tab);
  const int n = m.n, d = m.d, kin = mlp->kin, npad = mlp->npad, B = mlp->batch;
  const uint32_t nmask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint32_t C = h->v.chains;
  const uint32_t k0 = (uint32_t)h->v.seed, k1 = (uint32_t)(h->v.seed >> 32);
  const int T = 256;
  const int Ls = d - k + 1;
  cudaStream_t mst = mlp->st;
  mlp->st = st;
  cudaError_t e = cudaSuccess;
  const bool fused = mlp->kin <= 96 && mlp->npad <= 32;
  const uint32_t warps = h->v.groups * (uint32_t)d;
  unslice_kernel<<<(warps * 32 + T - 1) / T, T, 0, st>>>(h->v.state, n, d, h->v.groups, P);
  if (fused) {
    // one launch for log q of the current suffix, one per proposal layer
    e = mlp_fused_logq(mlp, P, m.beta, (int)C, k, lq, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(lqf, 0, (size_t)C * 4, st);
    if (e == cudaSuccess)
      e = mlp_fused_sample(mlp, P, Pn, m.beta, (int)C, k, k, d, lqf, k0, k1, move_dev, h->v.group0, st);
  } else {
    const uint64_t rows_total = (uint64_t)C * Ls;
    for (uint64_t r0 = 0; r0 < rows_total && e == cudaSuccess; r0 += B) {
      const int rows = (int)std::min<uint64_t>(B, rows_total - r0);
      rows_current_kernel<<<(rows + T - 1) / T, T, 0, st>>>(P, m.beta, n, d, kin, k, r0, rows, mlp->X);
      if ((e = mlp_forward_rows(mlp, rows)) != cudaSuccess) break;
      logq_current_kernel<<<(rows + T - 1) / T, T, 0, st>>>(mlp->logits, npad, P, n, d, k, r0, rows, lq);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(lqf, 0, (size_t)C * 4, st);
    for (int j = k; j <= d && e == cudaSuccess; ++j) {
      for (uint32_t c0 = 0; c0 < C && e == cudaSuccess; c0 += (uint32_t)B) {
        const int rows = (int)std::min<uint32_t>((uint32_t)B, C - c0);
        rows_proposal_kernel<<<(rows + T - 1) / T, T, 0, st>>>(P, Pn, m.beta, n, d, kin, k, j, c0,
                                                               rows, mlp->X);
        if ((e = mlp_forward_rows(mlp, rows)) != cudaSuccess) break;
        sample_kernel<<<(rows + T - 1) / T, T, 0, st>>>(mlp->logits, npad, n, d, j, c0, rows, k0, k1,
                                                        move_dev, h->v.group0, Pn, lqf);
      }
    }
  }
  if (e == cudaSuccess) {
    accept_kernel<<<(C + T - 1) / T, T, 0, st>>>(P, Pn, dtab, m.beta, nmask, d, k, (float)m.J, lq,
                                                 lqf, C, k0, k1, move_dev, h->v.group0, cnt);
    const uint32_t sw = h->v.groups * (uint32_t)Ls;
    slice_kernel<<<(sw * 32 + T - 1) / T, T, 0, st>>>(P, n, d, k, h->v.groups, h->v.state);
    mh_advance_kernel<<<1, 1, 0, st>>>(move_dev);
    e = cudaGetLastError();
  }
  mlp->st = mst;
  return e;
}

}  // namespace

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
  const MhLayout L = mh_layout(m.d, v.groups);
  if (ws_bytes < L.total) return PB_ERANGE;
  pb_mh* h = new (std::nothrow) pb_mh;
  if (!h) return PB_ENOMEM;
  h->run = run; h->mlp = mlp; h->model = model; h->v = v;
  h->ws = static_cast<char*>(d_ws); h->ws_bytes = ws_bytes; h->L = L;
  h->graphs.assign(m.d + 1, nullptr);
  const std::vector<LayerTab> tab = layer_table(m);
  cudaError_t e = cudaMemsetAsync(h->ws, 0, L.total, v.st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + L.tab, tab.data(), sizeof(LayerTab) * m.d, cudaMemcpyHostToDevice, v.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mlp->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.st);
  if (e == cudaSuccess) e = mlp_prepare();
  if (e != cudaSuccess) { delete h; return PB_ECUDA; }
  *out = h;
  return PB_OK;
}

// n_moves further moves, each replayed from a CUDA graph captured for its
// suffix start k* (asynchronous on the run's stream).
PB_API int pb_mh_moves(pb_mh* h, uint32_t n_moves) {
  if (!h) return PB_EINVAL;
  const int d = h->v.model->d;
  for (uint32_t i = 0; i < n_moves; ++i) {
    const uint32_t move = h->moves;
    const int k = 1 + (int)(splitmix(h->v.seed ^ (0xA5A5ull << 40) ^ move) % (uint64_t)d);
    cudaGraphExec_t& ex = h->graphs[k];
    if (!ex) {
      if (!h->cap_st && cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking) != cudaSuccess)
        return PB_ECUDA;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PB_ECUDA;
      cudaError_t e = enqueue_move(h, k, h->cap_st);
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
  unsigned long long acc = 0;
  uint32_t st = 0u;
  if (cudaMemcpyAsync(&acc, h->ws + h->L.cnt, 8, cudaMemcpyDeviceToHost, h->v.st) != cudaSuccess ||
      cudaMemcpyAsync(&st, h->mlp->status, 4, cudaMemcpyDeviceToHost, h->v.st) != cudaSuccess ||
      cudaStreamSynchronize(h->v.st) != cudaSuccess)
    return PB_ECUDA;
  if (moves) *moves = h->moves;
  if (accepted) *accepted = acc;
  // a bounded wait of the network's kernels ran out: the moves since are not valid
  return st != 0u ? (int)st : PB_OK;
}

PB_API void pb_mh_free(pb_mh* h) {
  if (!h) return;
  cudaStreamSynchronize(h->v.st);
  for (auto& g : h->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
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
  collect_kernel<<<(v.chains + T - 1) / T, T, 0, v.st>>>(
      P, reinterpret_cast<const LayerTab*>(ws + L.tab), m.beta, nmask, m.d, v.chains, d_paths,
      capacity, reinterpret_cast<unsigned long long*>(d_count));
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
