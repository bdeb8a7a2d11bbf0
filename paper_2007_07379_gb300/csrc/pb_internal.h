// Internal layout shared by the host compiler, the runtime and the kernels.
#pragma once
#include <cstddef>
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pbits.h"

namespace pb {

// Word indices in a chain group's shared-memory image: layer k word q sits
// at k*n + q (k = 0 is the clamped input), followed by a zero word and an
// all-ones word.
__host__ __device__ inline int zero_idx(int n, int d) { return (d + 1) * n; }
__host__ __device__ inline int ones_idx(int n, int d) { return (d + 1) * n + 1; }
__host__ __device__ inline int n_words(int n, int d) { return (d + 1) * n + 2; }

// One p-bit update (16 bytes).  Link i (i < m) demands the value
// r_i = W[a[i]] ^ W[b[i]]; the p-bit's violation count changes by
// v = sum_i (1 - 2 r_i) when it goes 0 -> 1.
struct Desc {
  uint16_t dst;   // word index of the p-bit (k*n + q)
  uint8_t mflag;  // bits 0-1: m (links), bit 2: link 0 is the p-bit's own link,
                  // bit 3: coupled (Metropolis acceptance, see Cpl),
                  // bit 4: general links (a Toffoli's, see GLink),
                  // bit 5: table acceptance (two-qubit tables, see TAcc)
  uint8_t pair;   // threshold pair: 0 (t0,t0) 1 (t1,t1) 2 (t2,t0) 3 (t3,t1)
  uint16_t a[3];
  uint16_t b[3];
};
static_assert(sizeof(Desc) == 16, "Desc must be 16 bytes");

// Record term of one p-bit (16 bytes): violation word W[vd]^W[va]^W[vb]
// (all ZERO when the p-bit has no own link; general-gate runs read
// W[vd]^W[va]^(W[vb]&W[vc]), vc = ONES except on a Toffoli target) and phase
// term w * (W[pa] & W[pb]) with w in {0, 1, 2, 4} units of pi/4.
struct Rec {
  uint16_t vd, va, vb;
  uint16_t pa, pb;
  uint16_t w;
  uint16_t vc, pad;
};
static_assert(sizeof(Rec) == 16, "Rec must be 16 bytes");

// Coupling of one p-bit to the neighbours of its coupled general gates
// (32 bytes, by p; models with PB_U gates only).  Category c = e_in + 2 e_out
// with e_in = x ^ W[win], e_out = x ^ W[wout] (win / wout = the p-bit's own
// word where it has no such neighbour): a proposed flip is accepted always
// (amask bit c) or when the tag-6 uniform is below A[c].  B: the exact
// sampler's threshold of a coupled output.  flags bit 0: the p-bit has a
// coupling; bit 1: it is the output of a coupled gate.
struct Cpl {
  uint16_t win, wout;
  uint32_t amask;
  uint32_t A[4];
  uint32_t B;
  uint32_t flags;
};
static_assert(sizeof(Cpl) == 32, "Cpl must be 32 bytes");

// General links of a p-bit next to a Toffoli gate (32 bytes, by p): link i
// demands r_i = W[a] ^ (W[b] & W[c]) and counts where W[e] is set (e = ZERO:
// no link; a plain link has c = e = ONES; a control's link through the
// target is active where the other control is 1).  Link 0 is the own link
// when the p-bit has one (its value for the initial path and the exact
// sampler).
struct GLink {
  uint16_t a[3], b[3], c[3], e[3];
  uint32_t pad[2];
};
static_assert(sizeof(GLink) == 32, "GLink must be 32 bytes");

// Metropolis acceptance of a p-bit next to two-qubit table gates (Eq. ET2),
// 544 bytes by p: a proposed flip of a chain is kept when bit idx of amask is
// set or the chain's tag-7 uniform is below thr[idx], idx = the bits of
// W[w[0..5]] at the chain (the in-table's other output and inputs, the
// out-table's other input and outputs; ZERO where absent) | old value << 6.
struct TAcc {
  uint16_t w[6];
  uint16_t pad[2];
  uint32_t amask[4];
  uint32_t thr[128];
};
static_assert(sizeof(TAcc) == 544, "TAcc must be 544 bytes");

// Record entry of a two-qubit table gate (80 bytes): inputs W[wx0], W[wx1],
// outputs W[wy0], W[wy1]; entry idx = x0 + 2 x1 + 4 (y0 + 2 y1): phase
// ph[idx] (2^-32 turn), zero entry (an invalid path) when bit idx of zmask.
struct TRec {
  uint16_t wx0, wx1, wy0, wy1;
  uint32_t zmask;
  uint32_t ph[16];
  uint32_t pad;
};
static_assert(sizeof(TRec) == 80, "TRec must be 80 bytes");

// Phase of one general gate (32 bytes): ph[2 y + x] = arg U_yx in units of
// 2^-32 turn, y = bit W[wout], x = bit W[win] of the chain.
struct UPh {
  uint32_t ph[4];
  uint16_t wout, win;
  uint32_t pad[3];
};
static_assert(sizeof(UPh) == 32, "UPh must be 32 bytes");

// Per-model device header (in the workspace).
struct ModelDev {
  int32_t n, d, nw;        // qubits, layers, words per group image
  int32_t h;
  uint32_t beta;
  uint32_t thr[4];
  int32_t col_off[5];      // descriptor ranges per colour class
  int32_t max_col;         // largest colour class
  int32_t wgt;             // 1: PB_U gates (complex phase sums, couplings)
  int32_t n_ug;            // PB_U gates (UPh entries)
  int32_t n_tr;            // two-qubit table gates (TRec entries)
  double log2z;            // log2 of the estimator scale
};

// Per-model run entry (device), one per model of a run.
struct RunModelDev {
  const ModelDev* model;
  const Desc* desc;        // n*d, ordered by colour class
  const Rec* rec;          // n*d
  uint32_t* state;         // groups * d * n words
  unsigned long long* hist;     // n_batches * bins * 8
  unsigned long long* valid;    // n_batches
  unsigned long long* samples;  // n_batches
  const uint32_t* alpha_sorted; // n_alphas (sorted)
  const int32_t* alpha_slot;    // original position of each sorted alpha
  double* amp;             // bins * 3 (re, im, se) output of the amplitude kernel
  int32_t n_alphas;        // 0 = full histogram
  uint32_t bins;
  uint32_t chains, groups, n_batches;
  uint32_t burn_in, record_every;
  uint32_t seed_lo, seed_hi;
  uint32_t group_base;     // first flat group index of this model in a launch
  uint32_t group0;         // global index of group 0 (Philox counter word 0)
  uint32_t hist_smem;      // 1: a CTA counts into shared memory and adds its
                           //    counts to `hist` once at the end of a launch
  int32_t amp_shift;       // amplitude scale 2^{h/2 + amp_shift} (-rank when clamped)
  // output-clamped exact sampler (PB_ELIM_CLAMP; else clamp_tab = nullptr):
  // per p-bit (1 + clamp_mw) words -- an H output's constant bit and its
  // mask over the clamp_nfree free draws
  const uint32_t* clamp_tab;
  int32_t clamp_mw, clamp_nfree, clamp_ok;  // clamp_ok = 0: alpha unreachable
  int32_t pad2;
  // models with PB_U gates (else nullptr): couplings by p, gate phases.
  // Their histogram slots per (batch, bin) are {re (double), im (double),
  // count (u64), compensation of re (double), compensation of im (double),
  // unused...} instead of 8 phase-class counters: the phase sums are
  // compensated (the sum is re + its compensation).
  const Cpl* cpl;
  const UPh* uph;
  const GLink* glk;        // models with Toffoli gates, else nullptr
  const TAcc* tacc;        // models with two-qubit table gates, else nullptr
  const TRec* trec;
};

// Workspace header at offset 0.
struct WsHeader {
  uint32_t status;         // 0 = ok, else a pb_status code set by a kernel
  uint32_t work_next;      // persistent scheduler counter
  uint32_t sweep0;         // absolute index of the next sweep
  uint32_t periods_left;   // learned runs: move periods still to run in a launch
  uint32_t pad[60];
};

// Dynamic shared memory the sweep and exact-sampler kernels may use per CTA
// (227 KB per block on sm_103a, less their static shared memory).
constexpr size_t kSweepSmemMax = 226 * 1024;
// Threads per sweep CTA in a run with general one-qubit gates (the general
// instantiation is compiled for at most this many).
constexpr int kSweepThreadsWgt = 512;
// Plain runs with the three-buffer production: at most 512 threads a CTA,
// so that the kernel gets up to 128 registers a thread (larger shapes take
// the two-buffer form, 608 threads and 96 registers).
constexpr int kSweepThreadsBal = 512;

constexpr uint32_t kTagSweep = 0;
constexpr uint32_t kTagInit = 1;
constexpr uint32_t kTagMH = 2;
constexpr uint32_t kTagElim = 4;  // exact sampler's H outputs (tag 3: training rows)
constexpr uint32_t kTagClamp = 5;  // free draws of the output-clamped exact sampler
constexpr uint32_t kTagCouple = 6;  // Metropolis acceptance of coupled p-bits
constexpr uint32_t kTagTable = 7;   // acceptance next to two-qubit tables (per-chain words)

}  // namespace pb

// Compiled model (host side of pb_model).
struct pb_model {
  int n = 0, d = 0;
  uint32_t beta = 0;
  double J = 0.0;
  uint32_t thr[4] = {0, 0, 0, 0};
  int h = 0, M = 0, rank = 0;
  int col_off[5] = {0, 0, 0, 0, 0};
  std::vector<int32_t> colour;        // [d][n]
  std::vector<pb::Desc> desc;         // colour-ordered
  std::vector<pb::Rec> rec;           // by p = (k-1) n + q
  std::vector<uint32_t> init;         // by p: 0xFFFFFFFF = free output, else a | b << 16
  std::vector<pb_gate> gates;
  // general one-qubit gates
  bool wgt = false;                   // any PB_U gate
  int n_u = 0, n_coupled = 0;
  double log2z = 0.0;
  std::vector<pb::Cpl> cpl;           // by p (wgt only)
  std::vector<pb::UPh> uph;           // one per PB_U gate
  int n_ccx = 0;                      // Toffoli gates
  std::vector<pb::GLink> glk;         // by p (Toffoli models only)
  int n_tab = 0;                      // two-qubit table gates
  std::vector<pb::TAcc> tacc;         // by p (table models only)
  std::vector<pb::TRec> trec;         // one per table gate
};

namespace pb {
// Philox calls the producers of a sweep launch make in one colour step for
// model m, nc colour steps per sweep: 3 per p-bit of the next class in one
// step (12 planes ahead, two buffers: general-gate runs, and plain runs
// whose tables leave no room for more), or 4 per p-bit spread evenly over
// the steps (16 planes ahead, three buffers: other plain runs); the larger
// of the two for plain runs, which take either.
inline int sweep_producers_wanted(const pb_model& m, int nc, bool wgt) {
  int maxcol = 1;
  for (int c = 0; c < 4; ++c) maxcol = std::max(maxcol, m.col_off[c + 1] - m.col_off[c]);
  if (wgt) return 3 * maxcol;
  return std::max(3 * maxcol, (4 * m.col_off[4] + nc - 1) / std::max(1, nc));
}
// Default producer count caps: 352, and 224 for plain runs with the three-
// buffer production (seven producer warps: with four consumer warps and the
// recorder, three warps per scheduler; measured 6 % faster than 352 on the
// mid workload, 2-4 % on the learned and large ones).
constexpr int kProducersMax = 352;
constexpr int kProducersBalanced = 224;
template <class Models>  // a container of pointers to models
inline int sweep_producers_wanted(const Models& ms, int nc, bool wgt) {
  int p = 32;
  for (auto& m : ms) p = std::max(p, sweep_producers_wanted(*m, nc, wgt));
  return p;
}
}  // namespace pb

// Proposal network (host side of pb_mlp): fp32 master weights, Adam state,
// bf16 copies for the tensor cores and the batch buffers of one call.
struct pb_mlp {
  int n = 0, d = 0, H = 0, kin = 0, npad = 0, batch = 0;
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  size_t off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0, n_params = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  __nv_bfloat16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W2t = nullptr, *W3t = nullptr;
  // W1, W2 (in K-chunks of 64) and W3 in the tensor cores' canonical K-major
  // shared-memory layout, loaded by the fused kernel with one bulk copy each
  __nv_bfloat16 *W1p = nullptr, *W2p = nullptr, *W3p = nullptr;
  __nv_bfloat16 *X = nullptr, *Xt = nullptr, *H1 = nullptr, *H1t = nullptr, *H2 = nullptr,
                *H2t = nullptr, *dY = nullptr, *dYt = nullptr, *dZ2 = nullptr, *dZ2t = nullptr,
                *dZ1 = nullptr, *dZ1t = nullptr;
  float *logits = nullptr, *target = nullptr, *loss = nullptr;
  // PB_ETIMEOUT once a bounded wait in one of this network's kernels expired
  // (a word of the workspace, zeroed at creation)
  uint32_t* status = nullptr;
  int step = 0;
};

namespace pb {
// Forward / backward of `rows` rows already staged in mlp->X (and
// mlp->target): logits in mlp->logits [rows x npad], gradients in mlp->g.
cudaError_t mlp_forward_rows(pb_mlp* p, int rows);
cudaError_t mlp_backward_rows(pb_mlp* p, int rows);
cudaError_t mlp_adam_step(pb_mlp* p, float lr);
cudaError_t mlp_prepare();
cudaError_t mlp_forward_fused(pb_mlp* p, int rows);
cudaError_t mlp_fused_logq(pb_mlp* p, const uint32_t* P, uint32_t beta, int chains, int k, float* lq,
                           cudaStream_t st);
cudaError_t mlp_fused_sample(pb_mlp* p, const uint32_t* P, uint32_t* Pn, uint32_t beta, int chains,
                             int k, int j, int jlast, float* lqf, uint32_t k0, uint32_t k1,
                             const uint32_t* move_dev, uint32_t group0, cudaStream_t st);
cudaError_t mlp_fused_logq_dev(pb_mlp* p, const uint32_t* P, uint32_t beta, int chains,
                               const int* k_dev, float* lq, cudaStream_t st);
cudaError_t mlp_fused_sample_dev(pb_mlp* p, const uint32_t* P, uint32_t* Pn, uint32_t beta,
                                 int chains, const int* k_dev, float* lqf, uint32_t k0, uint32_t k1,
                                 const uint32_t* move_dev, uint32_t group0, cudaStream_t st);

// Learned-proposal moves on one model (learned.cu): the run's chain words,
// the network and a device region of mh_region_bytes(d, groups) bytes
// (256-byte aligned) holding the per-chain words, log q terms, the move
// counters and the layer table.
struct MhCtx {
  const pb_model* model = nullptr;
  pb_mlp* mlp = nullptr;
  uint32_t* state = nullptr;  // [group][k-1][q] chain words of the model
  uint32_t chains = 0, groups = 0, group0 = 0;
  uint64_t seed = 0;
  char* ws = nullptr;
  // a second stream and two events: the log q of the current suffix runs
  // beside the proposal draw (mh_ctx_open / mh_ctx_close)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
// Counters at the start of a move region: proposals accepted, moves done.
struct MhCounters {
  unsigned long long accepted;
  uint32_t moves;
  int32_t k;  // suffix start of the current move
};
size_t mh_region_bytes(int d, uint32_t groups);
cudaError_t mh_ctx_open(MhCtx& c);
void mh_ctx_close(MhCtx& c);
// True when the network takes the fused inference kernel (k_in <= 96,
// n <= 32): then a move draws its suffix start on the device.
bool mh_fused(const pb_mlp* mlp);
// Zeroes the region and uploads the layer table (synchronous on st).
cudaError_t mh_region_init(const MhCtx& c, cudaStream_t st);
// Enqueues one move with its suffix start drawn on the device from the seed
// and the move counter (fused networks; capturable, no host synchronisation).
cudaError_t mh_enqueue_move_dev(const MhCtx& c, cudaStream_t st);

// What the learned-proposal code needs to know about one model of a run.
struct RunView {
  cudaStream_t st;
  uint32_t* state;  // [group][k-1][q] chain words
  const pb_model* model;
  uint32_t chains, groups, group0;
  uint64_t seed;
};
int run_view(const pb_run* r, int model, RunView* out);
}  // namespace pb
