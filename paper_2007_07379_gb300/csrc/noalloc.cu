// A plain Gibbs run that allocates no memory: its scratch (run header,
// tables, chain state, counters) lives in one file-scope device array.
//
// This serves callers that cannot allocate device memory at the point of the
// call: for example a plug-in whose host application owns every device
// allocation, or code running while a memory budget is frozen.  Such a
// caller passes only its inputs (a compiled model, a run configuration) and
// its outputs (device buffers for the counts); nothing is allocated here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "pb_internal.h"

namespace pb {
cudaError_t launch_init(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                        const uint32_t* const* d_init_tabs, size_t smem_bytes, WsHeader* hdr,
                        cudaStream_t st);
cudaError_t launch_sweeps(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                          uint32_t n_sweeps, int cons, int prod, int max_col, int nc,
                          size_t smem_bytes, WsHeader* hdr, cudaStream_t st, bool wgt = false,
                          bool ext = false, bool bal = false, bool dec = false);
size_t sweep_smem_bytes(int n, int d, int cons, int max_col, uint32_t hist_bins,
                        bool wgt = false, bool bal = false);
cudaError_t sweep_prepare();
}  // namespace pb

using namespace pb;

namespace {

// The scratch array: 16 MiB, held by every GPU that loads the library.
constexpr size_t kScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_pb_scratch[kScratchBytes];

// Per device, set up once with that device current: the device address of
// g_pb_scratch (the name itself is only a host-side stand-in) and the sweep
// kernels' shared-memory opt-in.  The cache assumes the device's context is
// not reset while the library is loaded (cudaDeviceReset would invalidate
// both; a process that resets a device must not call this entry point
// afterwards).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PB_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return PB_ERANGE;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pb_scratch) != cudaSuccess || p == nullptr) return PB_ECUDA;
    if (sweep_prepare() != cudaSuccess) return PB_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PB_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" PB_API int pb_gibbs_run_noalloc(const pb_model* m, const pb_run_cfg* cfg,
                                           uint32_t n_sweeps, unsigned long long* d_counts,
                                           unsigned long long* d_totals, uintptr_t stream) {
  if (!m || !cfg || !d_counts || !d_totals) return PB_EINVAL;
  if (cfg->sampler != PB_GIBBS || cfg->alphas != nullptr || cfg->n_alphas != 0) return PB_EINVAL;
  if (cfg->chains == 0 || cfg->record_every == 0) return PB_EINVAL;
  if (m->wgt) return PB_EINVAL;  // general one-qubit gates: use pb_run_create
  if (m->n > 16) return PB_ERANGE;
  if (n_sweeps > (1u << 26)) return PB_ERANGE;
  if ((uint64_t)cfg->group0 + (cfg->chains + 31) / 32 > 0xFFFFFFFFull) return PB_ERANGE;
  // The call copies its tables from host memory: it cannot be recorded into
  // a CUDA graph (the copies would point at this call's host buffers).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cap) != cudaSuccess)
    return PB_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return PB_ESTATE;

  const int n = m->n, d = m->d;
  const size_t npb = (size_t)n * d;
  const uint32_t groups = (cfg->chains + 31) / 32;
  const uint32_t bins = 1u << n;

  // Layout of the scratch (one model, one batch).
  size_t off = 0;
  const size_t o_hdr = off; off = align256(off + sizeof(WsHeader));
  const size_t o_rm = off; off = align256(off + sizeof(RunModelDev));
  const size_t o_iptr = off; off = align256(off + sizeof(uint32_t*));
  const size_t o_md = off; off = align256(off + sizeof(ModelDev));
  const size_t o_desc = off; off = align256(off + npb * sizeof(Desc));
  const size_t o_rec = off; off = align256(off + npb * sizeof(Rec));
  const size_t o_init = off; off = align256(off + npb * 4);
  const size_t o_state = off; off = align256(off + (size_t)groups * npb * 4);
  const size_t o_hist = off; off = align256(off + (size_t)bins * 8 * 8);
  const size_t o_cnt = off; off = align256(off + 2 * 8);
  if (off > kScratchBytes) return PB_ERANGE;

  void* base_v = nullptr;
  int rc = scratch_address(&base_v);
  if (rc != PB_OK) return rc;
  char* base = static_cast<char*>(base_v);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // Shape as for a single-model run.
  int maxcol = 1, nc = 2;  // largest class; colour steps per sweep
  for (int c = 0; c < 4; ++c) {
    maxcol = std::max(maxcol, m->col_off[c + 1] - m->col_off[c]);
    if (m->col_off[c + 1] > m->col_off[c]) nc = std::max(nc, c + 1);
  }
  auto up32 = [](int x) { return ((x + 31) / 32) * 32; };
  const int cons = std::max(32, std::min(224, up32(maxcol)));
  int prod = std::max(32, std::min(kProducersMax, up32(sweep_producers_wanted(*m, nc, false))));
  // histogram placement and plane buffers: the rules of a single-model run
  // (shared memory when its u32 counters take at most 128 KiB and the CTA
  // still fits; 16 planes ahead in three buffers when that fits with the
  // same placement)
  auto hist_fits = [&](bool bal) {
    const size_t smem0 = sweep_smem_bytes(n, d, cons, maxcol, 0, false, bal);
    return (size_t)bins * 32 <= (128u << 10) && smem0 + (size_t)bins * 32 <= kSweepSmemMax;
  };
  const bool hist_smem = hist_fits(false);
  const bool bal = hist_fits(true) == hist_smem &&
                   sweep_smem_bytes(n, d, cons, maxcol, hist_smem ? bins : 0, false, true) <= kSweepSmemMax;
  const size_t smem = sweep_smem_bytes(n, d, cons, maxcol, hist_smem ? bins : 0, false, bal);
  if (smem > kSweepSmemMax) return PB_ERANGE;
  if (bal) prod = std::min(prod, kProducersBalanced);  // cons + prod + 32 <= kSweepThreadsBal

  ModelDev md{};
  md.n = n;
  md.d = d;
  md.nw = n_words(n, d);
  md.h = m->h;
  md.beta = m->beta;
  for (int k = 0; k < 4; ++k) md.thr[k] = m->thr[k];
  for (int k = 0; k < 5; ++k) md.col_off[k] = m->col_off[k];
  md.max_col = maxcol;

  RunModelDev r{};
  r.model = reinterpret_cast<const ModelDev*>(base + o_md);
  r.desc = reinterpret_cast<const Desc*>(base + o_desc);
  r.rec = reinterpret_cast<const Rec*>(base + o_rec);
  r.state = reinterpret_cast<uint32_t*>(base + o_state);
  r.hist = reinterpret_cast<unsigned long long*>(base + o_hist);
  r.valid = reinterpret_cast<unsigned long long*>(base + o_cnt);
  r.samples = reinterpret_cast<unsigned long long*>(base + o_cnt + 8);
  r.alpha_sorted = nullptr;
  r.alpha_slot = nullptr;
  r.amp = nullptr;
  r.n_alphas = 0;
  r.bins = bins;
  r.chains = cfg->chains;
  r.groups = groups;
  r.n_batches = 1;
  r.burn_in = cfg->burn_in;
  r.record_every = cfg->record_every;
  r.seed_lo = (uint32_t)cfg->seed;
  r.seed_hi = (uint32_t)(cfg->seed >> 32);
  r.group_base = 0;
  r.group0 = cfg->group0;
  r.hist_smem = hist_smem ? 1u : 0u;
  const uint32_t* init_tab = reinterpret_cast<const uint32_t*>(base + o_init);

  // Every call starts from a cleared header (sweep index 0, status 0) and
  // cleared counters; the rest of the scratch is overwritten below.
  cudaError_t e;
  if ((e = cudaMemsetAsync(base, 0, o_desc, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + o_hist, 0, off - o_hist, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_md, &md, sizeof md, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_rm, &r, sizeof r, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_iptr, &init_tab, sizeof init_tab, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_desc, m->desc.data(), npb * sizeof(Desc), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_rec, m->rec.data(), npb * sizeof(Rec), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_init, m->init.data(), npb * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return PB_ECUDA;
  const RunModelDev* d_rm = reinterpret_cast<const RunModelDev*>(base + o_rm);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base + o_hdr);
  if ((e = launch_init(d_rm, 1, groups, reinterpret_cast<const uint32_t* const*>(base + o_iptr),
                       (size_t)n_words(n, d) * 4, hdr, st)) != cudaSuccess)
    return PB_ECUDA;
  if (n_sweeps > 0 &&
      (e = launch_sweeps(d_rm, 1, groups, n_sweeps, cons, prod, maxcol, nc, smem, hdr, st, false,
                         false, bal, bal && maxcol > cons)) != cudaSuccess)
    return PB_ECUDA;
  if ((e = cudaMemcpyAsync(d_counts, base + o_hist, (size_t)bins * 8 * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_totals, base + o_cnt, 2 * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return PB_ECUDA;
  (void)e;
  return PB_OK;
}
