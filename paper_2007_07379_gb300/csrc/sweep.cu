// Gibbs sweep, record and amplitude kernels (sm_103a).
//
// Layout: 32 chains are bit-sliced into one 32-bit word per p-bit (bit c =
// chain 32 g + c of group g).  A CTA owns one group at a time and keeps the
// group's image (all layers, (d+1) n words, plus a zero and an all-ones word)
// in shared memory for the whole launch; global memory sees the image only at
// the start and the end of a launch and the histogram atomics in between.
//
// One sweep = the model's colour classes in order (Fig. 2 Steps 1-2 for
// every p-bit; two to four classes, three on every workload circuit, from a
// DSATUR colouring of the p-bits' interaction graph at compile time); p-bits
// of one class share no link, so the threads of the CTA redraw a whole class
// in parallel.
// After each recorded sweep the CTA evaluates every chain's validity and path
// phase bit-sliced and adds one count to the bin (end state, phase class)
// (Fig. 2 Step 3).
#include <cuda_runtime.h>

#include <type_traits>

#include "pb_internal.h"
#include "philox.cuh"

namespace pb {

// ---------------------------------------------------------------------------
// Heat-bath draw for the 32 chains of one p-bit.
//
// Each chain compares its uniform u (bit 31-j = bit c of plane j) against a
// threshold t chosen per chain between tA (lanes in `sel`) and tB.  The
// comparison runs most significant plane first; a lane is decided at the
// first plane where its bit differs from the threshold's, and lanes with
// t = 2^31 (`tail0`) are decided by plane 0.  The result is neg ^ [u < t].
struct HbClass {
  uint32_t neg, sel, tail0, tA, tB;
};

// Four planes (one Philox output) of the comparison, planes 4 grp .. 4 grp+3.
__device__ __forceinline__ void compare4(uint32_t& lt, uint32_t& eq, const HbClass& k, uint4 r,
                                         uint32_t grp) {
  const uint32_t R[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (uint32_t w = 0; w < 4u; ++w) {
    const uint32_t j = grp * 4u + w;
    const uint32_t TA = (uint32_t)((int32_t)(k.tA << j) >> 31);
    const uint32_t TB = (uint32_t)((int32_t)(k.tB << j) >> 31);
    const uint32_t T = (k.sel & TA) | (~k.sel & TB);
    lt |= eq & ~R[w] & T;
    eq &= ~(R[w] ^ T);
  }
}

// Barrier `id` over the first `threads` threads of the CTA (whole warps).
__device__ __forceinline__ void bar_sync_first(uint32_t id, uint32_t threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Out-of-line Philox for the rarely taken paths (keeps the hot loop small).
__device__ __noinline__ uint4 philox_cold(uint4 c, uint32_t k0, uint32_t k1) {
  return philox4x32_10(c, k0, k1);
}

// Planes beyond the precomputed ones (rare): Philox calls grp0 .. 7.
__device__ __forceinline__ void compare_tail(uint32_t& lt, uint32_t& eq, const HbClass& k,
                                             uint32_t grp0, uint32_t g, uint32_t sweep, uint32_t p,
                                             uint32_t k0, uint32_t k1) {
#pragma unroll 1
  for (uint32_t grp = grp0; grp < 8u && eq != 0u; ++grp)
    compare4(lt, eq, k, philox_cold(make_uint4(g, sweep, p, grp), k0, k1), grp);
}

// Number of Philox calls computed ahead of a colour class: 12 planes for
// general-gate runs, 16 for plain runs (whose producers spread the work over
// the colour steps and have room for the fourth).
constexpr int kPre = 3;
constexpr int kPrePlain = 4;
// General-gate runs: Philox calls of the Metropolis acceptance draw (tag 6)
// computed ahead (12 planes) for the coupled p-bits among the first
// `consumers` of a class (the rest draw their own, out of line).
constexpr int kPreC = 3;

// Threshold pair of a p-bit with m links: tA for the lanes in `sel` (all
// links agree), tB for the others (see the consumer table set-up).
__device__ __forceinline__ uint32_t thr_a(int m, uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3) {
  return m == 0 ? t0 : (m == 1 ? t1 : (m == 2 ? t2 : t3));
}
__device__ __forceinline__ uint32_t thr_b(int m, uint32_t t0, uint32_t t1) {
  return (m == 0 || m == 2) ? t0 : t1;
}

// Comparison of the precomputed planes for any thresholds (small J), and
// the planes beyond them; out of line: taken rarely.
// np: the precomputed outputs R0 .. R{np-1} (3 or 4; R3 unused when 3).
__device__ __noinline__ uint32_t heat_bath_general(const HbClass k, uint4 R0, uint4 R1, uint4 R2,
                                                   uint4 R3, int np, uint32_t lt, uint32_t eq,
                                                   bool pre, uint32_t g, uint32_t sweep,
                                                   uint32_t pidx, uint32_t k0, uint32_t k1) {
  if (pre) {
    lt = 0u;
    eq = ~0u;
    compare4(lt, eq, k, R0, 0u);
    eq &= ~k.tail0;
    compare4(lt, eq, k, R1, 1u);
    compare4(lt, eq, k, R2, 2u);
    if (np > 3) compare4(lt, eq, k, R3, 3u);
  }
  compare_tail(lt, eq, k, (uint32_t)np, g, sweep, pidx, k0, k1);
  return lt;
}

// Thresholds for which the consumers take the short comparison below:
// thr1 < 2^24 and thr2 < 2^20 (thr3 <= thr2), i.e. on the first 12
// precomputed planes every threshold bit is 0 except the top bit of
// t0 = 2^31 and bits 23..20 of thr1 (planes 8..11).
struct FastThr {
  bool on;
  uint32_t U[4];  // ~0 where thr1 has a one bit on plane 8 + w, else 0
};
__device__ __forceinline__ FastThr fast_thresholds(uint32_t thr1, uint32_t thr2) {
  FastThr f;
  f.on = thr1 < (1u << 24) && thr2 < (1u << 20);
#pragma unroll
  for (int w = 0; w < 4; ++w) f.U[w] = ((thr1 >> (23 - w)) & 1u) ? ~0u : 0u;
  return f;
}

// New value of the 32 chains of one p-bit (Fig. 2 Steps 1-2) from its link
// demands r0..r2 (three-link form: m=0: 0,0,0  m=1: r0,r0,0  m=2: r0,r1,0
// m=3: r0,r1,r2), its masks Mk = [m == k] and its NP precomputed Philox
// outputs R.  Short form (F.on): plane 0 decides the t0 lanes (u < 2^31 iff
// its top bit is 0); on planes 1..7 every other threshold bit is 0, so a
// lane stays equal only while it draws zeros; on planes 8..11 the lanes
// compared with thr1 (L1) meet thr1's bits and the thr2 / thr3 lanes zeros.
// A lane is still equal after plane 11 with probability 2^-12, so about one
// p-bit in 128 (32 lanes) needs more: with NP = 4 the fourth output gives
// planes 12..15 inline (general comparison, no Philox call).  Lanes still
// equal after the precomputed planes, and every lane when the thresholds do
// not have that form, go to heat_bath_general.
template <int NP>
__device__ __forceinline__ uint32_t heat_bath_links(uint32_t r0, uint32_t r1, uint32_t r2, int m,
                                                    uint32_t M0, uint32_t M1, uint32_t M2,
                                                    uint32_t M3, const uint4 (&R)[NP],
                                                    const FastThr& F, uint32_t thr0,
                                                    uint32_t thr1, uint32_t thr2, uint32_t thr3,
                                                    uint32_t g, uint32_t sweep, uint32_t pidx,
                                                    uint32_t k0, uint32_t k1) {
  HbClass k;
  k.neg = (r0 & r1) | (r2 & (r0 | r1));
  k.sel = ~(r0 ^ r1) & (~(r1 ^ r2) | M2);
  k.tail0 = M0 | (M2 & ~k.sel);
  uint32_t lt = 0u, eq = ~0u;
  bool general = !F.on;
  if (F.on) {
    const uint32_t L1 = M1 | (M3 & ~k.sel);  // lanes compared with thr1
    lt = k.tail0 & ~R[0].x;
    eq = ~k.tail0 & ~(R[0].x | R[0].y | R[0].z | R[0].w | R[1].x | R[1].y | R[1].z | R[1].w);
    const uint32_t P[4] = {R[2].x, R[2].y, R[2].z, R[2].w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const uint32_t A = L1 & F.U[w];
      lt |= eq & ~P[w] & A;
      eq &= ~(P[w] ^ A);
    }
    if constexpr (NP > 3) {
      if (eq != 0u) {
        k.tA = thr_a(m, thr0, thr1, thr2, thr3);
        k.tB = thr_b(m, thr0, thr1);
        compare4(lt, eq, k, R[3], 3u);
      }
    }
    general = eq != 0u;
  }
  if (general) {
    k.tA = thr_a(m, thr0, thr1, thr2, thr3);
    k.tB = thr_b(m, thr0, thr1);
    lt = heat_bath_general(k, R[0], R[1], R[2], R[NP > 3 ? 3 : 2], NP, lt, eq, !F.on, g, sweep,
                           pidx, k0, k1);
  }
  return k.neg ^ lt;
}

// Metropolis acceptance of the proposed values `prop` of a coupled p-bit
// whose current values are `old` (general one-qubit gates, Eq. EB): a lane
// that would flip, of category c = e_in + 2 e_out (e_in = old ^ W[win],
// e_out = old ^ W[wout]), keeps the flip when amask bit c is set or its
// tag-6 uniform is below A[c] -- the bit-sliced comparison of
// compare4, planes most significant first, stopped once every lane is
// decided.  Out of line: only coupled p-bits of general-gate models.
// pre: the kPreC tag-6 Philox outputs computed ahead by the producers, or
// nullptr (all drawn here).  Inlined into the consumer's main pass (a call
// there costs more than the body: live registers around it), out of line
// for the rare extra p-bits.
// C: the p-bit's coupling entry; win_w / wout_w: W[C.win], W[C.wout] (the
// caller loads them ahead of the heat-bath draw).
__device__ __forceinline__ uint32_t couple_accept_body(const Cpl& C, uint32_t win_w,
                                                       uint32_t wout_w, uint32_t old, uint32_t prop,
                                                       const uint4* pre, uint32_t g,
                                                       uint32_t sweep, uint32_t p, uint32_t k0,
                                                       uint32_t k1) {
  const uint32_t flip = old ^ prop;
  if (flip == 0u) return old;
  const uint32_t e1 = old ^ win_w, e2 = old ^ wout_w;
  const uint32_t cat[4] = {~e1 & ~e2, e1 & ~e2, ~e1 & e2, e1 & e2};
  uint32_t always = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if ((C.amask >> i) & 1u) always |= cat[i];
  uint32_t eq = flip & ~always, lt = 0u;
#pragma unroll 1
  for (uint32_t grp = 0; grp < 8u && eq != 0u; ++grp) {
    const uint4 r = (pre != nullptr && grp < (uint32_t)kPreC)
                        ? pre[grp]
                        : philox_cold(make_uint4(g, sweep, p | (kTagCouple << 16), grp), k0, k1);
    const uint32_t R[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (uint32_t w = 0; w < 4u; ++w) {
      const uint32_t j = grp * 4u + w;
      uint32_t T = 0u;
#pragma unroll
      for (int i = 0; i < 4; ++i) T |= cat[i] & (uint32_t)((int32_t)(C.A[i] << j) >> 31);
      lt |= eq & ~R[w] & T;
      eq &= ~(R[w] ^ T);
    }
  }
  return old ^ (flip & (always | lt));
}
__device__ __noinline__ uint32_t couple_accept(const uint32_t* W, const Cpl* cpl, uint32_t old,
                                               uint32_t prop, const uint4* pre, uint32_t g,
                                               uint32_t sweep, uint32_t p, uint32_t k0,
                                               uint32_t k1) {
  const Cpl C = *cpl;
  return couple_accept_body(C, W[C.win], W[C.wout], old, prop, pre, g, sweep, p, k0, k1);
}

// Heat-bath draw of a p-bit with general links (next to a Toffoli gate): per
// lane the active links that demand 0 (z) and 1 (o) are counted in two-bit
// bit-sliced counters, v = z - o, and the new value is [v < 0] XOR
// [u < thr[|v|]] -- the plain rule with the link count varying by lane --
// from the same planes (the kPre precomputed Philox outputs of a general-
// gate run, then further ones of the same counter).  Out of line: only
// Toffoli-adjacent p-bits, which only general-gate runs have.
__device__ __noinline__ uint32_t glink_heat_bath(const uint32_t* W, const GLink* gp,
                                                 const uint4* rp, uint32_t thr0, uint32_t thr1,
                                                 uint32_t thr2, uint32_t thr3, uint32_t g,
                                                 uint32_t sweep, uint32_t pidx, uint32_t k0,
                                                 uint32_t k1) {
  const GLink G = *gp;
  uint32_t z0 = 0u, z1 = 0u, o0 = 0u, o1 = 0u;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const uint32_t act = W[G.e[l]];
    const uint32_t r = W[G.a[l]] ^ (W[G.b[l]] & W[G.c[l]]);
    const uint32_t one = act & r, zero = act & ~r;
    o1 |= o0 & one;  // counts stay <= 3: no carry out of bit 1
    o0 ^= one;
    z1 |= z0 & zero;
    z0 ^= zero;
  }
  const uint32_t neg = (o1 & ~z1) | (~(o1 ^ z1) & o0 & ~z0);  // o > z
  const uint32_t v0 = ~(o1 ^ z1) & ~(o0 ^ z0);                 // |v| = 0
  const uint32_t ozero = ~o1 & ~o0, zzero = ~z1 & ~z0;
  const uint32_t ge2 = (ozero & z1) | (zzero & o1);            // |v| >= 2
  const uint32_t v3 = (ozero & z1 & z0) | (zzero & o1 & o0);
  const uint32_t v2 = ge2 & ~v3, v1 = ~v0 & ~ge2;
  uint32_t lt = 0u, eq = ~0u;
#pragma unroll 1
  for (uint32_t grp = 0; grp < 8u && eq != 0u; ++grp) {
    const uint4 r = grp < (uint32_t)kPre ? rp[grp] : philox_cold(make_uint4(g, sweep, pidx, grp), k0, k1);
    const uint32_t R[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (uint32_t w = 0; w < 4u; ++w) {
      const uint32_t j = grp * 4u + w;
      const uint32_t T = (v0 & (uint32_t)((int32_t)(thr0 << j) >> 31)) |
                         (v1 & (uint32_t)((int32_t)(thr1 << j) >> 31)) |
                         (v2 & (uint32_t)((int32_t)(thr2 << j) >> 31)) |
                         (v3 & (uint32_t)((int32_t)(thr3 << j) >> 31));
      lt |= eq & ~R[w] & T;
      eq &= ~(R[w] ^ T);
    }
  }
  return neg ^ lt;
}

// Metropolis acceptance of a p-bit next to two-qubit table gates (Eq. ET2),
// one chain at a time: a lane that would flip keeps the flip when bit idx of
// the always-mask is set or its tag-7 uniform -- word (lane mod 4) of
// Philox(g, sweep, p | 7 << 16, lane / 4) -- is below thr[idx], idx = the
// lane's context bits | its old value << 6 (see TAcc).  Out of line: only
// p-bits next to a table.
__device__ __noinline__ uint32_t table_accept(const uint32_t* W, const TAcc* tp, uint32_t old,
                                              uint32_t prop, uint32_t g, uint32_t sweep,
                                              uint32_t p, uint32_t k0, uint32_t k1) {
  const uint32_t flip = old ^ prop;
  if (flip == 0u) return old;
  uint32_t cw[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) cw[i] = W[tp->w[i]];
  uint32_t acc = 0u;
#pragma unroll 1
  for (uint32_t grp = 0; grp < 8u; ++grp) {
    if (((flip >> (4u * grp)) & 0xFu) == 0u) continue;
    const uint4 r = philox_cold(make_uint4(g, sweep, p | (kTagTable << 16), grp), k0, k1);
    const uint32_t R[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (uint32_t w = 0; w < 4u; ++w) {
      const uint32_t l = 4u * grp + w;
      if (!((flip >> l) & 1u)) continue;
      uint32_t idx = ((old >> l) & 1u) << 6;
#pragma unroll
      for (int i = 0; i < 6; ++i) idx |= ((cw[i] >> l) & 1u) << i;
      if (((tp->amask[idx >> 5] >> (idx & 31u)) & 1u) || R[w] < tp->thr[idx]) acc |= 1u << l;
    }
  }
  return old ^ (flip & acc);
}

__device__ __forceinline__ void add3(uint32_t& f0, uint32_t& f1, uint32_t& f2, uint32_t x0,
                                     uint32_t x1, uint32_t x2) {
  const uint32_t c0 = f0 & x0;
  f0 ^= x0;
  const uint32_t t = f1 ^ x1;
  const uint32_t c1 = (f1 & x1) | (c0 & t);
  f1 = t ^ c0;
  f2 ^= x2 ^ c1;
}

__device__ __forceinline__ int find_model(const RunModelDev* rm, int n_models, uint32_t flat) {
  int lo = 0, hi = n_models - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rm[mid].group_base <= flat) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void set_status(WsHeader* hdr, int code) {
  if (hdr) atomicCAS(&hdr->status, 0u, (uint32_t)code);
}

// Compensated FP64 accumulation of the phase sums: *s += x by an atomic add,
// whose old value gives the exact rounding error of fl(old + x) (Knuth's
// two-sum), and that error (plus `carry`, a compensation brought along) is
// added to the compensation word *c.  The sum is *s + *c; the rounding of the
// big partial sums no longer accumulates over the samples.
__device__ __forceinline__ void atomic_add_comp(double* s, double* c, double x, double carry = 0.0) {
  const double old = atomicAdd(s, x);
  const double nw = old + x;
  const double bp = nw - old;
  const double err = (old - (nw - bp)) + (x - bp) + carry;
  if (err != 0.0) atomicAdd(c, err);
}

// CTA roles: `cons` consumer threads redraw the p-bits of the current colour
// class; `prod` producer threads compute the Philox planes of the next class,
// compared group by group with each p-bit's two thresholds,
// into shared memory; one recorder warp (the last) records the previous sweep.
struct Shape {
  int cons, prod;
};

// Consumer view of one p-bit of a colour class: byte offsets within the
// group image of the three link pairs and of the p-bit's own word, the link
// count m (the table set-up below gives every m the three-link form) and
// the masks Mk = (m == k ? ~0 : 0).
struct ClassEnt {
  uint32_t la[3], lb[3], dst, m;
  uint32_t M0, M1, M2, M3;
};
static_assert(sizeof(ClassEnt) == 48, "ClassEnt must be 48 bytes");

// Shared-memory image of one group: words (image_words) and two snapshots,
// descriptors, record terms, an optional histogram of hist_bins x 8 u32
// counters, the consumers' class table and the plane buffers: three of
// kPrePlain x max_col Philox outputs (plain runs), or two of kPre x max_col
// plus kPreC x cons acceptance outputs (general-gate runs).  The image holds the (d+1) n layer words,
// ZERO, ONES and one scratch word (the store target of consumers without a
// p-bit in a colour class), rounded up to 16 bytes.
__host__ __device__ inline int image_words(int n, int d) { return (n_words(n, d) + 1 + 3) & ~3; }

__host__ __device__ inline size_t group_smem_bytes(int n, int d, int cons, int max_col,
                                                   uint32_t hist_bins, bool wgt = false,
                                                   bool bal = false) {
  return (size_t)3 * image_words(n, d) * 4 + (size_t)n * d * sizeof(Desc) +
         (size_t)n * d * sizeof(Rec) + (((size_t)hist_bins * (wgt ? 10 : 8) + 3) & ~(size_t)3) * 4 +
         (size_t)4 * cons * sizeof(ClassEnt) +
         (wgt ? (size_t)2 * ((size_t)kPre * max_col + (size_t)kPreC * cons)
              : bal ? (size_t)3 * kPrePlain * max_col : (size_t)2 * kPre * max_col) * sizeof(uint4);
}

// 32 x 32 bit transpose across a warp: on entry lane r holds row r; on
// return lane c holds column c (bit r = bit c of row r).  Five butterfly
// steps, each swapping the off-diagonal blocks of the current block size.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
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

// Record of one sweep (Fig. 2 Step 3), computed by the recorder warp from a
// snapshot of the sweep's final state while the stage warps run the next
// sweep, pipelined over the colour stages: read() gathers, for a range of
// p-bits, the violation word and the phase (three bit planes, mod 8);
// reduce() combines the lanes and takes the last layer; bin() adds one count
// per valid chain to (end state alpha, phase class).
struct Recorder {
  uint32_t viol = 0u, f0 = 0u, f1 = 0u, f2 = 0u, lastw = 0u;
  uint32_t phi = 0u;  // general gates: this lane's chain's phase, 2^-32 turn

  __device__ void clear() { viol = f0 = f1 = f2 = phi = 0u; }

  // Two-qubit tables lo..hi-1: each adds its entry's phase for the lane's
  // chain, and a zero entry marks the chain's path invalid.
  __device__ void read_t(const uint32_t* S, const TRec* tr, int lo, int hi, int lane) {
    bool bad = false;
#pragma unroll 1
    for (int i = lo; i < hi; ++i) {
      const TRec& R = tr[i];
      const uint32_t idx = ((S[R.wx0] >> lane) & 1u) | (((S[R.wx1] >> lane) & 1u) << 1) |
                           (((S[R.wy0] >> lane) & 1u) << 2) | (((S[R.wy1] >> lane) & 1u) << 3);
      phi += R.ph[idx];
      bad = bad || ((R.zmask >> idx) & 1u);
    }
    viol |= __ballot_sync(0xffffffffu, bad);
  }

  // Phases of general gates lo..hi-1 for the lane's own chain, eight gates
  // per batch with every load of a batch issued before the first use.
  __device__ void read_u(const uint32_t* S, const UPh* uph, int lo, int hi, int lane) {
    int i = lo;
#pragma unroll 1
    for (; i + 8 <= hi; i += 8) {
      uint4 ph[8];
      uint32_t ww[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        ph[j] = *reinterpret_cast<const uint4*>(uph[i + j].ph);
        ww[j] = *reinterpret_cast<const uint32_t*>(&uph[i + j].wout);  // wout | win << 16
      }
      uint32_t y[8], x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        y[j] = (S[ww[j] & 0xFFFFu] >> lane) & 1u;
        x[j] = (S[ww[j] >> 16] >> lane) & 1u;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t a0 = y[j] ? ph[j].z : ph[j].x, a1 = y[j] ? ph[j].w : ph[j].y;
        phi += x[j] ? a1 : a0;
      }
    }
#pragma unroll 1
    for (; i < hi; ++i) {
      const UPh U = uph[i];
      const uint32_t y = (S[U.wout] >> lane) & 1u, x = (S[U.win] >> lane) & 1u;
      const uint32_t a0 = y ? U.ph[2] : U.ph[0], a1 = y ? U.ph[3] : U.ph[1];
      phi += x ? a1 : a0;
    }
  }

  // ANDV: general-gate runs, where a Toffoli target's term is
  // W[vd] ^ W[va] ^ (W[vb] & W[vc]) (vc = ONES elsewhere).
  template <bool ANDV = false>
  __device__ void read(const uint32_t* S, const Rec* srec, int lo, int hi, int lane) {
#pragma unroll 2
    for (int i = lo + lane; i < hi; i += 32) {
      const Rec R = srec[i];
      if constexpr (ANDV) viol |= S[R.vd] ^ S[R.va] ^ (S[R.vb] & S[R.vc]);
      else viol |= S[R.vd] ^ S[R.va] ^ S[R.vb];
      const uint32_t x = S[R.pa] & S[R.pb];
      add3(f0, f1, f2, (R.w & 1) ? x : 0u, (R.w & 2) ? x : 0u, (R.w & 4) ? x : 0u);
    }
  }

  __device__ void reduce(const uint32_t* S, int n, int d, int lane) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint32_t ov = __shfl_xor_sync(0xffffffffu, viol, off);
      const uint32_t o0 = __shfl_xor_sync(0xffffffffu, f0, off);
      const uint32_t o1 = __shfl_xor_sync(0xffffffffu, f1, off);
      const uint32_t o2 = __shfl_xor_sync(0xffffffffu, f2, off);
      viol |= ov;
      add3(f0, f1, f2, o0, o1, o2);
    }
    lastw = lane < n ? S[d * n + lane] : 0u;
  }

  // The phasor of this lane's record: the general gates' phases plus the
  // phase class (2^29 per pi/4), in FP32 (FP64 issues far slower on this
  // part): the angle rounds to 24 bits (<= pi 2^-24 rad) and sincospif adds
  // about one ulp, so each term is within 3e-7 of e^{i angle}.
  __device__ void phasor(uint32_t phase, double& cs, double& sn) const {
    const uint32_t ang = phi + (phase << 29);
    float snf, csf;
    sincospif((float)(int32_t)ang * 0x1p-31f, &snf, &csf);
    cs = (double)csf;
    sn = (double)snf;
  }

  // Few bins (<= 8): all lanes would hit a handful of FP64 counters, so the
  // warp sums each distinct bin's terms with shuffles and one lane adds them
  // (whole warp, convergent).
  __device__ void bin_few(const RunModelDev& rm, uint32_t batch, int lane, uint32_t* shist,
                          int bin) {
    const uint32_t phase = ((f0 >> lane) & 1u) | (((f1 >> lane) & 1u) << 1) |
                           (((f2 >> lane) & 1u) << 2);
    double cs, sn;
    phasor(phase, cs, sn);
    const bool has = bin >= 0;
    unsigned pending = __ballot_sync(0xffffffffu, has);
    while (pending) {
      const int leader = __ffs((int)pending) - 1;
      const int b = __shfl_sync(0xffffffffu, bin, leader);
      const bool mine = has && bin == b;
      const unsigned m = __ballot_sync(0xffffffffu, mine);
      double r = mine ? cs : 0.0, q = mine ? sn : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, off);
        q += __shfl_xor_sync(0xffffffffu, q, off);
      }
      if (lane == leader) {
        if (shist) {
          double* sd = reinterpret_cast<double*>(shist) + 4u * (uint32_t)b;
          atomic_add_comp(&sd[0], &sd[2], r);
          atomic_add_comp(&sd[1], &sd[3], q);
          atomicAdd(&shist[8u * rm.bins + (uint32_t)b], (uint32_t)__popc(m));
        } else {
          unsigned long long* c = rm.hist + ((size_t)batch * rm.bins + (uint32_t)b) * 8u;
          double* cd = reinterpret_cast<double*>(c);
          atomic_add_comp(&cd[0], &cd[3], r);
          atomic_add_comp(&cd[1], &cd[4], q);
          atomicAdd(c + 2, (unsigned long long)__popc(m));
        }
      }
      pending &= ~m;
    }
  }

  // WGT: models with general gates (rm.cpl set) add e^{i 2 pi phase} in FP64
  // (re, im, count per bin) instead of one count per phase class.
  template <bool WGT>
  __device__ void bin(const RunModelDev& rm, uint32_t g, uint32_t batch, int lane, uint32_t* shist,
                      unsigned long long& n_valid, unsigned long long& n_samples) {
    // lane = chain within the group; alpha bit q = bit `lane` of layer-d word q
    const uint32_t chain = g * 32u + (uint32_t)lane;
    const bool active = chain < rm.chains;
    const bool valid = active && !((viol >> lane) & 1u);
    const uint32_t alpha = warp_transpose32(lastw, lane);
    const uint32_t phase = ((f0 >> lane) & 1u) | (((f1 >> lane) & 1u) << 1) |
                           (((f2 >> lane) & 1u) << 2);
    int bin = -1;
    if (valid) {
      const int na = rm.n_alphas;
      if (na == 0) {
        bin = (int)alpha;
      } else {
        int lo = 0, hi = na - 1;
        while (lo <= hi) {
          const int mid = (lo + hi) >> 1;
          const uint32_t v = rm.alpha_sorted[mid];
          if (v == alpha) { bin = rm.alpha_slot[mid]; break; }
          if (v < alpha) lo = mid + 1; else hi = mid - 1;
        }
      }
    }
    if constexpr (WGT) {
      if (rm.cpl != nullptr && rm.bins <= 8u) {  // whole warp here: see bin_few
        bin_few(rm, batch, lane, shist, bin);
        bin = -1;
      }
    }
    if (bin >= 0) {
      bool done = false;
      if constexpr (WGT) {
        if (rm.cpl != nullptr) {
          double cs, sn;
          phasor(phase, cs, sn);
          if (shist) {
            double* sd = reinterpret_cast<double*>(shist) + 4u * (uint32_t)bin;
            atomic_add_comp(&sd[0], &sd[2], cs);
            atomic_add_comp(&sd[1], &sd[3], sn);
            atomicAdd(&shist[8u * rm.bins + (uint32_t)bin], 1u);
          } else {
            unsigned long long* c = rm.hist + ((size_t)batch * rm.bins + (uint32_t)bin) * 8u;
            double* cd = reinterpret_cast<double*>(c);
            atomic_add_comp(&cd[0], &cd[3], cs);
            atomic_add_comp(&cd[1], &cd[4], sn);
            atomicAdd(c + 2, 1ull);
          }
          done = true;
        }
      }
      if (!done) {
        if (shist) atomicAdd(&shist[(uint32_t)bin * 8u + phase], 1u);
        else atomicAdd(&rm.hist[((size_t)batch * rm.bins + (uint32_t)bin) * 8u + phase], 1ull);
      }
    }
    n_valid += __popc(__ballot_sync(0xffffffffu, valid));
    n_samples += __popc(__ballot_sync(0xffffffffu, active));
  }
};

// p-bits lo + first, lo + first + stride, ... < hi of a colour class from
// their descriptors (a class larger than the consumers; rare).  cpl: the
// coupling table of a general-gate model, else nullptr.  Output j of the
// class's k-th p-bit is cur[k NP + j] (pst = 1) or cur[j pst + k] (pst > 1:
// plane-major buffers).
template <int NP>
__device__ __forceinline__ void redraw_body(uint32_t* W, uint32_t* S, const Desc* sdesc,
                                            const uint4* cur, int pst, int lo, int first,
                                            int hi, int stride, int n, FastThr fast, uint32_t thr0,
                                            uint32_t thr1, uint32_t thr2, uint32_t thr3,
                                            uint32_t g, uint32_t sweep, uint32_t k0, uint32_t k1,
                                            const Cpl* cpl, const GLink* glk, const TAcc* tacc) {
  for (int i = lo + first; i < hi; i += stride) {
    Desc D = sdesc[i];
    if (D.mflag & 0x80) continue;
    const int m = D.mflag & 3;
    if (m == 1) { D.a[1] = D.a[0]; D.b[1] = D.b[0]; }
    const uint4* rp = cur + (i - lo) * (pst == 1 ? NP : 1);
    uint4 R[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) R[j] = rp[j * pst];
    const uint32_t r0 = W[D.a[0]] ^ W[D.b[0]];
    const uint32_t r1 = W[D.a[1]] ^ W[D.b[1]];
    const uint32_t r2 = W[D.a[2]] ^ W[D.b[2]];
    const uint32_t pidx = (uint32_t)(D.dst - n) | (kTagSweep << 16);
    uint32_t v = (glk && (D.mflag & 0x10))
                     ? glink_heat_bath(W, glk + (D.dst - n), rp, thr0, thr1, thr2, thr3, g, sweep,
                                       pidx, k0, k1)
                     : heat_bath_links<NP>(r0, r1, r2, m, m == 0 ? ~0u : 0u, m == 1 ? ~0u : 0u,
                                       m == 2 ? ~0u : 0u, m == 3 ? ~0u : 0u, R, fast, thr0, thr1,
                                       thr2, thr3, g, sweep, pidx, k0, k1);
    if (cpl && (D.mflag & 8)) {
      const uint32_t p = (uint32_t)(D.dst - n);
      v = couple_accept(W, cpl + p, W[D.dst], v, nullptr, g, sweep, p, k0, k1);
    }
    if (tacc && (D.mflag & 0x20)) {
      const uint32_t p = (uint32_t)(D.dst - n);
      v = table_accept(W, tacc + p, W[D.dst], v, g, sweep, p, k0, k1);
    }
    W[D.dst] = v;
    S[D.dst] = v;
  }
}

// Out-of-line entries (the plain one keeps the hot kernel's call site small:
// one argument more there costs register spills).  NP: Philox outputs
// computed ahead per p-bit.
template <int NP>
__device__ __noinline__ void redraw_extra(uint32_t* W, uint32_t* S, const Desc* sdesc,
                                          const uint4* cur, int pst, int lo, int first, int hi,
                                          int stride, int n, FastThr fast, uint32_t thr0,
                                          uint32_t thr1, uint32_t thr2, uint32_t thr3, uint32_t g,
                                          uint32_t sweep, uint32_t k0, uint32_t k1) {
  redraw_body<NP>(W, S, sdesc, cur, pst, lo, first, hi, stride, n, fast, thr0, thr1, thr2, thr3,
                  g, sweep, k0, k1, nullptr, nullptr, nullptr);
}
__device__ __noinline__ void redraw_extra_coupled(uint32_t* W, uint32_t* S, const Desc* sdesc,
                                                  const uint4* cur, int lo, int first, int hi,
                                                  int stride, int n, FastThr fast, uint32_t thr0,
                                                  uint32_t thr1, uint32_t thr2, uint32_t thr3,
                                                  uint32_t g, uint32_t sweep, uint32_t k0,
                                                  uint32_t k1, const Cpl* cpl, const GLink* glk,
                                                  const TAcc* tacc) {
  redraw_body<kPre>(W, S, sdesc, cur, 1, lo, first, hi, stride, n, fast, thr0, thr1, thr2, thr3,
                    g, sweep, k0, k1, cpl, glk, tacc);
}

// Runs `n_sweeps` sweeps (absolute indices sweep0...) of one chain group.
// NC = colour steps per sweep (2..4; the model's classes NC.. are empty).
// WGT: the instantiation for runs with general-gate models (coupled p-bits
// get the Metropolis acceptance, records add FP64 phases); plain models run
// through it unchanged.  EXT (with WGT): some model also has Toffoli links
// or two-qubit tables; without them those paths are compiled out, so the
// coupled-gate consumers and the recorder keep their shorter code.  BAL
// (plain runs whose tables leave room): 16 planes computed ahead per p-bit
// in three buffers, produced evenly over the colour steps; otherwise 12
// planes in two buffers, each class's produced during the step before.
template <int NC, bool WGT, bool EXT, bool BAL, bool DEC = false>
__device__ void run_group(const RunModelDev& rm_g, uint32_t g, uint32_t sweep0, uint32_t n_sweeps,
                          Shape sh, int max_col_all, uint32_t* smem, WsHeader* hdr) {
  // run and model constants held in registers for the whole launch
  const RunModelDev rm = rm_g;
  const ModelDev& md = *rm.model;  // a reference: a struct copy here costs 1.5 % of sweep time
  const int n = md.n, d = md.d, nw = md.nw;
  const int npb = n * d;
  const int tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const bool recorder = warp == nwarps - 1;
  const bool consumer = tid < sh.cons;
  const bool producer = !consumer && !recorder;
  const int ptid = tid - sh.cons;

  const bool wgt_m = WGT && rm.cpl != nullptr;
  const int nug = md.n_ug;
  const int iw = image_words(n, d);
  uint32_t* W = smem;
  // snapshots of the final state of even / odd sweeps at smem + iw (1 + parity)
  Desc* sdesc = reinterpret_cast<Desc*>(smem + 3 * iw);
  Rec* srec = reinterpret_cast<Rec*>(sdesc + npb);
  uint32_t* after_rec = reinterpret_cast<uint32_t*>(srec + npb);
  uint32_t* shist = rm.hist_smem ? after_rec : nullptr;
  // per bin: 8 u32 phase-class counters, or (general gates) 4 doubles (re,
  // im and their compensations) and a u32 count (10 words with padding)
  // (rounded up to 16 bytes: the class table and the plane buffers follow)
  const uint32_t hist_words = (rm.bins * (wgt_m ? 10u : 8u) + 3u) & ~3u;
  ClassEnt* sclass = reinterpret_cast<ClassEnt*>(after_rec + (rm.hist_smem ? hist_words : 0u));
  // plane buffers, each [max_col][KP] sweep-draw outputs, then (general-
  // gate runs) [cons][kPreC] acceptance outputs of the class's first cons
  // p-bits: three with BAL (producers up to two steps ahead), else two (one
  // step ahead)
  uint4* planes = reinterpret_cast<uint4*>(sclass + 4 * sh.cons);
  static_assert(!(WGT && BAL), "balanced production: plain runs only");
  constexpr int KP = BAL ? kPrePlain : kPre;  // Philox outputs computed ahead per p-bit
  // Output j of a class's k-th p-bit: [k KP + j] (48-byte rows, conflict-free
  // for 16-byte loads across a warp), or with BAL [j max_col + k] (plane-
  // major: 64-byte rows would put 16 lanes on the same four banks).
  const int pst = BAL ? max_col_all : 1;
  auto pidx_of = [&](int k, int j) { return BAL ? j * max_col_all + k : k * KP + j; };
  const int acc_off = max_col_all * KP;
  const int pbuf = acc_off + (WGT ? sh.cons * kPreC : 0);

  // ---- load the group image and the tables
  const uint32_t* gstate = rm.state + (size_t)g * npb;
#pragma unroll 1
  for (int i = tid; i < nw; i += T) {
    uint32_t v;
    if (i < n) v = ((md.beta >> i) & 1u) ? ~0u : 0u;        // clamped input layer
    else if (i < (d + 1) * n) v = gstate[i - n];
    else v = (i == zero_idx(n, d)) ? 0u : ~0u;
    W[i] = v;
    smem[iw + i] = v;
    smem[2 * iw + i] = v;
  }
#pragma unroll 1
  for (int i = tid; i < npb; i += T) {
    Desc D = rm.desc[i];
    bool ok = D.dst < nw;
#pragma unroll
    for (int l = 0; l < 3; ++l) ok = ok && D.a[l] < nw && D.b[l] < nw;
    if (!EXT && (D.mflag & 0x30)) ok = false;  // Toffoli / table p-bit: needs EXT
    if (!ok) {  // never write through a bad index: the entry is skipped
      set_status(hdr, PB_EINVAL);
      D.mflag = 0x80;
    }
    sdesc[i] = D;
    Rec R = rm.rec[i];
    if (R.vd >= nw || R.va >= nw || R.vb >= nw || R.pa >= nw || R.pb >= nw || (WGT && R.vc >= nw)) {
      set_status(hdr, PB_EINVAL);
      R.vd = R.va = R.vb = R.pa = R.pb = (uint16_t)zero_idx(n, d);
      R.vc = (uint16_t)ones_idx(n, d);
      R.w = 0;
    }
    srec[i] = R;
  }
  if (shist) {
#pragma unroll 1
    for (uint32_t i = tid; i < hist_words; i += T) shist[i] = 0u;
  }
  if (wgt_m) {
    // coupling and phase tables index the image: a bad table is reported,
    // never followed (the whole group returns before any work)
    int bad = 0;
#pragma unroll 1
    for (int i = tid; i < npb; i += T) bad |= (rm.cpl[i].win >= nw || rm.cpl[i].wout >= nw) ? 1 : 0;
#pragma unroll 1
    for (int i = tid; i < nug; i += T) bad |= (rm.uph[i].win >= nw || rm.uph[i].wout >= nw) ? 1 : 0;
    if (rm.tacc) {
#pragma unroll 1
      for (int i = tid; i < npb; i += T)
        for (int l = 0; l < 6; ++l) bad |= rm.tacc[i].w[l] >= nw ? 1 : 0;
#pragma unroll 1
      for (int i = tid; i < md.n_tr; i += T)
        bad |= (rm.trec[i].wx0 >= nw || rm.trec[i].wx1 >= nw || rm.trec[i].wy0 >= nw ||
                rm.trec[i].wy1 >= nw) ? 1 : 0;
    }
    if (rm.glk)
#pragma unroll 1
      for (int i = tid; i < npb; i += T)
        for (int l = 0; l < 3; ++l)
          bad |= (rm.glk[i].a[l] >= nw || rm.glk[i].b[l] >= nw || rm.glk[i].c[l] >= nw ||
                  rm.glk[i].e[l] >= nw) ? 1 : 0;
    if (__syncthreads_or(bad)) {
      if (tid == 0) set_status(hdr, PB_EINVAL);
      return;
    }
  }
  __syncthreads();

  const uint32_t thr0 = md.thr[0], thr1 = md.thr[1], thr2 = md.thr[2], thr3 = md.thr[3];
  const uint32_t k0 = rm.seed_lo, k1 = rm.seed_hi;
  const uint32_t batch = g % rm.n_batches;
  const uint32_t gglob = g + rm.group0;
  int col_lo[4], col_hi[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) { col_lo[c] = md.col_off[c]; col_hi[c] = md.col_off[c + 1]; }

  // Consumer class table (branch-free form): consumers without a p-bit get a
  // dummy with links to ZERO that stores into the scratch word; a single link
  // is duplicated so that the majority of (r0, r1, r2) is the demanded value
  // for every link count m:  m=0: 0,0,0  m=1: r0,r0,0  m=2: r0,r1,0  m=3: r0,r1,r2.
  if (consumer) {
    const uint16_t scratch = (uint16_t)nw;
    const uint16_t zw = (uint16_t)zero_idx(n, d);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = col_lo[c] + tid;
      bool has = i < col_hi[c];
      Desc D = sdesc[has ? i : 0];
      has = has && !(D.mflag & 0x80);
      if (!has) {
        D.dst = scratch;
        D.mflag = 0;
#pragma unroll
        for (int l = 0; l < 3; ++l) { D.a[l] = zw; D.b[l] = zw; }
      }
      const int m = D.mflag & 3;
      if (m == 1) { D.a[1] = D.a[0]; D.b[1] = D.b[0]; }
      ClassEnt E;
      // plain runs: link words as shared-window addresses (no add per load)
      const uint32_t lbase = WGT ? 0u : (uint32_t)__cvta_generic_to_shared(W);
#pragma unroll
      for (int l = 0; l < 3; ++l) { E.la[l] = lbase + 4u * D.a[l]; E.lb[l] = lbase + 4u * D.b[l]; }
      E.dst = 4u * D.dst;
      E.m = (uint32_t)m;
      if (WGT && (D.mflag & 8)) E.m |= 0x100u;     // coupled: Metropolis acceptance
      if (EXT && (D.mflag & 0x10)) E.m |= 0x200u;  // general links (Toffoli)
      if (EXT && (D.mflag & 0x20)) E.m |= 0x400u;  // table acceptance
      E.M0 = m == 0 ? ~0u : 0u;
      E.M1 = m == 1 ? ~0u : 0u;
      E.M2 = m == 2 ? ~0u : 0u;
      E.M3 = m == 3 ? ~0u : 0u;
      sclass[c * sh.cons + tid] = E;
    }
  }
  // Producers: the Philox outputs of class C at sweep `sw` into `buf`
  // (three-buffer runs: with the group's round keys computed once).
  [[maybe_unused]] PhiloxGroup pg;
  if constexpr (BAL) pg = philox_group(gglob, k0, k1);
  auto produce = [&](auto cc, uint32_t sw, uint4* buf) {
    constexpr int C = decltype(cc)::value;
    const int lo = col_lo[C], K = col_hi[C] - lo;
    const int nsw = K * KP;
    const int nacc = WGT ? (K < sh.cons ? K : sh.cons) * kPreC : 0;
#pragma unroll 1
    for (int u = ptid; u < nsw + nacc; u += sh.prod) {
      if (!WGT || u < nsw) {
        const int i = u / KP, j = u - i * KP;
        const uint32_t p = (uint32_t)(sdesc[lo + i].dst - n) | (kTagSweep << 16);
        buf[pidx_of(i, j)] = philox4x32_10(make_uint4(gglob, sw, p, (uint32_t)j), k0, k1);
      } else {  // acceptance draws: coupled p-bits only
        const int a = u - nsw, i = a / kPreC, j = a - i * kPreC;
        const Desc& D = sdesc[lo + i];
        if (D.mflag & 8)
          buf[acc_off + a] = philox4x32_10(
              make_uint4(gglob, sw, (uint32_t)(D.dst - n) | (kTagCouple << 16), (uint32_t)j), k0, k1);
      }
    }
  };
  if (producer && n_sweeps > 0u) produce(std::integral_constant<int, 0>{}, sweep0, planes);
  __syncthreads();

  // BAL: production spread evenly over the colour steps.  The units
  // of a sweep are its U Philox outputs (KP a p-bit) in step order; step t
  // needs its own before it starts, and the three buffers hold steps t (being
  // read), t + 1 and t + 2.  During step t the producers take the next units
  // of the stream up to max(D(t + 2), pp + B) and at most D(t + 3), B = U /
  // NC a step (D(t): units of the steps before t; pp: units produced so
  // far, kept relative to the current sweep's first unit).  With classes of
  // 116, 91 and 33 p-bits this is 320 outputs a step instead of 364, 132 and
  // 464 for the next step alone.
  [[maybe_unused]] const uint32_t U = (uint32_t)(KP * col_hi[NC - 1]);  // every p-bit is in one class
  [[maybe_unused]] const uint32_t B = (U + NC - 1) / NC;
  [[maybe_unused]] uint32_t pp = (uint32_t)(KP * col_hi[0]);  // units of step 0, produced above

  const FastThr fast = fast_thresholds(thr1, thr2);
  Recorder rec;
  unsigned long long n_valid = 0ull, n_samples = 0ull;  // recorder warp only
  auto recorded = [&](uint32_t t) {
    return t >= rm.burn_in && (rm.record_every == 1u || (t - rm.burn_in) % rm.record_every == 0);
  };

  // One colour class C of sweep sweep0 + s: consumers redraw it from plane
  // buffer C & 1, producers fill the other buffer for the next class, the
  // recorder works on the previous sweep's snapshot; then one barrier.
  [[maybe_unused]] ClassEnt En{};  // DEC consumers: the coming step's table entry
  if (DEC && consumer) En = sclass[tid];
  auto step = [&](auto cc, uint32_t s) {
    constexpr int C = decltype(cc)::value;
    const uint32_t sweep = sweep0 + s;
    uint32_t* S = smem + iw * (1 + (s & 1u));
    // plane buffer of global step s NC + C
    const uint32_t gstep = s * (uint32_t)NC + (uint32_t)C;
    // (with three colour steps a sweep, step C's buffer is C)
    const uint32_t cslot = BAL ? (NC == 3 ? (uint32_t)C : gstep % 3u) : (gstep & 1u);
    const uint4* cur = planes + cslot * pbuf;
    if (consumer) {
      const int lo = col_lo[C], hi = col_hi[C], K = hi - lo;
      // the first p-bit of every consumer from its table entry; warps with no
      // p-bit in this class skip it (their entries are dummies)
      if (warp * 32 < K) {
        const ClassEnt E = DEC ? En : sclass[C * sh.cons + tid];
        const uint4* rp = cur + pidx_of(tid < K ? tid : 0, 0);  // dummies: any planes
        uint4 R[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) R[j] = rp[j * pst];
        const char* Wb = reinterpret_cast<const char*>(W);
        auto word = [&](uint32_t off) { return *reinterpret_cast<const uint32_t*>(Wb + off); };
        auto link = [&](uint32_t a) {  // plain runs: a is a shared-window address
          if constexpr (WGT) return word(a);
          uint32_t x;
          asm volatile("ld.shared.u32 %0, [%1];" : "=r"(x) : "r"(a));
          return x;
        };
        const uint32_t r0 = link(E.la[0]) ^ link(E.lb[0]);
        const uint32_t r1 = link(E.la[1]) ^ link(E.lb[1]);
        const uint32_t r2 = link(E.la[2]) ^ link(E.lb[2]);
        const uint32_t pidx = (E.dst / 4u - (uint32_t)n) | (kTagSweep << 16);
        // coupled p-bit: its coupling entry and neighbour words, loaded
        // ahead so that their latency overlaps the heat-bath draw
        [[maybe_unused]] Cpl Cp{};
        [[maybe_unused]] uint32_t old_w = 0u, win_w = 0u, wout_w = 0u;
        if constexpr (WGT) {
          if (E.m & 0x100u) {
            Cp = rm.cpl[E.dst / 4u - (uint32_t)n];
            old_w = word(E.dst);
            win_w = W[Cp.win];
            wout_w = W[Cp.wout];
          }
        }
        uint32_t v;
        if (EXT && (E.m & 0x200u))
          v = glink_heat_bath(W, rm.glk + (E.dst / 4u - (uint32_t)n), rp, thr0, thr1, thr2, thr3,
                              gglob, sweep, pidx, k0, k1);
        else
          v = heat_bath_links<KP>(r0, r1, r2, (int)(WGT ? (E.m & 3u) : E.m), E.M0, E.M1, E.M2, E.M3, R,
                              fast, thr0, thr1, thr2, thr3, gglob, sweep, pidx, k0, k1);
        if constexpr (WGT) {
          if (E.m & 0x100u) {
            const uint32_t p = E.dst / 4u - (uint32_t)n;
            v = couple_accept_body(Cp, win_w, wout_w, old_w, v, cur + acc_off + tid * kPreC,
                                   gglob, sweep, p, k0, k1);
          }
          if (EXT && (E.m & 0x400u)) {  // a second acceptance factor: the tables' energy
            const uint32_t p = E.dst / 4u - (uint32_t)n;
            v = table_accept(W, rm.tacc + p, word(E.dst), v, gglob, sweep, p, k0, k1);
          }
        }
        *reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(W) + E.dst) = v;
        *reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(S) + E.dst) = v;
      }
      // further p-bits (a class larger than the consumers) from the descriptors
      if (K > sh.cons) {
        if constexpr (WGT)
          redraw_extra_coupled(W, S, sdesc, cur, lo, tid + sh.cons, hi, sh.cons, n, fast, thr0,
                               thr1, thr2, thr3, gglob, sweep, k0, k1, rm.cpl,
                               EXT ? rm.glk : nullptr, EXT ? rm.tacc : nullptr);
        else
          redraw_extra<KP>(W, S, sdesc, cur, pst, lo, tid + sh.cons, hi, sh.cons, n, fast, thr0, thr1, thr2,
                       thr3, gglob, sweep, k0, k1);
      }
      // DEC: the next step's table entry, loaded before the barrier so that
      // the step after it starts with the link loads
      if constexpr (DEC) En = sclass[((C + 1) % NC) * sh.cons + tid];
    } else if (producer) {
      if constexpr (!BAL) {
        // the next step: class C + 1 of this sweep, or class 0 of the next one
        const uint32_t nxt = gstep + 1u;
        if constexpr (C + 1 < NC) {
          produce(std::integral_constant<int, C + 1>{}, sweep, planes + (nxt & 1u) * pbuf);
        } else {
          if (s + 1u < n_sweeps)
            produce(std::integral_constant<int, 0>{}, sweep + 1u, planes + (nxt & 1u) * pbuf);
        }
      } else {
        // steps gstep + 1 and gstep + 2: classes C1, C2 of sweeps s + c1, s + c2
        constexpr int C1 = (C + 1) % NC, C2 = (C + 2) % NC, C3 = (C + 3) % NC;
        constexpr uint32_t c1 = (C + 1) / NC, c2 = (C + 2) / NC, c3 = (C + 3) / NC;
        const uint32_t d1 = c1 * U + (uint32_t)(KP * col_lo[C1]);  // D(t + k) - D(sweep s)
        const uint32_t d2 = c2 * U + (uint32_t)(KP * col_lo[C2]);
        uint32_t lim = c3 * U + (uint32_t)(KP * col_lo[C3]);
        if (s + 1u >= n_sweeps && lim > U) lim = U;  // no unit past the launch
        uint32_t tgt = pp + B > d2 ? pp + B : d2;
        if (tgt > lim) tgt = lim;
#pragma unroll 1
        for (uint32_t u = pp + (uint32_t)ptid; u < tgt; u += (uint32_t)sh.prod) {
          const bool second = u >= d2;
          const uint32_t r = u - (second ? d2 : d1);  // unit within its step
          const uint32_t i = r / (uint32_t)KP, j = r - i * (uint32_t)KP;
          const int lo = second ? col_lo[C2] : col_lo[C1];
          const uint32_t sw = sweep + (second ? c2 : c1);
          const uint32_t slot = NC == 3 ? (second ? (uint32_t)((C + 2) % 3) : (uint32_t)((C + 1) % 3))
                                        : (gstep + (second ? 2u : 1u)) % 3u;
          const uint32_t p = (uint32_t)(sdesc[lo + (int)i].dst - n) | (kTagSweep << 16);
          planes[slot * (uint32_t)pbuf + j * (uint32_t)max_col_all + i] =
              philox4x32_10_group(pg, sw, p, j);
        }
        pp = tgt;
      }
    } else {
      // records run one sweep behind: the record of sweep s-1 reads its
      // snapshot in NC-1 parts (steps 0..NC-2 of sweep s), then reduces and
      // bins (step NC-1).  General-gate runs, and plain runs with DEC: the
      // recorder takes no part in the colour steps' barriers, only in the
      // sweep's last one (it reads the previous sweep's snapshot, which no
      // consumer writes during this sweep, at its own pace; measured 3-4 %
      // faster on general_mid and on the large workload, whose classes take
      // two consumer passes, and slower on the plain mid circuit, whose
      // steps it then crowds).
      if (s > 0u && recorded(sweep - 1u)) {
        const uint32_t* Sp = smem + iw * (1 + ((s + 1u) & 1u));
        if constexpr (C == 0) rec.clear();
        if constexpr (C + 1 < NC) {
          // part C of the records: one share in step 0 (the largest class,
          // the most consumer warps), two in each later step
          constexpr int D = 2 * (NC - 1) - 1, B0 = C == 0 ? 0 : 2 * C - 1, B1 = 2 * C + 1;
          rec.read<EXT>(Sp, srec, B0 * npb / D, B1 * npb / D, lane);
          if (wgt_m) rec.read_u(Sp, rm.uph, B0 * nug / D, B1 * nug / D, lane);
          if (EXT && rm.trec) rec.read_t(Sp, rm.trec, B0 * md.n_tr / D, B1 * md.n_tr / D, lane);
        } else {
          rec.reduce(Sp, n, d, lane);
          rec.bin<WGT>(rm_g, g, batch, lane, shist, n_valid, n_samples);
        }
      }
    }
    if constexpr ((WGT || DEC) && C + 1 < NC) {
      if (!recorder) bar_sync_first(1u, (uint32_t)(sh.cons + sh.prod));
    } else {
      __syncthreads();  // (the sweep's end: snapshots change parity)
    }
  };
#pragma unroll 1
  for (uint32_t s = 0; s < n_sweeps; ++s) {
    step(std::integral_constant<int, 0>{}, s);
    step(std::integral_constant<int, 1>{}, s);
    if constexpr (NC > 2) step(std::integral_constant<int, 2>{}, s);
    if constexpr (NC > 3) step(std::integral_constant<int, 3>{}, s);
    if constexpr (BAL) pp -= U;  // production pointer relative to the next sweep
  }
  // the record still in flight: the last sweep's
  if (recorder) {
    if (n_sweeps > 0 && recorded(sweep0 + n_sweeps - 1)) {
      const uint32_t* Sl = smem + iw * (1 + ((n_sweeps - 1u) & 1u));
      rec.clear();
      rec.read<EXT>(Sl, srec, 0, npb, lane);
      if (wgt_m) rec.read_u(Sl, rm.uph, 0, nug, lane);
      if (EXT && rm.trec) rec.read_t(Sl, rm.trec, 0, md.n_tr, lane);
      rec.reduce(Sl, n, d, lane);
      rec.bin<WGT>(rm_g, g, batch, lane, shist, n_valid, n_samples);
    }
  }
  __syncthreads();

  // ---- write the group image back, add the counts of this launch
  uint32_t* out = rm.state + (size_t)g * npb;
#pragma unroll 1
  for (int i = tid; i < npb; i += T) out[i] = W[n + i];
  if (shist && wgt_m) {  // (re, im, comp re, comp im) doubles per bin, then u32 counts
    const double* sd = reinterpret_cast<const double*>(shist);
#pragma unroll 1
    for (uint32_t i = tid; i < rm.bins; i += T) {
      const uint32_t cn = shist[8u * rm.bins + i];
      if (!cn) continue;
      unsigned long long* c = rm.hist + ((size_t)batch * rm.bins + i) * 8u;
      double* cd = reinterpret_cast<double*>(c);
      atomic_add_comp(&cd[0], &cd[3], sd[4u * i], sd[4u * i + 2u]);
      atomic_add_comp(&cd[1], &cd[4], sd[4u * i + 1u], sd[4u * i + 3u]);
      atomicAdd(c + 2, (unsigned long long)cn);
    }
  } else if (shist) {
    unsigned long long* gh = rm.hist + (size_t)batch * rm.bins * 8u;
#pragma unroll 1
    for (uint32_t i = tid; i < rm.bins * 8u; i += T)
      if (shist[i]) atomicAdd(&gh[i], (unsigned long long)shist[i]);
  }
  if (recorder && lane == 0) {
    if (n_valid) atomicAdd(&rm_g.valid[batch], n_valid);
    if (n_samples) atomicAdd(&rm_g.samples[batch], n_samples);
  }
  __syncthreads();
}

// One CTA per chain group of every model of the run (flat group index).
constexpr int kMaxThreads = 608;  // 224 consumers + 352 producers + 1 recorder warp
// General-gate runs: at most 512 threads, so that the longer consumer and
// recorder paths get 128 registers.
constexpr int kMaxThreadsWgt = 512;

template <int NC, bool WGT, bool EXT, bool BAL, bool DEC = false>
__global__ void __launch_bounds__(WGT ? kMaxThreadsWgt : (BAL ? kSweepThreadsBal : kMaxThreads)) sweep_kernel(const RunModelDev* __restrict__ rm,
                                                     int n_models, uint32_t total_groups,
                                                     uint32_t n_sweeps, Shape sh, int max_col,
                                                     WsHeader* hdr) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t sweep0 = hdr->sweep0;
  const uint32_t flat = blockIdx.x;
  if (flat >= total_groups) return;
  const int mi = find_model(rm, n_models, flat);
  const RunModelDev& r = rm[mi];
  const uint32_t g = flat - r.group_base;
  if (g >= r.groups) return;
  run_group<NC, WGT, EXT, BAL, DEC>(r, g, sweep0, n_sweeps, sh, max_col, smem, hdr);
}

// Persistent form: a fixed grid pops (model, group) items from a
// cost-ordered work list with one atomic counter.  No CTA waits on another.
template <int NC, bool BAL>
__global__ void __launch_bounds__(BAL ? kSweepThreadsBal : kMaxThreads) sweep_persistent_kernel(
    const RunModelDev* __restrict__ rm, int n_models, const uint32_t* __restrict__ work,
    uint32_t n_work, uint32_t n_sweeps, Shape sh, int max_col, WsHeader* hdr) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t sweep0 = hdr->sweep0;
  __shared__ uint32_t item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(&hdr->work_next, 1u);
    __syncthreads();
    const uint32_t it = item;
    __syncthreads();
    if (it >= n_work) break;
    const uint32_t flat = work[it];
    const int mi = find_model(rm, n_models, flat);
    const RunModelDev& r = rm[mi];
    const uint32_t g = flat - r.group_base;
    if (g < r.groups) run_group<NC, false, false, BAL>(r, g, sweep0, n_sweeps, sh, max_col, smem, hdr);
  }
}

// ---------------------------------------------------------------------------
// Initial chains: a valid path with random H outputs (tag-1 stream), every
// other bit its deterministic value, layer by layer.
__global__ void init_kernel(const RunModelDev* __restrict__ rm, int n_models,
                            uint32_t total_groups, const uint32_t* const* __restrict__ init_tabs,
                            WsHeader* hdr) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t flat = blockIdx.x;
  if (flat >= total_groups) return;
  const int mi = find_model(rm, n_models, flat);
  const RunModelDev& r = rm[mi];
  const uint32_t g = flat - r.group_base;
  if (g >= r.groups) return;
  const ModelDev* mp = r.model;
  const int n = mp->n, d = mp->d, nw = mp->nw;
  const uint32_t* itab = init_tabs[mi];  // per p-bit: 0xFFFFFFFF = H, else a | b << 16
  uint32_t* W = smem;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) {
    uint32_t v = 0u;
    if (i < n) v = ((mp->beta >> i) & 1u) ? ~0u : 0u;
    else if (i == ones_idx(n, d)) v = ~0u;
    W[i] = v;
  }
  __syncthreads();
  for (int k = 1; k <= d; ++k) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int p = (k - 1) * n + q;
      const uint32_t e = itab[p];
      uint32_t v;
      if (e == 0xFFFFFFFFu) {
        v = philox4x32_10(make_uint4(g + r.group0, 0u, (uint32_t)p | (kTagInit << 16), 0u),
                          r.seed_lo, r.seed_hi).x;
      } else if (e == 0xFFFFFFFEu) {  // Toffoli target: its own general link
        const GLink* G = r.glk ? r.glk + p : nullptr;
        if (!G || G->a[0] >= nw || G->b[0] >= nw || G->c[0] >= nw) { set_status(hdr, PB_EINVAL); v = 0u; }
        else v = W[G->a[0]] ^ (W[G->b[0]] & W[G->c[0]]);
      } else {
        const uint32_t a = e & 0xFFFFu, b = e >> 16;
        if ((int)a >= nw || (int)b >= nw) { set_status(hdr, PB_EINVAL); v = 0u; }
        else v = W[a] ^ W[b];
      }
      W[k * n + q] = v;
    }
    __syncthreads();
  }
  uint32_t* out = r.state + (size_t)g * n * d;
  for (int i = threadIdx.x; i < n * d; i += blockDim.x) out[i] = W[n + i];
}

// ---------------------------------------------------------------------------
// Exact path sampler on the eliminated network (R2; Appendix: without the
// link constraints the non-H bits are functions of the previous layer and
// each H output is a fair coin).  Each recorded sample draws a fresh path
// from the clamped input, layer by layer -- an H output (k, q) of chain c at
// sample t is bit (c mod 32) of word 0 of Philox(c / 32, t, p | 4 << 16, 0),
// every other bit the XOR of two words given by the init table -- and
// records it (Fig. 2 Step 3; every path is valid).  One CTA per chain group;
// warp w of the NW takes the launch's samples w, w + NW, ... in its own
// shared-memory image; lane q writes word q of a layer.  The samples are
// independent, so NW only sets how much latency a CTA can hide: the run
// takes 32 warps when its groups do not fill the SMs, 16 or 8 when they do.
// Output-clamped models (clamp_tab set): the sample's free draws z_b are
// bit c % 32 of word b % 4 of Philox(c / 32, t, (b / 4) | 5 << 16, 0), and an
// H output is its table constant XOR the z_b of its mask (GF(2) elimination
// on the host), so every path ends at the clamped output.
// WGT: the instantiation for runs with general-gate models (coupled coins,
// phasor records); plain runs take the plain one.
template <bool WGT, int NW>
__global__ void __launch_bounds__(NW * 32) elim_kernel(
    const RunModelDev* __restrict__ rm, int n_models, uint32_t total_groups,
    const uint32_t* const* __restrict__ init_tabs, uint32_t n_sweeps, int wstride, WsHeader* hdr) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t sweep0 = hdr->sweep0;
  const uint32_t flat = blockIdx.x;
  if (flat >= total_groups) return;
  const int mi = find_model(rm, n_models, flat);
  const RunModelDev& r = rm[mi];
  const uint32_t g = flat - r.group_base;
  if (g >= r.groups) return;
  const ModelDev md = *r.model;
  const int n = md.n, d = md.d, nw = md.nw, npb = n * d;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* W = smem + warp * wstride;       // path image
  uint32_t* Z = W + image_words(n, d);       // free draws of a clamped sample
  const uint32_t* ctab = r.clamp_tab;
  const int cmw = r.clamp_mw, nfree = r.clamp_nfree;
  if (ctab && (!r.clamp_ok || image_words(n, d) + nfree > wstride)) {
    if (!r.clamp_ok) return;  // unreachable output: nothing to draw
    if (threadIdx.x == 0) set_status(hdr, PB_EINVAL);
    return;
  }
  const uint32_t* itab = init_tabs[mi];  // per p-bit: 0xFFFFFFFF = H, else a | b << 16
  // record terms index the image: a bad table is reported, never followed
  int bad = 0;
  for (int i = threadIdx.x; i < npb; i += blockDim.x) {
    const Rec R = r.rec[i];
    bad |= (R.vd >= nw || R.va >= nw || R.vb >= nw || R.pa >= nw || R.pb >= nw ||
            (WGT && R.vc >= nw)) ? 1 : 0;
  }
  if (WGT && r.cpl)
    for (int i = threadIdx.x; i < md.n_ug; i += blockDim.x)
      bad |= (r.uph[i].win >= nw || r.uph[i].wout >= nw) ? 1 : 0;
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) set_status(hdr, PB_EINVAL);
    return;
  }
  for (int i = lane; i < nw; i += 32) {
    uint32_t v = 0u;
    if (i < n) v = ((md.beta >> i) & 1u) ? ~0u : 0u;  // clamped input layer
    else if (i == ones_idx(n, d)) v = ~0u;
    W[i] = v;
  }
  __syncwarp();
  auto recorded = [&](uint32_t t) {
    return t >= r.burn_in && (r.record_every == 1u || (t - r.burn_in) % r.record_every == 0);
  };
  const uint32_t gglob = g + r.group0, batch = g % r.n_batches;
  Recorder rec;
  unsigned long long n_valid = 0ull, n_samples = 0ull;
#pragma unroll 1
  for (uint32_t i = (uint32_t)warp; i < n_sweeps; i += (uint32_t)NW) {
    const uint32_t t = sweep0 + i;
    if (!recorded(t)) continue;
    if (ctab) {
#pragma unroll 1
      for (int b0 = 4 * lane; b0 < nfree; b0 += 128) {
        const uint4 z = philox4x32_10(make_uint4(gglob, t, (uint32_t)(b0 >> 2) | (kTagClamp << 16), 0u),
                                      r.seed_lo, r.seed_hi);
        Z[b0] = z.x;
        if (b0 + 1 < nfree) Z[b0 + 1] = z.y;
        if (b0 + 2 < nfree) Z[b0 + 2] = z.z;
        if (b0 + 3 < nfree) Z[b0 + 3] = z.w;
      }
      __syncwarp();
    }
#pragma unroll 1
    for (int k = 1; k <= d; ++k) {
      if (lane < n) {
        const int p = (k - 1) * n + lane;
        const uint32_t e = itab[p];
        uint32_t v;
        if (e == 0xFFFFFFFFu && ctab) {
          const uint32_t* ce = ctab + (size_t)p * (1 + cmw);
          v = ce[0] ? ~0u : 0u;
          for (int w = 0; w < cmw; ++w) {
            uint32_t msk = ce[1 + w];
            while (msk) {
              const int b = 32 * w + __ffs((int)msk) - 1;
              if (b < nfree) v ^= Z[b];
              msk &= msk - 1u;
            }
          }
        } else if (WGT && e == 0xFFFFFFFFu && r.cpl && (r.cpl[p].flags & 2u)) {
          // coupled general gate: s_in ^ [u < B], u from the tag-4 planes of
          // this p-bit, most significant first, compared bit-sliced
          const uint32_t B = r.cpl[p].B;
          uint32_t lt = 0u, eq = ~0u;
#pragma unroll 1
          for (uint32_t grp = 0; grp < 8u && eq != 0u; ++grp) {
            const uint4 rr = philox4x32_10(make_uint4(gglob, t, (uint32_t)p | (kTagElim << 16), grp),
                                           r.seed_lo, r.seed_hi);
            const uint32_t R[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
            for (uint32_t w = 0; w < 4u; ++w) {
              const uint32_t Tb = (uint32_t)((int32_t)(B << (grp * 4u + w)) >> 31);
              lt |= eq & ~R[w] & Tb;
              eq &= ~(R[w] ^ Tb);
            }
          }
          v = W[p] ^ lt;  // W[(k-1) n + q]: the gate's input bit
        } else if (e == 0xFFFFFFFFu) {
          v = philox4x32_10(make_uint4(gglob, t, (uint32_t)p | (kTagElim << 16), 0u), r.seed_lo,
                            r.seed_hi).x;
        } else if (WGT && e == 0xFFFFFFFEu) {  // Toffoli target: its own general link
          const GLink* G = r.glk ? r.glk + p : nullptr;
          if (!G || G->a[0] >= nw || G->b[0] >= nw || G->c[0] >= nw) { set_status(hdr, PB_EINVAL); v = 0u; }
          else v = W[G->a[0]] ^ (W[G->b[0]] & W[G->c[0]]);
        } else {
          const uint32_t a = e & 0xFFFFu, b = e >> 16;
          if ((int)a >= nw || (int)b >= nw) { set_status(hdr, PB_EINVAL); v = 0u; }
          else v = W[a] ^ W[b];
        }
        W[k * n + lane] = v;
      }
      __syncwarp();
    }
    rec.clear();
    rec.read<WGT>(W, r.rec, 0, npb, lane);
    if (WGT && r.cpl) rec.read_u(W, r.uph, 0, md.n_ug, lane);
    rec.reduce(W, n, d, lane);
    rec.bin<WGT>(r, g, batch, lane, nullptr, n_valid, n_samples);
    __syncwarp();
  }
  if (lane == 0) {
    if (n_valid) atomicAdd(&r.valid[batch], n_valid);
    if (n_samples) atomicAdd(&r.samples[batch], n_samples);
  }
  // the group's state: the path of the launch's last recorded sample
  int last = -1;
  for (int i = (int)n_sweeps - 1; i >= 0; --i)
    if (recorded(sweep0 + (uint32_t)i)) { last = i; break; }
  if (last >= 0 && warp == last % NW) {
    uint32_t* out = r.state + (size_t)g * npb;
    for (int i = lane; i < npb; i += 32) out[i] = W[n + i];
  }
}

// ---------------------------------------------------------------------------
// Amplitudes (Eq. U23 with uniform valid paths, exact integer phase classes):
//   Z = sum_b cnt_b w^b = (c0 - c4) + (c1 - c3 - c5 + c7)/sqrt2
//                      + i[(c2 - c6) + (c1 + c3 - c5 - c7)/sqrt2]
//   psi = 2^{h/2} Z / valid.
// The standard error comes from batch means over chain groups (Eq. U26),
// with compensated (Kahan) FP64 accumulation of the batch sums.
struct Kahan {
  double s = 0.0, c = 0.0;
  __device__ void add(double x) {
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

__device__ inline void phase_sum(const unsigned long long* c, double& re, double& im) {
  const long long c0 = (long long)c[0], c1 = (long long)c[1], c2 = (long long)c[2],
                  c3 = (long long)c[3], c4 = (long long)c[4], c5 = (long long)c[5],
                  c6 = (long long)c[6], c7 = (long long)c[7];
  const double inv_sqrt2 = 0.70710678118654752440;
  re = (double)(c0 - c4) + (double)(c1 - c3 - c5 + c7) * inv_sqrt2;
  im = (double)(c2 - c6) + (double)(c1 + c3 - c5 - c7) * inv_sqrt2;
}

// Phase sum of one batch's bin: the 8 exact classes, or (general gates) the
// FP64 (re, im) slots.
__device__ inline void batch_sum(const RunModelDev& rm, bool wgt, uint32_t b, uint32_t bin,
                                 double& re, double& im) {
  const unsigned long long* c = rm.hist + ((size_t)b * rm.bins + bin) * 8u;
  if (wgt) {  // the compensated sums: sum + compensation
    re = __longlong_as_double((long long)c[0]) + __longlong_as_double((long long)c[3]);
    im = __longlong_as_double((long long)c[1]) + __longlong_as_double((long long)c[4]);
  } else {
    phase_sum(c, re, im);
  }
}

// One warp per bin, the lanes over the batches (lane b takes batches b,
// b + 32, ...): the counts (or phase sums) and valid totals of every batch
// are summed by warp reductions, then each lane adds its batches' terms of
// the batch-means variance (one FP64 division a batch, the terms summed by
// a compensated add per lane and a warp reduction).
__global__ void amplitude_kernel(const RunModelDev* __restrict__ rm_all, int model) {
  const RunModelDev& rm = rm_all[model];
  const uint32_t bin = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (bin >= rm.bins) return;  // whole warp
  const int h = rm.model->h;
  const bool wgt = rm.model->wgt != 0;
  // 2^{h/2} (Clifford+T: every valid path has |U_C| = 2^{-h/2}); general
  // gates: 2^{log2z}, the sum of |U_C| over all paths (FP64 issues slowly on
  // this part: one lane evaluates the warp-uniform factors)
  double scale_h = 0.0;
  if (lane == 0)
    scale_h = wgt ? exp2(rm.model->log2z + (double)rm.amp_shift)
                  : exp2(0.5 * (double)h + (double)rm.amp_shift);
  scale_h = __shfl_sync(0xffffffffu, scale_h, 0);
  unsigned long long tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double wre = 0.0, wim = 0.0;
  unsigned long long vtot = 0;
  for (uint32_t b = (uint32_t)lane; b < rm.n_batches; b += 32u) {
    if (wgt) {
      double x, y;
      batch_sum(rm, true, b, bin, x, y);
      wre += x;
      wim += y;
    } else {
      const unsigned long long* c = rm.hist + ((size_t)b * rm.bins + bin) * 8u;
#pragma unroll
      for (int k = 0; k < 8; ++k) tot[k] += c[k];
    }
    vtot += rm.valid[b];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    vtot += __shfl_xor_sync(0xffffffffu, vtot, off);
    if (wgt) {
      wre += __shfl_xor_sync(0xffffffffu, wre, off);
      wim += __shfl_xor_sync(0xffffffffu, wim, off);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], off);
    }
  }
  double re = 0.0, im = 0.0, se = 0.0;
  if (vtot > 0) {
    if (wgt) {
      re = wre;
      im = wim;
    } else {
      phase_sum(tot, re, im);
    }
    double f = 0.0, inv_vtot = 0.0;
    if (lane == 0) {
      f = scale_h / (double)vtot;
      inv_vtot = 1.0 / (double)vtot;
    }
    f = __shfl_sync(0xffffffffu, f, 0);
    inv_vtot = __shfl_sync(0xffffffffu, inv_vtot, 0);
    re *= f;
    im *= f;
    uint32_t nb = 0;
    Kahan acc;
    for (uint32_t b = (uint32_t)lane; b < rm.n_batches; b += 32u) {
      const unsigned long long vb = rm.valid[b];
      if (vb == 0) continue;
      ++nb;
      double br, bi;
      batch_sum(rm, wgt, b, bin, br, bi);
      const double fb = scale_h / (double)vb;
      br = br * fb - re;
      bi = bi * fb - im;
      const double w = (double)vb * inv_vtot;
      acc.add(w * w * (br * br + bi * bi));
    }
    double var = acc.s - acc.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      var += __shfl_xor_sync(0xffffffffu, var, off);
      nb += __shfl_xor_sync(0xffffffffu, nb, off);
    }
    if (lane == 0) se = nb > 1 ? sqrt(var * (double)nb / (double)(nb - 1)) : 0.0;
  }
  if (lane == 0) {
    double* out = rm.amp + (size_t)bin * 3u;
    out[0] = re;
    out[1] = im;
    out[2] = se;
  }
}

// L2 normalisation over the recorded bins (Fig. 2 Step 4), one CTA.
__global__ void normalize_kernel(const RunModelDev* __restrict__ rm_all, int model) {
  const RunModelDev& rm = rm_all[model];
  __shared__ double part[1024];
  Kahan acc;
  for (uint32_t i = threadIdx.x; i < rm.bins; i += blockDim.x) {
    const double* a = rm.amp + (size_t)i * 3u;
    acc.add(a[0] * a[0] + a[1] * a[1]);
  }
  part[threadIdx.x] = acc.s;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  const double norm = sqrt(part[0]);
  if (norm <= 0.0) return;
  const double inv = 1.0 / norm;
  for (uint32_t i = threadIdx.x; i < rm.bins; i += blockDim.x) {
    double* a = rm.amp + (size_t)i * 3u;
    a[0] *= inv;
    a[1] *= inv;
    a[2] *= inv;
  }
}

__global__ void philox_fill_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                   uint32_t count, uint32_t* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = philox4x32_10(c, k0, k1);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// ---------------------------------------------------------------------------
// Host-side launchers (called by the runtime).
cudaError_t launch_init(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                        const uint32_t* const* d_init_tabs, size_t smem_bytes, WsHeader* hdr,
                        cudaStream_t st) {
  init_kernel<<<total_groups, 32, smem_bytes, st>>>(d_rm, n_models, total_groups, d_init_tabs, hdr);
  return cudaGetLastError();
}

// Sweep index advance after a launch (the sweep kernels read hdr->sweep0, so
// one captured graph replays correctly any number of times).
__global__ void advance_kernel(WsHeader* hdr, uint32_t n_sweeps) { hdr->sweep0 += n_sweeps; }
__global__ void reset_work_kernel(WsHeader* hdr) { hdr->work_next = 0u; }

// nc: colour steps per sweep (the largest over the launch's models; 2..4).
// wgt: some model has general gates (the WGT instantiation); ext: some model
// has Toffoli links or two-qubit tables (EXT).
cudaError_t launch_sweeps(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                          uint32_t n_sweeps, int cons, int prod, int max_col, int nc,
                          size_t smem_bytes, WsHeader* hdr, cudaStream_t st, bool wgt, bool ext,
                          bool bal, bool dec) {
  const int threads = cons + prod + 32;
  const Shape sh{cons, prod};
  auto go = [&](auto kern) {
    kern<<<total_groups, threads, smem_bytes, st>>>(d_rm, n_models, total_groups, n_sweeps, sh,
                                                    max_col, hdr);
  };
  if (wgt && ext) {
    if (nc <= 2) go(sweep_kernel<2, true, true, false>);
    else if (nc == 3) go(sweep_kernel<3, true, true, false>);
    else go(sweep_kernel<4, true, true, false>);
  } else if (wgt) {
    if (nc <= 2) go(sweep_kernel<2, true, false, false>);
    else if (nc == 3) go(sweep_kernel<3, true, false, false>);
    else go(sweep_kernel<4, true, false, false>);
  } else if (bal && dec) {
    if (nc <= 2) go(sweep_kernel<2, false, false, true, true>);
    else if (nc == 3) go(sweep_kernel<3, false, false, true, true>);
    else go(sweep_kernel<4, false, false, true, true>);
  } else if (bal) {
    if (nc <= 2) go(sweep_kernel<2, false, false, true>);
    else if (nc == 3) go(sweep_kernel<3, false, false, true>);
    else go(sweep_kernel<4, false, false, true>);
  } else {
    if (nc <= 2) go(sweep_kernel<2, false, false, false>);
    else if (nc == 3) go(sweep_kernel<3, false, false, false>);
    else go(sweep_kernel<4, false, false, false>);
  }
  advance_kernel<<<1, 1, 0, st>>>(hdr, n_sweeps);
  return cudaGetLastError();
}

cudaError_t launch_sweeps_persistent(const RunModelDev* d_rm, int n_models, const uint32_t* d_work,
                                     uint32_t n_work, uint32_t n_sweeps, int cons, int prod,
                                     int max_col, int nc, int grid, size_t smem_bytes,
                                     WsHeader* hdr, cudaStream_t st, bool bal) {
  const int threads = cons + prod + 32;
  // the work counter is cleared by a kernel (a graph may hold this launch
  // inside a device-side loop, whose body takes kernels)
  reset_work_kernel<<<1, 1, 0, st>>>(hdr);
  const Shape sh{cons, prod};
  auto go = [&](auto kern) {
    kern<<<grid, threads, smem_bytes, st>>>(d_rm, n_models, d_work, n_work, n_sweeps, sh, max_col,
                                            hdr);
  };
  if (bal) {
    if (nc <= 2) go(sweep_persistent_kernel<2, true>);
    else if (nc == 3) go(sweep_persistent_kernel<3, true>);
    else go(sweep_persistent_kernel<4, true>);
  } else {
    if (nc <= 2) go(sweep_persistent_kernel<2, false>);
    else if (nc == 3) go(sweep_persistent_kernel<3, false>);
    else go(sweep_persistent_kernel<4, false>);
  }
  advance_kernel<<<1, 1, 0, st>>>(hdr, n_sweeps);
  return cudaGetLastError();
}

// smem_bytes from elim_smem_bytes(.., warps): `warps` (8, 16 or 32) equal
// per-warp regions.
cudaError_t launch_elim(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                        const uint32_t* const* d_init_tabs, uint32_t n_sweeps, size_t smem_bytes,
                        WsHeader* hdr, cudaStream_t st, bool wgt, int warps) {
  if (warps != 8 && warps != 16 && warps != 32) return cudaErrorInvalidValue;
  const int wstride = (int)(smem_bytes / (4 * (size_t)warps));
  auto go = [&](auto kern) {
    kern<<<total_groups, warps * 32, smem_bytes, st>>>(d_rm, n_models, total_groups, d_init_tabs,
                                                       n_sweeps, wstride, hdr);
  };
  if (wgt) {
    if (warps == 32) go(elim_kernel<true, 32>);
    else if (warps == 16) go(elim_kernel<true, 16>);
    else go(elim_kernel<true, 8>);
  } else {
    if (warps == 32) go(elim_kernel<false, 32>);
    else if (warps == 16) go(elim_kernel<false, 16>);
    else go(elim_kernel<false, 8>);
  }
  advance_kernel<<<1, 1, 0, st>>>(hdr, n_sweeps);
  return cudaGetLastError();
}

// Per warp: the path image and up to `zwords` free draws (16-byte multiples).
size_t elim_smem_bytes(int n, int d, int zwords, int warps) {
  return (size_t)warps * (size_t)(image_words(n, d) + ((zwords + 3) & ~3)) * 4;
}

cudaError_t launch_amplitudes(const RunModelDev* d_rm, int model, uint32_t bins, int l2,
                              cudaStream_t st) {
  // one warp a bin, eight bins a CTA
  const uint32_t per_cta = 8;
  amplitude_kernel<<<(bins + per_cta - 1) / per_cta, 32 * per_cta, 0, st>>>(d_rm, model);
  if (l2) normalize_kernel<<<1, 1024, 0, st>>>(d_rm, model);
  return cudaGetLastError();
}

cudaError_t launch_philox_fill(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t count,
                               uint32_t* out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  philox_fill_kernel<<<(count + 255) / 256, 256, 0, st>>>(ctr, k0, k1, count, out);
  return cudaGetLastError();
}

size_t sweep_smem_bytes(int n, int d, int cons, int max_col, uint32_t hist_bins, bool wgt,
                        bool bal) {
  return group_smem_bytes(n, d, cons, max_col, hist_bins, wgt && !bal, bal && !wgt);
}

// Opt the sweep kernels into large dynamic shared memory (called once per
// run, outside any stream capture).
cudaError_t sweep_prepare() {
  const int big = (int)kSweepSmemMax;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(sweep_kernel<2, false, false, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<3, false, false, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<4, false, false, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<2, false, false, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<3, false, false, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<4, false, false, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<2, false, false, true, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<3, false, false, true, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<4, false, false, true, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<2, true, false, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<3, true, false, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<4, true, false, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<2, true, true, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<3, true, true, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_kernel<4, true, true, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_persistent_kernel<2, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_persistent_kernel<3, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_persistent_kernel<4, false>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_persistent_kernel<2, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_persistent_kernel<3, true>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(sweep_persistent_kernel<4, true>, a, big)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(elim_kernel<false, 8>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(elim_kernel<false, 16>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(elim_kernel<false, 32>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(elim_kernel<true, 8>, a, big)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(elim_kernel<true, 16>, a, big)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(elim_kernel<true, 32>, a, big);
}

int sweep_max_blocks_per_sm(int threads, size_t smem, bool bal) {
  int blocks = 0;
  const cudaError_t e =
      bal ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, sweep_persistent_kernel<4, true>,
                                                          threads, smem)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, sweep_persistent_kernel<4, false>,
                                                          threads, smem);
  return e == cudaSuccess ? blocks : 1;
}

}  // namespace pb
