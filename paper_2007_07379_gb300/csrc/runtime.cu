// Host side of the C ABI: the circuit compiler (gate list -> p-bit tables),
// workspace layout, run objects, CUDA-graph replay and result read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "pb_internal.h"

namespace pb {
cudaError_t launch_init(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                        const uint32_t* const* d_init_tabs, size_t smem_bytes, WsHeader* hdr,
                        cudaStream_t st);
cudaError_t launch_sweeps(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                          uint32_t n_sweeps, int cons, int prod, int max_col, int nc,
                          size_t smem_bytes, WsHeader* hdr, cudaStream_t st, bool wgt = false,
                          bool ext = false, bool bal = false, bool dec = false);
cudaError_t launch_sweeps_persistent(const RunModelDev* d_rm, int n_models, const uint32_t* d_work,
                                     uint32_t n_work, uint32_t n_sweeps, int cons, int prod,
                                     int max_col, int nc, int grid, size_t smem_bytes,
                                     WsHeader* hdr, cudaStream_t st, bool bal);
cudaError_t launch_elim(const RunModelDev* d_rm, int n_models, uint32_t total_groups,
                        const uint32_t* const* d_init_tabs, uint32_t n_sweeps, size_t smem_bytes,
                        WsHeader* hdr, cudaStream_t st, bool wgt, int warps);
size_t elim_smem_bytes(int n, int d, int zwords, int warps);
cudaError_t launch_amplitudes(const RunModelDev* d_rm, int model, uint32_t bins, int l2,
                              cudaStream_t st);
cudaError_t launch_philox_fill(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t count,
                               uint32_t* out, cudaStream_t st);
size_t sweep_smem_bytes(int n, int d, int cons, int max_col, uint32_t hist_bins,
                        bool wgt = false, bool bal = false);
cudaError_t sweep_prepare();
int sweep_max_blocks_per_sm(int threads, size_t smem, bool bal);
}  // namespace pb

using namespace pb;

namespace {

// Gate occupying (layer, qubit): kind and partner / role.
struct Slot {
  int op = -1;       // -1 identity wire
  int partner = -1;  // other qubit of a 2-qubit gate
  bool target = false;  // CNOT target
  int ukind = 0;     // PB_U: kUDiag, kUAnti or kUCoupled
  double a = 0.0, b = 0.0, K = 0.0;  // PB_U magnitudes and coupling
  int gi = -1;       // gate row
  int u2o = 0;       // PB_U2: 0 on q0, 1 on q1 (this qubit's output and input index);
                     // PB_CCX: 0, 1 on the controls q0, q1, 2 on the target q2
};

// A PB_U2 gate's permutation and the affine map of its output bits:
// output o = cbit[o] XOR (input 0 if dmask[o] & 1) XOR (input 1 if dmask[o] & 2).
struct U2Map {
  int perm[4] = {0, 0, 0, 0};
  int dmask[2] = {0, 0}, cbit[2] = {0, 0};
};

// PB_U2 matrix (32 doubles: Re/Im of <y|U|x>, row-major 4x4), unitary within
// 1e-9.  Exactly one nonzero per column: an affine permutation (u filled;
// returns 1) unless an output equals the complement of the XOR of both
// inputs (returns 0: rejected).  More than one nonzero in some column: a
// table gate (returns 2).  Not unitary: 0.
int classify_u2(const double* m, U2Map& u) {
  auto re = [&](int y, int x) { return m[2 * (4 * y + x)]; };
  auto im = [&](int y, int x) { return m[2 * (4 * y + x) + 1]; };
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double sr = 0.0, si = 0.0;  // (U^dagger U)_ij
      for (int y = 0; y < 4; ++y) {
        sr += re(y, i) * re(y, j) + im(y, i) * im(y, j);
        si += re(y, i) * im(y, j) - im(y, i) * re(y, j);
      }
      if (!(std::fabs(sr - (i == j ? 1.0 : 0.0)) <= 1e-9) || !(std::fabs(si) <= 1e-9)) return 0;
    }
  for (int x = 0; x < 4; ++x) {
    int nz = 0;
    for (int y = 0; y < 4; ++y)
      if (re(y, x) != 0.0 || im(y, x) != 0.0) {
        u.perm[x] = y;
        ++nz;
      }
    if (nz != 1) return 2;
  }
  for (int o = 0; o < 2; ++o) {
    const int c = (u.perm[0] >> o) & 1;
    const int al = ((u.perm[1] >> o) & 1) ^ c, be = ((u.perm[2] >> o) & 1) ^ c;
    if ((((u.perm[3] >> o) & 1) ^ c) != (al ^ be)) return 0;
    u.dmask[o] = al | (be << 1);
    u.cbit[o] = c;
    if (u.dmask[o] == 0 || (u.dmask[o] == 3 && c)) return 0;
  }
  return 1;
}

constexpr int kU2Table = 4;  // Slot.ukind of a two-qubit table gate

enum { kUDiag = 1, kUAnti = 2, kUCoupled = 3 };

// Kind of a PB_U matrix (8 doubles: Re/Im of U00, U01, U10, U11, row =
// output) with its magnitudes a = (|U00|+|U11|)/2, b = (|U01|+|U10|)/2 and
// coupling K = ln(a/b) (Eq. EB for a unitary); -1 when it is not unitary
// within 1e-9 or has a single zero entry.
int classify_u(const double* m, double& a, double& b, double& K) {
  auto re = [&](int y, int x) { return m[2 * (2 * y + x)]; };
  auto im = [&](int y, int x) { return m[2 * (2 * y + x) + 1]; };
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double sr = 0.0, si = 0.0;  // (U^dagger U)_ij
      for (int y = 0; y < 2; ++y) {
        sr += re(y, i) * re(y, j) + im(y, i) * im(y, j);
        si += re(y, i) * im(y, j) - im(y, i) * re(y, j);
      }
      if (!(std::fabs(sr - (i == j ? 1.0 : 0.0)) <= 1e-9) || !(std::fabs(si) <= 1e-9)) return -1;
    }
  auto zero = [&](int y, int x) { return re(y, x) == 0.0 && im(y, x) == 0.0; };
  a = 0.5 * (std::hypot(re(0, 0), im(0, 0)) + std::hypot(re(1, 1), im(1, 1)));
  b = 0.5 * (std::hypot(re(0, 1), im(0, 1)) + std::hypot(re(1, 0), im(1, 0)));
  K = 0.0;
  const bool z00 = zero(0, 0), z01 = zero(0, 1), z10 = zero(1, 0), z11 = zero(1, 1);
  if (z01 && z10 && !z00 && !z11) return kUDiag;
  if (z00 && z11 && !z01 && !z10) return kUAnti;
  if (z00 || z01 || z10 || z11) return -1;
  K = std::log(a / b);
  return kUCoupled;
}

// floor(2^32 x) for x >= 0, capped at 2^32 - 1 (a uniform u accepts when u < it).
uint32_t u32_threshold(double x) {
  const double t = std::floor(x * 4294967296.0);
  return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

// arg z in units of 2^-32 turn (mod 2^32).
uint32_t fixed_turns(double re, double im) {
  const double t = std::atan2(im, re) / (2.0 * M_PI);  // [-1/2, 1/2]
  return (uint32_t)(uint64_t)(int64_t)std::llround(t * 4294967296.0);
}

// GF(2) rank of the rows (bitsets over the H variables), by inserting each
// row into an XOR basis keyed by its highest set bit.
int gf2_rank_rows(const std::vector<std::vector<uint64_t>>& rows, int nbits) {
  const int nw = (nbits + 63) / 64;
  std::vector<std::vector<uint64_t>> basis(nbits);
  std::vector<bool> have(nbits, false);
  int rank = 0;
  for (auto row : rows) {
    row.resize(nw, 0);
    for (int b = nbits - 1; b >= 0; --b) {
      if (!((row[b >> 6] >> (b & 63)) & 1ull)) continue;
      if (!have[b]) {
        basis[b] = row;
        have[b] = true;
        ++rank;
        break;
      }
      for (int w = 0; w < nw; ++w) row[w] ^= basis[b][w];
    }
  }
  return rank;
}

}  // namespace

extern "C" {

PB_API int pb_version(void) { return 1; }

PB_API const char* pb_strerror(int s) {
  switch (s) {
    case PB_OK: return "ok";
    case PB_EINVAL: return "invalid argument";
    case PB_ERANGE: return "size out of range";
    case PB_ENOMEM: return "out of host memory";
    case PB_ECUDA: return "CUDA runtime error";
    case PB_ETIMEOUT: return "device wait timed out";
    case PB_ESTATE: return "invalid state for this call";
  }
  return "unknown status";
}

PB_API int pb_compile(int n, int d, const pb_gate* gates, int n_gates, uint32_t input_bits,
                      double J, pb_model** out) {
  return pb_compile_u(n, d, gates, n_gates, nullptr, input_bits, J, out);
}

PB_API int pb_compile_u(int n, int d, const pb_gate* gates, int n_gates, const double* mats,
                        uint32_t input_bits, double J, pb_model** out) {
  return pb_compile_g(n, d, gates, n_gates, mats, 8, input_bits, J, out);
}

PB_API int pb_compile_g(int n, int d, const pb_gate* gates, int n_gates, const double* mats,
                        int stride, uint32_t input_bits, double J, pb_model** out) {
  if (!out) return PB_EINVAL;
  if (stride < 8) return PB_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 32 || d < 1 || d > 64) return PB_ERANGE;
  if (n_gates < 0 || (n_gates > 0 && !gates)) return PB_EINVAL;
  if (!(J >= 0.0) || !std::isfinite(J)) return PB_EINVAL;
  if (n < 32 && (input_bits >> n) != 0) return PB_EINVAL;

  std::vector<Slot> slot((size_t)d * n);
  std::vector<U2Map> u2map((size_t)std::max(n_gates, 1));
  for (int i = 0; i < n_gates; ++i) {
    const pb_gate& g = gates[i];
    if (g.op < PB_H || g.op > PB_CCX || g.layer < 0 || g.layer >= d) return PB_EINVAL;
    if (g.q0 < 0 || g.q0 >= n) return PB_EINVAL;
    const bool two = g.op == PB_CNOT || g.op == PB_CZ || g.op == PB_U2 || g.op == PB_CCX;
    if (two && (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)) return PB_EINVAL;
    if (g.op == PB_CCX) {
      if (g.q2 < 0 || g.q2 >= n || g.q2 == g.q0 || g.q2 == g.q1) return PB_EINVAL;
      Slot& s2 = slot[(size_t)g.layer * n + g.q2];
      if (s2.op != -1) return PB_EINVAL;
      s2.op = g.op;
      s2.gi = i;
      s2.u2o = 2;
    }
    Slot& s0 = slot[(size_t)g.layer * n + g.q0];
    if (s0.op != -1) return PB_EINVAL;
    s0.op = g.op;
    s0.gi = i;
    if (g.op == PB_U) {
      if (!mats) return PB_EINVAL;
      s0.ukind = classify_u(mats + (size_t)stride * i, s0.a, s0.b, s0.K);
      if (s0.ukind < 0) return PB_EINVAL;
    }
    if (g.op == PB_U2) {
      if (!mats || stride < 32) return PB_EINVAL;
      const int k = classify_u2(mats + (size_t)stride * i, u2map[i]);
      if (k == 0) return PB_EINVAL;
      if (k == 2) s0.ukind = kU2Table;
    }
    if (two) {
      Slot& s1 = slot[(size_t)g.layer * n + g.q1];
      if (s1.op != -1) return PB_EINVAL;
      s0.partner = g.q1;
      s1.op = g.op;
      s1.partner = g.q0;
      s1.target = (g.op == PB_CNOT);
      s1.gi = i;
      s1.u2o = 1;
      s1.ukind = s0.ukind;
    }
  }

  std::unique_ptr<pb_model> m(new (std::nothrow) pb_model);
  if (!m) return PB_ENOMEM;
  m->n = n;
  m->d = d;
  m->beta = input_bits;
  m->J = J;
  m->gates.assign(gates, gates + n_gates);
  // Heat-bath thresholds: P(1) = 1 / (1 + e^{J v}) for a violation change v.
  m->thr[0] = 0x80000000u;
  for (int v = 1; v <= 3; ++v) {
    double t = std::floor(4294967296.0 / (1.0 + std::exp(J * (double)v)));
    m->thr[v] = (uint32_t)std::min(t, 4294967295.0);
  }

  const uint16_t Z = (uint16_t)zero_idx(n, d), O = (uint16_t)ones_idx(n, d);
  auto at = [&](int layer, int q) -> const Slot& { return slot[(size_t)layer * n + q]; };
  auto word = [&](int k, int q) -> uint16_t { return (uint16_t)(k * n + q); };
  // free outputs: H and coupled PB_U; the second word of a single-input
  // link: the CNOT control (target), ONES (anti-diagonal PB_U: NOT), ZERO
  auto table = [](const Slot& s) { return s.op == PB_U2 && s.ukind == kU2Table; };
  auto is_free = [&](const Slot& s) {
    return s.op == PB_H || (s.op == PB_U && s.ukind == kUCoupled) || table(s);
  };
  auto coupled = [](const Slot& s) { return s.op == PB_U && s.ukind == kUCoupled; };
  for (int i = 0; i < n_gates; ++i) {
    if (gates[i].op == PB_U || gates[i].op == PB_U2) {
      m->wgt = true;
      ++m->n_u;
      m->n_coupled += coupled(at(gates[i].layer, gates[i].q0)) ? 1 : 0;
    }
    if (gates[i].op == PB_CCX) {  // general links: the general-gate kernels
      m->wgt = true;
      ++m->n_ccx;
    }
    if (gates[i].op == PB_U2 && table(at(gates[i].layer, gates[i].q0))) ++m->n_tab;
  }
  if (m->n_ccx) m->glk.assign((size_t)n * d, GLink{});
  if (m->n_tab) m->tacc.assign((size_t)n * d, TAcc{});
  // energy -ln|U(y, x)| of a table gate's entry, J for a zero entry (Appendix)
  auto tab_energy = [&](int gi, int y, int x) {
    const double* mu = mats + (size_t)stride * gi;
    const double mag = std::hypot(mu[2 * (4 * y + x)], mu[2 * (4 * y + x) + 1]);
    return mag > 0.0 ? -std::log(mag) : J;
  };

  const int npb = n * d;
  std::vector<Desc> by_p(npb);
  m->rec.assign(npb, Rec{});
  m->init.assign(npb, 0xFFFFFFFFu);
  m->colour.assign(npb, 0);
  for (int k = 1; k <= d; ++k) {
    for (int q = 0; q < n; ++q) {
      const int p = (k - 1) * n + q;
      Desc D;
      D.dst = word(k, q);
      for (int l = 0; l < 3; ++l) { D.a[l] = Z; D.b[l] = Z; }
      int m_links = 0;
      bool own = false;
      // own link: gate layer k-1 produces s_k
      const Slot& prod = at(k - 1, q);
      auto second = [&](const Slot& s, int layer) -> uint16_t {
        if (s.op == PB_CNOT && s.target) return word(layer, s.partner);
        if (s.op == PB_U && s.ukind == kUAnti) return O;
        if (s.op == PB_X) return O;
        return Z;
      };
      // qubit of input u (0: q0, 1: q1) of the PB_U2 on this slot
      auto u2q = [&](const Slot& s, int u) { return ((s.u2o == 0) == (u == 0)) ? q : s.partner; };
      if (prod.op == PB_U2 && !table(prod)) {  // own link: this output's affine map
        const U2Map& um = u2map[prod.gi];
        const int o = prod.u2o, dm = um.dmask[o];
        own = true;
        if (dm == 3) {
          D.a[m_links] = word(k - 1, u2q(prod, 0));
          D.b[m_links] = word(k - 1, u2q(prod, 1));
        } else {
          D.a[m_links] = word(k - 1, u2q(prod, dm == 1 ? 0 : 1));
          D.b[m_links] = um.cbit[o] ? O : Z;
        }
        ++m_links;
      } else if (!is_free(prod)) {
        own = true;
        D.a[m_links] = word(k - 1, q);
        D.b[m_links] = second(prod, k - 1);
        ++m_links;
      }
      bool tgt_next = false;
      if (k < d && at(k, q).op == PB_U2 && !table(at(k, q))) {
        // the outputs of the next layer's PB_U2 whose map reads this input
        const Slot& cons = at(k, q);
        const U2Map& um = u2map[cons.gi];
        const int me = cons.u2o;
        for (int o = 0; o < 2; ++o) {
          if (!((um.dmask[o] >> me) & 1)) continue;
          const int qo = (o == me) ? q : cons.partner;  // the qubit carrying output o
          D.a[m_links] = word(k + 1, qo);
          D.b[m_links] = um.dmask[o] == 3 ? word(k, cons.partner) : (um.cbit[o] ? O : Z);
          ++m_links;
        }
        tgt_next = me == 1 && (um.dmask[0] == 3 || um.dmask[1] == 3);
      } else if (k < d) {
        const Slot& cons = at(k, q);  // gate layer k consumes s_k
        if (!is_free(cons)) {         // the wire's next bit demands s_k[q]
          D.a[m_links] = word(k + 1, q);
          D.b[m_links] = second(cons, k);
          ++m_links;
        }
        if (cons.op == PB_CNOT && !cons.target) {  // control: the target's next bit
          D.a[m_links] = word(k + 1, cons.partner);
          D.b[m_links] = word(k, cons.partner);
          ++m_links;
        }
        tgt_next = cons.op == PB_CNOT && cons.target;
      }
      D.mflag = (uint8_t)(m_links | (own ? 4 : 0));
      // Toffoli: every link of its target output and of its inputs in the
      // general form r = W[a] ^ (W[b] & W[c]), counted where W[e]
      const bool ccx_out = prod.op == PB_CCX && prod.u2o == 2;
      const bool ccx_in = k < d && at(k, q).op == PB_CCX;
      bool ccx_target_out = false;
      if (ccx_out || ccx_in) {
        GLink G{};
        for (int l = 0; l < 3; ++l) G.a[l] = G.b[l] = G.c[l] = G.e[l] = Z;
        int nl = 0;
        auto add = [&](uint16_t a, uint16_t b, uint16_t c, uint16_t e) {
          G.a[nl] = a; G.b[nl] = b; G.c[nl] = c; G.e[nl] = e;
          ++nl;
        };
        if (ccx_out) {  // own: t' = t ^ (c0 & c1)
          const pb_gate& tg = gates[prod.gi];
          add(word(k - 1, tg.q2), word(k - 1, tg.q0), word(k - 1, tg.q1), O);
          ccx_target_out = true;
        } else if (own) {
          add(D.a[0], D.b[0], O, O);
        }
        if (ccx_in) {
          const Slot& cons = at(k, q);
          const pb_gate& tg = gates[cons.gi];
          if (cons.u2o == 2) {  // target input: t = t' ^ (c0 & c1)
            add(word(k + 1, tg.q2), word(k, tg.q0), word(k, tg.q1), O);
          } else {              // a control: its copy, and t' ^ t where the other control is 1
            add(word(k + 1, q), Z, O, O);
            add(word(k + 1, tg.q2), word(k, tg.q2), O, word(k, cons.u2o == 0 ? tg.q1 : tg.q0));
          }
        } else {
          for (int l = own ? 1 : 0; l < m_links; ++l) add(D.a[l], D.b[l], O, O);
        }
        m->glk[(size_t)(k - 1) * n + q] = G;
        D.mflag |= 0x10;
        own = own || ccx_out;
        tgt_next = ccx_in && at(k, q).u2o == 2;
      }
      if (m->wgt) {  // couplings of the p-bit (Metropolis acceptance table)
        Cpl C{};
        C.win = C.wout = D.dst;
        double kin = 0.0, kout = 0.0;
        if (coupled(prod)) {
          C.win = word(k - 1, q);
          kin = prod.K;
          C.flags |= 3u;
          C.B = u32_threshold(prod.b / (prod.a + prod.b));
        }
        if (k < d && coupled(at(k, q))) {
          C.wout = word(k + 1, q);
          kout = at(k, q).K;
          C.flags |= 1u;
        }
        for (int c = 0; c < 4; ++c) {
          const int ein = c & 1, eout = c >> 1;
          const double dk = kin * (double)(1 - 2 * ein) + kout * (double)(1 - 2 * eout);
          if (dk <= 0.0) C.amask |= 1u << c;
          else C.A[c] = u32_threshold(std::exp(-dk));
        }
        if (C.flags & 1u) D.mflag |= 8;
        m->cpl.push_back(C);
      }
      const bool tin = table(prod), tout = k < d && table(at(k, q));
      if (tin || tout) {  // Metropolis acceptance on the tables' energy
        TAcc A{};
        for (int l = 0; l < 6; ++l) A.w[l] = Z;
        int o = 0, iu = 0, gin = -1, gout = -1;
        if (tin) {  // this bit is output o of the table of layer k-1
          gin = prod.gi;
          const pb_gate& tg = gates[gin];
          o = prod.u2o;
          A.w[0] = word(k, o == 0 ? tg.q1 : tg.q0);  // the other output
          A.w[1] = word(k - 1, tg.q0);
          A.w[2] = word(k - 1, tg.q1);
        }
        if (tout) {  // input iu of the table of layer k
          const Slot& cs = at(k, q);
          gout = cs.gi;
          const pb_gate& tg = gates[gout];
          iu = cs.u2o;
          A.w[3] = word(k, iu == 0 ? tg.q1 : tg.q0);  // the other input
          A.w[4] = word(k + 1, tg.q0);
          A.w[5] = word(k + 1, tg.q1);
        }
        for (int idx = 0; idx < 128; ++idx) {
          const int ci = idx & 7, co = (idx >> 3) & 7, dir = idx >> 6;
          double din = 0.0, dout = 0.0;
          if (tin) {
            const int yo = ci & 1, xi = (ci >> 1) & 3;
            const int y1 = o == 0 ? 1 + 2 * yo : yo + 2, y0 = o == 0 ? 2 * yo : yo;
            din = tab_energy(gin, y1, xi) - tab_energy(gin, y0, xi);
          }
          if (tout) {
            const int xo = co & 1, yi = (co >> 1) & 3;
            const int x1 = iu == 0 ? 1 + 2 * xo : xo + 2, x0 = iu == 0 ? 2 * xo : xo;
            dout = tab_energy(gout, yi, x1) - tab_energy(gout, yi, x0);
          }
          const double de = din + dout;
          const double dt = dir == 0 ? de : -de;
          if (dt <= 0.0) A.amask[idx >> 5] |= 1u << (idx & 31);
          else A.thr[idx] = u32_threshold(std::exp(-dt));
        }
        m->tacc[(size_t)(k - 1) * n + q] = A;
        D.mflag |= 0x20;
      }
      static const uint8_t pair_of_m[4] = {0, 1, 2, 3};
      D.pair = pair_of_m[m_links];
      by_p[p] = D;
      m->colour[p] = 2 * ((k % 2) == 0) + (tgt_next ? 1 : 0);

      Rec R{};
      R.vd = R.va = R.vb = Z;
      R.vc = O;
      R.pa = R.pb = Z;
      R.w = 0;
      if (ccx_target_out) {  // violation t' ^ t ^ (c0 & c1); the initial value from link 0
        const GLink& G = m->glk[(size_t)(k - 1) * n + q];
        R.vd = D.dst;
        R.va = G.a[0];
        R.vb = G.b[0];
        R.vc = G.c[0];
        m->init[p] = 0xFFFFFFFEu;
      } else if (own) {
        R.vd = D.dst;
        R.va = D.a[0];
        R.vb = D.b[0];
        m->init[p] = (uint32_t)D.a[0] | ((uint32_t)D.b[0] << 16);
      }
      switch (prod.op) {
        case PB_H: R.w = 4; R.pa = word(k - 1, q); R.pb = word(k, q); break;
        case PB_S: R.w = 2; R.pa = word(k - 1, q); R.pb = O; break;
        case PB_T: R.w = 1; R.pa = word(k - 1, q); R.pb = O; break;
        case PB_CZ:
          if (q < prod.partner) { R.w = 4; R.pa = word(k - 1, q); R.pb = word(k - 1, prod.partner); }
          break;
        default: break;
      }
      m->rec[p] = R;
    }
  }
  // Colour classes: p-bits that share a link interact; a p-bit's neighbours
  // are the p-bit words among its link demands W[a_l] ^ W[b_l].  DSATUR
  // (Brelaz) with fixed tie-breaks: the uncoloured p-bit with the most
  // distinct neighbour colours, then the most neighbours, then the lowest p,
  // takes the smallest colour its neighbours lack.  More than four colours
  // (not met in practice: at most six neighbours) falls back to the fixed
  // classes 2 [k even] + [CNOT target in layer k+1] set above.
  {
    std::vector<std::vector<int>> nb(npb);
    auto join = [&](int p, int u) {
      if (std::find(nb[p].begin(), nb[p].end(), u) == nb[p].end()) nb[p].push_back(u);
    };
    for (int p = 0; p < npb; ++p) {
      const pb::Desc& D = by_p[p];
      if (D.mflag & 0x10) {  // general links: every word of every link
        const GLink& G = m->glk[p];
        for (int l = 0; l < 3; ++l)
          for (int w : {(int)G.a[l], (int)G.b[l], (int)G.c[l], (int)G.e[l]})
            if (w >= n && w < (d + 1) * n && w - n != p) join(p, w - n);
        continue;
      }
      for (int l = 0; l < (D.mflag & 3); ++l)
        for (int w : {(int)D.a[l], (int)D.b[l]})
          if (w >= n && w < (d + 1) * n && w - n != p) join(p, w - n);
    }
    // a coupled PB_U in layer L >= 1 joins p-bits (L, q) and (L + 1, q)
    for (int L = 1; L < d; ++L)
      for (int q = 0; q < n; ++q)
        if (coupled(at(L, q))) {
          join((L - 1) * n + q, L * n + q);
          join(L * n + q, (L - 1) * n + q);
        }
    // a two-qubit table joins its outputs and inputs pairwise
    for (int i = 0; i < n_gates; ++i) {
      const pb_gate& tg = gates[i];
      if (tg.op != PB_U2 || !table(at(tg.layer, tg.q0))) continue;
      std::vector<int> vs = {tg.layer * n + tg.q0, tg.layer * n + tg.q1};
      if (tg.layer >= 1) {
        vs.push_back((tg.layer - 1) * n + tg.q0);
        vs.push_back((tg.layer - 1) * n + tg.q1);
      }
      for (int a : vs)
        for (int b : vs)
          if (a != b) join(a, b);
    }
    std::vector<int> col(npb, -1);
    std::vector<uint32_t> seen(npb, 0u);
    int ncol = 0;
    for (int step = 0; step < npb; ++step) {
      int best = -1, bsat = -1, bdeg = -1;
      for (int v = 0; v < npb; ++v) {
        if (col[v] >= 0) continue;
        const int sat = __builtin_popcount(seen[v]);
        if (sat > bsat || (sat == bsat && (int)nb[v].size() > bdeg)) {
          best = v;
          bsat = sat;
          bdeg = (int)nb[v].size();
        }
      }
      int c = 0;
      while (c < 32 && ((seen[best] >> c) & 1u)) ++c;
      col[best] = c;
      ncol = std::max(ncol, c + 1);
      for (int u : nb[best]) seen[u] |= 1u << c;
    }
    if (ncol <= 4)
      for (int p = 0; p < npb; ++p) m->colour[p] = col[p];
    else if (m->n_ccx || m->n_tab)  // the fixed classes cannot separate a four-bit factor
      return PB_ERANGE;
  }

  // colour-ordered descriptors
  for (int c = 0; c < 4; ++c) {
    m->col_off[c] = (int)m->desc.size();
    for (int p = 0; p < npb; ++p)
      if (m->colour[p] == c) m->desc.push_back(by_p[p]);
  }
  m->col_off[4] = (int)m->desc.size();

  // general gates: phases (units of 2^-32 turn) and the estimator scale
  // log2z = h/2 + sum over coupled gates of log2(a + b), in gate order
  double l2z = 0.0;
  for (int i = 0; i < n_gates; ++i) {
    const pb_gate& g = gates[i];
    if (g.op == PB_H) l2z += 0.5;
    if (g.op == PB_U2 && table(at(g.layer, g.q0))) {  // a table: 16 phases, zero entries
      TRec R{};
      const double* mu = mats + (size_t)stride * i;
      for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x) {
          const double re = mu[2 * (4 * y + x)], im = mu[2 * (4 * y + x) + 1];
          R.ph[x + 4 * y] = fixed_turns(re, im);
          if (re == 0.0 && im == 0.0) R.zmask |= 1u << (x + 4 * y);
        }
      R.wx0 = word(g.layer, g.q0);
      R.wx1 = word(g.layer, g.q1);
      R.wy0 = word(g.layer + 1, g.q0);
      R.wy1 = word(g.layer + 1, g.q1);
      m->trec.push_back(R);
      continue;
    }
    if (g.op == PB_U2) {  // phase of the column taken: arg U(pi(x), x), x = x_{q0} + 2 x_{q1}
      UPh P{};
      const double* mu = mats + (size_t)stride * i;
      for (int x = 0; x < 4; ++x) {
        const int y = u2map[i].perm[x];
        P.ph[x] = fixed_turns(mu[2 * (4 * y + x)], mu[2 * (4 * y + x) + 1]);
      }
      P.win = word(g.layer, g.q0);   // bit x_{q0}: the recorder's "x"
      P.wout = word(g.layer, g.q1);  // bit x_{q1}: the recorder's "y" (ph[2 y + x])
      m->uph.push_back(P);
      continue;
    }
    if (g.op != PB_U) continue;
    const Slot& s = at(g.layer, g.q0);
    if (s.ukind == kUCoupled) l2z += std::log2(s.a + s.b);
    UPh P{};
    const double* mu = mats + (size_t)stride * i;
    for (int y = 0; y < 2; ++y)
      for (int x = 0; x < 2; ++x) P.ph[2 * y + x] = fixed_turns(mu[2 * (2 * y + x)], mu[2 * (2 * y + x) + 1]);
    P.wout = word(g.layer + 1, g.q0);
    P.win = word(g.layer, g.q0);
    m->uph.push_back(P);
  }
  // tables: the columns of |U| need not share one sum, so sum |U_C| has no
  // closed form; the estimate is read L2-normalised
  m->log2z = m->n_tab ? std::nan("") : l2z;

  // h, M and the GF(2) rank of the free outputs (H, coupled PB_U) -> s_d
  int h = 0;
  for (int i = 0; i < n_gates; ++i) h += gates[i].op == PB_H;
  m->h = h;
  m->M = npb - h - m->n_coupled;
  if (m->n_ccx) {
    m->rank = -1;  // a Toffoli makes the wires non-affine in the free outputs
  } else {
    const int nvar = h + m->n_coupled;
    std::vector<std::vector<uint64_t>> wire(n, std::vector<uint64_t>((nvar + 63) / 64 + 1, 0));
    int var = 0;
    for (int L = 0; L < d; ++L) {
      std::vector<std::vector<uint64_t>> nxt = wire;
      for (int q = 0; q < n; ++q) {
        const Slot& s = at(L, q);
        if (is_free(s)) {
          std::fill(nxt[q].begin(), nxt[q].end(), 0);
          nxt[q][var >> 6] |= 1ull << (var & 63);
          ++var;
        } else if (s.op == PB_CNOT && s.target) {
          for (size_t w = 0; w < nxt[q].size(); ++w) nxt[q][w] = wire[q][w] ^ wire[s.partner][w];
        } else if (s.op == PB_U2 && !table(s)) {  // the linear part of this output's affine map
          const int dm = u2map[s.gi].dmask[s.u2o];
          const int qa = s.u2o == 0 ? q : s.partner, qb = s.u2o == 0 ? s.partner : q;  // q0, q1
          for (size_t w = 0; w < nxt[q].size(); ++w)
            nxt[q][w] = ((dm & 1) ? wire[qa][w] : 0ull) ^ ((dm & 2) ? wire[qb][w] : 0ull);
        }
      }
      wire.swap(nxt);
    }
    m->rank = nvar > 0 ? gf2_rank_rows(wire, nvar) : 0;
  }
  *out = m.release();
  return PB_OK;
}

PB_API int pb_model_info(const pb_model* m, pb_model_info_t* info) {
  if (!m || !info) return PB_EINVAL;
  info->n = m->n;
  info->d = m->d;
  info->n_pbits = m->n * (m->d + 1);
  info->h = m->h;
  info->M = m->M;
  info->rank = m->rank;
  info->J = m->J;
  info->input_bits = m->beta;
  for (int i = 0; i < 4; ++i) {
    info->thr[i] = m->thr[i];
    info->colour_size[i] = m->col_off[i + 1] - m->col_off[i];
  }
  info->n_u = m->n_u;
  info->n_coupled = m->n_coupled;
  info->log2z = m->wgt ? m->log2z : 0.5 * m->h;
  return PB_OK;
}

PB_API int pb_model_colours(const pb_model* m, int32_t* colour) {
  if (!m || !colour) return PB_EINVAL;
  std::memcpy(colour, m->colour.data(), m->colour.size() * sizeof(int32_t));
  return PB_OK;
}

PB_API void pb_model_free(pb_model* m) { delete m; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Runs.
namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

struct ModelSlots {
  size_t model_dev, desc, rec, init, state, hist, valid, samples, alpha_sorted, alpha_slot, amp,
      clamp, cpl, uph, glk, tacc, trec;
  size_t mh;  // PB_LEARNED: the model's move region (mh_region_bytes), else unused
  uint32_t bins, groups, n_batches;
  int clamp_mw;  // mask words per p-bit of the clamp table (0: not clamped)
};

// Output clamping for the exact sampler (PB_ELIM_CLAMP).  The wire bits are
// affine over GF(2) in the H outputs x (in p order): s_d = A x + c.  A and c
// come from h + 1 evaluations of the init table (one chain, bit values), and
// the paths to alpha solve A x = alpha + c.  Gauss-Jordan on the augmented
// rows (bitsets) gives the unique reduced row echelon form; the free
// variables (non-pivot columns, increasing) take the draws z_b, each pivot
// variable its row's right-hand side XOR the free variables in its row.
struct ClampTable {
  bool ok = false;
  int rank = 0, nfree = 0;
  std::vector<uint32_t> tab;  // per p-bit: constant, then mw mask words
};

ClampTable build_clamp(const pb_model& m, uint32_t alpha, int mw) {
  const int n = m.n, d = m.d, npb = n * d, nw = n_words(n, d);
  std::vector<int> hp;  // p of the j-th H output
  for (int p = 0; p < npb; ++p)
    if (m.init[p] == 0xFFFFFFFFu) hp.push_back(p);
  const int h = (int)hp.size();
  auto end_state = [&](const std::vector<uint8_t>& x) {
    std::vector<uint8_t> W(nw, 0);
    for (int q = 0; q < n; ++q) W[q] = (uint8_t)((m.beta >> q) & 1u);
    W[ones_idx(n, d)] = 1;
    int j = 0;
    for (int p = 0; p < npb; ++p) {
      const uint32_t e = m.init[p];
      W[n + p] = e == 0xFFFFFFFFu ? x[j++] : (uint8_t)(W[e & 0xFFFFu] ^ W[e >> 16]);
    }
    uint32_t s = 0;
    for (int q = 0; q < n; ++q) s |= (uint32_t)W[d * n + q] << q;
    return s;
  };
  const int words = (h + 1 + 63) / 64;  // augmented row: h columns + right-hand side
  std::vector<std::vector<uint64_t>> row(n, std::vector<uint64_t>(words, 0));
  auto get = [&](int q, int c) { return (int)((row[q][c >> 6] >> (c & 63)) & 1u); };
  auto set = [&](int q, int c) { row[q][c >> 6] |= 1ull << (c & 63); };
  std::vector<uint8_t> x(h, 0);
  const uint32_t c0 = end_state(x);
  for (int j = 0; j < h; ++j) {
    x[j] = 1;
    const uint32_t cj = end_state(x) ^ c0;
    x[j] = 0;
    for (int q = 0; q < n; ++q)
      if ((cj >> q) & 1u) set(q, j);
  }
  for (int q = 0; q < n; ++q)
    if (((alpha ^ c0) >> q) & 1u) set(q, h);
  std::vector<int> pivot;
  int r = 0;
  for (int j = 0; j < h && r < n; ++j) {
    int piv = -1;
    for (int q = r; q < n; ++q)
      if (get(q, j)) { piv = q; break; }
    if (piv < 0) continue;
    std::swap(row[piv], row[r]);
    for (int q = 0; q < n; ++q)
      if (q != r && get(q, j))
        for (int w = 0; w < words; ++w) row[q][w] ^= row[r][w];
    pivot.push_back(j);
    ++r;
  }
  ClampTable t;
  t.rank = r;
  t.ok = true;
  for (int q = r; q < n; ++q)
    if (get(q, h)) t.ok = false;
  std::vector<int> free_of(h, -1), row_of(h, -1);
  for (int i = 0; i < r; ++i) row_of[pivot[i]] = i;
  for (int j = 0; j < h; ++j)
    if (row_of[j] < 0) free_of[j] = t.nfree++;
  t.tab.assign((size_t)npb * (1 + mw), 0u);
  for (int j = 0; j < h; ++j) {
    uint32_t* e = &t.tab[(size_t)hp[j] * (1 + mw)];
    if (free_of[j] >= 0) {
      const int b = free_of[j];
      e[1 + b / 32] |= 1u << (b % 32);
    } else {
      const int i = row_of[j];
      e[0] = (uint32_t)get(i, h);
      for (int c = 0; c < h; ++c)
        if (free_of[c] >= 0 && get(i, c)) e[1 + free_of[c] / 32] |= 1u << (free_of[c] % 32);
    }
  }
  return t;
}

struct Layout {
  size_t hdr = 0, rm = 0, init_ptrs = 0, work = 0, total = 0;
  std::vector<ModelSlots> ms;
};

int check_cfg(const pb_model* m, const pb_run_cfg& c) {
  if (!m) return PB_EINVAL;
  if (c.chains == 0 || c.record_every == 0) return PB_EINVAL;
  if ((uint64_t)c.group0 + (c.chains + 31) / 32 > 0xFFFFFFFFull) return PB_ERANGE;
  if (c.sampler != PB_GIBBS && c.sampler != PB_LEARNED && c.sampler != PB_ELIM &&
      c.sampler != PB_ELIM_CLAMP)
    return PB_EINVAL;
  // the learned proposal: a network for this circuit that the fused kernel
  // takes (its suffix start is drawn on the device), a move period, and a
  // model whose acceptance needs the J energy only
  if (c.sampler == PB_LEARNED) {
    const pb_mlp* mlp = c.proposal;
    if (!mlp || c.mh_every == 0 || m->wgt || mlp->n != m->n || mlp->d != m->d || !mh_fused(mlp))
      return PB_EINVAL;
  }
  if (c.sampler == PB_ELIM_CLAMP && (c.alphas == nullptr || c.n_alphas != 1)) return PB_EINVAL;
  // clamping assumes uniform free outputs: no coupled general gate
  if (c.sampler == PB_ELIM_CLAMP && (m->n_coupled > 0 || m->n_ccx > 0)) return PB_EINVAL;
  // tables: Gibbs only (the exact sampler would need closed-form column sums)
  if (c.sampler != PB_GIBBS && m->n_tab > 0) return PB_EINVAL;
  if (c.alphas == nullptr) {
    if (c.n_alphas != 0) return PB_EINVAL;
    if (m->n > 22) return PB_ERANGE;
  } else {
    if (c.n_alphas <= 0) return PB_EINVAL;
    for (int i = 0; i < c.n_alphas; ++i)
      if (m->n < 32 && (c.alphas[i] >> m->n) != 0) return PB_EINVAL;
  }
  return PB_OK;
}

uint32_t auto_batches(uint32_t groups, uint32_t bins) {
  uint32_t b = std::min<uint32_t>(groups, 32);
  // keep the per-batch histograms within 64 MiB
  while (b > 1 && (uint64_t)b * bins * 64 > (64ull << 20)) b >>= 1;
  return std::max<uint32_t>(b, 1);
}

int plan(pb_model* const* models, const pb_run_cfg* cfgs, int nm, Layout& L) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    size_t at = off;
    off += std::max<size_t>(bytes, 1);
    return at;
  };
  L.hdr = take(sizeof(WsHeader));
  L.rm = take(sizeof(RunModelDev) * nm);
  L.init_ptrs = take(sizeof(uint32_t*) * nm);
  uint32_t total_groups = 0;
  L.ms.resize(nm);
  for (int i = 0; i < nm; ++i) {
    const pb_model* m = models[i];
    const pb_run_cfg& c = cfgs[i];
    int rc = check_cfg(m, c);
    if (rc != PB_OK) return rc;
    ModelSlots& s = L.ms[i];
    const size_t npb = (size_t)m->n * m->d;
    s.groups = (c.chains + 31) / 32;
    s.bins = c.alphas ? (uint32_t)c.n_alphas : (1u << m->n);
    s.n_batches = c.n_batches ? std::min<uint32_t>(c.n_batches, s.groups) : auto_batches(s.groups, s.bins);
    total_groups += s.groups;
    s.model_dev = take(sizeof(ModelDev));
    s.desc = take(npb * sizeof(Desc));
    s.rec = take(npb * sizeof(Rec));
    s.init = take(npb * sizeof(uint32_t));
    s.state = take((size_t)s.groups * npb * 4);
    s.hist = take((size_t)s.n_batches * s.bins * 8 * 8);
    s.valid = take((size_t)s.n_batches * 8);
    s.samples = take((size_t)s.n_batches * 8);
    s.alpha_sorted = take((size_t)(c.alphas ? c.n_alphas : 0) * 4);
    s.alpha_slot = take((size_t)(c.alphas ? c.n_alphas : 0) * 4);
    s.amp = take((size_t)s.bins * 3 * 8);
    s.clamp_mw = c.sampler == PB_ELIM_CLAMP ? std::max(1, (m->h + 31) / 32) : 0;
    s.clamp = take(npb * (size_t)(1 + s.clamp_mw) * 4 * (s.clamp_mw > 0 ? 1 : 0));
    s.cpl = take(m->wgt ? npb * sizeof(Cpl) : 0);
    s.uph = take(m->uph.size() * sizeof(UPh));
    s.glk = take(m->glk.size() * sizeof(GLink));
    s.tacc = take(m->tacc.size() * sizeof(TAcc));
    s.trec = take(m->trec.size() * sizeof(TRec));
    s.mh = take(c.sampler == PB_LEARNED ? mh_region_bytes(m->d, s.groups) : 0);
  }
  L.work = take((size_t)total_groups * 4);
  L.total = align_up(off, 256);
  return PB_OK;
}

}  // namespace

struct pb_run {
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int nm = 0;
  std::vector<std::shared_ptr<pb_model>> models;  // private copies
  std::vector<pb_run_cfg> cfgs;
  Layout L;
  std::vector<RunModelDev> rm;
  uint32_t total_groups = 0;
  int threads = 32;
  int cons = 32, prod = 32, max_col = 1, blocks_per_sm = 0;
  size_t smem = 0;
  bool persistent = false;
  bool wgt = false;        // some model has PB_U gates (the general-gate kernels)
  bool ext = false;        // some model has Toffoli links or two-qubit tables
  bool bal = false;        // plain run with 16 planes ahead, produced evenly over the steps
  bool dec = false;        // (with bal) the recorder outside the colour steps' barriers
  int nc = 2;              // colour steps per sweep (largest over the models)
  bool elim = false;       // exact-sampler run: i.i.d. paths instead of sweeps
  size_t elim_smem = 0;
  int elim_warps = 8;      // exact samplers: warps per CTA (8, 16 or 32)
  std::vector<std::vector<uint32_t>> clamp_keep;
  int grid = 0;
  uint64_t sweeps_done = 0;
  double flips_per_sweep = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t cap_st = nullptr;  // private stream for graph capture (the caller's
                                  // stream may be the legacy default stream)
  bool timed = false;
  double last_flips = 0.0;
  std::map<uint32_t, cudaGraphExec_t> graphs;
  // PB_LEARNED models: their move contexts (mlp == nullptr for the others),
  // the common move period and a device counter of the loop's periods
  std::vector<MhCtx> mh;
  bool learned = false;
  uint32_t mh_every = 0;
  ~pb_run() {
    for (MhCtx& x : mh) mh_ctx_close(x);
  }
  WsHeader* hdr() const { return reinterpret_cast<WsHeader*>(ws + L.hdr); }
  RunModelDev* d_rm() const { return reinterpret_cast<RunModelDev*>(ws + L.rm); }
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PB_OK : PB_ECUDA; }

// The device-side loop of a learned run's launch: the count of move periods
// is set at the start, and the last kernel of each period counts down and
// tells the graph's while node whether to run another.
__global__ void periods_init_kernel(WsHeader* hdr, uint32_t periods) { hdr->periods_left = periods; }
__global__ void periods_step_kernel(WsHeader* hdr, cudaGraphConditionalHandle loop) {
  const uint32_t left = hdr->periods_left - 1u;
  hdr->periods_left = left;
  cudaGraphSetConditional(loop, left > 0u ? 1u : 0u);
}

// The launches of n sweeps of every model (no moves), in stream order.
cudaError_t enqueue_sweeps(pb_run* r, uint32_t n_sweeps, cudaStream_t st) {
  if (r->elim)
    return launch_elim(r->d_rm(), r->nm, r->total_groups,
                       reinterpret_cast<const uint32_t* const*>(r->ws + r->L.init_ptrs), n_sweeps,
                       r->elim_smem, r->hdr(), st, r->wgt, r->elim_warps);
  if (r->persistent)
    return launch_sweeps_persistent(r->d_rm(), r->nm, reinterpret_cast<const uint32_t*>(r->ws + r->L.work),
                                    r->total_groups, n_sweeps, r->cons, r->prod, r->max_col, r->nc,
                                    r->grid, r->smem, r->hdr(), st, r->bal);
  return launch_sweeps(r->d_rm(), r->nm, r->total_groups, n_sweeps, r->cons, r->prod, r->max_col,
                       r->nc, r->smem, r->hdr(), st, r->wgt, r->ext, r->bal, r->dec);
}

// Graph of n sweeps of a learned run (Fig. 2 Step 1 with the network as the
// proposal, interleaved with the heat-bath sweeps): n / mh_every periods of
// [one suffix move of every PB_LEARNED model, mh_every sweeps] run by a
// while node on the device, then n mod mh_every sweeps without a move.
cudaError_t build_learned_graph(pb_run* r, uint32_t n_sweeps, cudaStream_t cap, cudaGraph_t* out) {
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  const uint32_t periods = n_sweeps / r->mh_every, rem = n_sweeps % r->mh_every;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  auto fail = [&](cudaError_t err) {
    cudaGraphDestroy(g);
    return err;
  };
  cudaGraphNode_t last = nullptr;
  if (periods > 0) {
    if ((e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, mode)) != cudaSuccess) return fail(e);
    periods_init_kernel<<<1, 1, 0, cap>>>(r->hdr(), periods);
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) return fail(e != cudaSuccess ? e : e2);
    size_t nn = 1;
    cudaGraphNode_t init = nullptr;
    if ((e = cudaGraphGetNodes(g, &init, &nn)) != cudaSuccess || nn != 1) return fail(cudaErrorUnknown);
    cudaGraphConditionalHandle loop;
    if ((e = cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess)
      return fail(e);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond = nullptr;
    if ((e = cudaGraphAddNode(&cond, g, &init, nullptr, 1, &cp)) != cudaSuccess) return fail(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, mode)) != cudaSuccess)
      return fail(e);
    for (const MhCtx& x : r->mh)
      if (x.mlp && e == cudaSuccess) e = mh_enqueue_move_dev(x, cap);
    if (e == cudaSuccess) e = enqueue_sweeps(r, r->mh_every, cap);
    if (e == cudaSuccess) {
      periods_step_kernel<<<1, 1, 0, cap>>>(r->hdr(), loop);
      e = cudaGetLastError();
    }
    e2 = cudaStreamEndCapture(cap, &body);
    if (e != cudaSuccess || e2 != cudaSuccess) return fail(e != cudaSuccess ? e : e2);
    last = cond;
  }
  if (rem > 0) {
    if ((e = cudaStreamBeginCaptureToGraph(cap, g, last ? &last : nullptr, nullptr, last ? 1 : 0, mode)) !=
        cudaSuccess)
      return fail(e);
    e = enqueue_sweeps(r, rem, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) return fail(e != cudaSuccess ? e : e2);
  }
  *out = g;
  return cudaSuccess;
}

// Applies a CTA shape (consumer and producer threads, multiples of 32) to
// the run: shared-memory size, histogram placement and the persistent grid.
void apply_shape(pb_run* r, int cons, int prod, int blocks_per_sm) {
  int maxcol = 1;
  for (auto& m : r->models)
    for (int c = 0; c < 4; ++c) maxcol = std::max(maxcol, m->col_off[c + 1] - m->col_off[c]);
  r->cons = cons;
  r->prod = prod;
  r->max_col = maxcol;
  r->threads = cons + prod + 32;
  // Shared-memory histograms: counted per CTA, added to the global counters
  // once per launch.  Used when the bins fit (up to 4096 bins for one
  // circuit, 1024 per circuit in a batch so that several CTAs share an SM;
  // 32 bytes a bin, 40 with general gates); otherwise the record adds to
  // global memory directly.
  const size_t cap_bins = r->nm == 1 ? 4096u : 1024u;
  auto layout = [&](bool bal, std::vector<char>& use) {
    size_t smem = 0;
    use.assign(r->nm, 0);
    for (int i = 0; i < r->nm; ++i) {
      const pb_model& m = *r->models[i];
      const uint32_t bins = r->L.ms[i].bins;
      use[i] = bins <= cap_bins &&
               sweep_smem_bytes(m.n, m.d, cons, maxcol, bins, r->wgt, bal) <= kSweepSmemMax;
      smem = std::max(smem, sweep_smem_bytes(m.n, m.d, cons, maxcol, use[i] ? bins : 0, r->wgt, bal));
    }
    return smem;
  };
  r->persistent = r->nm > 1;
  if (const char* e = std::getenv("PB_PERSISTENT")) r->persistent = std::atoi(e) != 0;
  if (r->wgt) r->persistent = false;  // general-gate sweeps: one CTA per group
  // Plain runs take the balanced production (16 planes ahead, three plane
  // buffers) when its tables fit with the same histogram placement and, on
  // a persistent grid, the same CTAs per SM; otherwise 12 planes in two.
  std::vector<char> use_s, use_b;
  const size_t smem_s = layout(false, use_s);
  bool bal = false;
  size_t smem_b = 0;
  if (!r->wgt) {
    smem_b = layout(true, use_b);
    bal = smem_b <= kSweepSmemMax && use_b == use_s && r->threads <= kSweepThreadsBal;
    if (bal && r->persistent)
      bal = sweep_max_blocks_per_sm(r->threads, smem_b, true) >=
            sweep_max_blocks_per_sm(r->threads, smem_s, false);
    if (const char* e = std::getenv("PB_BALANCED")) bal = bal && std::atoi(e) != 0;
  }
  const std::vector<char>& use = bal ? use_b : use_s;
  for (int i = 0; i < r->nm; ++i) r->rm[i].hist_smem = use[i] ? 1u : 0u;
  const size_t smem = bal ? smem_b : smem_s;
  r->bal = bal;
  // the recorder outside the colour steps' barriers where some class takes
  // more than one consumer pass (single-grid plain runs)
  r->dec = bal && !r->wgt && !r->persistent && maxcol > cons;
  r->smem = smem;
  r->grid = 0;
  if (r->persistent) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = sweep_max_blocks_per_sm(r->threads, smem, r->bal);
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
    r->grid = std::max(1, sms * std::max(1, per_sm));
    r->grid = (int)std::min<uint32_t>((uint32_t)r->grid, r->total_groups);
  }
  r->blocks_per_sm = blocks_per_sm;
}

// Default launch shape: consumers = the largest colour class rounded up to
// a warp (one p-bit per consumer per class), capped at 224; producers = one
// per Philox call of a colour step (sweep_producers_wanted), capped at 352,
// or at 224 when the run takes the three-buffer production; plus one
// recorder warp.  Environment overrides PB_CONS, PB_PROD (multiples of 32).
void choose_shape(pb_run* r) {
  int maxcol = 1;
  for (auto& m : r->models)
    for (int c = 0; c < 4; ++c) maxcol = std::max(maxcol, m->col_off[c + 1] - m->col_off[c]);
  auto up32 = [](int x) { return ((x + 31) / 32) * 32; };
  int cons = std::max(32, std::min(224, up32(maxcol)));
  const int want = up32(sweep_producers_wanted(r->models, r->nc, r->wgt));
  int prod = std::max(32, std::min(kProducersMax, want));
  if (const char* e = std::getenv("PB_CONS")) {
    int v = std::atoi(e);
    if (v >= 32 && v <= 224 && v % 32 == 0) cons = v;
  }
  bool fixed_prod = false;
  if (const char* e = std::getenv("PB_PROD")) {
    int v = std::atoi(e);
    if (v >= 32 && v <= 352 && v % 32 == 0) { prod = v; fixed_prod = true; }
  }
  if (r->wgt) prod = std::max(32, std::min(prod, kSweepThreadsWgt - 32 - cons));
  if (!r->wgt && !fixed_prod && prod > kProducersBalanced) {
    // the three-buffer form with its producer count where it applies, else
    // the two-buffer form with the larger one
    apply_shape(r, cons, kProducersBalanced, 0);
    if (r->bal) prod = kProducersBalanced;
    else apply_shape(r, cons, prod, 0);
  } else {
    apply_shape(r, cons, prod, 0);
  }
  // a shape whose tables do not fit: fewer consumers (their class table and
  // acceptance planes shrink; the class runs in more passes)
  while (r->smem > kSweepSmemMax && cons > 32) {
    cons -= 32;
    apply_shape(r, cons, prod, 0);
  }
}

}  // namespace

extern "C" {

PB_API int pb_workspace_bytes(pb_model* const* models, const pb_run_cfg* cfgs, int n_models,
                              size_t* bytes) {
  if (!models || !cfgs || n_models < 1 || !bytes) return PB_EINVAL;
  Layout L;
  int rc = plan(models, cfgs, n_models, L);
  if (rc != PB_OK) return rc;
  *bytes = L.total;
  return PB_OK;
}

PB_API int pb_run_create(pb_model* const* models, const pb_run_cfg* cfgs, int n_models,
                         void* d_workspace, size_t workspace_bytes, uintptr_t stream,
                         pb_run** out) {
  if (!out) return PB_EINVAL;
  *out = nullptr;
  if (!models || !cfgs || n_models < 1 || !d_workspace) return PB_EINVAL;
  if (((uintptr_t)d_workspace & 255u) != 0) return PB_EINVAL;
  std::unique_ptr<pb_run> r(new (std::nothrow) pb_run);
  if (!r) return PB_ENOMEM;
  int rc = plan(models, cfgs, n_models, r->L);
  if (rc != PB_OK) return rc;
  if (workspace_bytes < r->L.total) return PB_ERANGE;
  r->st = reinterpret_cast<cudaStream_t>(stream);
  r->ws = static_cast<char*>(d_workspace);
  r->ws_bytes = workspace_bytes;
  r->nm = n_models;
  r->cfgs.assign(cfgs, cfgs + n_models);
  for (int i = 0; i < n_models; ++i) r->models.emplace_back(new pb_model(*models[i]));
  // one sampler family per run: Gibbs, or the exact samplers
  auto exact = [](int smp) { return smp == PB_ELIM || smp == PB_ELIM_CLAMP; };
  for (int i = 1; i < n_models; ++i)
    if (exact(cfgs[i].sampler) != exact(cfgs[0].sampler)) return PB_EINVAL;
  r->elim = exact(cfgs[0].sampler);
  for (auto& m : r->models) r->wgt = r->wgt || m->wgt;
  for (auto& m : r->models) r->ext = r->ext || m->n_ccx > 0 || m->n_tab > 0;
  for (auto& m : r->models)
    for (int c = 0; c < 4; ++c)
      if (m->col_off[c + 1] > m->col_off[c]) r->nc = std::max(r->nc, c + 1);

  cudaStream_t st = r->st;
  char* ws = r->ws;
  // Zero the header and every counter; tables are uploaded below.
  cudaError_t e = cudaMemsetAsync(ws, 0, r->L.total, st);
  if (e != cudaSuccess) return PB_ECUDA;

  std::vector<const uint32_t*> init_ptrs(n_models);
  std::vector<uint32_t> work;
  std::vector<std::pair<double, uint32_t>> cost;
  uint32_t base = 0;
  r->rm.resize(n_models);
  std::vector<std::vector<uint32_t>> sorted_alpha(n_models);
  std::vector<std::vector<int32_t>> slot_alpha(n_models);
  for (int i = 0; i < n_models; ++i) {
    const pb_model& m = *r->models[i];
    const pb_run_cfg& c = r->cfgs[i];
    const ModelSlots& s = r->L.ms[i];
    ModelDev md{};
    md.n = m.n;
    md.d = m.d;
    md.nw = n_words(m.n, m.d);
    md.h = m.h;
    md.beta = m.beta;
    for (int k = 0; k < 4; ++k) md.thr[k] = m.thr[k];
    for (int k = 0; k < 5; ++k) md.col_off[k] = m.col_off[k];
    md.max_col = 0;
    for (int k = 0; k < 4; ++k) md.max_col = std::max(md.max_col, m.col_off[k + 1] - m.col_off[k]);
    md.wgt = m.wgt ? 1 : 0;
    md.n_ug = (int32_t)m.uph.size();
    md.n_tr = (int32_t)m.trec.size();
    md.log2z = m.n_tab ? 0.0 : m.log2z;  // tables: unit scale, read L2-normalised
    const size_t npb = (size_t)m.n * m.d;
    if ((e = cudaMemcpyAsync(ws + s.model_dev, &md, sizeof md, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + s.desc, m.desc.data(), npb * sizeof(Desc), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + s.rec, m.rec.data(), npb * sizeof(Rec), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + s.init, m.init.data(), npb * 4, cudaMemcpyHostToDevice, st)))
      return PB_ECUDA;
    if (m.wgt &&
        ((e = cudaMemcpyAsync(ws + s.cpl, m.cpl.data(), npb * sizeof(Cpl), cudaMemcpyHostToDevice, st)) ||
         (!m.uph.empty() && (e = cudaMemcpyAsync(ws + s.uph, m.uph.data(), m.uph.size() * sizeof(UPh),
                                                 cudaMemcpyHostToDevice, st))) ||
         (!m.glk.empty() && (e = cudaMemcpyAsync(ws + s.glk, m.glk.data(), m.glk.size() * sizeof(GLink),
                                                 cudaMemcpyHostToDevice, st))) ||
         (!m.tacc.empty() && (e = cudaMemcpyAsync(ws + s.tacc, m.tacc.data(), m.tacc.size() * sizeof(TAcc),
                                                  cudaMemcpyHostToDevice, st))) ||
         (!m.trec.empty() && (e = cudaMemcpyAsync(ws + s.trec, m.trec.data(), m.trec.size() * sizeof(TRec),
                                                  cudaMemcpyHostToDevice, st)))))
      return PB_ECUDA;
    if (c.alphas) {
      std::vector<int32_t> idx(c.n_alphas);
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(),
                       [&](int a, int b) { return c.alphas[a] < c.alphas[b]; });
      for (int k = 0; k < c.n_alphas; ++k) {
        sorted_alpha[i].push_back(c.alphas[idx[k]]);
        slot_alpha[i].push_back(idx[k]);
      }
      // a repeated alpha would split its counts; reject it
      for (int k = 1; k < c.n_alphas; ++k)
        if (sorted_alpha[i][k] == sorted_alpha[i][k - 1]) return PB_EINVAL;
      if ((e = cudaMemcpyAsync(ws + s.alpha_sorted, sorted_alpha[i].data(), c.n_alphas * 4,
                               cudaMemcpyHostToDevice, st)) ||
          (e = cudaMemcpyAsync(ws + s.alpha_slot, slot_alpha[i].data(), c.n_alphas * 4,
                               cudaMemcpyHostToDevice, st)))
        return PB_ECUDA;
    }
    RunModelDev& d = r->rm[i];
    std::memset(&d, 0, sizeof d);
    d.model = reinterpret_cast<const ModelDev*>(ws + s.model_dev);
    d.desc = reinterpret_cast<const Desc*>(ws + s.desc);
    d.rec = reinterpret_cast<const Rec*>(ws + s.rec);
    d.state = reinterpret_cast<uint32_t*>(ws + s.state);
    d.hist = reinterpret_cast<unsigned long long*>(ws + s.hist);
    d.valid = reinterpret_cast<unsigned long long*>(ws + s.valid);
    d.samples = reinterpret_cast<unsigned long long*>(ws + s.samples);
    d.alpha_sorted = reinterpret_cast<const uint32_t*>(ws + s.alpha_sorted);
    d.alpha_slot = reinterpret_cast<const int32_t*>(ws + s.alpha_slot);
    d.amp = reinterpret_cast<double*>(ws + s.amp);
    d.n_alphas = c.alphas ? c.n_alphas : 0;
    d.bins = s.bins;
    d.chains = c.chains;
    d.groups = s.groups;
    d.n_batches = s.n_batches;
    d.burn_in = c.burn_in;
    d.record_every = c.record_every;
    d.seed_lo = (uint32_t)c.seed;
    d.seed_hi = (uint32_t)(c.seed >> 32);
    d.group_base = base;
    d.group0 = c.group0;
    if (m.wgt) {
      d.cpl = reinterpret_cast<const Cpl*>(ws + s.cpl);
      d.uph = reinterpret_cast<const UPh*>(ws + s.uph);
      if (!m.glk.empty()) d.glk = reinterpret_cast<const GLink*>(ws + s.glk);
      if (!m.tacc.empty()) {
        d.tacc = reinterpret_cast<const TAcc*>(ws + s.tacc);
        d.trec = reinterpret_cast<const TRec*>(ws + s.trec);
      }
    }
    if (c.sampler == PB_ELIM_CLAMP) {
      ClampTable t = build_clamp(m, c.alphas[0], s.clamp_mw);
      if ((e = cudaMemcpyAsync(ws + s.clamp, t.tab.data(), t.tab.size() * 4, cudaMemcpyHostToDevice,
                               st)) != cudaSuccess)
        return PB_ECUDA;
      r->clamp_keep.push_back(std::move(t.tab));  // host copy outlives the async copy
      d.clamp_tab = reinterpret_cast<const uint32_t*>(ws + s.clamp);
      d.clamp_mw = s.clamp_mw;
      d.clamp_nfree = t.nfree;
      d.clamp_ok = t.ok ? 1 : 0;
      d.amp_shift = -t.rank;
    }
    init_ptrs[i] = reinterpret_cast<const uint32_t*>(ws + s.init);
    for (uint32_t g = 0; g < s.groups; ++g) cost.push_back({(double)npb, base + g});
    base += s.groups;
    r->flips_per_sweep += (double)c.chains * (double)npb;
  }
  r->total_groups = base;
  // Learned models: one move period for the run; their move regions.
  r->mh.assign(n_models, MhCtx{});
  for (int i = 0; i < n_models; ++i) {
    const pb_run_cfg& c = r->cfgs[i];
    if (c.sampler != PB_LEARNED) continue;
    if (r->learned && c.mh_every != r->mh_every) return PB_EINVAL;
    r->learned = true;
    r->mh_every = c.mh_every;
    MhCtx& x = r->mh[i];
    x.model = r->models[i].get();
    x.mlp = const_cast<pb_mlp*>(c.proposal);
    x.state = r->rm[i].state;
    x.chains = c.chains;
    x.groups = r->L.ms[i].groups;
    x.group0 = c.group0;
    x.seed = c.seed;
    x.ws = ws + r->L.ms[i].mh;
  }
  // Exact samplers: warps per CTA.  Samples are independent, so a CTA with
  // more warps hides more latency; 32 while the groups leave SMs free, 16 up
  // to two groups per SM, else 8 (several CTAs per SM do the same), and
  // fewer when the per-warp images do not fit.
  if (r->elim) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int ew = r->total_groups <= (uint32_t)sms ? 32 : (r->total_groups <= 2u * (uint32_t)sms ? 16 : 8);
    auto smem_for = [&](int w) {
      size_t b = 0;
      for (auto& m : r->models) b = std::max(b, elim_smem_bytes(m->n, m->d, (m->h + 3) & ~3, w));
      return b;
    };
    while (ew > 8 && smem_for(ew) > kSweepSmemMax) ew /= 2;
    r->elim_warps = ew;
    r->elim_smem = smem_for(ew);
  }
  // Work list for the persistent launch: longest first (LPT order).
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<double, uint32_t>& a, const std::pair<double, uint32_t>& b) {
                     return a.first > b.first;
                   });
  for (auto& c : cost) work.push_back(c.second);
  if (sweep_prepare() != cudaSuccess) return PB_ECUDA;
  choose_shape(r.get());
  if (r->smem > kSweepSmemMax || r->elim_smem > kSweepSmemMax) return PB_ERANGE;
  if ((e = cudaMemcpyAsync(ws + r->L.rm, r->rm.data(), sizeof(RunModelDev) * n_models,
                           cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(ws + r->L.init_ptrs, init_ptrs.data(), sizeof(uint32_t*) * n_models,
                           cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(ws + r->L.work, work.data(), work.size() * 4, cudaMemcpyHostToDevice, st)))
    return PB_ECUDA;
  size_t init_smem = 0;
  for (auto& m : r->models) init_smem = std::max(init_smem, (size_t)n_words(m->n, m->d) * 4);
  e = launch_init(r->d_rm(), n_models, r->total_groups,
                  reinterpret_cast<const uint32_t* const*>(ws + r->L.init_ptrs), init_smem,
                  r->hdr(), st);
  if (e != cudaSuccess) return PB_ECUDA;
  if (r->learned) {
    if (mlp_prepare() != cudaSuccess) return PB_ECUDA;
    for (MhCtx& x : r->mh)
      if (x.mlp && (mh_ctx_open(x) != cudaSuccess || mh_region_init(x, st) != cudaSuccess))
        return PB_ECUDA;  // the run's destructor closes what was opened
  }
  // host copies must outlive the (possibly staged) async copies
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PB_ECUDA;
  if (cudaEventCreate(&r->ev0) != cudaSuccess || cudaEventCreate(&r->ev1) != cudaSuccess)
    return PB_ECUDA;
  *out = r.release();
  return PB_OK;
}

PB_API int pb_run_sweeps(pb_run* r, uint32_t n_sweeps) {
  if (!r) return PB_EINVAL;
  if (n_sweeps == 0) return PB_OK;
  if (r->sweeps_done + n_sweeps > 0xFFFFFFFFull) return PB_ERANGE;
  if (n_sweeps > (1u << 26)) return PB_ERANGE;  // per-launch u32 shared counters
  cudaGraphExec_t exec = nullptr;
  auto it = r->graphs.find(n_sweeps);
  if (it != r->graphs.end()) {
    exec = it->second;
  } else {
    cudaGraph_t graph = nullptr;
    if (!r->cap_st && cudaStreamCreateWithFlags(&r->cap_st, cudaStreamNonBlocking) != cudaSuccess)
      return PB_ECUDA;
    cudaError_t e;
    if (r->learned) {
      if (build_learned_graph(r, n_sweeps, r->cap_st, &graph) != cudaSuccess) return PB_ECUDA;
    } else {
      e = cudaStreamBeginCapture(r->cap_st, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return PB_ECUDA;
      e = enqueue_sweeps(r, n_sweeps, r->cap_st);
      cudaError_t e2 = cudaStreamEndCapture(r->cap_st, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return PB_ECUDA;
      }
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return PB_ECUDA;
    r->graphs[n_sweeps] = exec;
  }
  cudaEventRecord(r->ev0, r->st);
  cudaError_t e = cudaGraphLaunch(exec, r->st);
  cudaEventRecord(r->ev1, r->st);
  if (e != cudaSuccess) return PB_ECUDA;
  r->sweeps_done += n_sweeps;
  r->timed = true;
  r->last_flips = r->flips_per_sweep * n_sweeps;
  return PB_OK;
}

PB_API int pb_run_wait(pb_run* r) {
  if (!r) return PB_EINVAL;
  cudaError_t e = cudaStreamSynchronize(r->st);
  if (e != cudaSuccess) return PB_ECUDA;
  uint32_t status = 0;
  e = cudaMemcpy(&status, &r->hdr()->status, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return PB_ECUDA;
  // learned runs: an expired bounded wait in a network's kernels
  for (const MhCtx& x : r->mh) {
    if (!x.mlp || status != 0) continue;
    if (cudaMemcpy(&status, x.mlp->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
  }
  return status == 0 ? PB_OK : (int)status;
}

PB_API int pb_run_moves(pb_run* r, int model, uint64_t* moves, uint64_t* accepted) {
  if (!r || model < 0 || model >= r->nm) return PB_EINVAL;
  const MhCtx& x = r->mh[model];
  if (!x.mlp) return PB_ESTATE;  // not a PB_LEARNED model
  MhCounters c{};
  if (cudaStreamSynchronize(r->st) != cudaSuccess ||
      cudaMemcpy(&c, x.ws, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PB_ECUDA;
  if (moves) *moves = c.moves;
  if (accepted) *accepted = c.accepted;
  return PB_OK;
}

PB_API int pb_run_phase_sums(const pb_run* r, int model, double* re, double* im, uint64_t* counts,
                             uint64_t* valid_total, uint64_t* samples_total) {
  if (!r || model < 0 || model >= r->nm) return PB_EINVAL;
  const ModelSlots& s = r->L.ms[model];
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  std::vector<uint64_t> h((size_t)s.n_batches * s.bins * 8);
  if (cudaMemcpy(h.data(), r->ws + s.hist, h.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PB_ECUDA;
  const bool wgt = r->models[model]->wgt;
  for (uint32_t i = 0; i < s.bins; ++i) {
    double sr = 0.0, si = 0.0;
    uint64_t cn = 0;
    for (uint32_t b = 0; b < s.n_batches; ++b) {
      const uint64_t* c = &h[((size_t)b * s.bins + i) * 8];
      if (wgt) {  // compensated sums: slot 3 / 4 hold the compensations of re / im
        double x, y, cx, cy;
        std::memcpy(&x, &c[0], 8);
        std::memcpy(&y, &c[1], 8);
        std::memcpy(&cx, &c[3], 8);
        std::memcpy(&cy, &c[4], 8);
        sr += x + cx;
        si += y + cy;
        cn += c[2];
      } else {
        for (int k = 0; k < 8; ++k) {
          sr += (double)c[k] * std::cos(M_PI / 4.0 * k);
          si += (double)c[k] * std::sin(M_PI / 4.0 * k);
          cn += c[k];
        }
      }
    }
    if (re) re[i] = sr;
    if (im) im[i] = si;
    if (counts) counts[i] = cn;
  }
  std::vector<uint64_t> v(s.n_batches);
  if (valid_total) {
    if (cudaMemcpy(v.data(), r->ws + s.valid, s.n_batches * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PB_ECUDA;
    *valid_total = std::accumulate(v.begin(), v.end(), (uint64_t)0);
  }
  if (samples_total) {
    if (cudaMemcpy(v.data(), r->ws + s.samples, s.n_batches * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PB_ECUDA;
    *samples_total = std::accumulate(v.begin(), v.end(), (uint64_t)0);
  }
  return PB_OK;
}

PB_API int pb_run_histogram(const pb_run* r, int model, uint64_t* counts, uint64_t* valid_total,
                            uint64_t* samples_total) {
  if (!r || model < 0 || model >= r->nm) return PB_EINVAL;
  const ModelSlots& s = r->L.ms[model];
  if (r->models[model]->wgt && counts) return PB_ESTATE;  // phase sums, not classes
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  if (counts) {
    std::vector<uint64_t> h((size_t)s.n_batches * s.bins * 8);
    if (cudaMemcpy(h.data(), r->ws + s.hist, h.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PB_ECUDA;
    std::memset(counts, 0, (size_t)s.bins * 8 * 8);
    for (uint32_t b = 0; b < s.n_batches; ++b)
      for (size_t i = 0; i < (size_t)s.bins * 8; ++i) counts[i] += h[(size_t)b * s.bins * 8 + i];
  }
  std::vector<uint64_t> v(s.n_batches);
  if (valid_total) {
    if (cudaMemcpy(v.data(), r->ws + s.valid, s.n_batches * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PB_ECUDA;
    *valid_total = std::accumulate(v.begin(), v.end(), (uint64_t)0);
  }
  if (samples_total) {
    if (cudaMemcpy(v.data(), r->ws + s.samples, s.n_batches * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PB_ECUDA;
    *samples_total = std::accumulate(v.begin(), v.end(), (uint64_t)0);
  }
  return PB_OK;
}

PB_API int pb_run_amplitudes(const pb_run* r, int model, int l2_normalize, double* re, double* im,
                             double* se) {
  if (!r || model < 0 || model >= r->nm || !re || !im) return PB_EINVAL;
  if (r->models[model]->n_tab && !l2_normalize) return PB_ESTATE;  // no closed-form scale
  const ModelSlots& s = r->L.ms[model];
  cudaError_t e = launch_amplitudes(r->d_rm(), model, s.bins, l2_normalize, r->st);
  if (e != cudaSuccess) return PB_ECUDA;
  std::vector<double> a((size_t)s.bins * 3);
  e = cudaMemcpyAsync(a.data(), r->ws + s.amp, a.size() * 8, cudaMemcpyDeviceToHost, r->st);
  if (e != cudaSuccess) return PB_ECUDA;
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  for (uint32_t i = 0; i < s.bins; ++i) {
    re[i] = a[(size_t)i * 3];
    im[i] = a[(size_t)i * 3 + 1];
    if (se) se[i] = a[(size_t)i * 3 + 2];
  }
  return PB_OK;
}

PB_API int pb_run_get_state(const pb_run* r, int model, uint32_t* words, size_t bytes) {
  if (!r || model < 0 || model >= r->nm || !words) return PB_EINVAL;
  const ModelSlots& s = r->L.ms[model];
  const size_t need = (size_t)s.groups * r->models[model]->n * r->models[model]->d * 4;
  if (bytes < need) return PB_ERANGE;
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  return cuda_status(cudaMemcpy(words, r->ws + s.state, need, cudaMemcpyDeviceToHost));
}

PB_API int pb_run_set_state(pb_run* r, int model, const uint32_t* words, size_t bytes) {
  if (!r || model < 0 || model >= r->nm || !words) return PB_EINVAL;
  const ModelSlots& s = r->L.ms[model];
  const size_t need = (size_t)s.groups * r->models[model]->n * r->models[model]->d * 4;
  if (bytes < need) return PB_ERANGE;
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  return cuda_status(cudaMemcpy(r->ws + s.state, words, need, cudaMemcpyHostToDevice));
}

// Sets the CTA shape of a run (cached graphs are rebuilt on the next call).
PB_API int pb_run_set_shape(pb_run* r, int consumers, int producers, int blocks_per_sm) {
  if (!r) return PB_EINVAL;
  if (consumers < 32 || consumers > 224 || consumers % 32) return PB_EINVAL;
  if (producers < 32 || producers > 352 || producers % 32) return PB_EINVAL;
  if (blocks_per_sm < 0) return PB_EINVAL;
  if (r->wgt && consumers + producers + 32 > kSweepThreadsWgt) return PB_ERANGE;
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  const int c0 = r->cons, p0 = r->prod, b0 = r->blocks_per_sm;
  apply_shape(r, consumers, producers, blocks_per_sm);
  if (r->smem > kSweepSmemMax) {  // the shape does not fit: keep the old one
    apply_shape(r, c0, p0, b0);
    return PB_ERANGE;
  }
  for (auto& kv : r->graphs) cudaGraphExecDestroy(kv.second);
  r->graphs.clear();
  if (cudaMemcpy(r->ws + r->L.rm, r->rm.data(), sizeof(RunModelDev) * r->nm, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return PB_ECUDA;
  return PB_OK;
}

PB_API int pb_run_get_shape(const pb_run* r, int* consumers, int* producers, int* blocks_per_sm,
                            int* grid) {
  if (!r) return PB_EINVAL;
  if (consumers) *consumers = r->cons;
  if (producers) *producers = r->prod;
  if (blocks_per_sm) *blocks_per_sm = r->blocks_per_sm;
  if (grid) *grid = r->grid;
  return PB_OK;
}

// Autotuner: times `trial_sweeps` sweeps for each candidate CTA shape on the
// run itself, restoring the run's state after every trial, and keeps the
// fastest.  With cache_path, a previous result for the same set of (n, d,
// chains) is reused without trials and new results are appended.
PB_API int pb_run_tune(pb_run* r, uint32_t trial_sweeps, const char* cache_path, double* best_ms) {
  if (!r || trial_sweeps == 0) return PB_EINVAL;
  if (r->elim) {  // one fixed shape
    if (best_ms) *best_ms = 0.0;
    return PB_OK;
  }
  // key: the run's shapes
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
  for (int i = 0; i < r->nm; ++i) {
    mix((uint64_t)r->models[i]->n);
    mix((uint64_t)r->models[i]->d);
    mix((uint64_t)r->cfgs[i].chains);
  }
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      unsigned long long k;
      int c, p, b;
      double ms;
      int found = 0, bc = 0, bp = 0, bb = 0;
      double bms = 0;
      while (std::fscanf(f, "%llx %d %d %d %lf", &k, &c, &p, &b, &ms) == 5)
        if (k == key) { found = 1; bc = c; bp = p; bb = b; bms = ms; }
      std::fclose(f);
      if (found) {
        if (best_ms) *best_ms = bms;
        return pb_run_set_shape(r, bc, bp, bb);
      }
    }
  }
  size_t need = 0;
  int rc = pb_run_checkpoint(r, nullptr, 0, &need);
  if (rc != PB_OK) return rc;
  std::vector<char> blob(need);
  if ((rc = pb_run_checkpoint(r, blob.data(), need, &need)) != PB_OK) return rc;
  const uint64_t sweeps_before = r->sweeps_done;
  int maxcol = 1;
  for (auto& m : r->models)
    for (int c = 0; c < 4; ++c) maxcol = std::max(maxcol, m->col_off[c + 1] - m->col_off[c]);
  const int up = ((maxcol + 31) / 32) * 32;
  std::vector<int> cons_c, prod_c, bpsm_c = {0};
  for (int c : {64, 128, 224})
    if (c <= std::max(64, up)) cons_c.push_back(c);
  const int pw = sweep_producers_wanted(r->models, r->nc, r->wgt);
  for (int p : {96, 192, 224, 352})
    if (p <= std::max(96, ((pw + 31) / 32) * 32)) prod_c.push_back(p);
  if (r->nm > 1) bpsm_c = {1, 2, 0};
  double best = 1e30;
  int bc = r->cons, bp = r->prod, bb = r->blocks_per_sm;
  for (int c : cons_c)
    for (int p : prod_c)
      for (int b : bpsm_c) {
        rc = pb_run_set_shape(r, c, p, b);
        if (rc == PB_ERANGE) continue;  // a shape that does not fit in shared memory
        if (rc != PB_OK) return rc;
        // first launch builds the graph; time the second
        if ((rc = pb_run_sweeps(r, trial_sweeps)) != PB_OK) return rc;
        if ((rc = pb_run_sweeps(r, trial_sweeps)) != PB_OK) return rc;
        pb_run_stats_t st;
        if ((rc = pb_run_stats(r, &st)) != PB_OK) return rc;
        if (st.last_ms < best) { best = st.last_ms; bc = c; bp = p; bb = b; }
        if ((rc = pb_run_restore(r, blob.data(), blob.size())) != PB_OK) return rc;
        r->sweeps_done = sweeps_before;
      }
  if ((rc = pb_run_set_shape(r, bc, bp, bb)) != PB_OK) return rc;
  if (best_ms) *best_ms = best;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%llx %d %d %d %.6f\n", (unsigned long long)key, bc, bp, bb, best);
      std::fclose(f);
    }
  }
  return PB_OK;
}

PB_API int pb_run_stats(pb_run* r, pb_run_stats_t* st) {
  if (!r || !st) return PB_EINVAL;
  st->sweeps_done = r->sweeps_done;
  st->flips = r->flips_per_sweep * (double)r->sweeps_done;
  st->last_ms = 0.0;
  st->flips_per_s = 0.0;
  if (r->timed) {
    if (cudaEventSynchronize(r->ev1) != cudaSuccess) return PB_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r->ev0, r->ev1) != cudaSuccess) return PB_ECUDA;
    st->last_ms = ms;
    st->flips_per_s = ms > 0 ? r->last_flips / (ms * 1e-3) : 0.0;
  }
  return PB_OK;
}

// Checkpoint blob: magic, sweep index, then per model: state, hist, valid, samples.
PB_API int pb_run_checkpoint(const pb_run* r, void* host_buf, size_t bytes, size_t* bytes_needed) {
  if (!r) return PB_EINVAL;
  size_t need = 16;
  for (int i = 0; i < r->nm; ++i) {
    const ModelSlots& s = r->L.ms[i];
    need += (size_t)s.groups * r->models[i]->n * r->models[i]->d * 4 +
            (size_t)s.n_batches * s.bins * 64 + (size_t)s.n_batches * 16 +
            (r->mh[i].mlp ? sizeof(MhCounters) : 0);  // learned: the move counters
  }
  if (bytes_needed) *bytes_needed = need;
  if (!host_buf) return PB_OK;
  if (bytes < need) return PB_ERANGE;
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  char* p = static_cast<char*>(host_buf);
  uint64_t magic = 0x706269747343504bull;  // "pbitsCPK"
  std::memcpy(p, &magic, 8);
  uint64_t sw = r->sweeps_done;
  std::memcpy(p + 8, &sw, 8);
  p += 16;
  for (int i = 0; i < r->nm; ++i) {
    const ModelSlots& s = r->L.ms[i];
    const size_t sb = (size_t)s.groups * r->models[i]->n * r->models[i]->d * 4;
    const size_t hb = (size_t)s.n_batches * s.bins * 64;
    if (cudaMemcpy(p, r->ws + s.state, sb, cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
    p += sb;
    if (cudaMemcpy(p, r->ws + s.hist, hb, cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
    p += hb;
    if (cudaMemcpy(p, r->ws + s.valid, s.n_batches * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
    p += s.n_batches * 8;
    if (cudaMemcpy(p, r->ws + s.samples, s.n_batches * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
    p += s.n_batches * 8;
    if (r->mh[i].mlp) {
      if (cudaMemcpy(p, r->mh[i].ws, sizeof(MhCounters), cudaMemcpyDeviceToHost) != cudaSuccess) return PB_ECUDA;
      p += sizeof(MhCounters);
    }
  }
  return PB_OK;
}

PB_API int pb_run_restore(pb_run* r, const void* host_buf, size_t bytes) {
  if (!r || !host_buf) return PB_EINVAL;
  size_t need = 0;
  int rc = pb_run_checkpoint(r, nullptr, 0, &need);
  if (rc != PB_OK) return rc;
  if (bytes < need) return PB_ERANGE;
  const char* p = static_cast<const char*>(host_buf);
  uint64_t magic = 0, sw = 0;
  std::memcpy(&magic, p, 8);
  std::memcpy(&sw, p + 8, 8);
  if (magic != 0x706269747343504bull || sw > 0xFFFFFFFFull) return PB_EINVAL;
  p += 16;
  if (cudaStreamSynchronize(r->st) != cudaSuccess) return PB_ECUDA;
  for (int i = 0; i < r->nm; ++i) {
    const ModelSlots& s = r->L.ms[i];
    const size_t sb = (size_t)s.groups * r->models[i]->n * r->models[i]->d * 4;
    const size_t hb = (size_t)s.n_batches * s.bins * 64;
    if (cudaMemcpy(r->ws + s.state, p, sb, cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
    p += sb;
    if (cudaMemcpy(r->ws + s.hist, p, hb, cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
    p += hb;
    if (cudaMemcpy(r->ws + s.valid, p, s.n_batches * 8, cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
    p += s.n_batches * 8;
    if (cudaMemcpy(r->ws + s.samples, p, s.n_batches * 8, cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
    p += s.n_batches * 8;
    if (r->mh[i].mlp) {
      if (cudaMemcpy(r->mh[i].ws, p, sizeof(MhCounters), cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
      p += sizeof(MhCounters);
    }
  }
  uint32_t sw32 = (uint32_t)sw;
  if (cudaMemcpy(&r->hdr()->sweep0, &sw32, 4, cudaMemcpyHostToDevice) != cudaSuccess) return PB_ECUDA;
  r->sweeps_done = sw;
  return PB_OK;
}

PB_API void pb_run_free(pb_run* r) {
  if (!r) return;
  cudaStreamSynchronize(r->st);
  for (auto& kv : r->graphs) cudaGraphExecDestroy(kv.second);
  if (r->cap_st) cudaStreamDestroy(r->cap_st);
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
  delete r;
}

}  // extern "C"

namespace pb {
int run_view(const pb_run* r, int model, RunView* out) {
  if (!r || !out || model < 0 || model >= r->nm) return PB_EINVAL;
  if (r->elim) return PB_EINVAL;  // moves act on Gibbs chains
  // the learned move's acceptance knows the J energy only
  if (r->models[model]->wgt) return PB_EINVAL;
  out->st = r->st;
  out->state = r->rm[model].state;
  out->model = r->models[model].get();
  out->chains = r->cfgs[model].chains;
  out->groups = r->rm[model].groups;
  out->group0 = r->cfgs[model].group0;
  out->seed = r->cfgs[model].seed;
  return PB_OK;
}
}  // namespace pb

extern "C" {

PB_API int pb_philox_fill(const uint32_t* d_ctr, uint32_t k0, uint32_t k1, uint32_t count,
                          uint32_t* d_out, uintptr_t stream) {
  if ((!d_ctr || !d_out) && count) return PB_EINVAL;
  cudaError_t e = launch_philox_fill(d_ctr, k0, k1, count, d_out, reinterpret_cast<cudaStream_t>(stream));
  return cuda_status(e);
}

}  // extern "C"
