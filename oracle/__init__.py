"""CPU oracle for the p-bit Feynman-path sampler (arXiv 2007.07379).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; never by the product
package.  It shares no code with the CUDA library.  ``oracle.c`` holds the
plain C implementation (FP64 state vector, exact path sum, reference Gibbs
sampler, Philox4x32-10); this module compiles it with gcc on first use and
wraps it with ctypes.  ``mlp.py`` holds the FP64 numpy MLP reference.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "general.c"), os.path.join(_HERE, "shor.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

H, S, T, CNOT, CZ, U, X, U2, CCX = 0, 1, 2, 3, 4, 5, 6, 7, 8


def build(force: bool = False) -> str:
    """Compile oracle.c, general.c and shor.c into liboracle.so (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < max(os.path.getmtime(s) for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
             "-fPIC", "-shared"] + _SRCS + ["-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.orc_philox4x32_10.restype = None
            for name in ("orc_statevector", "orc_pathsum_exact", "orc_gf2_rank", "orc_reach",
                         "orc_colour", "orc_gibbs", "orc_elim", "orc_elim_clamped", "orc_violations", "orc_path_phase",
                         "orc_thresholds", "orc_u_statevector", "orc_u_pathstats", "orc_u_gibbs",
                         "orc_u_elim", "orc_u_log2z", "orc_shor_columns", "orc_shor_prob_at",
                         "orc_u_colour"):
                getattr(lib, name).restype = ctypes.c_int
            lib.orc_modexp.restype = ctypes.c_uint64
            lib.orc_modexp.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _gates(gates) -> np.ndarray:
    """Gate rows (op, layer, q0, q1[, q2]) as int32 [n, 5] (q2 = -1 when absent)."""
    a = np.asarray(gates, dtype=np.int32)
    if a.size == 0:
        return np.zeros((0, 5), dtype=np.int32)
    if a.ndim == 1:
        a = a.reshape(-1, 4)
    if a.shape[1] == 4:
        a = np.concatenate([a, -np.ones((len(a), 1), dtype=np.int32)], axis=1)
    return np.ascontiguousarray(a)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def statevector(n: int, d: int, gates, beta: int = 0) -> np.ndarray:
    """FP64 state vector psi_alpha = U_{alpha,beta} (Eq. U), complex128[2^n]."""
    lib = _load()
    g = _gates(gates)
    re = np.zeros(1 << n)
    im = np.zeros(1 << n)
    rc = lib.orc_statevector(n, d, _p(g), len(g), ctypes.c_uint32(beta), _p(re), _p(im))
    if rc != 0:
        raise ValueError(f"orc_statevector failed ({rc})")
    return re + 1j * im


def pathsum_exact(n: int, d: int, gates, beta: int = 0):
    """Exact path sum: (cnt int64[2^n, 8], h); U_alpha = 2^{-h/2} sum_b cnt[alpha,b] w^b."""
    lib = _load()
    g = _gates(gates)
    cnt = np.zeros((1 << n, 8), dtype=np.int64)
    h = ctypes.c_int(0)
    rc = lib.orc_pathsum_exact(n, d, _p(g), len(g), ctypes.c_uint32(beta), _p(cnt), ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"orc_pathsum_exact failed ({rc})")
    return cnt, h.value


def phase_counts_to_complex(cnt: np.ndarray, h: int) -> np.ndarray:
    """2^{-h/2} sum_b cnt[..., b] e^{i pi b / 4} in FP64."""
    w = np.exp(1j * np.pi * np.arange(8) / 4.0)
    return (cnt.astype(np.float64) @ w) * 2.0 ** (-h / 2.0)


def gf2_rank(n: int, d: int, gates):
    """(h, rank) of the GF(2) map from H outputs to the last layer."""
    lib = _load()
    g = _gates(gates)
    h = ctypes.c_int(0)
    r = ctypes.c_int(0)
    rc = lib.orc_gf2_rank(n, d, _p(g), len(g), ctypes.byref(h), ctypes.byref(r))
    if rc != 0:
        raise ValueError(f"orc_gf2_rank failed ({rc})")
    return h.value, r.value


def valid_paths_per_output(n: int, d: int, gates, alphas=None, beta: int = 0) -> np.ndarray:
    """N_alpha, the number of valid paths ending at alpha (float64; 2^{h-rank}
    for an output in the affine image of the H outputs, else 0), for every
    alpha in `alphas` (default: all 2^n outputs)."""
    lib = _load()
    g = _gates(gates)
    h = ctypes.c_int(0)
    r = ctypes.c_int(0)
    c = ctypes.c_uint32(0)
    masks = np.zeros(32, dtype=np.uint32)
    rc = lib.orc_reach(n, d, _p(g), len(g), ctypes.c_uint32(beta), ctypes.byref(h), ctypes.byref(r),
                       ctypes.byref(c), _p(masks))
    if rc != 0:
        raise ValueError(f"orc_reach failed ({rc})")
    a = np.arange(1 << n, dtype=np.uint64) if alphas is None else np.asarray(alphas, dtype=np.uint64)
    x = a ^ np.uint64(c.value)
    ok = np.ones(len(a), dtype=bool)
    for m in masks[:n - r.value]:
        v = x & np.uint64(m)
        par = np.zeros(len(a), dtype=np.uint64)
        while np.any(v):
            par ^= v & np.uint64(1)
            v >>= np.uint64(1)
        ok &= par == 0
    return np.where(ok, 2.0 ** (h.value - r.value), 0.0)


def thresholds(J: float) -> np.ndarray:
    lib = _load()
    thr = np.zeros(4, dtype=np.uint32)
    rc = lib.orc_thresholds(ctypes.c_double(J), _p(thr))
    if rc != 0:
        raise ValueError("bad J")
    return thr


def colour(n: int, d: int, gates) -> np.ndarray:
    """Colour class (0..3) of every p-bit, shape [d, n] (row k-1 = layer k):
    the sweep visits the classes in increasing order."""
    lib = _load()
    g = _gates(gates)
    col = np.zeros((d, n), dtype=np.int32)
    rc = lib.orc_colour(n, d, _p(g), len(g), _p(col))
    if rc <= 0:
        raise ValueError("orc_colour failed")
    return col


def gibbs(n: int, d: int, gates, *, J: float, seed: int, chains: int, sweeps: int,
          beta: int = 0, chain0: int = 0, sweep0: int = 0, burn_in: int = 0,
          record_every: int = 1, state: np.ndarray | None = None, alphas=None):
    """Reference Gibbs run.  Returns dict(state[chains, d] u32, cnt[bins, 8] u64,
    valid, samples).  ``state=None`` starts from fresh valid paths (init=1)."""
    lib = _load()
    g = _gates(gates)
    init = 1 if state is None else 0
    st = np.zeros((chains, d), dtype=np.uint32) if state is None else \
        np.ascontiguousarray(state, dtype=np.uint32).copy()
    assert st.shape == (chains, d)
    if alphas is None:
        bins = 1 << n
        al = None
    else:
        al = np.ascontiguousarray(alphas, dtype=np.uint32)
        bins = len(al)
    cnt = np.zeros((bins, 8), dtype=np.uint64)
    valid = ctypes.c_uint64(0)
    samples = ctypes.c_uint64(0)
    rc = lib.orc_gibbs(n, d, _p(g), len(g), ctypes.c_uint32(beta), ctypes.c_double(J),
                       ctypes.c_uint64(seed), ctypes.c_uint32(chain0), ctypes.c_uint32(chains),
                       ctypes.c_uint32(sweep0), ctypes.c_uint32(sweeps), ctypes.c_uint32(burn_in),
                       ctypes.c_uint32(record_every), init, _p(st),
                       None if al is None else _p(al), 0 if al is None else len(al),
                       _p(cnt), ctypes.byref(valid), ctypes.byref(samples))
    if rc != 0:
        raise ValueError(f"orc_gibbs failed ({rc})")
    return {"state": st, "cnt": cnt, "valid": valid.value, "samples": samples.value}


def elim(n: int, d: int, gates, *, seed: int, chains: int, sweeps: int, beta: int = 0,
         chain0: int = 0, sweep0: int = 0, burn_in: int = 0, record_every: int = 1, alphas=None):
    """Exact i.i.d. path sampler on the eliminated network (R2).  Returns
    dict(state[chains, d] u32 = each chain's last drawn path, cnt[bins, 8]
    u64, valid, samples)."""
    lib = _load()
    g = _gates(gates)
    st = np.zeros((chains, d), dtype=np.uint32)
    if alphas is None:
        bins = 1 << n
        al = None
    else:
        al = np.ascontiguousarray(alphas, dtype=np.uint32)
        bins = len(al)
    cnt = np.zeros((bins, 8), dtype=np.uint64)
    valid = ctypes.c_uint64(0)
    samples = ctypes.c_uint64(0)
    rc = lib.orc_elim(n, d, _p(g), len(g), ctypes.c_uint32(beta), ctypes.c_uint64(seed),
                      ctypes.c_uint32(chain0), ctypes.c_uint32(chains), ctypes.c_uint32(sweep0),
                      ctypes.c_uint32(sweeps), ctypes.c_uint32(burn_in), ctypes.c_uint32(record_every),
                      _p(st), None if al is None else _p(al), 0 if al is None else len(al),
                      _p(cnt), ctypes.byref(valid), ctypes.byref(samples))
    if rc != 0:
        raise ValueError(f"orc_elim failed ({rc})")
    return {"state": st, "cnt": cnt, "valid": valid.value, "samples": samples.value}


def elim_clamped(n: int, d: int, gates, *, alpha: int, seed: int, chains: int, sweeps: int,
                 beta: int = 0, chain0: int = 0, sweep0: int = 0, burn_in: int = 0,
                 record_every: int = 1):
    """Exact sampler with the end state clamped to alpha.  Returns
    dict(state, cnt[8] u64, samples, consistent, nfree, rank)."""
    lib = _load()
    g = _gates(gates)
    st = np.zeros((chains, d), dtype=np.uint32)
    cnt = np.zeros(8, dtype=np.uint64)
    samples = ctypes.c_uint64(0)
    cons, nfree, rank = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rc = lib.orc_elim_clamped(n, d, _p(g), len(g), ctypes.c_uint32(beta), ctypes.c_uint32(alpha),
                              ctypes.c_uint64(seed), ctypes.c_uint32(chain0), ctypes.c_uint32(chains),
                              ctypes.c_uint32(sweep0), ctypes.c_uint32(sweeps), ctypes.c_uint32(burn_in),
                              ctypes.c_uint32(record_every), _p(st), _p(cnt), ctypes.byref(samples),
                              ctypes.byref(cons), ctypes.byref(nfree), ctypes.byref(rank))
    if rc != 0:
        raise ValueError(f"orc_elim_clamped failed ({rc})")
    return {"state": st, "cnt": cnt, "samples": samples.value, "consistent": bool(cons.value),
            "nfree": nfree.value, "rank": rank.value}


def clamped_amplitude(cnt8: np.ndarray, samples: int, h: int, rank: int) -> complex:
    """2^{h/2 - r} sum_phi cnt[phi] w^phi / T (0 when nothing was drawn)."""
    if samples == 0:
        return 0j
    w = np.exp(1j * np.pi / 4 * np.arange(8))
    return complex(2.0 ** (h / 2 - rank) * np.sum(np.asarray(cnt8, dtype=np.float64) * w) / samples)


def violations(n: int, d: int, gates, state: np.ndarray, beta: int = 0) -> np.ndarray:
    lib = _load()
    g = _gates(gates)
    st = np.ascontiguousarray(state, dtype=np.uint32)
    out = np.zeros(st.shape[0], dtype=np.int32)
    rc = lib.orc_violations(n, d, _p(g), len(g), ctypes.c_uint32(beta), ctypes.c_uint32(st.shape[0]),
                            _p(st), _p(out))
    if rc != 0:
        raise ValueError("orc_violations failed")
    return out


def path_phase(n: int, d: int, gates, path, beta: int = 0) -> int:
    lib = _load()
    g = _gates(gates)
    p = np.ascontiguousarray(path, dtype=np.uint32)
    return lib.orc_path_phase(n, d, _p(g), len(g), ctypes.c_uint32(beta), _p(p))


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(t: int) -> int:
    """Threads of the oracle's OpenMP loops from now on; returns the count."""
    return _load().orc_set_num_threads(int(t))


def estimate_amplitudes(cnt: np.ndarray, valid: int, h: int) -> np.ndarray:
    """Eq. U23 with uniform valid paths: psi_hat = 2^{h/2} sum_b cnt[.,b] w^b / valid."""
    w = np.exp(1j * np.pi * np.arange(8) / 4.0)
    return (cnt.astype(np.float64) @ w) * (2.0 ** (h / 2.0)) / max(valid, 1)


# ---- general one-qubit gates (general.c)

def _mats(gates, mats, mats2=None) -> np.ndarray:
    """Gate matrices as float64 [n_gates, 32]: a U row's first 8 entries are
    Re/Im of U00, U01, U10, U11 (rows = output bit, from `mats` [ng, 2, 2]);
    a U2 row holds Re/Im of its 4x4 matrix row-major (from `mats2`
    [ng, 4, 4], basis index x_{q0} + 2 x_{q1}); other rows are ignored."""
    g = _gates(gates)
    m = np.zeros((len(g), 32), dtype=np.float64)
    if mats is not None:
        c = np.asarray(mats, dtype=np.complex128).reshape(len(g), 4)
        m[:, 0:8:2] = c.real
        m[:, 1:8:2] = c.imag
    if mats2 is not None:
        c2 = np.asarray(mats2, dtype=np.complex128).reshape(len(g), 16)
        rows = g[:, 0] == U2
        m[rows, 0::2] = c2[rows].real
        m[rows, 1::2] = c2[rows].imag
    return np.ascontiguousarray(m)


def u_statevector(n: int, d: int, gates, mats, beta: int = 0, mats2=None) -> np.ndarray:
    """FP64 state vector of a circuit with general gates (ops U, X, U2)."""
    lib = _load()
    g = _gates(gates)
    m = _mats(g, mats, mats2)
    re = np.zeros(1 << n)
    im = np.zeros(1 << n)
    rc = lib.orc_u_statevector(n, d, _p(g), len(g), _p(m), ctypes.c_uint32(beta), _p(re), _p(im))
    if rc != 0:
        raise ValueError(f"orc_u_statevector failed ({rc})")
    return re + 1j * im


def u_pathstats(n: int, d: int, gates, mats, beta: int = 0, mats2=None) -> dict:
    """Brute-force path sum per output: U (complex), zabs = sum |U_C|,
    s2 = sum |U_C|^2, npath = nonzero paths; std_weighted = sqrt(zabs^2 - |U|^2)
    and std_uniform = sqrt(npath s2 - |U|^2) (Eq. U30, paths to each output)."""
    lib = _load()
    g = _gates(gates)
    m = _mats(g, mats, mats2)
    N = 1 << n
    ure, uim, zabs, s2 = (np.zeros(N) for _ in range(4))
    npath = np.zeros(N, dtype=np.uint64)
    rc = lib.orc_u_pathstats(n, d, _p(g), len(g), _p(m), ctypes.c_uint32(beta), _p(ure), _p(uim),
                             _p(zabs), _p(s2), _p(npath))
    if rc != 0:
        raise ValueError(f"orc_u_pathstats failed ({rc})")
    U = ure + 1j * uim
    a2 = np.abs(U) ** 2
    return {"U": U, "zabs": zabs, "s2": s2, "npath": npath,
            "std_weighted": np.sqrt(np.maximum(zabs ** 2 - a2, 0.0)),
            "std_uniform": np.sqrt(np.maximum(npath.astype(np.float64) * s2 - a2, 0.0))}


def u_log2z(n: int, d: int, gates, mats, mats2=None) -> float:
    lib = _load()
    g = _gates(gates)
    m = _mats(g, mats, mats2)
    out = ctypes.c_double(0.0)
    rc = lib.orc_u_log2z(n, d, _p(g), len(g), _p(m), ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"orc_u_log2z failed ({rc})")
    return out.value


def _u_run(fn, n, d, gates, mats, chains, alphas, extra_args, state_arg, mats2=None):
    lib = _load()
    g = _gates(gates)
    m = _mats(g, mats, mats2)
    if alphas is None:
        bins, al = 1 << n, None
    else:
        al = np.ascontiguousarray(alphas, dtype=np.uint32)
        bins = len(al)
    sre, sim = np.zeros(bins), np.zeros(bins)
    cnt = np.zeros(bins, dtype=np.uint64)
    valid, samples, l2z = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_double(0.0)
    rc = getattr(lib, fn)(n, d, _p(g), len(g), _p(m), *extra_args, state_arg,
                          None if al is None else _p(al), 0 if al is None else len(al),
                          _p(sre), _p(sim), _p(cnt), ctypes.byref(valid), ctypes.byref(samples),
                          ctypes.byref(l2z))
    if rc != 0:
        raise ValueError(f"{fn} failed ({rc})")
    return {"sum": sre + 1j * sim, "cnt": cnt, "valid": valid.value, "samples": samples.value,
            "log2z": l2z.value}


def u_gibbs(n: int, d: int, gates, mats, *, J: float, seed: int, chains: int, sweeps: int,
            beta: int = 0, chain0: int = 0, sweep0: int = 0, burn_in: int = 0,
            record_every: int = 1, state: np.ndarray | None = None, alphas=None,
            mats2=None) -> dict:
    """Reference Gibbs run with general one-qubit gates (proposal by heat-bath
    on the J energy, Metropolis acceptance on the coupling energy).  Returns
    dict(state, sum = sum of e^{i arg U_C} per bin, cnt, valid, samples, log2z);
    psi = 2^log2z sum / valid."""
    init = 1 if state is None else 0
    st = np.zeros((chains, d), dtype=np.uint32) if state is None else \
        np.ascontiguousarray(state, dtype=np.uint32).copy()
    args = (ctypes.c_uint32(beta), ctypes.c_double(J), ctypes.c_uint64(seed), ctypes.c_uint32(chain0),
            ctypes.c_uint32(chains), ctypes.c_uint32(sweep0), ctypes.c_uint32(sweeps),
            ctypes.c_uint32(burn_in), ctypes.c_uint32(record_every), init)
    out = _u_run("orc_u_gibbs", n, d, gates, mats, chains, alphas, args, _p(st), mats2)
    out["state"] = st
    return out


def u_elim(n: int, d: int, gates, mats, *, seed: int, chains: int, sweeps: int, beta: int = 0,
           chain0: int = 0, sweep0: int = 0, burn_in: int = 0, record_every: int = 1,
           alphas=None, mats2=None) -> dict:
    """Exact i.i.d. sampler with general one-qubit gates; outputs as u_gibbs
    (state = each chain's last drawn path)."""
    st = np.zeros((chains, d), dtype=np.uint32)
    args = (ctypes.c_uint32(beta), ctypes.c_uint64(seed), ctypes.c_uint32(chain0),
            ctypes.c_uint32(chains), ctypes.c_uint32(sweep0), ctypes.c_uint32(sweeps),
            ctypes.c_uint32(burn_in), ctypes.c_uint32(record_every))
    out = _u_run("orc_u_elim", n, d, gates, mats, chains, alphas, args, _p(st), mats2)
    out["state"] = st
    return out


def u_estimate(run: dict) -> np.ndarray:
    """psi_hat = 2^log2z * (sum of phases) / valid (Eq. U23 with p_C ~ |U_C|)."""
    return run["sum"] * (2.0 ** run["log2z"]) / max(run["valid"], 1)


# ---- column sampling of the period-finding circuit (shor.c)

def modexp(a: int, x: int, N: int) -> int:
    return int(_load().orc_modexp(a, x, N))


def shor_columns(N: int, a: int, n: int, x) -> tuple[np.ndarray, np.ndarray]:
    """prob[k] = sum_y |sum_{i: y_i = y} 2^{-n/2} e^{2 pi i k x_i / 2^n}|^2 / T for
    k < 2^n (n <= 24), and y_i = a^{x_i} mod N."""
    lib = _load()
    xs = np.ascontiguousarray(x, dtype=np.uint32)
    prob = np.zeros(1 << n)
    y = np.zeros(len(xs), dtype=np.uint64)
    rc = lib.orc_shor_columns(ctypes.c_uint64(N), ctypes.c_uint64(a), n, _p(xs),
                              ctypes.c_uint32(len(xs)), _p(prob), _p(y))
    if rc != 0:
        raise ValueError(f"orc_shor_columns failed ({rc})")
    return prob, y


def shor_prob_at(N: int, a: int, n: int, x, ks) -> np.ndarray:
    """prob at the given k values (any n <= 32)."""
    lib = _load()
    xs = np.ascontiguousarray(x, dtype=np.uint32)
    kk = np.ascontiguousarray(ks, dtype=np.uint64)
    out = np.zeros(len(kk))
    rc = lib.orc_shor_prob_at(ctypes.c_uint64(N), ctypes.c_uint64(a), n, _p(xs),
                              ctypes.c_uint32(len(xs)), _p(kk), ctypes.c_uint32(len(kk)), _p(out))
    if rc != 0:
        raise ValueError(f"orc_shor_prob_at failed ({rc})")
    return out


def u_colour(n: int, d: int, gates, mats=None, mats2=None) -> np.ndarray:
    """Colour classes [d, n] of a general circuit (the sweep order)."""
    lib = _load()
    g = _gates(gates)
    m = _mats(g, mats, mats2)
    col = np.zeros((d, n), dtype=np.int32)
    rc = lib.orc_u_colour(n, d, _p(g), len(g), _p(m), _p(col))
    if rc <= 0:
        raise ValueError("orc_u_colour failed")
    return col
