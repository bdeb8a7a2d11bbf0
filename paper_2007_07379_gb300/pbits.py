"""Python binding of the C ABI in ``include/pbits.h`` (ctypes; marshalling only).

Every step of the sampler runs in ``libpbits.so``; PyTorch supplies device
memory (the run workspace) and the CUDA stream.  Loading fails loudly when
the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpbits.so")

PB_OK, PB_EINVAL, PB_ERANGE, PB_ENOMEM, PB_ECUDA, PB_ETIMEOUT, PB_ESTATE = 0, -1, -2, -3, -4, -5, -6
PB_GIBBS, PB_LEARNED, PB_ELIM, PB_ELIM_CLAMP = 0, 1, 2, 3
PB_U, PB_X, PB_U2, PB_CCX = 5, 6, 7, 8

_lib = None


class PbError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code) if _lib else code} ({code})")


class pb_gate(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("layer", ctypes.c_int32), ("q0", ctypes.c_int32),
                ("q1", ctypes.c_int32), ("q2", ctypes.c_int32)]


class pb_model_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("d", ctypes.c_int32), ("n_pbits", ctypes.c_int32),
                ("h", ctypes.c_int32), ("M", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("J", ctypes.c_double), ("input_bits", ctypes.c_uint32),
                ("thr", ctypes.c_uint32 * 4), ("colour_size", ctypes.c_int32 * 4),
                ("n_u", ctypes.c_int32), ("n_coupled", ctypes.c_int32), ("log2z", ctypes.c_double)]


class pb_run_cfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("chains", ctypes.c_uint32), ("burn_in", ctypes.c_uint32),
                ("record_every", ctypes.c_uint32), ("n_batches", ctypes.c_uint32),
                ("alphas", ctypes.POINTER(ctypes.c_uint32)), ("n_alphas", ctypes.c_int32),
                ("sampler", ctypes.c_int32), ("proposal", ctypes.c_void_p),
                ("mh_every", ctypes.c_uint32), ("group0", ctypes.c_uint32)]


class pb_run_stats_t(ctypes.Structure):
    _fields_ = [("sweeps_done", ctypes.c_uint64), ("flips", ctypes.c_double),
                ("last_ms", ctypes.c_double), ("flips_per_s", ctypes.c_double)]


# Exported entry points: name -> (restype, argtypes).  Tests check that the
# library exports every one of them.
_VP = ctypes.c_void_p
_SIGS = {
    "pb_version": (ctypes.c_int, []),
    "pb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pb_compile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(pb_gate), ctypes.c_int,
                                  ctypes.c_uint32, ctypes.c_double, ctypes.POINTER(_VP)]),
    "pb_compile_u": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(pb_gate), ctypes.c_int,
                                    _VP, ctypes.c_uint32, ctypes.c_double, ctypes.POINTER(_VP)]),
    "pb_compile_g": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(pb_gate), ctypes.c_int,
                                    _VP, ctypes.c_int, ctypes.c_uint32, ctypes.c_double,
                                    ctypes.POINTER(_VP)]),
    "pb_model_info": (ctypes.c_int, [_VP, ctypes.POINTER(pb_model_info_t)]),
    "pb_model_colours": (ctypes.c_int, [_VP, _VP]),
    "pb_model_free": (None, [_VP]),
    "pb_workspace_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(pb_run_cfg), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "pb_run_create": (ctypes.c_int, [_VP, ctypes.POINTER(pb_run_cfg), ctypes.c_int, _VP,
                                     ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(_VP)]),
    "pb_run_sweeps": (ctypes.c_int, [_VP, ctypes.c_uint32]),
    "pb_run_wait": (ctypes.c_int, [_VP]),
    "pb_run_moves": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(ctypes.c_uint64)]),
    "pb_run_histogram": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "pb_run_phase_sums": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "pb_run_amplitudes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "pb_run_get_state": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_size_t]),
    "pb_run_set_state": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_size_t]),
    "pb_run_stats": (ctypes.c_int, [_VP, ctypes.POINTER(pb_run_stats_t)]),
    "pb_run_checkpoint": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "pb_run_restore": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "pb_run_free": (None, [_VP]),
    "pb_run_set_shape": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pb_run_get_shape": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pb_run_tune": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]),
    "pb_philox_fill": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _VP,
                                      ctypes.c_void_p]),
    "pb_gibbs_run_noalloc": (ctypes.c_int, [_VP, ctypes.POINTER(pb_run_cfg), ctypes.c_uint32, _VP, _VP,
                                            ctypes.c_void_p]),
    "pb_mlp_workspace_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "pb_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     _VP, ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(_VP)]),
    "pb_mlp_info": (ctypes.c_int, [_VP, _VP]),
    "pb_mlp_status": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "pb_selftest_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, _VP]),
    "pb_mlp_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "pb_mlp_grads": (ctypes.c_int, [_VP, _VP]),
    "pb_mlp_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    "pb_mlp_backward": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "pb_mlp_forward_fused": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    "pb_mlp_adam": (ctypes.c_int, [_VP, ctypes.c_float]),
    "pb_mlp_free": (None, [_VP]),
    "pb_mh_workspace_bytes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "pb_mh_create": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)]),
    "pb_mh_moves": (ctypes.c_int, [_VP, ctypes.c_uint32]),
    "pb_mh_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "pb_mh_free": (None, [_VP]),
    "pb_run_collect_paths": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_size_t, _VP, ctypes.c_uint64,
                                            _VP]),
    "pb_mlp_train_paths": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_float, ctypes.c_uint64, _VP]),
    "pb_shor_workspace_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]),
    "pb_shor_columns": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _VP, ctypes.c_uint32,
                                       _VP, ctypes.c_size_t, _VP, _VP, ctypes.c_void_p]),
    "pb_shor_peaks": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, _VP, ctypes.c_size_t, _VP,
                                     ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "pb_gemm_bf16": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_float, ctypes.c_void_p]),
}


def load(path: str = LIB_PATH):
    """Load libpbits.so (raises if it is missing: build it with
    ``python -m paper_2007_07379_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: the CUDA library has not been built "
                      "(python -m paper_2007_07379_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue  # reported by exported_symbols()
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols(path: str = LIB_PATH) -> dict[str, bool]:
    lib = ctypes.CDLL(path)
    return {name: hasattr(lib, name) for name in _SIGS}


def selftest_wait(arrive: bool, max_iters: int) -> int:
    """The library's bounded mbarrier wait on its own (pb_selftest_wait):
    PB_OK when the barrier was arrived on, PB_ETIMEOUT when it was not."""
    v = ctypes.c_int(0)
    _check(load().pb_selftest_wait(1 if arrive else 0, ctypes.c_uint32(max_iters), ctypes.byref(v)),
           "pb_selftest_wait")
    return v.value


def strerror(code: int) -> str:
    return load().pb_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != PB_OK:
        raise PbError(rc, what)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def gate_array(gates) -> ctypes.Array:
    """Gate rows (op, layer, q0, q1[, q2]) as pb_gate structs (q2 = -1 when
    the rows have four columns)."""
    g = np.asarray(gates, dtype=np.int32)
    if g.size == 0:
        g = np.zeros((0, 5), dtype=np.int32)
    elif g.ndim == 1:
        g = g.reshape(-1, 4)
    arr = (pb_gate * max(len(g), 1))()
    for i, row in enumerate(g):
        q2 = int(row[4]) if len(row) > 4 else -1
        arr[i] = pb_gate(int(row[0]), int(row[1]), int(row[2]), int(row[3]), q2)
    return arr, len(g)


def mat_array(n_gates: int, mats, mats2=None) -> np.ndarray:
    """Gate matrices as the float64 rows of pb_compile_g: one-qubit matrices
    (complex [n_gates, 2, 2], rows = output bit) in the first 8 entries of a
    row; with mats2 (complex [n_gates, 4, 4], basis index x_{q0} + 2 x_{q1})
    32 entries per row, the 4x4 row-major."""
    w = 32 if mats2 is not None else 8
    m = np.zeros((max(n_gates, 1), w), dtype=np.float64)
    if mats is not None and n_gates:
        c = np.asarray(mats, dtype=np.complex128).reshape(n_gates, 4)
        m[:n_gates, 0:8:2] = c.real
        m[:n_gates, 1:8:2] = c.imag
    if mats2 is not None and n_gates:
        c2 = np.asarray(mats2, dtype=np.complex128).reshape(n_gates, 16)
        m[:n_gates, 0::2] = np.where(np.abs(c2) > 0, c2.real, m[:n_gates, 0::2])
        m[:n_gates, 1::2] = np.where(np.abs(c2) > 0, c2.imag, m[:n_gates, 1::2])
    return np.ascontiguousarray(m)


class Model:
    """A compiled circuit (pb_compile; pb_compile_u when `mats` gives the
    matrices of PB_U gates, complex [n_gates, 2, 2])."""

    def __init__(self, n: int, d: int, gates, J: float, input_bits: int = 0, mats=None,
                 mats2=None):
        lib = load()
        arr, ng = gate_array(gates)
        h = ctypes.c_void_p()
        g5 = np.asarray(gates)
        toffoli = g5.size > 0 and g5.ndim == 2 and np.any(g5[:, 0] == PB_CCX)
        if mats is None and mats2 is None and not toffoli:
            _check(lib.pb_compile(n, d, arr, ng, ctypes.c_uint32(input_bits), ctypes.c_double(J),
                                  ctypes.byref(h)), "pb_compile")
        else:
            m = mat_array(ng, mats, mats2)
            _check(lib.pb_compile_g(n, d, arr, ng, _ptr(m), m.shape[1], ctypes.c_uint32(input_bits),
                                    ctypes.c_double(J), ctypes.byref(h)), "pb_compile_g")
        self._h = h
        self.n, self.d = n, d

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = pb_model_info_t()
        _check(load().pb_model_info(self._h, ctypes.byref(inf)), "pb_model_info")
        return {"n": inf.n, "d": inf.d, "n_pbits": inf.n_pbits, "h": inf.h, "M": inf.M,
                "rank": inf.rank, "J": inf.J, "input_bits": inf.input_bits,
                "thr": list(inf.thr), "colour_size": list(inf.colour_size),
                "n_u": inf.n_u, "n_coupled": inf.n_coupled, "log2z": inf.log2z}

    def colours(self) -> np.ndarray:
        out = np.zeros((self.d, self.n), dtype=np.int32)
        _check(load().pb_model_colours(self._h, _ptr(out)), "pb_model_colours")
        return out

    def close(self):
        if self._h:
            load().pb_model_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class RunCfg:
    seed: int
    chains: int
    burn_in: int = 0
    record_every: int = 1
    n_batches: int = 0
    alphas: np.ndarray | None = None
    sampler: int = PB_GIBBS
    proposal: object = None
    mh_every: int = 1
    group0: int = 0


def _cfg_array(cfgs: list[RunCfg]):
    arr = (pb_run_cfg * len(cfgs))()
    keep = []
    for i, c in enumerate(cfgs):
        al = None
        if c.alphas is not None:
            al = np.ascontiguousarray(c.alphas, dtype=np.uint32)
            keep.append(al)
        arr[i] = pb_run_cfg(c.seed & ((1 << 64) - 1), c.chains, c.burn_in, c.record_every, c.n_batches,
                            al.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if al is not None else None,
                            0 if al is None else len(al), c.sampler,
                            c.proposal.handle if c.proposal is not None else None, c.mh_every,
                            c.group0)
    return arr, keep


def workspace_bytes(models: list[Model], cfgs: list[RunCfg]) -> int:
    lib = load()
    mh = (ctypes.c_void_p * len(models))(*[m.handle.value for m in models])
    ca, keep = _cfg_array(cfgs)
    out = ctypes.c_size_t(0)
    _check(lib.pb_workspace_bytes(mh, ca, len(models), ctypes.byref(out)), "pb_workspace_bytes")
    return out.value


class Run:
    """A set of chains on the GPU (pb_run_create ... pb_run_free).

    The workspace is a torch uint8 CUDA tensor owned by this object; the
    stream is torch's current stream unless one is given.
    """

    def __init__(self, models: list[Model], cfgs: list[RunCfg], stream=None, workspace=None):
        import torch
        lib = load()
        self.models = list(models)
        self.cfgs = list(cfgs)
        nbytes = workspace_bytes(self.models, self.cfgs)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if workspace.numel() < nbytes or workspace.data_ptr() % 256:
            raise ValueError("workspace too small or not 256-byte aligned")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        mh = (ctypes.c_void_p * len(models))(*[m.handle.value for m in models])
        ca, keep = _cfg_array(self.cfgs)
        h = ctypes.c_void_p()
        _check(lib.pb_run_create(mh, ca, len(models), ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel(), ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(h)), "pb_run_create")
        self._h = h

    def bins(self, model: int = 0) -> int:
        c = self.cfgs[model]
        return len(c.alphas) if c.alphas is not None else (1 << self.models[model].n)

    def groups(self, model: int = 0) -> int:
        return (self.cfgs[model].chains + 31) // 32

    def sweeps(self, n: int):
        _check(load().pb_run_sweeps(self._h, n), "pb_run_sweeps")

    def wait(self):
        _check(load().pb_run_wait(self._h), "pb_run_wait")

    def moves(self, model: int = 0):
        """(moves done, proposals accepted) of a PB_LEARNED model."""
        mv, acc = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load().pb_run_moves(self._h, model, ctypes.byref(mv), ctypes.byref(acc)), "pb_run_moves")
        return mv.value, acc.value

    def histogram(self, model: int = 0):
        cnt = np.zeros((self.bins(model), 8), dtype=np.uint64)
        v = ctypes.c_uint64(0)
        s = ctypes.c_uint64(0)
        _check(load().pb_run_histogram(self._h, model, _ptr(cnt), ctypes.byref(v), ctypes.byref(s)),
               "pb_run_histogram")
        return cnt, v.value, s.value

    def phase_sums(self, model: int = 0):
        """(sums complex[bins] = sum of e^{i arg U_C} over valid samples per bin,
        counts u64[bins], valid, samples) -- any model."""
        b = self.bins(model)
        re, im = np.zeros(b), np.zeros(b)
        cnt = np.zeros(b, dtype=np.uint64)
        v = ctypes.c_uint64(0)
        s = ctypes.c_uint64(0)
        _check(load().pb_run_phase_sums(self._h, model, _ptr(re), _ptr(im), _ptr(cnt), ctypes.byref(v),
                                        ctypes.byref(s)), "pb_run_phase_sums")
        return re + 1j * im, cnt, v.value, s.value

    def amplitudes(self, model: int = 0, l2_normalize: bool = False):
        b = self.bins(model)
        re, im, se = np.zeros(b), np.zeros(b), np.zeros(b)
        _check(load().pb_run_amplitudes(self._h, model, int(l2_normalize), _ptr(re), _ptr(im), _ptr(se)),
               "pb_run_amplitudes")
        return re + 1j * im, se

    def get_state(self, model: int = 0) -> np.ndarray:
        m = self.models[model]
        out = np.zeros((self.groups(model), m.d, m.n), dtype=np.uint32)
        _check(load().pb_run_get_state(self._h, model, _ptr(out), out.nbytes), "pb_run_get_state")
        return out

    def set_state(self, words: np.ndarray, model: int = 0):
        w = np.ascontiguousarray(words, dtype=np.uint32)
        _check(load().pb_run_set_state(self._h, model, _ptr(w), w.nbytes), "pb_run_set_state")

    def stats(self) -> dict:
        st = pb_run_stats_t()
        _check(load().pb_run_stats(self._h, ctypes.byref(st)), "pb_run_stats")
        return {"sweeps_done": st.sweeps_done, "flips": st.flips, "last_ms": st.last_ms,
                "flips_per_s": st.flips_per_s}

    def set_shape(self, consumers: int, producers: int, blocks_per_sm: int = 0):
        _check(load().pb_run_set_shape(self._h, consumers, producers, blocks_per_sm), "pb_run_set_shape")

    def shape(self) -> dict:
        v = [ctypes.c_int(0) for _ in range(4)]
        _check(load().pb_run_get_shape(self._h, *[ctypes.byref(x) for x in v]), "pb_run_get_shape")
        return {"consumers": v[0].value, "producers": v[1].value, "blocks_per_sm": v[2].value,
                "grid": v[3].value}

    def tune(self, trial_sweeps: int = 200, cache_path: str | None = None) -> float:
        ms = ctypes.c_double(0)
        _check(load().pb_run_tune(self._h, trial_sweeps, cache_path.encode() if cache_path else None,
                                  ctypes.byref(ms)), "pb_run_tune")
        return ms.value

    def checkpoint(self) -> bytes:
        lib = load()
        need = ctypes.c_size_t(0)
        _check(lib.pb_run_checkpoint(self._h, None, 0, ctypes.byref(need)), "pb_run_checkpoint")
        buf = np.zeros(need.value, dtype=np.uint8)
        _check(lib.pb_run_checkpoint(self._h, _ptr(buf), buf.nbytes, ctypes.byref(need)),
               "pb_run_checkpoint")
        return buf.tobytes()

    def restore(self, blob: bytes):
        buf = np.frombuffer(blob, dtype=np.uint8).copy()
        _check(load().pb_run_restore(self._h, _ptr(buf), buf.nbytes), "pb_run_restore")

    def close(self):
        if getattr(self, "_h", None):
            load().pb_run_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unslice_state(words: np.ndarray, chains: int) -> np.ndarray:
    """Chain-sliced words [groups, d, n] -> per-chain layer words [chains, d]
    (bit q of row k-1 = p-bit (k, q)).  Pure data movement."""
    G, d, n = words.shape
    out = np.zeros((G * 32, d), dtype=np.uint32)
    for q in range(n):
        bits = ((words[:, :, q][:, None, :] >> np.arange(32, dtype=np.uint32)[None, :, None]) & 1)
        out |= (bits.reshape(G * 32, d).astype(np.uint32) << np.uint32(q))
    return out[:chains]


def slice_state(per_chain: np.ndarray, n: int) -> np.ndarray:
    """Inverse of unslice_state (chains padded with zero to a multiple of 32)."""
    C, d = per_chain.shape
    G = (C + 31) // 32
    pad = np.zeros((G * 32, d), dtype=np.uint32)
    pad[:C] = per_chain
    pad = pad.reshape(G, 32, d)
    out = np.zeros((G, d, n), dtype=np.uint32)
    for q in range(n):
        bits = (pad >> np.uint32(q)) & 1  # [G, 32, d]
        out[:, :, q] = np.sum(bits.astype(np.uint64) << np.arange(32, dtype=np.uint64)[None, :, None],
                              axis=1).astype(np.uint32)
    return out


def philox_fill(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32-10 of each counter row on the device (test hook)."""
    import torch
    c = torch.as_tensor(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32)).cuda()
    out = torch.empty_like(c)
    st = torch.cuda.current_stream()
    _check(load().pb_philox_fill(ctypes.c_void_p(c.data_ptr()), key[0], key[1], c.shape[0],
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)),
           "pb_philox_fill")
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def gibbs_run_noalloc(model: Model, cfg: RunCfg, n_sweeps: int, counts, totals, stream=None):
    """One plain Gibbs run whose scratch is the library's fixed device array
    (pb_gibbs_run_noalloc).  `counts` (2^n * 8) and `totals` (2) are the
    caller's int64 CUDA tensors; they hold the histogram and (valid, samples)
    once the stream reaches the end of the call."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    ca, keep = _cfg_array([cfg])
    _check(load().pb_gibbs_run_noalloc(model.handle, ca, n_sweeps, ctypes.c_void_p(counts.data_ptr()),
                                       ctypes.c_void_p(totals.data_ptr()),
                                       ctypes.c_void_p(st.cuda_stream)), "pb_gibbs_run_noalloc")


EPI_RELU, EPI_OUT_BF16, EPI_ACCUM, EPI_MASK = 1, 2, 4, 8


def gemm_bf16(A, B, D, bias=None, mask=None, flags: int = 0, alpha: float = 1.0, stream=None):
    """D = epilogue(alpha * A @ B^T) on the tensor cores (pb_gemm_bf16).
    A [M, K], B [N, K] bf16 CUDA tensors (row-major); D [M, N] fp32 or bf16."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    M, K = A.shape
    N = B.shape[0]
    _check(load().pb_gemm_bf16(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                               B.stride(0), ctypes.c_void_p(D.data_ptr()), D.stride(0),
                               ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
                               ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
                               mask.stride(0) if mask is not None else 0, M, N, K, flags, alpha,
                               ctypes.c_void_p(st.cuda_stream)), "pb_gemm_bf16")


class Mlp:
    """The proposal network (pb_mlp_*); workspace is a torch CUDA tensor."""

    def __init__(self, n: int, d: int, hidden: int = 256, batch: int = 4096, seed: int = 1, stream=None):
        import torch
        lib = load()
        nb = ctypes.c_size_t(0)
        _check(lib.pb_mlp_workspace_bytes(n, d, hidden, batch, ctypes.byref(nb)), "pb_mlp_workspace_bytes")
        self.workspace = torch.zeros(nb.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.pb_mlp_create(n, d, hidden, batch, ctypes.c_uint64(seed), ctypes.c_void_p(self.workspace.data_ptr()),
                                 nb.value, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "pb_mlp_create")
        self._h = h
        dims = np.zeros(6, dtype=np.int32)
        _check(lib.pb_mlp_info(h, _ptr(dims)), "pb_mlp_info")
        self.n, self.d, self.hidden, self.k_in, self.batch, self.n_params = [int(x) for x in dims]
        self.npad = ((n + 15) // 16) * 16

    @property
    def handle(self):
        return self._h

    def params(self) -> dict:
        flat = np.zeros(self.n_params, dtype=np.float32)
        _check(load().pb_mlp_params(self._h, _ptr(flat), 1), "pb_mlp_params")
        return self._unflat(flat)

    def set_params(self, p: dict):
        _check(load().pb_mlp_params(self._h, _ptr(self._flat(p)), 0), "pb_mlp_params")

    def status(self, clear: bool = False) -> int:
        """PB_OK, or PB_ETIMEOUT once a bounded wait in one of the network's
        kernels ran out (pb_mlp_status; synchronizes the network's stream)."""
        v = ctypes.c_int(0)
        _check(load().pb_mlp_status(self._h, 1 if clear else 0, ctypes.byref(v)), "pb_mlp_status")
        return v.value

    def grads(self) -> dict:
        flat = np.zeros(self.n_params, dtype=np.float32)
        _check(load().pb_mlp_grads(self._h, _ptr(flat)), "pb_mlp_grads")
        return self._unflat(flat)

    def _shapes(self):
        H, k, npd = self.hidden, self.k_in, self.npad
        return [("W1", (H, k)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (npd, H)), ("b3", (npd,))]

    def _unflat(self, flat):
        out, o = {}, 0
        for name, shp in self._shapes():
            size = int(np.prod(shp))
            out[name] = flat[o:o + size].reshape(shp).astype(np.float64)
            o += size
        return out

    def _flat(self, p):
        return np.concatenate([np.asarray(p[name], dtype=np.float32).reshape(-1) for name, _ in self._shapes()])

    def forward(self, x_bf16):
        import torch
        rows = x_bf16.shape[0]
        out = torch.empty(rows, self.n, dtype=torch.float32, device="cuda")
        _check(load().pb_mlp_forward(self._h, ctypes.c_void_p(x_bf16.data_ptr()), rows,
                                     ctypes.c_void_p(out.data_ptr())), "pb_mlp_forward")
        return out

    def forward_fused(self, x_bf16):
        import torch
        rows = x_bf16.shape[0]
        out = torch.empty(rows, self.n, dtype=torch.float32, device="cuda")
        _check(load().pb_mlp_forward_fused(self._h, ctypes.c_void_p(x_bf16.data_ptr()), rows,
                                           ctypes.c_void_p(out.data_ptr())), "pb_mlp_forward_fused")
        return out

    def backward(self, x_bf16, target):
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        _check(load().pb_mlp_backward(self._h, ctypes.c_void_p(x_bf16.data_ptr()),
                                      ctypes.c_void_p(target.data_ptr()), x_bf16.shape[0],
                                      ctypes.c_void_p(loss.data_ptr())), "pb_mlp_backward")
        return loss

    def adam(self, lr: float):
        _check(load().pb_mlp_adam(self._h, ctypes.c_float(lr)), "pb_mlp_adam")

    def close(self):
        if getattr(self, "_h", None):
            load().pb_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Learned:
    """Learned-proposal sampler on one model of a run (pb_mh_*): path
    collection, Metropolis-Hastings suffix moves with the network."""

    def __init__(self, run: Run, mlp: Mlp, model: int = 0):
        import torch
        self.run, self.mlp, self.model = run, mlp, model
        nb = ctypes.c_size_t(0)
        _check(load().pb_mh_workspace_bytes(run._h, model, ctypes.byref(nb)), "pb_mh_workspace_bytes")
        self.workspace = torch.zeros(nb.value, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check(load().pb_mh_create(run._h, model, mlp.handle, ctypes.c_void_p(self.workspace.data_ptr()),
                                   self.workspace.numel(), ctypes.byref(h)), "pb_mh_create")
        self._h = h

    def step(self, n_moves: int = 1):
        _check(load().pb_mh_moves(self._h, n_moves), "pb_mh_moves")

    def stats(self):
        mv, acc = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load().pb_mh_stats(self._h, ctypes.byref(mv), ctypes.byref(acc)), "pb_mh_stats")
        return mv.value, acc.value

    @property
    def moves(self):
        return self.stats()[0]

    @property
    def accepted(self):
        return self.stats()[1]

    @property
    def proposed(self):
        return self.stats()[0] * self.run.cfgs[self.model].chains

    def collect(self, paths, count):
        """Append the valid chain paths to `paths` (int32 [cap, d] CUDA tensor);
        `count` is an int64 [1] CUDA tensor holding the fill level."""
        _check(load().pb_run_collect_paths(self.run._h, self.model, ctypes.c_void_p(self.workspace.data_ptr()),
                                           self.workspace.numel(), ctypes.c_void_p(paths.data_ptr()),
                                           paths.shape[0], ctypes.c_void_p(count.data_ptr())),
               "pb_run_collect_paths")

    def close(self):
        if getattr(self, "_h", None):
            load().pb_mh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def train_on_paths(mlp: Mlp, paths, n_paths: int, beta: int, steps: int, rows: int, lr: float, seed: int):
    """Adam steps on uniform (path, layer) batches; returns the per-step losses."""
    import torch
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    _check(load().pb_mlp_train_paths(mlp.handle, ctypes.c_void_p(paths.data_ptr()), n_paths, beta, steps,
                                     rows, ctypes.c_float(lr), ctypes.c_uint64(seed),
                                     ctypes.c_void_p(losses.data_ptr())), "pb_mlp_train_paths")
    return losses


class ShorColumns:
    """Column sampling of the period-finding circuit (pb_shor_columns): the
    device buffers (torch) and the calls."""

    def __init__(self, n: int, T: int, stream=None):
        import torch
        lib = load()
        self.n, self.T = n, T
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nb = ctypes.c_size_t(0)
        _check(lib.pb_shor_workspace_bytes(n, T, ctypes.byref(nb)), "pb_shor_workspace_bytes")
        self.ws = torch.empty(max(nb.value, 256 + 8 * 4096), dtype=torch.uint8, device="cuda")
        self.prob = torch.empty(1 << n, dtype=torch.float64, device="cuda")

    def run(self, N: int, a: int, x, want_y: bool = False):
        """Fills self.prob (device); returns y_i (host u64) when want_y."""
        xs = np.ascontiguousarray(x, dtype=np.uint32)
        assert len(xs) == self.T
        y = np.zeros(self.T, dtype=np.uint64) if want_y else None
        _check(load().pb_shor_columns(ctypes.c_uint64(N), ctypes.c_uint64(a), self.n, _ptr(xs),
                                      ctypes.c_uint32(self.T), ctypes.c_void_p(self.ws.data_ptr()),
                                      self.ws.numel(), ctypes.c_void_p(self.prob.data_ptr()),
                                      None if y is None else _ptr(y),
                                      ctypes.c_void_p(self.stream.cuda_stream)), "pb_shor_columns")
        return y

    def peaks(self, threshold: float, max_positions: int = 4096):
        """(count, positions u64 (first max_positions, increasing), max prob)."""
        pos = np.zeros(max(max_positions, 1), dtype=np.uint64)
        c = ctypes.c_uint32(0)
        mx = ctypes.c_double(0.0)
        _check(load().pb_shor_peaks(ctypes.c_void_p(self.prob.data_ptr()), self.n, ctypes.c_double(threshold),
                                    ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), _ptr(pos),
                                    ctypes.c_uint32(max_positions), ctypes.byref(c), ctypes.byref(mx),
                                    ctypes.c_void_p(self.stream.cuda_stream)), "pb_shor_peaks")
        return c.value, pos[:min(c.value, max_positions)], mx.value
