"""Host-side checks of the C ABI (no GPU): the library loads, exports every
entry point that include/pbits.h declares, and its circuit compiler agrees
with the oracle's independent derivations."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import build, pbits
from paper_2007_07379_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pbits.load()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"PB_API\s+[^;(]*?\b(pb_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert len(names) >= 18
    import ctypes
    lib = ctypes.CDLL(pbits.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert names <= set(pbits._SIGS), names - set(pbits._SIGS)


@pytest.mark.parametrize("n,d,seed", [(3, 4, 0), (12, 20, 1000), (16, 24, 3000), (24, 32, 4000), (7, 13, 5)])
def test_compile_matches_oracle(n, d, seed):
    g = W.random_circuit(n, d, seed)
    J = W.default_J(n, d, g)
    m = pbits.Model(n, d, g, J)
    info = m.info()
    h, rank = oracle.gf2_rank(n, d, g)
    assert info["h"] == h and info["rank"] == rank and info["M"] == n * d - h
    assert info["n_pbits"] == n * (d + 1)
    assert list(info["thr"]) == [int(x) for x in oracle.thresholds(J)]
    assert np.array_equal(m.colours(), oracle.colour(n, d, g))
    assert sum(info["colour_size"]) == n * d


def test_compile_rejects_bad_input():
    ok = np.array([(W.H, 0, 0, -1)], dtype=np.int32)
    with pytest.raises(pbits.PbError) as e:
        pbits.Model(33, 4, ok, 3.0)
    assert e.value.code == pbits.PB_ERANGE
    with pytest.raises(pbits.PbError) as e:
        pbits.Model(2, 65, ok, 3.0)
    assert e.value.code == pbits.PB_ERANGE
    bad = [
        [(7, 0, 0, -1)],                     # unknown op
        [(W.H, 0, 2, -1)],                   # qubit out of range
        [(W.H, 0, 0, -1), (W.S, 0, 0, -1)],  # qubit used twice in a layer
        [(W.CNOT, 0, 1, 1)],                 # control == target
        [(W.CZ, 3, 0, 1)],                   # layer out of range
    ]
    for rows in bad:
        with pytest.raises(pbits.PbError) as e:
            pbits.Model(2, 2, np.array(rows, dtype=np.int32), 3.0)
        assert e.value.code == pbits.PB_EINVAL
    with pytest.raises(pbits.PbError):
        pbits.Model(2, 2, ok, -1.0)
    with pytest.raises(pbits.PbError):
        pbits.Model(2, 2, ok, 3.0, input_bits=4)


def test_workspace_sizing_and_cfg_checks():
    g = W.random_circuit(5, 6, 1)
    m = pbits.Model(5, 6, g, 3.0)
    b1 = pbits.workspace_bytes([m], [pbits.RunCfg(seed=1, chains=64)])
    b2 = pbits.workspace_bytes([m], [pbits.RunCfg(seed=1, chains=6400)])
    assert b2 > b1 > 0 and b1 % 256 == 0
    with pytest.raises(pbits.PbError):
        pbits.workspace_bytes([m], [pbits.RunCfg(seed=1, chains=0)])
    with pytest.raises(pbits.PbError):
        pbits.workspace_bytes([m], [pbits.RunCfg(seed=1, chains=32, record_every=0)])
    with pytest.raises(pbits.PbError):
        pbits.workspace_bytes([m], [pbits.RunCfg(seed=1, chains=32, alphas=np.array([40], np.uint32))])


def test_slice_roundtrip():
    rng = np.random.default_rng(0)
    per = rng.integers(0, 1 << 7, size=(70, 5), dtype=np.uint32)
    w = pbits.slice_state(per, 7)
    assert w.shape == (3, 5, 7)
    assert np.array_equal(pbits.unslice_state(w, 70), per)


@pytest.mark.parametrize("n,d,seed", [(3, 5, 4), (6, 10, 8), (12, 20, 1000), (5, 8, 21)])
def test_compile_general_gates_matches_oracle(n, d, seed):
    """X and two-qubit permutation gates: the colour classes (the sweep
    order the parity tests rely on) equal the oracle's; info counts them."""
    g, m2 = W.random_two_qubit_circuit(n, d, seed, frac=0.8)
    m = pbits.Model(n, d, g, 3.0, mats2=m2)
    assert np.array_equal(m.colours(), oracle.u_colour(n, d, g, None, m2))
    inf = m.info()
    assert inf["n_u"] == int(np.sum(g[:, 0] == W.U2))
    assert inf["log2z"] == 0.5 * int(np.sum(g[:, 0] == W.H))
    gu, mu = W.random_general_circuit(n, d, seed, frac_u=0.4)
    mm = pbits.Model(n, d, gu, 3.0, mats=mu)
    assert np.array_equal(mm.colours(), oracle.u_colour(n, d, gu, mu))


def test_compile_rejects_unrepresentable_two_qubit_gates():
    g = np.array([[W.U2, 0, 0, 1]], dtype=np.int32)
    m = np.zeros((4, 4), dtype=np.complex128)
    for x in range(4):
        x1, x2 = x & 1, x >> 1
        m[(1 ^ x1 ^ x2) | (x2 << 1), x] = 1
    for bad in (m, 2 * W.swap_matrix()):
        with pytest.raises(pbits.PbError):
            pbits.Model(2, 1, g, 3.0, mats2=bad[None])
    pbits.Model(2, 1, g, 3.0, mats2=W.swap_matrix()[None])
    # a non-permutation unitary is a table gate (Eq. ET2): no closed-form scale
    h = np.kron(np.eye(2), np.array([[1, 1], [1, -1]]) / np.sqrt(2))
    assert np.isnan(pbits.Model(2, 1, g, 3.0, mats2=h[None]).info()["log2z"])


@pytest.mark.parametrize("n,d,seed", [(3, 5, 2), (6, 8, 5), (12, 20, 1000)])
def test_compile_table_gates_matches_oracle(n, d, seed):
    g, m2 = W.random_table_circuit(n, d, seed)
    m = pbits.Model(n, d, g, 3.0, mats2=m2)
    assert np.array_equal(m.colours(), oracle.u_colour(n, d, g, None, m2))
    assert np.isnan(m.info()["log2z"])


@pytest.mark.parametrize("n,d,seed", [(4, 5, 2), (6, 8, 3), (12, 20, 1000)])
def test_compile_toffoli_matches_oracle(n, d, seed):
    g = W.random_ccx_circuit(n, d, seed, frac=0.9)
    assert np.sum(g[:, 0] == W.CCX) > 0
    m = pbits.Model(n, d, g, 3.0)
    assert np.array_equal(m.colours(), oracle.u_colour(n, d, g))
    assert m.info()["rank"] == -1


def test_selftest_wait_rejects_bad_arguments_before_any_launch():
    """Argument checks of pb_selftest_wait come before any CUDA call."""
    import ctypes
    lib = pbits.load()
    v = ctypes.c_int(7)
    assert lib.pb_selftest_wait(0, ctypes.c_uint32(0), ctypes.byref(v)) == pbits.PB_EINVAL
    assert lib.pb_selftest_wait(0, ctypes.c_uint32((1 << 20) + 1), ctypes.byref(v)) == pbits.PB_EINVAL
    assert lib.pb_selftest_wait(1, ctypes.c_uint32(10), None) == pbits.PB_EINVAL
    assert lib.pb_mlp_status(None, 0, ctypes.byref(v)) == pbits.PB_EINVAL
    assert v.value == 7
