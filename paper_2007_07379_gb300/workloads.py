"""Seeded synthetic inputs: random Clifford+T circuits and the five workloads.

This module holds input generation only (no sampling, energy or phase
arithmetic).  The CUDA path and the CPU oracle both take its gate lists.

Generator (the paper names no circuit family; this is the stated reading):
per layer, the qubits are visited in a seeded random order; each qubit not yet
used in the layer draws a gate uniformly from {H, S, T, CNOT, CZ}; a 2-qubit
draw takes a partner uniformly among the still-free qubits (CNOT control and
target in random order); with no free partner the draw is redone among the
1-qubit gates.  Every qubit is acted on once per layer.  Randomness is
SplitMix64(seed).

A gate is the row ``(op, layer, q0, q1)``: ``op`` in H=0, S=1, T=2, CNOT=3,
CZ=4; ``layer`` in ``[0, d)`` maps the state after ``layer`` gate layers to
the next; for CNOT ``q0`` is the control and ``q1`` the target; a 1-qubit gate
has ``q1 = -1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

H, S, T, CNOT, CZ, U, X, U2, CCX = 0, 1, 2, 3, 4, 5, 6, 7, 8
GATE_NAMES = {H: "H", S: "S", T: "T", CNOT: "CNOT", CZ: "CZ", U: "U", X: "X", U2: "U2", CCX: "CCX"}
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        """Uniform integer in [0, m) by rejection."""
        if m <= 0:
            raise ValueError("m must be positive")
        limit = (1 << 64) - ((1 << 64) % m)
        while True:
            x = self.next()
            if x < limit:
                return x % m


def random_circuit(n: int, d: int, seed: int, one_gate_per_layer: bool = False) -> np.ndarray:
    """Seeded random Clifford+T circuit, int32[n_gates, 4] rows (op, layer, q0, q1).

    ``one_gate_per_layer`` is the alternative reading (a single random gate per
    layer, the other qubits idle); the graded workloads never use it.
    """
    if not (1 <= n <= 32 and 1 <= d <= 64):
        raise ValueError("need 1 <= n <= 32 and 1 <= d <= 64")
    rng = SplitMix64(seed)
    rows = []
    for layer in range(d):
        if one_gate_per_layer:
            op = rng.below(5) if n >= 2 else rng.below(3)
            q0 = rng.below(n)
            if op in (CNOT, CZ):
                q1 = rng.below(n - 1)
                q1 = q1 + 1 if q1 >= q0 else q1
                rows.append((op, layer, q0, q1))
            else:
                rows.append((op, layer, q0, -1))
            continue
        order = list(range(n))
        for i in range(n - 1, 0, -1):  # Fisher-Yates
            j = rng.below(i + 1)
            order[i], order[j] = order[j], order[i]
        free = [True] * n
        for q in order:
            if not free[q]:
                continue
            op = rng.below(5)
            partners = [p for p in range(n) if free[p] and p != q]
            if op in (CNOT, CZ) and not partners:
                op = rng.below(3)
            if op in (CNOT, CZ):
                p = partners[rng.below(len(partners))]
                a, b = (q, p) if rng.below(2) == 0 else (p, q)
                rows.append((op, layer, a, b))
                free[q] = free[p] = False
            else:
                rows.append((op, layer, q, -1))
                free[q] = False
    return np.asarray(rows, dtype=np.int32).reshape(-1, 4)


def rotated_h(theta: float) -> np.ndarray:
    """The rotated Hadamard of Eq. HadT, [[cos t, sin t], [sin t, -cos t]]
    (rows = output bit): t = pi/4 is H, t = pi/2 the classical NOT."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, s], [s, -c]], dtype=np.complex128)


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    """The usual three-angle one-qubit unitary
    [[cos(t/2), -e^{i lam} sin(t/2)], [e^{i phi} sin(t/2), e^{i(phi+lam)} cos(t/2)]]."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


# Two-qubit gates as 4x4 matrices, rows = output, basis index x_{q0} + 2 x_{q1}
# (the order 00, 10, 01, 11 of Eq. ET2).

def swap_matrix() -> np.ndarray:
    m = np.zeros((4, 4), dtype=np.complex128)
    for x in range(4):
        y = ((x & 1) << 1) | (x >> 1)
        m[y, x] = 1.0
    return m


def exchange_matrix(gamma: float) -> np.ndarray:
    """The Appendix's two-qubit exchange operator J12:
    diag(e^{i g/2}, e^{-i g/2}, e^{-i g/2}, e^{i g/2})."""
    return np.diag(np.exp(0.5j * gamma * np.array([1, -1, -1, 1]))).astype(np.complex128)


def iswap_matrix() -> np.ndarray:
    m = swap_matrix()
    m[2, 1] = m[1, 2] = 1j
    return m


def cphase_matrix(theta: float) -> np.ndarray:
    return np.diag([1, 1, 1, np.exp(1j * theta)]).astype(np.complex128)


def cnot_matrix(control_is_q0: bool = True) -> np.ndarray:
    m = np.zeros((4, 4), dtype=np.complex128)
    for x in range(4):
        c, t = (x & 1, x >> 1) if control_is_q0 else (x >> 1, x & 1)
        t ^= c
        y = (c | (t << 1)) if control_is_q0 else (t | (c << 1))
        m[y, x] = 1.0
    return m


def random_two_qubit_circuit(n: int, d: int, seed: int, frac: float = 0.5):
    """random_circuit(n, d, seed) with each CNOT / CZ replaced, with
    probability frac, by a U2 gate drawn from {SWAP, exchange J12(g), iSWAP,
    controlled phase(t), CNOT with the control on q1} (angles uniform in
    [0, 2 pi)) and each one-qubit gate replaced, with probability frac / 4,
    by X.  Returns (gates, mats2) with mats2 complex128[n_gates, 4, 4]."""
    g = random_circuit(n, d, seed).copy()
    rng = SplitMix64(seed ^ 0x51A7)
    mats2 = np.zeros((len(g), 4, 4), dtype=np.complex128)

    def unif() -> float:
        return (rng.next() >> 11) * (2.0 ** -53)

    for i in range(len(g)):
        if g[i, 0] in (CNOT, CZ) and unif() < frac:
            kind = rng.below(5)
            ang = 2 * np.pi * unif()
            mats2[i] = (swap_matrix(), exchange_matrix(ang), iswap_matrix(), cphase_matrix(ang),
                        cnot_matrix(False))[kind]
            g[i, 0] = U2
        elif g[i, 0] in (H, S, T) and unif() < frac / 4:
            g[i, 0] = X
    return g, mats2


def random_ccx_circuit(n: int, d: int, seed: int, frac: float = 0.5) -> np.ndarray:
    """random_circuit(n, d, seed) where, in each layer with probability frac,
    three qubits that carry one-qubit gates there are replaced by a Toffoli
    (controls the first two, target the third, in the layer's random
    order).  int32[n_gates, 5] rows (op, layer, q0, q1, q2)."""
    g = random_circuit(n, d, seed)
    rng = SplitMix64(seed ^ 0xCC0)
    rows = []
    for layer in range(d):
        lg = [tuple(int(v) for v in r) + (-1,) for r in g if r[1] == layer]
        ones = [r for r in lg if r[0] in (H, S, T)]
        if len(ones) >= 3 and (rng.next() >> 11) * (2.0 ** -53) < frac:
            pick = []
            pool = list(ones)
            for _ in range(3):
                pick.append(pool.pop(rng.below(len(pool))))
            lg = [r for r in lg if r not in pick]
            lg.append((CCX, layer, pick[0][2], pick[1][2], pick[2][2]))
        rows.extend(lg)
    return np.asarray(rows, dtype=np.int32).reshape(-1, 5)


def random_unitary4(rng: "SplitMix64") -> np.ndarray:
    """A 4x4 unitary with no zero entry: QR of a complex matrix of entries
    uniform in the unit square (SplitMix64 draws), phases fixed by R's
    diagonal."""
    def unif() -> float:
        return (rng.next() >> 11) * (2.0 ** -53)
    a = np.array([[unif() - 0.5 + 1j * (unif() - 0.5) for _ in range(4)] for _ in range(4)])
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def random_table_circuit(n: int, d: int, seed: int, frac: float = 0.6):
    """random_circuit(n, d, seed) with each CNOT / CZ replaced, with
    probability frac, by a random dense two-qubit unitary (a table gate,
    Eq. ET2), alternating with the controlled-H (a table with zeros).
    Returns (gates, mats2)."""
    g = random_circuit(n, d, seed).copy()
    rng = SplitMix64(seed ^ 0x7AB1E)
    mats2 = np.zeros((len(g), 4, 4), dtype=np.complex128)
    ch = np.eye(4, dtype=np.complex128)
    ch[np.ix_([1, 3], [1, 3])] = np.array([[1, 1], [1, -1]]) / np.sqrt(2)  # H on q1 if q0 = 1
    k = 0
    for i in range(len(g)):
        if g[i, 0] in (CNOT, CZ) and (rng.next() >> 11) * (2.0 ** -53) < frac:
            mats2[i] = random_unitary4(rng) if k % 2 == 0 else ch
            g[i, 0] = U2
            k += 1
    return g, mats2


def rotated_h_chain(d: int, theta: float):
    """n = 1, d rotated Hadamards in series (Sec. 4.2, Fig. 5): (gates, mats)
    with mats complex128[d, 2, 2]."""
    g = np.asarray([(U, k, 0, -1) for k in range(d)], dtype=np.int32).reshape(-1, 4)
    return g, np.stack([rotated_h(theta)] * d)


def random_general_circuit(n: int, d: int, seed: int, frac_u: float = 0.3):
    """random_circuit(n, d, seed) with each one-qubit gate replaced, with
    probability frac_u, by a U gate of three angles drawn uniformly in
    [0, 2 pi) (SplitMix64(seed ^ 0x9E37)).  Returns (gates, mats), mats
    complex128[n_gates, 2, 2] (zero rows for the other gates)."""
    g = random_circuit(n, d, seed).copy()
    rng = SplitMix64(seed ^ 0x9E37)
    mats = np.zeros((len(g), 2, 2), dtype=np.complex128)

    def unif() -> float:
        return (rng.next() >> 11) * (2.0 ** -53)

    for i in range(len(g)):
        if g[i, 0] in (H, S, T) and unif() < frac_u:
            g[i, 0] = U
            mats[i] = u3(2 * np.pi * unif(), 2 * np.pi * unif(), 2 * np.pi * unif())
    return g, mats


def hadamard_chain(d: int) -> np.ndarray:
    """n = 1, d Hadamard gates in series (Sec. 4, Fig. 3/4)."""
    return np.asarray([(H, k, 0, -1) for k in range(d)], dtype=np.int32).reshape(-1, 4)


def ghz(n: int) -> np.ndarray:
    """H on qubit 0 then a CNOT ladder 0->1->...->n-1 (d = n layers)."""
    rows = [(H, 0, 0, -1)] + [(CNOT, k, k - 1, k) for k in range(1, n)]
    return np.asarray(rows, dtype=np.int32).reshape(-1, 4)


def chains_for(n: int) -> int:
    """Batched workload chain count: max(256, 2^ceil(n/2))."""
    return max(256, 1 << ((n + 1) // 2))


def default_J(n: int, d: int, gates) -> float:
    """J = ln(M / ln 2), M = number of linked (non-H) p-bits: the stationary
    fraction of valid paths, (1 + e^{-J})^{-M}, is then close to 1/2.  U
    gates count as free outputs here (most are coupled)."""
    h = int(np.sum(np.isin(np.asarray(gates)[:, 0], (H, U))))
    M = max(n * d - h, 1)
    return float(np.log(max(M / np.log(2.0), 1.0 + 1e-9)))


@dataclass
class Workload:
    name: str
    n: int
    d: int
    gates: np.ndarray
    chains: int
    sweeps: int
    seed: int
    J: float
    alphas: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n_pbits(self) -> int:
        return self.n * (self.d + 1)


def tiny() -> Workload:
    """n=3, d=4 (15 p-bits), 1024 chains x 1e4 sweeps."""
    g = random_circuit(3, 4, seed=0)
    return Workload("tiny", 3, 4, g, chains=1024, sweeps=10_000, seed=0x5EED, J=default_J(3, 4, g))


def mid() -> Workload:
    """n=12, d=20 (252 p-bits), 4096 chains x 1e5 sweeps, full 2^12 histogram."""
    g = random_circuit(12, 20, seed=1000)
    return Workload("mid", 12, 20, g, chains=4096, sweeps=100_000, seed=0x5EED + 1,
                    J=default_J(12, 20, g))


def general_mid() -> Workload:
    """The mid circuit (n=12, d=20, seed 1000) with 30 % of its one-qubit
    gates replaced by random three-angle unitaries (Eq. EB gates with real
    couplings and phases off the pi/4 grid); 4096 chains.  extra["mats"]
    holds the gate matrices."""
    g, mats = random_general_circuit(12, 20, seed=1000, frac_u=0.3)
    return Workload("general_mid", 12, 20, g, chains=4096, sweeps=10_000, seed=0x5EED + 5,
                    J=default_J(12, 20, g), extra={"mats": mats})


def batched(count: int = 256) -> list[Workload]:
    """256 circuits, n ~ U[6,20], d ~ U[8,40], chains max(256, 2^ceil(n/2)), 1e4 sweeps."""
    rng = SplitMix64(2000)
    out = []
    for i in range(count):
        n = 6 + rng.below(15)
        d = 8 + rng.below(33)
        g = random_circuit(n, d, seed=2000 + i)
        out.append(Workload(f"batched_{i}", n, d, g, chains=chains_for(n), sweeps=10_000,
                            seed=0x5EED + i, J=default_J(n, d, g)))
    return out


def learned() -> Workload:
    """n=16, d=24 circuit for the learned proposal (MLP hidden 256)."""
    g = random_circuit(16, 24, seed=3000)
    return Workload("learned", 16, 24, g, chains=4096, sweeps=10_000, seed=0x5EED + 3,
                    J=default_J(16, 24, g), extra={"hidden": 256, "train_paths": 1_000_000})


def learned_sparse() -> Workload:
    """n=16, d=24 under the alternative reading "one random gate per layer"
    (few H gates: the error target is reachable and plain Gibbs must walk a
    defect along each wire to change a path)."""
    g = random_circuit(16, 24, seed=3000, one_gate_per_layer=True)
    return Workload("learned_sparse", 16, 24, g, chains=4096, sweeps=10_000, seed=0x5EED + 3,
                    J=default_J(16, 24, g), extra={"hidden": 256, "train_paths": 1_000_000})


def large() -> Workload:
    """n=24, d=32 (24*33 = 792 p-bits), 65536 chains, 64 output amplitudes alpha in 0..63."""
    g = random_circuit(24, 32, seed=4000)
    return Workload("large", 24, 32, g, chains=65536, sweeps=10_000, seed=0x5EED + 4,
                    J=default_J(24, 32, g), alphas=np.arange(64, dtype=np.uint32))


# ---- column sampling of the period-finding circuit (Sec. 5.2)

@dataclass
class ShorWorkload:
    name: str
    N: int
    a: int
    n: int           # bits of the first register (t = n = ceil(log2 N), Sec. 5.2)
    T: int           # column samples
    seed: int
    r: int           # the known order of a mod N (for checking only)

    def columns(self) -> np.ndarray:
        return shor_columns(self.n, self.T, self.seed)


def shor_columns(n: int, T: int, seed: int) -> np.ndarray:
    """T column indices uniform in [0, 2^n): the top n bits of SplitMix64(seed)
    draws, uint32."""
    rng = SplitMix64(seed)
    return np.asarray([rng.next() >> (64 - n) for _ in range(T)], dtype=np.uint32)


def shor_paper() -> ShorWorkload:
    """f(x) = 10424^x mod 98743069 (27 bits, order 78) with 250 column samples
    (Sec. 5.3: 250 columns of 2^27, about 5923 s on one laptop core)."""
    return ShorWorkload("shor_78", 98743069, 10424, 27, 250, 0x5EED + 6, 78)


def shor_table1(gamma: int = 3) -> ShorWorkload:
    """The Table 1 case: N = 961307 (20 bits), a = 5, order 479568, with
    gamma * r column samples (Sec. 5.2: T = gamma r, 2 <= gamma <= 4)."""
    return ShorWorkload("shor_table1", 961307, 5, 20, gamma * 479568, 0x5EED + 7, 479568)
