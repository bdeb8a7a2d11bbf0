#!/usr/bin/env python
"""Throughput benchmark of the plain Gibbs path (p-bit flips/s).

Workload: the mid circuit (random Clifford+T, n = 12 qubits, d = 20 layers,
252 p-bits), 4096 chains, 1e5 sweeps in total.  A step is one pass of the hot
path over the batch of chains: `--sweeps-per-step` Gibbs sweeps of every chain
with a record (validity, phase, histogram bin) after each sweep, then the
amplitude reduction of the 4096-bin histogram and its read-back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank owns its own 4096 chains (global chain groups offset
by rank, weak scaling) and the ranks combine their integer histograms with one
all-reduce after the timed steps.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2007_07379_gb300 import workloads as W  # noqa: E402

METRIC = "p-bit flips/s; wall time to 1% amplitude error (learned vs plain Gibbs)"
UNIT = "flips/s"

# Algorithmic integer work of one 32-chain word update, in 32-lane integer
# instruction slots: expected Philox4x32-10 calls of the most-significant-
# first comparison (each plane decides a chain with probability 1/2, calls of
# 4 planes continue while any of the 32 chains is undecided) x (20 widening
# multiplies + 20 three-input XORs per call + 4 planes x 4 slots of
# comparison) + 12 slots of links and store; plus the record (8 slots per
# p-bit word) every sweep.  The multiplies run on the integer multiply pipe,
# everything else on the integer logic pipe; each pipe issues 64 lanes per
# clock per SM (2 warp-instructions), so the logic pipe, which carries most
# of the work, is the bound.
PHILOX_MUL_SLOTS = 20
PHILOX_XOR_SLOTS = 20
PLANE_SLOTS = 4
LINK_SLOTS = 12
RECORD_SLOTS = 8
LOGIC_LANES_PER_SM = 64


def expected_calls(lanes: int = 32) -> float:
    return sum(1.0 - (1.0 - 2.0 ** (-4 * c)) ** lanes for c in range(0, 9))


def alg_slots_per_word() -> float:
    """All algorithmic integer slots (both pipes) per 32-chain word."""
    return (expected_calls(32) * (PHILOX_MUL_SLOTS + PHILOX_XOR_SLOTS + 4 * PLANE_SLOTS)
            + LINK_SLOTS + RECORD_SLOTS)


def alg_logic_slots_per_word() -> float:
    """Algorithmic slots on the integer logic pipe per 32-chain word."""
    return expected_calls(32) * (PHILOX_XOR_SLOTS + 4 * PLANE_SLOTS) + LINK_SLOTS + RECORD_SLOTS


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def gpu_id(dev) -> str:
    """nvidia-smi identifier (UUID) of a torch device."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _oracle_gibbs(oracle, wl, **kw):
    """The oracle's reference Gibbs sampler for the workload (the general-gate
    one when the circuit has gate matrices)."""
    if "mats" in wl.extra:
        return oracle.u_gibbs(wl.n, wl.d, wl.gates, wl.extra["mats"], J=wl.J, seed=wl.seed, **kw)
    return oracle.gibbs(wl.n, wl.d, wl.gates, J=wl.J, seed=wl.seed, **kw)


def cpu_oracle_rate(wl, budget_s: float = 10.0, chains: int | None = None, threads: int | None = None):
    """The oracle's reference Gibbs sampler on a bounded sample of the same
    workload (host cores, OpenMP over chains, about `budget_s` seconds; all
    the host's threads, or `threads`).  Returns (flips/s, cores, sample)."""
    import oracle
    n, d = wl.n, wl.d
    all_threads = oracle.num_threads()
    if threads is not None:
        oracle.set_num_threads(threads)
    try:
        return _cpu_oracle_rate(oracle, wl, n, d, budget_s, chains)
    finally:
        oracle.set_num_threads(all_threads)


def _cpu_oracle_rate(oracle, wl, n, d, budget_s, chains):
    c = chains or 128
    t0 = time.perf_counter()
    _oracle_gibbs(oracle, wl, chains=c, sweeps=20)
    dt = max(time.perf_counter() - t0, 1e-3)
    sweeps = max(2, int(budget_s / dt * 20))
    sweeps = min(sweeps, 200_000)
    t0 = time.perf_counter()
    _oracle_gibbs(oracle, wl, chains=c, sweeps=sweeps)
    dt = time.perf_counter() - t0
    flips = c * sweeps * n * d
    return flips / dt, oracle.num_threads(), f"{c} chains x {sweeps} sweeps of the {wl.name} circuit ({dt:.1f} s)"


def run_reference(args, wl):
    """Reference arm: the CPU oracle as it stands, on the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    n, d = wl.n, wl.d
    c = 64
    per_step = max(2, args.ref_sweeps)
    for _ in range(args.warmup):
        _oracle_gibbs(oracle, wl, chains=c, sweeps=1)
    times = []
    state = None
    for k in range(args.steps):
        t0 = time.perf_counter()
        r = _oracle_gibbs(oracle, wl, chains=c, sweeps=per_step, sweep0=k * per_step, state=state)
        state = r["state"]
        times.append(time.perf_counter() - t0)
    flips = c * per_step * n * d * args.steps
    value = flips / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": _config(wl, args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{c} chains x {per_step} sweeps per step of the {wl.name} circuit"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _model(pbits, wl):
    """The workload's compiled circuit (general one-qubit gates when it has
    gate matrices)."""
    return pbits.Model(wl.n, wl.d, wl.gates, wl.J, mats=wl.extra.get("mats"))


def _config(wl, args, world):
    kind = ("random Clifford+T + 30% random one-qubit unitaries" if "mats" in wl.extra
            else "random Clifford+T")
    return {"workload": f"{wl.name}: {kind} n={wl.n} d={wl.d} ({wl.n_pbits} p-bits), "
                        f"{wl.chains} chains per GPU, {args.sweeps_per_step} sweeps per step, J={wl.J:.4f}",
            "n": wl.n, "d": wl.d, "chains_per_gpu": wl.chains, "sweeps_per_step": args.sweeps_per_step,
            "circuit_seed": 1000, "philox_key": wl.seed, "parallelism": f"chains sharded over {world} GPU(s)",
            "l2": "flushed (256 MiB write) between timed steps; working set is on-chip by design"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps-per-step", type=int, default=10_000)
    ap.add_argument("--ref-sweeps", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--learned-seconds", type=float, default=8.0)
    ap.add_argument("--moves-only", type=int, default=0, metavar="K",
                    help="run K learned suffix moves (pb_mh_moves, one plain graph per move) on the "
                         "learned workload with an untrained network and exit: a profiling target")
    ap.add_argument("--moves-workload", default="learned", choices=["learned", "large"],
                    help="workload of --moves-only")
    ap.add_argument("--workload", default="mid", choices=["mid", "general_mid"],
                    help="headline circuit: mid (Clifford+T) or general_mid (30%% of the "
                         "one-qubit gates random unitaries)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3

    if args.moves_only:
        moves_only(args.moves_only, args.moves_workload)
        return
    wl = W.mid() if args.workload == "mid" else W.general_mid()
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    from paper_2007_07379_gb300 import pbits

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    pbits.load()

    stream = torch.cuda.Stream(device=dev)
    groups = (wl.chains + 31) // 32
    S = args.sweeps_per_step
    with torch.cuda.stream(stream):
        model = _model(pbits, wl)
        info = model.info()
        cfg = pbits.RunCfg(seed=wl.seed, chains=wl.chains, group0=rank * groups)
        run = pbits.Run([model], [cfg], stream=stream)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        for _ in range(args.warmup):
            run.sweeps(S)
            run.amplitudes()
        torch.cuda.synchronize(dev)

        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sweep_ms = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(gpu_id(dev)) as clk:
            for k in range(args.steps):
                flush.fill_(k & 0xFF)  # evict L2 between timed steps (outside the events)
                ev[k][0].record(stream)
                run.sweeps(S)
                run.amplitudes()  # reduction kernel + read-back; synchronises the stream
                ev[k][1].record(stream)
                sweep_ms.append(run.stats()["last_ms"])
            torch.cuda.synchronize(dev)
        step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
        # the single exchange of the method: integer sum of the histograms
        from paper_2007_07379_gb300 import dist as D
        cnt, valid, samples = run.histogram()
        D.allreduce_histogram(cnt, valid, samples, device=dev)
    flips_per_step = wl.chains * info["n"] * info["d"] * S
    value = world * flips_per_step * args.steps / total_s
    clocks = clk.summary()

    # roofline of the dominant kernel (the sweep launch): algorithmic logic-
    # pipe lane operations per launch / its duration, against the logic pipe
    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sms * LOGIC_LANES_PER_SM * sm_max * 1e6
    words_per_launch = groups * wl.n * wl.d * S
    alg_ops = words_per_launch * alg_logic_slots_per_word()
    launch_s = statistics.mean(sweep_ms) / 1e3
    achieved = alg_ops / launch_s
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "T int32 logic ops/s", "frac": achieved / peak_ops, "traffic": None,
                "peak_basis": f"{sms} SMs x {LOGIC_LANES_PER_SM} int32 logic lanes per clock "
                              f"x {sm_max:.0f} MHz ({peak_kind} sm_max)",
                "kernel": "sweep_kernel", "launch_ms": statistics.mean(sweep_ms),
                "alg_logic_ops_per_flip": alg_logic_slots_per_word() / 32,
                "alg_mul_ops_per_flip": expected_calls(32) * PHILOX_MUL_SLOTS / 32,
                "frac_of_issue": words_per_launch * alg_slots_per_word() / launch_s
                / (sms * 128 * sm_max * 1e6)}
    prof = os.path.join(ROOT, "profiles", "sweep_kernel_mid_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                tr = json.load(f)
            # the stored capture covers one launch of its own sweep count
            if tr.get("kernel_rev") == kernel_rev() and tr.get("sweeps_per_launch") == S:
                roofline["traffic"] = tr["dram_bytes_read_per_launch"] + tr["dram_bytes_write_per_launch"]
        except Exception:
            pass

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(wl, rank, groups, S, dev, stream, world)

    extra = {}
    if rank == 0 and not args.no_extra:
        extra["batched"] = batched_measurement(dev, stream)
        extra["elim"] = elim_measurement(dev, stream)
        extra["large"] = large_measurement(dev, stream)
        extra["general"] = general_measurement(dev, stream)
        extra["shor"] = shor_measurement(dev, stream)

    learned = None
    if rank == 0 and not args.no_learned:
        learned = [learned_comparison(dev, stream, seconds=args.learned_seconds, wl=w)
                   for w in (W.learned(), W.learned_sparse())]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_oracle_rate(wl)
        v1, _, sample1 = cpu_oracle_rate(wl, budget_s=6.0, chains=32, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": _config(wl, args, world), "clocks": clocks, "e2e": e2e,
            "gpu_launches": 3 * args.steps, "roofline": roofline, "cpu_baseline": cpu,
            "samples_per_s": world * wl.chains * S * args.steps / total_s,
            "learned_vs_plain": learned,
            "other_workloads": extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _top16(name: str):
    """The 16 outputs of largest |psi| of a learned workload and their exact
    amplitudes (tests/golden/learned_top16.json, written from the FP64 state
    vector by tests/golden/make_learned_top16.py)."""
    with open(os.path.join(ROOT, "tests", "golden", "learned_top16.json")) as f:
        d = json.load(f)[name]
    return np.array(d["alphas"], dtype=np.int64), np.array(d["re"]) + 1j * np.array(d["im"])


def _eps_curve(run, chunk: int, seconds: float, alphas, exact):
    """Error eps(t) = max over the 16 outputs of |psi_hat - psi|, read after
    1, 2, 4, ... pb_run_sweeps calls of `chunk` sweeps (or samples) and at
    the end; t = the summed device time of those calls (CUDA events around
    each graph replay), until `seconds` of device time."""
    pts, t, k, nxt = [], 0.0, 0, 1
    wall0 = time.perf_counter()
    while True:
        run.sweeps(chunk)
        t += run.stats()["last_ms"] / 1e3
        k += 1
        last = t >= seconds or time.perf_counter() - wall0 > 3 * seconds + 30
        if k == nxt or last:
            psi, _ = run.amplitudes()
            pts.append((t, float(np.abs(psi[alphas] - exact).max())))
            nxt *= 2
        if last:
            return pts, k


def _eps_fit(pts, eps: float):
    """Least-squares fit of log eps = log A - log t / 2 (the 1/sqrt(T) law of
    Eq. U26) over the points in the last 64th of the time range and on, and
    the time to eps it gives, (A / eps)^2; the free-slope fit beside it; the
    first measured time with eps(t) <= eps, if any."""
    t = np.array([p[0] for p in pts])
    e = np.array([p[1] for p in pts])
    use = (t >= t[-1] / 64) & (e > 0)
    A = float(np.exp(np.mean(np.log(e[use]) + 0.5 * np.log(t[use]))))
    slope = float(np.polyfit(np.log(t[use]), np.log(e[use]), 1)[0]) if use.sum() >= 2 else None
    hit = [float(tt) for tt, ee in pts if ee <= eps]
    return {"A": A, "t_to_eps_s": (A / eps) ** 2, "free_slope": slope,
            "t_first_below_eps_s": hit[0] if hit else None, "eps_final": float(e[-1]),
            "t_final_s": float(t[-1]), "points": [[float(a), float(b)] for a, b in pts]}


def moves_only(k: int, workload: str = "learned"):
    """K learned suffix moves on the learned workload (4096 chains) or the
    large one (65536 chains), hidden 256, untrained network (the cost of a
    move does not depend on the weights), each a replay of the move graph;
    prints the mean time."""
    import torch
    from paper_2007_07379_gb300 import pbits
    wl = W.large() if workload == "large" else W.learned()
    pbits.load()
    m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
    net = pbits.Mlp(wl.n, wl.d, hidden=256, batch=4096, seed=3)
    run = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, alphas=wl.alphas)])
    mh = pbits.Learned(run, net)
    mh.step(2)
    run.wait()
    t0 = time.perf_counter()
    mh.step(k)
    run.wait()
    print(json.dumps({"workload": workload, "moves": k,
                      "ms_per_move": 1e3 * (time.perf_counter() - t0) / k}), flush=True)


def learned_comparison(dev, stream, seconds: float = 8.0, train_paths: int = 1_000_000,
                       train_steps: int = 3000, wl=None):
    """Wall time to 1 % amplitude error, learned proposal vs plain Gibbs (and
    the exact i.i.d. sampler as the ceiling), on the learned workload (n=16,
    d=24, 4096 chains).  The error is measured against the exact amplitudes:
    eps(t) = max over the 16 largest |psi_alpha| of |psi_hat - psi|, read at
    doubling intervals for `seconds` of device time per sampler; eps(t) is
    fitted with the 1/sqrt(t) law and extrapolated to eps = 0.01.  The
    network is trained first on valid paths of plain Gibbs (time reported
    separately); the learned sampler is the PB_LEARNED run mode, one suffix
    move before every sweep, all in one graph per call."""
    import torch
    from paper_2007_07379_gb300 import pbits
    wl = wl or W.learned()
    n, d = wl.n, wl.d
    alphas, exact = _top16(wl.name)
    eps = 0.01
    out = {"workload": f"{wl.name}: random Clifford+T n={n} d={d}, {wl.chains} chains, hidden 256",
           "eps": eps, "error": "max |psi_hat - psi| over the 16 largest |psi| (FP64 state vector)",
           "top16_abs_psi": float(np.abs(exact).max())}
    with torch.cuda.stream(stream):
        model = pbits.Model(n, d, wl.gates, wl.J)
        # 1. collect valid paths from plain Gibbs and train the network
        t0 = time.perf_counter()
        src = pbits.Run([model], [pbits.RunCfg(seed=wl.seed + 100, chains=wl.chains)], stream=stream)
        net = pbits.Mlp(n, d, hidden=256, batch=4096, seed=21, stream=stream)
        coll = pbits.Learned(src, net)
        cap = train_paths
        paths = torch.zeros((cap, d), dtype=torch.int32, device=dev)
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        src.sweeps(200)
        while int(count.item()) < cap:
            src.sweeps(2)
            coll.collect(paths, count)
        t_collect = time.perf_counter() - t0
        t0 = time.perf_counter()
        losses = pbits.train_on_paths(net, paths, cap, 0, steps=train_steps, rows=4096, lr=1e-3, seed=5)
        torch.cuda.synchronize(dev)
        t_train = time.perf_counter() - t0
        lc = losses.cpu().numpy()
        out.update({"train_paths": cap, "train_steps": train_steps, "collect_s": t_collect,
                    "train_s": t_train, "loss_first": float(lc[:10].mean()), "loss_last": float(lc[-10:].mean()),
                    "h": model.info()["h"]})
        del paths

        def arm(sampler, chunk, **kw):
            run = pbits.Run([model], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, n_batches=32,
                                                   sampler=sampler, **kw)], stream=stream)
            pts, calls = _eps_curve(run, chunk, seconds, alphas, exact)
            res = _eps_fit(pts, eps)
            res["sweeps_or_samples"] = calls * chunk
            if sampler == pbits.PB_LEARNED:
                mv, acc = run.moves()
                res["moves"] = mv
                res["accept"] = acc / max(mv * wl.chains, 1)
                res["ms_per_move_and_sweep"] = 1e3 * res["t_final_s"] / max(mv, 1)
            return res

        out["plain"] = arm(pbits.PB_GIBBS, 200)
        out["learned"] = arm(pbits.PB_LEARNED, 20, proposal=net, mh_every=1)
        out["elim"] = arm(pbits.PB_ELIM, 200)
        out["ratio_plain_over_learned"] = out["plain"]["t_to_eps_s"] / out["learned"]["t_to_eps_s"]
        out["ratio_elim_over_learned"] = out["elim"]["t_to_eps_s"] / out["learned"]["t_to_eps_s"]
        # the learned arm's time with its training included, for the same error
        out["ratio_plain_over_learned_with_training"] = out["plain"]["t_to_eps_s"] / (
            out["learned"]["t_to_eps_s"] + t_collect + t_train)
    return out


def elim_measurement(dev, stream, samples: int = 10_000):
    """Exact i.i.d. path sampler (PB_ELIM) on the mid workload: path samples
    per second and the equivalent p-bit assignments per second."""
    import torch
    from paper_2007_07379_gb300 import pbits
    wl = W.mid()
    with torch.cuda.stream(stream):
        m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
        run = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, sampler=pbits.PB_ELIM)],
                        stream=stream)
        run.sweeps(samples)
        run.wait()
        best = None
        for _ in range(3):
            run.sweeps(samples)
            run.wait()
            ms = run.stats()["last_ms"]
            best = ms if best is None else min(best, ms)
        # one amplitude with the end state clamped (psi_0): its SE at this
        # budget and the time to an absolute error (1 SE) of 1e-2 and 1e-3
        runc = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, n_batches=32,
                                            alphas=np.array([0], dtype=np.uint32),
                                            sampler=pbits.PB_ELIM_CLAMP)], stream=stream)
        runc.sweeps(samples)
        runc.wait()
        runc.sweeps(samples)
        runc.wait()
        ms_c = runc.stats()["last_ms"]
        _, se_c = runc.amplitudes()
        _, se_u = run.amplitudes()
    t_c = 2 * ms_c / 1e3  # both launches recorded
    return {"workload": f"mid (n={wl.n}, d={wl.d}), {wl.chains} chains, exact i.i.d. paths",
            "samples": samples, "launch_ms": best,
            "paths_per_s": wl.chains * samples / (best / 1e3),
            "pbit_assignments_per_s": wl.chains * wl.n * wl.d * samples / (best / 1e3),
            "clamped_psi0": {"launch_ms": ms_c, "se": float(se_c[0]),
                             # the unclamped run recorded 4 launches, this one 2
                             "se_unclamped_same_samples": float(se_u[0]) * np.sqrt(2.0),
                             "t_to_1e-2_s": t_c * (float(se_c[0]) / 1e-2) ** 2,
                             "t_to_1e-3_s": t_c * (float(se_c[0]) / 1e-3) ** 2}}


def general_measurement(dev, stream, sweeps: int = 2000, samples: int = 2000):
    """General one-qubit gates (Eq. EB): the mid circuit with 30 % of its
    one-qubit gates random unitaries.  Gibbs sweeps (heat-bath proposal,
    Metropolis acceptance of coupled p-bits, FP64 phase sums) and the exact
    sampler, against the same shape of plain Clifford+T circuit."""
    import torch
    from paper_2007_07379_gb300 import pbits
    wl = W.general_mid()
    pl = W.mid()

    def best_ms(run, k):
        run.sweeps(k)
        run.wait()
        out = None
        for _ in range(3):
            run.sweeps(k)
            run.wait()
            ms = run.stats()["last_ms"]
            out = ms if out is None else min(out, ms)
        return out

    with torch.cuda.stream(stream):
        m = pbits.Model(wl.n, wl.d, wl.gates, wl.J, mats=wl.extra["mats"])
        inf = m.info()
        g_ms = best_ms(pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains)], stream=stream),
                       sweeps)
        e_ms = best_ms(pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains,
                                                    sampler=pbits.PB_ELIM)], stream=stream), samples)
        mp = pbits.Model(pl.n, pl.d, pl.gates, pl.J)
        p_ms = best_ms(pbits.Run([mp], [pbits.RunCfg(seed=pl.seed, chains=pl.chains)], stream=stream),
                       sweeps)
    flips = wl.chains * wl.n * wl.d * sweeps
    return {"workload": "general_mid: mid (n=12, d=20) with 30% of one-qubit gates random unitaries, "
                        "4096 chains",
            "u_gates": inf["n_u"], "coupled": inf["n_coupled"], "sweeps": sweeps,
            "launch_ms": g_ms, "flips_per_s": flips / (g_ms * 1e-3),
            "plain_mid_flips_per_s": flips / (p_ms * 1e-3),
            "elim_paths_per_s": wl.chains * samples / (e_ms * 1e-3)}


def shor_measurement(dev, stream):
    """Column sampling of the period-finding circuit (Sec. 5.2): the paper's
    27-bit example (order 78, 250 columns; 5923 s on one laptop core) and
    the Table 1 case (N = 961307, order 479568, T = 3 r; 32 hours there).
    Time of one pb_shor_columns call from host column indices to the device
    distribution (modular powers, sort, column walk), the order read off as
    the number of peaks above 2.2 / 2^n, and the column walk's FP32 rate."""
    import torch
    from paper_2007_07379_gb300 import pbits
    out = {}
    peak_fp32 = None
    props = torch.cuda.get_device_properties(dev)
    peaks, _ = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_fp32 = props.multi_processor_count * 128 * sm_max * 1e6  # FP32 lanes per clock
    for wl in (W.shor_paper(), W.shor_table1(3)):
        x = wl.columns()
        with torch.cuda.stream(stream):
            sc = pbits.ShorColumns(wl.n, wl.T, stream=stream)
            sc.run(wl.N, wl.a, x)
            stream.synchronize()
            best = None
            for _ in range(3):
                t0 = time.perf_counter()
                sc.run(wl.N, wl.a, x)
                stream.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            M = 2 ** wl.n
            count, _, mx = sc.peaks(2.2 / M, 0)
        steps = float(M) * wl.T  # (k, sample) pairs
        # per pair one complex multiply-add: 4 FP32 lane operations
        out[wl.name] = {"N": wl.N, "a": wl.a, "n": wl.n, "T": wl.T, "order": wl.r,
                        "peaks_found": count, "call_s": best, "pairs_per_s": steps / best,
                        "fp32_frac_lower_bound": steps * 4 / best / peak_fp32,
                        "paper_s": 5923.0 if wl.name == "shor_78" else 32 * 3600.0}
        del sc
        torch.cuda.empty_cache()
    return out


def batched_measurement(dev, stream, sweeps: int = 10_000):
    """The batched workload: 256 random circuits (n in [6,20], d in [8,40],
    chains max(256, 2^ceil(n/2))), 1e4 sweeps each, in one persistent,
    graph-captured launch with an autotuned CTA shape."""
    import torch
    from paper_2007_07379_gb300 import pbits
    wls = W.batched()
    with torch.cuda.stream(stream):
        models = [pbits.Model(w.n, w.d, w.gates, w.J) for w in wls]
        cfgs = [pbits.RunCfg(seed=w.seed, chains=w.chains) for w in wls]
        run = pbits.Run(models, cfgs, stream=stream)
        t0 = time.perf_counter()
        run.tune(trial_sweeps=50)
        t_tune = time.perf_counter() - t0
        run.sweeps(sweeps)
        run.wait()
        ms = run.stats()["last_ms"]
    flips = sum(w.chains * w.n * w.d for w in wls) * sweeps
    return {"workload": "batched: 256 random Clifford+T circuits, n~U[6,20], d~U[8,40], "
                        "chains max(256, 2^ceil(n/2)), 1e4 sweeps, one persistent launch",
            "circuits": len(wls), "chains": sum(w.chains for w in wls), "sweeps": sweeps,
            "launch_ms": ms, "flips_per_s": flips / (ms * 1e-3), "tune_s": t_tune,
            "shape": run.shape()}


def large_measurement(dev, stream, sweeps: int = 2000, moves: int = 40):
    """The large workload: n=24, d=32 (792 p-bits), 65536 chains, 64 output
    amplitudes; plain sweeps, the PB_LEARNED run mode (a suffix move before
    every sweep, one graph per call) and the moves alone (pb_mh_moves, one
    graph per move, CUDA events); untrained network: the cost of a move does
    not depend on the weights."""
    import torch
    from paper_2007_07379_gb300 import pbits
    wl = W.large()
    with torch.cuda.stream(stream):
        m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
        run = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, alphas=wl.alphas)],
                        stream=stream)
        run.sweeps(200)
        run.sweeps(sweeps)
        run.wait()
        ms = run.stats()["last_ms"]
        net = pbits.Mlp(wl.n, wl.d, hidden=256, batch=4096, seed=3, stream=stream)
        lr = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, alphas=wl.alphas,
                                          sampler=pbits.PB_LEARNED, proposal=net, mh_every=1)],
                       stream=stream)
        lr.sweeps(moves)
        lr.wait()
        lr.sweeps(moves)
        lr.wait()
        ms_l = lr.stats()["last_ms"]
        run.sweeps(1)
        run.wait()
        one = run.stats()["last_ms"]
        mh = pbits.Learned(run, net)
        mh.step(2)
        run.wait()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mh.step(moves)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_mv = e0.elapsed_time(e1) / moves
    flips = wl.chains * wl.n * wl.d * sweeps
    return {"workload": "large: random Clifford+T n=24 d=32 (792 p-bits), 65536 chains, 64 amplitudes",
            "sweeps": sweeps, "launch_ms": ms, "flips_per_s": flips / (ms * 1e-3),
            "ms_per_mh_move": ms_mv,
            "learned_run_ms_per_move_and_sweep": ms_l / moves,
            "one_sweep_launch_ms": one}


def kernel_rev() -> str:
    """Hash of the sources that make up the sweep kernel (ties a stored ncu
    traffic figure to the kernel it was measured on)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("sweep.cu", "philox.cuh", "pb_internal.h"):
        with open(os.path.join(ROOT, "paper_2007_07379_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measure_e2e(wl, rank, groups, S, dev, stream, world):
    """Same metric through the C ABI from host buffers: each step compiles the
    host gate list, creates the run (tables copied host -> device, chains
    initialised), runs S sweeps and copies the amplitudes back to the host."""
    import torch
    from paper_2007_07379_gb300 import pbits
    steps = 3
    cfg = pbits.RunCfg(seed=wl.seed, chains=wl.chains, group0=rank * groups)
    nbytes = None
    times = []
    h2d = d2h = 0
    with torch.cuda.stream(stream):
        for k in range(steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            model = _model(pbits, wl)
            if nbytes is None:
                nbytes = pbits.workspace_bytes([model], [cfg])
                ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            run = pbits.Run([model], [cfg], stream=stream, workspace=ws)
            run.sweeps(S)
            psi, se = run.amplitudes()
            dt = time.perf_counter() - t0
            run.close()
            model.close()
            if k > 0:  # first pass warms the graph cache and allocator
                times.append(dt)
            npb = wl.n * wl.d
            h2d = npb * (16 + 16 + 4) + 256 + 256 + 8
            d2h = psi.size * 3 * 8
    t = sum(times)
    if world > 1:
        tt = torch.tensor([t], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t = float(tt.item())
    value = world * wl.chains * wl.n * wl.d * S * steps / t
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": steps, "what": "pb_compile + pb_run_create + sweeps + pb_run_amplitudes"}


if __name__ == "__main__":
    main()
