#!/usr/bin/env python
"""Benchmark: merged Pauli products per second for H*H on one GB300.

A step is one canonical product C = H*H (outer product of every term pair,
then sort by symplectic key and merge duplicates, PauLIB Sec. III-H / IV-C)
of a seeded, synthetic Jordan-Wigner-shaped Hamiltonian, with the inputs
already resident in HBM.  Between timed steps a 512 MiB buffer is written to
flush L2 (the inputs are smaller than L2).  The device time of each step is
taken with CUDA events on the stream the library launches on.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "merged Pauli products/s (H·H), mixed vs FP64 at equal error; % of roofline"
UNIT = "products/s"
HBM_PEAK_FALLBACK = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
PIPELINE_SRC = os.path.join(ROOT, "paper_2605_25974_gb300", "csrc", "paulib_pipeline.cuh")

WORKLOADS = {
    "jw_hh_n200_m30000": dict(n=200, m=30000, seed=401),
    "jw_hh_n100_m20000": dict(n=100, m=20000, seed=301),
    "jw_hh_n100_m2000": dict(n=100, m=2000, seed=301),
    "jw_hh_n200_m6000": dict(n=200, m=6000, seed=401),
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device="cpu"):
    """The slowest rank's value (the job is as slow as its slowest replica);
    every rank gets it.  One all-reduce when world > 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (ms)."""
    return units_per_rank * world / (ms / 1e3)


def make_workload(name):
    from paper_2605_25974_gb300 import workloads as wl
    cfg = WORKLOADS[name]
    h = wl.jw(n=cfg["n"], m=cfg["m"], seed=cfg["seed"])
    return h


# ------------------------------------------------------------------ CPU oracle leg

def cpu_info():
    """Host CPU model and logical core count."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count() or 1}


def oracle_rate(h, budget_s=10.0, threads=1):
    """The oracle as it stands on a bounded sample: the canonical product of
    the first m' terms of H with themselves, m' chosen so one run takes about
    budget_s.  threads=1 runs the plain ordered-map mode; more threads run
    the oracle's multi-threaded sort-and-merge mode over the whole key
    range."""
    from oracle import pauli_oracle
    pauli_oracle._load()

    def run(mp):
        s = h.subset(slice(0, mp))
        t0 = time.perf_counter()
        if threads == 1:
            pauli_oracle.multiply_canonical(h.n, s.as_tuple(), s.as_tuple())
        else:
            pauli_oracle.multiply_canonical_range(h.n, s.as_tuple(), s.as_tuple(), None, None, threads)
        return time.perf_counter() - t0

    probe = 300 if threads == 1 else 1200
    t = run(probe)
    rate = probe * probe / max(t, 1e-6)
    mp = int(min(h.m, max(probe, (rate * budget_s) ** 0.5)))
    t = run(mp)
    mode = "ordered-map mode" if threads == 1 else "multi-threaded sort-and-merge mode"
    return {"value": mp * mp / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "canonical product of the first %d terms of H with themselves (%d products, %.1f s, %s)"
                      % (mp, mp * mp, t, mode)}, mp


def oracle_baselines(h, budget_s=10.0):
    """Single-core and all-core oracle rates with the host's CPU model."""
    info = cpu_info()
    one, _ = oracle_rate(h, budget_s, 1)
    allc, _ = oracle_rate(h, budget_s, info["nproc"])
    out = dict(allc)
    out["cpu"] = info["model"]
    out["nproc"] = info["nproc"]
    out["single_core"] = one
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    h = make_workload(args.workload)
    from oracle import pauli_oracle
    info = cpu_info()
    threads = info["nproc"]
    base, mp = oracle_rate(h, budget_s=min(8.0, 150.0 / max(1, args.steps + args.warmup)), threads=threads)
    s = h.subset(slice(0, mp))
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pauli_oracle.multiply_canonical_range(h.n, s.as_tuple(), s.as_tuple(), None, None, threads)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = mp * mp / (ms / 1e3)
    base["value"] = value
    base["cpu"] = info["model"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "terms": h.m, "n_qubits": h.n, "sample_terms": mp},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def traffic_per_product(stage, n):
    """DRAM bytes per product of a stage's kernels from the committed ncu
    summary, or None when the summary is missing, is for another size, or was
    taken on another version of the pipeline source (hash mismatch)."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        with open(PIPELINE_SRC, "rb") as f:
            src_hash = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, ValueError):
        return None, None
    e = d.get("stages", {}).get("%s_n%d" % (stage, n))
    if not e or d.get("pipeline_sha256_16") != src_hash:
        return None, d.get("pipeline_sha256_16")
    return float(e["bytes_per_product"]), src_hash


# ------------------------------------------------------------------ GPU leg

def timed_events(fn, stream, flush, reps, warm=2):
    """Mean device time (ms) of fn() between CUDA events on `stream`, with L2
    flushed before each timed call; fn returns an object with close()."""
    import torch
    for _ in range(warm):
        fn().close()
    ts = []
    for k in range(reps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        o.close()
    return statistics.mean(ts)


def measure_outer_product(paulib, gh, gh2, h, stream, flush, reps, hbm_peak, peak_src):
    """The raw outer product alone (every pair's key, exact phase and
    coefficient, written at j*|A| + i): an HBM-write-bound kernel."""
    W = h.x.shape[0]
    WP = 1
    while WP < W:
        WP *= 2
    products = h.m * h.m
    ms = timed_events(lambda: paulib.multiply(gh, gh2, "fp64", canonical=False), stream, flush, reps)
    # compulsory bytes: the product records written (2*WP key words, complex128,
    # the X^x Z^z phase byte and the stored phase byte); the inputs are read once
    bytes_out = products * (16 * WP + 16 + 2)
    bytes_in = 2 * h.m * (16 * WP + 16 + 1)
    gbs = (bytes_out + bytes_in) / (ms / 1e3) / 1e9
    return {"ms_per_step": ms, "value": products / (ms / 1e3), "unit": UNIT,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "peak_source": peak_src,
                         "bytes_per_product": 16 * WP + 16 + 2}}


def measure_propagation(paulib, stream, flush, reps, hbm_peak, peak_src, m=8_000_000, n=500):
    """Pauli-propagation steps on an 8M-term, 500-qubit sum of random strings
    of weight <= 32: one 100-gate Clifford list applied in place (Sec. III-B;
    each term is read and written once per list) and one rotation step
    exp(-i theta P / 2) with merge and truncation."""
    import numpy as np
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(601)
    x, z = wl.low_weight_terms(rng, n, m, 32)
    s = wl.SumArrays(n, x, z, wl.coeffs_loguniform(rng, m))
    g = paulib.PauliSum.from_arrays(s)
    WP = 1
    while WP < s.x.shape[0]:
        WP *= 2
    gates = []
    for _ in range(100):
        kind = ["h", "s", "cnot", "cz"][int(rng.integers(0, 4))]
        q1 = int(rng.integers(0, n))
        q2 = int((q1 + 1 + rng.integers(0, n - 1)) % n)
        gates.append((kind, q1, q2))

    class _NoClose:
        def close(self):
            pass

    def clifford():
        paulib.apply_clifford(g, gates, stream=stream)
        return _NoClose()

    ms_c = timed_events(clifford, stream, flush, reps)
    # compulsory bytes: every term's key, coefficient and phase byte read, then key,
    # coefficient and phase byte written
    per_term = 2 * (16 * WP + 16 + 1)
    gbs = m * per_term / (ms_c / 1e3) / 1e9
    res = {"terms": m, "n_qubits": n,
           "clifford": {"gates": len(gates), "ms_per_call": ms_c, "terms_per_s": m / (ms_c / 1e3),
                        "gate_terms_per_s": m * len(gates) / (ms_c / 1e3),
                        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                     "frac": gbs / hbm_peak, "peak_source": peak_src, "bytes_per_term": per_term}}}
    # one gate (H on qubit 137): the one-word kernel, which reads each term's
    # x and z word of that qubit (two 32-byte sectors) and its phase byte, and
    # writes only what changes; the compulsory bytes counted are those reads
    one = [("h", 137, 0)]

    def clifford1():
        paulib.apply_clifford(g, one, stream=stream)
        return _NoClose()

    ms_1 = timed_events(clifford1, stream, flush, reps)
    per_term1 = 2 * 32 + 1
    gbs1 = m * per_term1 / (ms_1 / 1e3) / 1e9
    res["clifford_single_gate"] = {"gate": "h 137", "ms_per_call": ms_1, "terms_per_s": m / (ms_1 / 1e3),
                                   "roofline": {"bound": "hbm", "achieved": gbs1, "peak": hbm_peak, "unit": "GB/s",
                                                "frac": gbs1 / hbm_peak, "peak_source": peak_src,
                                                "bytes_per_term": per_term1}}
    # rotation: a weight-250 generator anti-commutes with about half the terms
    pb = wl.SumArrays(n, *wl.low_weight_terms(wl.rng_for(602), n, 1, 250), np.ones(1, np.complex128))
    px, pz = pb.x[:, 0], pb.z[:, 0]
    out = paulib.rotate(g, px, pz, 0.1, 1e-9)
    u = out.n_terms
    out.close()
    ms_r = timed_events(lambda: paulib.rotate(g, px, pz, 0.1, 1e-9), stream, flush, max(2, reps // 2))
    res["rotation"] = {"theta": 0.1, "threshold": 1e-9, "ms_per_step": ms_r, "terms_in": m, "terms_out": int(u),
                       "terms_per_s": m / (ms_r / 1e3)}
    # the same step on the canonical form of the sum (as in a propagation run,
    # where every step's input is the previous step's canonical output): only
    # the partners are sorted, then merged with the already sorted terms
    cg = paulib.compress(g)
    out = paulib.rotate(cg, px, pz, 0.1, 1e-9)
    uc = out.n_terms
    out.close()
    ms_rc = timed_events(lambda: paulib.rotate(cg, px, pz, 0.1, 1e-9), stream, flush, max(2, reps // 2))
    res["rotation_canonical_input"] = {"theta": 0.1, "threshold": 1e-9, "ms_per_step": ms_rc,
                                       "terms_in": int(cg.n_terms), "terms_out": int(uc),
                                       "terms_per_s": cg.n_terms / (ms_rc / 1e3)}
    cg.close()
    # element-wise products of two 8M-term lists (the paper's single multiplication, in bulk)
    xb, zb = wl.low_weight_terms(wl.rng_for(603), n, m, 32)
    gb = paulib.PauliSum.from_arrays(wl.SumArrays(n, xb, zb, wl.coeffs_loguniform(wl.rng_for(604), m)))
    ms_p = timed_events(lambda: paulib.multiply_pairwise(g, gb), stream, flush, reps)
    per_pair = 2 * (16 * WP + 16 + 1) + (16 * WP + 16 + 2)  # both inputs read, one raw product written
    gbp = m * per_pair / (ms_p / 1e3) / 1e9
    res["pairwise"] = {"pairs": m, "ms_per_call": ms_p, "ns_per_product": ms_p * 1e6 / m,
                       "products_per_s": m / (ms_p / 1e3),
                       "roofline": {"bound": "hbm", "achieved": gbp, "peak": hbm_peak, "unit": "GB/s",
                                    "frac": gbp / hbm_peak, "peak_source": peak_src, "bytes_per_product": per_pair}}
    gb.close()
    g.close()
    return res


def measure_grouping(paulib, stream, reps, sizes=(200, 500, 1000, 2000, 20000), n=500):
    """Greedy commutation grouping (Sec. V-D) of random 500-qubit sums, at the
    paper's grouping sizes (200 to 2,000 terms, Sec. VI-C) and one larger sum:
    the whole call (anti-commutation bits, the greedy walk, the group count
    read back to the host, the CSR listing), timed with CUDA events around it
    and with the host clock."""
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    out = {"n_qubits": n, "paper_cpu_ms": {"200": 0.05, "2000": 5.6}, "sizes": {}}
    for m in sizes:
        g = paulib.PauliSum.from_arrays(wl.grouping(m, n=n))
        for _ in range(3):
            paulib.group_commuting(g, csr=True, stream=stream)
        ev, wall = [], []
        ng = 0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            _, ng, _, _ = paulib.group_commuting(g, csr=True, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            wall.append((time.perf_counter() - t0) * 1e3)
            ev.append(e0.elapsed_time(e1))
        ms = statistics.median(ev)
        out["sizes"][str(m)] = {"groups": ng, "ms_per_call": ms, "ms_per_call_host": statistics.median(wall),
                                "us_per_term": ms * 1e3 / m}
        g.close()
    return out


def measure_batched(paulib, stream, flush, reps, problems=4096):
    """Batched products (4,096 independent sum x sum products shaped like
    Pauli-propagation steps) as one prepared plan replayed from a CUDA graph,
    against the plain FP64 form: one paulib_multiply call per product."""
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    t0 = time.perf_counter()
    pairs = wl.batch(problems=problems)
    gen_s = time.perf_counter() - t0
    As = [paulib.PauliSum.from_arrays(a) for a, _ in pairs]
    Bs = [paulib.PauliSum.from_arrays(b) for _, b in pairs]
    products = int(sum(a.m * b.m for a, b in pairs))
    res = {"problems": problems, "products": products, "n_qubits": pairs[0][0].n,
           "generation_s": gen_s}
    res["method"] = "persistent kernel (one launch); general pipeline timed beside it"
    for prec, general in (("fp32_fp64merge", 0), ("fp64", 0), ("fp32_fp64merge", 1)):
        paulib.set_debug(3, general)  # plans made now take the general pipeline when set
        plan = paulib.BatchPlan(As, Bs, prec, stream=stream)
        paulib.set_debug(3, 0)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.launch(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        ts = []
        cur = torch.cuda.current_stream()
        for k in range(reps):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            g.replay()
            e1.record(cur)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.mean(ts)
        outs = plan.outputs(stream=cur)
        res[("general_pipeline_graph_" if general else "graph_") + prec] = {
            "ms_per_step": ms, "value": products / (ms / 1e3), "distinct_out": int(sum(o.n_terms for o in outs))}
        del outs
        plan.close()
        del g
    # plain FP64 form: one canonical multiply per product, back to back
    torch.cuda.synchronize()
    for i in range(min(64, problems)):
        paulib.multiply(As[i], Bs[i], "fp64").close()
    torch.cuda.synchronize()
    flush.fill_(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(problems):
        paulib.multiply(As[i], Bs[i], "fp64").close()
    torch.cuda.synchronize()
    seq_ms = (time.perf_counter() - t0) * 1e3
    res["sequential_fp64"] = {"ms_per_step": seq_ms, "value": products / (seq_ms / 1e3),
                              "note": "one paulib_multiply per product; each call synchronises once"}
    res["speedup_vs_sequential_fp64"] = seq_ms / res["graph_fp32_fp64merge"]["ms_per_step"]
    res["speedup_fp64_graph_vs_sequential_fp64"] = seq_ms / res["graph_fp64"]["ms_per_step"]
    res["speedup_vs_general_pipeline"] = (res["general_pipeline_graph_fp32_fp64merge"]["ms_per_step"] /
                                          res["graph_fp32_fp64merge"]["ms_per_step"])
    # compulsory HBM bytes: every operand term read once (16 words of key at
    # n=500, FP32 coefficient copy, phase byte), every merged term written once
    wp_words = 16
    terms_in = sum(a.m + b.m for a, b in pairs)
    bytes_io = terms_in * (8 * wp_words + 8 + 1) + res["graph_fp32_fp64merge"]["distinct_out"] * (8 * wp_words + 16 + 1)
    peak, kind = measured_peaks()
    bound_ms = bytes_io / (peak * 1e9) * 1e3
    res["roofline"] = {"bound": "hbm", "compulsory_bytes": bytes_io, "hbm_bound_ms": bound_ms,
                       "frac": bound_ms / res["graph_fp32_fp64merge"]["ms_per_step"], "peak_GBs": peak,
                       "peak_kind": kind}
    for t in As + Bs:
        t.close()
    return res


def measure_tiny(paulib, stream, reps=200):
    """64 x 64 terms at n=20 (every qubit uniform over I, X, Y, Z): one
    canonical product is launch-latency bound; device time from CUDA events
    and host time per call (the call synchronises once)."""
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    ga, gb = paulib.PauliSum.from_arrays(a), paulib.PauliSum.from_arrays(b)
    for _ in range(10):
        paulib.multiply(ga, gb).close()
    torch.cuda.synchronize()
    ev, wall = [], []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        o = paulib.multiply(ga, gb)
        e1.record(stream)
        torch.cuda.synchronize()
        wall.append((time.perf_counter() - t0) * 1e6)
        ev.append(e0.elapsed_time(e1) * 1e3)
        u = o.n_terms
        o.close()
    ga.close()
    gb.close()
    us = statistics.median(ev)
    return {"workload": "tiny_n20_64x64", "products": a.m * b.m, "distinct_out": int(u), "us_per_call": us,
            "us_per_call_host": statistics.median(wall), "value": a.m * b.m / (us * 1e-6), "unit": UNIT}


def measure_streaming(paulib, stream, hbm_peak, strings=256, reps=2):
    """A 1,000,000-term sum at n=500 times 256 single strings of coefficient 1,
    one canonical output per string (each a permutation of the sum's terms,
    re-sorted).  Compulsory traffic: the input once, every output term
    written once."""
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    t0 = time.perf_counter()
    A, singles = wl.stream(m=1_000_000, strings=strings)
    gen_s = time.perf_counter() - t0
    ga = paulib.PauliSum.from_arrays(A)
    gs = [paulib.PauliSum.from_arrays(s) for s in singles]
    paulib.multiply(ga, gs[0]).close()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for g in gs:
            paulib.multiply(ga, g).close()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    products = A.m * strings
    WP = 8
    term = 16 * WP + 16 + 1
    bound_ms = 1e3 * (A.m * term + products * term) / (hbm_peak * 1e9)
    # the same 256 products as one batch (the persistent batched kernel: one
    # launch, a CTA per string), timed as a prepared plan
    plan = paulib.BatchPlan([ga] * strings, gs, "fp64")
    tb = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.launch(stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1))
    outs = plan.outputs(stream=stream)
    bterms = int(sum(o.n_terms for o in outs))
    del outs
    plan.close()
    bms = statistics.median(tb)
    for g in gs:
        g.close()
    ga.close()
    return {"workload": "stream_n500_1m_x256", "products": products, "ms_per_pass": ms,
            "value": products / (ms / 1e3), "unit": UNIT, "hbm_bound_ms": bound_ms,
            "frac_of_hbm_bound": bound_ms / ms, "generation_s": gen_s,
            "note": "256 canonical products, one call per string, back to back on one stream",
            "one_batched_call": {"ms_per_pass": bms, "value": products / (bms / 1e3), "distinct_out": bterms,
                                 "frac_of_hbm_bound": bound_ms / bms,
                                 "note": "the 256 products as one prepared batch plan (persistent kernel)"}}


def measure_hh(paulib, name, stream, flush, steps, warmup):
    """Canonical H*H over all ordered pairs (two handles) for one workload:
    device time per step and the library's per-stage times."""
    import torch
    h = make_workload(name)
    g1, g2 = paulib.PauliSum.from_arrays(h), paulib.PauliSum.from_arrays(h)
    for _ in range(warmup):
        paulib.multiply(g1, g2).close()
    torch.cuda.synchronize()
    paulib.timing_read(reset=True)
    paulib.timing_enable(True)
    ts = []
    for k in range(steps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = paulib.multiply(g1, g2)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        u = o.n_terms
        o.close()
    paulib.timing_enable(False)
    stage_ms, _ = paulib.timing_read(reset=True)
    g1.close()
    g2.close()
    ms = statistics.mean(ts)
    return {"workload": name, "products": h.m * h.m, "distinct_out": int(u), "ms_per_step": ms,
            "value": h.m * h.m / (ms / 1e3), "unit": UNIT,
            "stage_ms_per_step": {k: v / steps for k, v in stage_ms.items() if v}}


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2605_25974_gb300 import paulib
    paulib.load()
    if args.coarse_factor > 0:
        paulib.set_tuning(0, args.coarse_factor, 0, 0, 0)
    if args.method >= 0:
        paulib.set_slot_tuning(0, args.method)
    gsizes = tuple(int(v) for v in args.grouping_sizes.split(","))
    stream = torch.cuda.current_stream()
    hbm_peak, peak_src = measured_peaks()
    if args.peaks:
        if rank == 0:
            print(json.dumps({"pipe_peaks": paulib.measure_peaks(stream)}), flush=True)
        return
    if args.kernels_case:
        # small case for kernel profiles: a raw and a canonical H*H of the
        # 6,000-term n=200 Jordan-Wigner-shaped H, twice (a few GB on the device)
        hs = make_workload("jw_hh_n200_m6000")
        g1, g2 = paulib.PauliSum.from_arrays(hs), paulib.PauliSum.from_arrays(hs)
        for _ in range(2):
            paulib.multiply(g1, g2, canonical=False).close()
            o = paulib.multiply(g1, g2)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"kernels_case": "jw_hh_n200_m6000", "distinct_out": o.n_terms}), flush=True)
            o.close()
        return
    if args.batched_case:
        # small case for the persistent batched kernel's profile: 512
        # propagation-shaped problems at n=500 (about 5.5e6 products), one
        # plan launched twice
        from paper_2605_25974_gb300 import workloads as wl
        pairs = wl.batch(problems=512)
        As = [paulib.PauliSum.from_arrays(a) for a, _ in pairs]
        Bs = [paulib.PauliSum.from_arrays(b) for _, b in pairs]
        plan = paulib.BatchPlan(As, Bs, "fp32_fp64merge")
        plan.launch()
        outs = plan.outputs()
        if rank == 0:
            print(json.dumps({"batched_case": "batch_n500_512", "products": int(sum(a.m * b.m for a, b in pairs)),
                              "distinct_out": int(sum(o.n_terms for o in outs))}), flush=True)
        plan.close()
        return
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    if args.only_propagation:
        # the gate, rotation and pair-product leg alone (for profiling its kernels)
        res = measure_propagation(paulib, stream, flush, max(3, args.steps), hbm_peak, peak_src)
        if rank == 0:
            print(json.dumps({"propagation": res}), flush=True)
        return
    if args.only_grouping:
        if rank == 0:
            print(json.dumps({"grouping": measure_grouping(paulib, stream, max(5, args.steps), gsizes)}), flush=True)
        return

    h = make_workload(args.workload)
    products = h.m * h.m
    W = h.x.shape[0]
    WP = 1
    while WP < W:
        WP *= 2

    # Two handles holding the same sum: the headline runs the general
    # ordered-pair product over all |H|^2 pairs.  multiply(gh, gh) with one
    # handle takes the symmetric path (pairs i <= j), reported separately.
    gh = paulib.PauliSum.from_arrays(h)
    gh2 = paulib.PauliSum.from_arrays(h)

    def step(prec="fp64", same=False):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = paulib.multiply(gh, gh if same else gh2, prec)
        e1.record(stream)
        return out, e0, e1

    for _ in range(args.warmup):
        out, _, _ = step()
        U = out.n_terms
        out.close()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    paulib.timing_read(reset=True)
    paulib.timing_enable(True)
    step_ms = []
    for k in range(args.steps):
        flush.fill_(k)
        out, e0, e1 = step()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        U = out.n_terms
        out.close()
    torch.cuda.synchronize()
    paulib.timing_enable(False)
    stage_ms, stage_launches = paulib.timing_read(reset=True)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(step_ms), world, "cuda")
    value = job_rate(products, world, ms)
    method = paulib.last_canon_method()

    # ---- the same product through one handle (symmetric pairs i <= j)
    for _ in range(2):
        o, _, _ = step(same=True)
        o.close()
    sym_ms = []
    for k in range(max(2, args.steps // 2)):
        flush.fill_(k)
        o, e0, e1 = step(same=True)
        torch.cuda.synchronize()
        sym_ms.append(e0.elapsed_time(e1))
        assert o.n_terms == U
        o.close()
    sms_ = statistics.mean(sym_ms)
    symmetric = {"ms_per_step": sms_, "value": products / (sms_ / 1e3), "speedup_vs_ordered": ms / sms_,
                 "pair_evaluations": h.m * (h.m + 1) // 2}

    # ---- mixed precision on the same input: speed, and each mode's merged
    # coefficients against the FP64 oracle on sampled output strings
    rng = np.random.default_rng(11)
    pos = np.unique(rng.integers(0, U, 120))
    sampled = {}

    def sample_values(o, name):
        vals = np.zeros(len(pos), np.complex128)
        qx = np.zeros((W, len(pos)), np.uint64)
        qz = np.zeros((W, len(pos)), np.uint64)
        for t, p in enumerate(pos):
            x, z, c, _ = o.export_range(int(p), 1)
            qx[:, t], qz[:, t], vals[t] = x[:, 0], z[:, 0], c[0]
        sampled[name] = (qx, qz, vals)

    o, _, _ = step("fp64")
    sample_values(o, "fp64")
    o.close()
    precision = {}
    for prec in ("fp32_fp64merge", "fp32_twosum"):
        for _ in range(2):
            o, _, _ = step(prec)
            o.close()
        tms = []
        for k in range(max(2, args.steps // 2)):
            flush.fill_(k)
            o, e0, e1 = step(prec)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
            if k == 0:
                assert o.n_terms == U
                sample_values(o, prec)
                assert np.array_equal(sampled[prec][0], sampled["fp64"][0]), "mixed-precision key set differs"
            o.close()
        pm = statistics.mean(tms)
        precision[prec] = {"ms_per_step": pm, "value": products / (pm / 1e3), "speedup_vs_fp64": ms / pm}
    from oracle import pauli_oracle
    qx, qz, _ = sampled["fp64"]
    oc, oabs, _ = pauli_oracle.query_product_coeffs(h.n, h.as_tuple(), h.as_tuple(), qx, qz)
    live = np.abs(oc) > 1e-12  # cancelled strings get absolute errors only
    for name in ("fp64", "fp32_fp64merge", "fp32_twosum"):
        c = sampled[name][2]
        err = np.maximum(np.abs(c.real - oc.real), np.abs(c.imag - oc.imag))
        sc = err / oabs
        rel = err[live] / np.abs(oc[live])
        stats = {"samples": int(len(pos)), "max_err_over_sum_abs": float(sc.max()),
                 "p99_err_over_sum_abs": float(np.quantile(sc, 0.99)),
                 "median_err_over_sum_abs": float(np.median(sc)), "max_abs_err": float(err.max()),
                 "max_rel_err": float(rel.max()) if live.any() else 0.0,
                 "median_rel_err": float(np.median(rel)) if live.any() else 0.0}
        if name == "fp64":
            precision["fp64_vs_oracle"] = stats
        else:
            precision[name]["error_vs_oracle"] = stats
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers, on the same
    # two-handle ordered-pair path as the headline
    hx = torch.from_numpy(h.x.view(np.int64)).pin_memory()
    hz = torch.from_numpy(h.z.view(np.int64)).pin_memory()
    hc = torch.from_numpy(h.c.view(np.float64)).pin_memory()
    ox = torch.empty((W, U), dtype=torch.int64).pin_memory()
    oz = torch.empty((W, U), dtype=torch.int64).pin_memory()
    oc_ = torch.empty((U, 2), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + max(2, args.steps // 2)):
        flush.fill_(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g1 = paulib.PauliSum.create(h.n, hx, hz, hc, stream=stream)
        g2 = paulib.PauliSum.create(h.n, hx, hz, hc, stream=stream)
        o = paulib.multiply(g1, g2, "fp64")
        o.export(ox, oz, oc_, None, stream=stream)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) * 1e3
        if k >= args.warmup:
            e2e_ms.append(dt)
        o.close()
        g1.close()
        g2.close()
    e2e = max_over_ranks(statistics.mean(e2e_ms), world, "cuda")
    h2d = 2 * (hx.numel() * 8 + hz.numel() * 8 + hc.numel() * 8)
    d2h = (ox.numel() + oz.numel() + oc_.numel()) * 8
    del ox, oz, oc_

    # ---- roofline of the dominant stage (the kernels of the stage that takes
    # most device time), from CUDA events recorded on the launching stream
    peaks = paulib.measure_peaks(stream)
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    dom_ms = stage_ms[dom] / args.steps
    term_bytes = 16 * WP + 16 + 1  # key words, complex128, phase byte
    stage_bytes = {
        "count": products * 2,                       # one coarse range id per product
        "scatter": products * (2 + 4),               # range id in, record out
        "level2": products * (4 + 2 + 4),            # one split pass: record in, child id, record out
        "leaf": products * 4 + U * (16 * WP + 16),   # records in, merged terms out (staged)
        "compact": products + U * (2 * (16 * WP + 16) + 1),  # flags, staged terms in, terms out
        "split": products * (4 + 2),                 # slot sort: records in, slot ids out
        "place": products * (4 + 2 + 16 * WP + 16),  # records and slot ids in, terms out
    }
    bytes_per = stage_bytes.get(dom, products * 4)
    kernels = {"leaf": "k_leaf_warp + k_leaf_block", "level2": "k_level2", "count": "k_count_prod",
               "scatter": "k_scatter", "compact": "k_flag_count + k_compact", "split": "k_slot_split + k_slot_locate",
               "place": "k_slot_place"}
    roof = {"bound": "hbm", "achieved": bytes_per / (dom_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "peak_source": peak_src, "stage": dom, "kernel": kernels.get(dom, dom), "bytes_per_step": bytes_per,
            "kernel_ms_per_step": dom_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    tpp, src_hash = traffic_per_product(dom, h.n)
    roof["traffic"] = tpp * products if tpp is not None else None
    roof["traffic_source"] = ("profiles/traffic.json (ncu, pipeline source %s)" % src_hash) if tpp is not None \
        else "none for the current pipeline source"
    if dom in ("leaf", "level2"):
        # these stages gather both factors' key words (and, in the leaf, the
        # coefficients) from L2-resident tables, once per record per pass
        gathered = products * 2 * (16 * WP + (16 if dom == "leaf" else 0))
        l2 = peaks["l2_gather64_bytes_per_s"] / 1e9
        roof["l2_gather_bytes"] = gathered
        roof["l2_gather_GBs"] = gathered / (dom_ms / 1e3) / 1e9
        roof["l2_gather_peak_GBs"] = l2
        roof["l2_gather_frac"] = roof["l2_gather_GBs"] / l2
    roof["stage_ms_per_step"] = {k: v / args.steps for k, v in stage_ms.items() if v}
    # whole-step bound of the method: compulsory traffic (inputs once, merged
    # terms once; the sort's intermediate traffic is overhead), the FP64
    # work (per product: complex product 2 MUL + 2 FMA, merge 2 ADD) and the
    # integer work of key and phase (per product: 2*WP 64-bit XOR + the
    # bit-sliced |x&z| counter, about 6*WP three-input logic ops on 32-bit
    # halves, and 4 population counts), each over its measured pipe rate
    t_hbm = (2 * h.m * term_bytes + U * term_bytes) / (hbm_peak * 1e9)
    t_fp64 = products * 6 / peaks["fp64_fma_per_s"]
    t_int = products * 6 * WP / peaks["lop3_per_s"]
    t_popc = products * 4 / peaks["popc_per_s"]
    bounds = {"hbm": t_hbm, "fp64": t_fp64, "int": t_int, "popc": t_popc}
    roof["step_bound_ms"] = {k: 1e3 * v for k, v in bounds.items()}
    roof["step_binding"] = max(bounds, key=bounds.get)
    roof["step_frac"] = 1e3 * max(bounds.values()) / ms
    roof["pipe_peaks"] = peaks

    outer = measure_outer_product(paulib, gh, gh2, h, stream, flush, max(2, args.steps // 2), hbm_peak, peak_src)
    gh.close()
    gh2.close()
    tiny = measure_tiny(paulib, stream)
    workloads = {"tiny": tiny}
    if not args.no_streaming:
        workloads["streaming"] = measure_streaming(paulib, stream, hbm_peak)
    if args.workload != "jw_hh_n100_m20000" and not args.no_n100:
        workloads["jw_hh_n100_m20000"] = measure_hh(paulib, "jw_hh_n100_m20000", stream, flush,
                                                   max(3, args.steps // 2), 2)
    batched = None
    if not args.no_batched:
        batched = measure_batched(paulib, stream, flush, max(3, args.steps // 2))
    propagation = None
    if not args.no_propagation:
        propagation = measure_propagation(paulib, stream, flush, max(3, args.steps // 2), hbm_peak, peak_src)
    grouping = None
    if not args.no_grouping:
        grouping = measure_grouping(paulib, stream, max(5, args.steps), gsizes)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_qubits": h.n, "terms": h.m, "products": products,
                       "distinct_out": U, "parallelism": "replicas" if world > 1 else "single",
                       "canonical_method": "range sort" if method[0] == 1 else "slot sort",
                       "l2": "512 MiB flush between timed steps"},
            "roofline": roof, "outer_product": outer, "precision": precision, "symmetric": symmetric,
            "workloads": workloads, "batched": batched, "propagation": propagation, "grouping": grouping,
            "e2e": {"value": job_rate(products, world, e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e,
                    "path": "two handles created from pinned host buffers, ordered-pair product, export"},
            "gpu_launches": int(sum(stage_launches.values())),
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baselines(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="jw_hh_n200_m30000", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-products leg")
    ap.add_argument("--no-propagation", action="store_true", help="skip the gate and rotation leg")
    ap.add_argument("--no-grouping", action="store_true", help="skip the commutation-grouping leg")
    ap.add_argument("--only-grouping", action="store_true", help="run the commutation-grouping leg alone")
    ap.add_argument("--only-propagation", action="store_true", help="run the gate, rotation and pair-product leg alone")
    ap.add_argument("--grouping-sizes", default="200,500,1000,2000,20000",
                    help="term counts of the grouping leg (comma separated)")
    ap.add_argument("--no-streaming", action="store_true", help="skip the 1M-term x 256-string streaming leg")
    ap.add_argument("--no-n100", action="store_true", help="skip the n=100 H*H leg")
    ap.add_argument("--peaks", action="store_true", help="print the measured pipe rates and exit")
    ap.add_argument("--kernels-case", action="store_true",
                    help="run the small kernel-profiling case (raw and canonical H*H, n=200, 6,000 terms) and exit")
    ap.add_argument("--batched-case", action="store_true",
                    help="run the small batched-kernel profiling case (512 problems at n=500) and exit")
    ap.add_argument("--method", type=int, default=-1,
                    help="canonicalisation method (0 slot sort, 1 range sort; -1: library default)")
    ap.add_argument("--coarse-factor", type=int, default=0,
                    help="first-level fan-out of the canonicalisation (0: library default); for profiling "
                         "small cases with the range mix of large ones")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
