"""Autotuner for the canonicalisation pipeline.

Times canonical products on representative inputs while sweeping the
pipeline's tunables one at a time (coordinate descent from the defaults):

* coarse_factor      -- first-level key ranges target coarse_factor x the
                        shared-memory leaf capacity records (the fan-out of the
                        first level against the depth of in-CTA splitting);
* oversample         -- splitter sample size per first-level range;
* count_ctas_per_sm  -- CTAs per SM of the first-level counting kernel (its
                        product-tile grid);
* range_ctas_per_sm  -- CTAs per SM of the range sort/merge kernel;
* the canonicalisation method (range sort or slot sort) and, for the slot
  sort, its mean slot size.

Cases: H*H for Jordan-Wigner-shaped sums at n=100 and n=200 (4- and 8-word
keys), and batched products shaped like Pauli-propagation steps at n=500,
timed as prepared plans: on the general pipeline (18-word keys with the
problem prefix) and on the persistent batched kernel, whose leaf capacity
and split fan-out are swept too (written as a line "batch leaf_cap
split_fan").  Results never depend on these settings; only speed does.
The best setting per key width is written as lines "key_words
coarse_factor oversample count_ctas_per_sm range_ctas_per_sm method
leaf_cap slot_target slot_oversample", the format the library reads from
the file named by PAULIB_TUNE_FILE.

    python -m paper_2605_25974_gb300.autotune --out tune.txt [--quick]
"""
from __future__ import annotations

import argparse
import statistics

from . import paulib, workloads


SPACE = {
    "coarse_factor": [8, 16, 32, 64, 128],
    "oversample": [16, 32, 64],
    "count_ctas_per_sm": [2, 4, 8],
    "range_ctas_per_sm": [1, 2],
}
DEFAULT = {"coarse_factor": 32, "oversample": 64, "count_ctas_per_sm": 8, "range_ctas_per_sm": 2,
           "method": 1, "leaf_cap": 0, "slot_target": 0, "slot_oversample": 0}
BATCH_SPACE = {"leaf_cap": [0, 256, 512], "split_fan": [1, 2, 3, 4]}
BATCH_DEFAULT = {"leaf_cap": 0, "split_fan": 2}
# smaller leaves than the default make slots oversized (the multi-pass path,
# which serialises the leaves after it): the slot sort is tuned around its
# default leaf
SLOT_SPACE = {"slot_target": [0, 120, 300]}


def _key_words(n_qubits: int, batched: bool = False) -> int:
    w = (n_qubits + 63) // 64
    wp = 1
    while wp < w:
        wp *= 2
    return 2 * wp + (2 if batched else 0)


def _timed(run, reps: int) -> float:
    import torch
    s = torch.cuda.current_stream()
    run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        run()
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def product_case(a, b):
    def run():
        paulib.multiply(a, b).close()
    return run


def batch_case(As, Bs):
    plan = {"p": None}

    def run():
        if plan["p"] is None:  # a plan is laid out for the settings in force when it is made
            plan["p"] = paulib.BatchPlan(As, Bs, "fp32_fp64merge")
        plan["p"].launch()

    def reset():
        if plan["p"] is not None:
            plan["p"].close()
            plan["p"] = None
    return run, reset


def apply(kw: int, cfg: dict):
    paulib.set_tuning(kw, cfg["coarse_factor"], cfg["oversample"], cfg["count_ctas_per_sm"],
                      cfg["range_ctas_per_sm"])
    paulib.set_slot_tuning(kw, cfg["method"], cfg["leaf_cap"], cfg["slot_target"], cfg["slot_oversample"])


def tune_one(kw: int, run, reps: int, log, reset=None, methods=(1, 0)) -> dict:
    def measure(cfg):
        apply(kw, cfg)
        if reset:
            reset()
        return _timed(run, reps)

    best = dict(DEFAULT)
    best_t = measure(best)
    log("key_words %d default %.3f ms" % (kw, best_t))
    for name, values in SPACE.items():
        for v in values:
            if v == best[name]:
                continue
            cfg = dict(best, **{name: v})
            t = measure(cfg)
            log("  %s=%d: %.3f ms" % (name, v, t))
            if t < best_t * 0.98:
                best, best_t = cfg, t
    if 0 in methods:
        for tgt in SLOT_SPACE["slot_target"]:
            cfg = dict(best, method=0, slot_target=tgt)
            t = measure(cfg)
            log("  slot sort, slot_target=%d: %.3f ms" % (tgt, t))
            if t < best_t * 0.98:
                best, best_t = cfg, t
    apply(kw, best)
    log("key_words %d best %s %.3f ms" % (kw, best, best_t))
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="paulib_tune.txt")
    ap.add_argument("--quick", action="store_true", help="smaller inputs (a few minutes)")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    paulib.load()
    lines = ["# key_words coarse_factor oversample count_ctas_per_sm range_ctas_per_sm "
             "method leaf_cap slot_target slot_oversample"]

    def emit(kw, best):
        lines.append("%d %d %d %d %d %d %d %d %d" % (
            kw, best["coarse_factor"], best["oversample"], best["count_ctas_per_sm"], best["range_ctas_per_sm"],
            best["method"], best["leaf_cap"], best["slot_target"], best["slot_oversample"]))

    m100, m200 = (6000, 4000) if args.quick else (20000, 30000)
    for n, m in ((100, m100), (200, m200)):
        h = workloads.jw(n=n, m=m, seed=300 + n)
        a, b = paulib.PauliSum.from_arrays(h), paulib.PauliSum.from_arrays(h)
        emit(_key_words(n), tune_one(_key_words(n), product_case(a, b), args.reps, print))
        a.close()
        b.close()
    # batched products on the general pipeline (the persistent kernel has no
    # setting here; batches with right operands above its size take this path)
    pairs = workloads.batch(problems=512 if args.quick else 4096)
    As = [paulib.PauliSum.from_arrays(x) for x, _ in pairs]
    Bs = [paulib.PauliSum.from_arrays(y) for _, y in pairs]
    paulib.set_debug(3, 1)
    try:
        run, reset = batch_case(As, Bs)
        emit(_key_words(500, True), tune_one(_key_words(500, True), run, args.reps, print, reset, methods=(1,)))
        reset()
    finally:
        paulib.set_debug(3, 0)
    # the persistent kernel's own sizes
    best, best_t = dict(BATCH_DEFAULT), None
    run, reset = batch_case(As, Bs)

    def measure(cfg):
        paulib.set_batch_tuning(cfg["leaf_cap"], cfg["split_fan"])
        reset()
        return _timed(run, args.reps)
    best_t = measure(best)
    print("persistent batched kernel default %.3f ms" % best_t)
    for name, values in BATCH_SPACE.items():
        for v in values:
            if v == best[name]:
                continue
            cfg = dict(best, **{name: v})
            t = measure(cfg)
            print("  %s=%d: %.3f ms" % (name, v, t))
            if t < best_t * 0.98:
                best, best_t = cfg, t
    reset()
    paulib.set_batch_tuning(best["leaf_cap"], best["split_fan"])
    print("persistent batched kernel best %s %.3f ms" % (best, best_t))
    lines.append("batch %d %d" % (best["leaf_cap"], best["split_fan"]))
    for s in As + Bs:
        s.close()
    with open(args.out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", args.out)


if __name__ == "__main__":
    main()
