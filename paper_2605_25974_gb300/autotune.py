"""Autotuner for the canonicalisation pipeline.

Times the canonical product on representative inputs while sweeping the
pipeline's tunables one at a time (coordinate descent from the defaults):

* coarse_factor      -- first-level key ranges target coarse_factor x the
                        shared-memory leaf capacity records (the fan-out of the
                        first level against the depth of in-CTA splitting);
* oversample         -- splitter sample size per first-level range;
* count_ctas_per_sm  -- CTAs per SM of the first-level counting kernel (its
                        product-tile grid);
* range_ctas_per_sm  -- CTAs per SM of the range sort/merge kernel.

Results never depend on these; only speed does.  The best setting per key
width is written as lines "key_words coarse_factor oversample
count_ctas_per_sm range_ctas_per_sm", the format the library reads from the
file named by PAULIB_TUNE_FILE.

    python -m paper_2605_25974_gb300.autotune --out tune.txt [--quick]
"""
from __future__ import annotations

import argparse
import statistics

from . import paulib, workloads


SPACE = {
    "coarse_factor": [4, 8, 16, 32, 64],
    "oversample": [16, 32, 64],
    "count_ctas_per_sm": [2, 4, 8],
    "range_ctas_per_sm": [1, 2],
}
DEFAULT = {"coarse_factor": 32, "oversample": 32, "count_ctas_per_sm": 4, "range_ctas_per_sm": 2}


def _key_words(n_qubits: int, batched: bool = False) -> int:
    w = (n_qubits + 63) // 64
    wp = 1
    while wp < w:
        wp *= 2
    return 2 * wp + (2 if batched else 0)


def time_product(a, b, reps: int = 3) -> float:
    import torch
    s = torch.cuda.current_stream()
    out = paulib.multiply(a, b)
    out.close()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        out = paulib.multiply(a, b)
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        out.close()
    return statistics.median(ts)


def tune_one(kw: int, a, b, reps: int, log) -> dict:
    best = dict(DEFAULT)

    def apply(cfg):
        paulib.set_tuning(kw, cfg["coarse_factor"], cfg["oversample"], cfg["count_ctas_per_sm"],
                          cfg["range_ctas_per_sm"])

    apply(best)
    best_t = time_product(a, b, reps)
    log("key_words %d default %.3f ms" % (kw, best_t))
    for name, values in SPACE.items():
        for v in values:
            if v == best[name]:
                continue
            cfg = dict(best)
            cfg[name] = v
            apply(cfg)
            t = time_product(a, b, reps)
            log("  %s=%d: %.3f ms" % (name, v, t))
            if t < best_t * 0.98:
                best, best_t = cfg, t
        apply(best)
    log("key_words %d best %s %.3f ms" % (kw, best, best_t))
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="paulib_tune.txt")
    ap.add_argument("--quick", action="store_true", help="smaller inputs (a minute or two)")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    paulib.load()
    cases = []
    m100, m200 = (6000, 4000) if args.quick else (20000, 30000)
    for n, m in ((100, m100), (200, m200)):
        h = workloads.jw(n=n, m=m, seed=300 + n)
        cases.append((_key_words(n), paulib.PauliSum.from_arrays(h), paulib.PauliSum.from_arrays(h)))
    lines = ["# key_words coarse_factor oversample count_ctas_per_sm range_ctas_per_sm"]
    for kw, a, b in cases:
        best = tune_one(kw, a, b, args.reps, print)
        lines.append("%d %d %d %d %d" % (kw, best["coarse_factor"], best["oversample"], best["count_ctas_per_sm"],
                                         best["range_ctas_per_sm"]))
        a.close()
        b.close()
    with open(args.out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", args.out)


if __name__ == "__main__":
    main()
