"""Re-measure the small-omega chunk table of the FP32 path on this GPU.

For every omega count n = 1..64 it times the field kernel of one chunk of n
uniform omegas (chunk planning off), on the broadband mirror and beam at
256 x 256 nodes and 4160 focal points, then finds for every n the split into
chunks that minimises the summed field time, charging each extra chunk 2% of
a 32-omega chunk.  It prints the first chunk of each best split as the
kFirstChunk table of csrc/sc_batch.cpp.

    python -m paper_1609_08146_gb300.tune_chunks
"""
from __future__ import annotations

import numpy as np


def measure(n_max: int = 64, reps: int = 3) -> dict:
    """Field-kernel throughput (evals/s) of one chunk of n omegas."""
    import torch

    import paper_1609_08146_gb300 as sc
    from paper_1609_08146_gb300 import workloads as wl

    w = wl.broadband(256, 8)
    ctx = sc.Context(0)
    try:
        m = w["mirror"]
        mir = ctx.mirror(m["f"], m["r_min"], m["r_max"], m["n_r"], m["n_theta"], rim=m["rim"])
        b = w["beam"]
        inc = ctx.incident(profile=b["profile"], w0=b["w0"], pol=b["pol"], spectrum=w["spectrum"])
        pts = torch.tensor(w["points"], device="cuda")
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
        rate = {}
        for n in range(1, n_max + 1):
            om = wl.uniform_omegas(n)
            for _ in range(2):
                ctx.eval(mir, inc, om, pts)
            ctx.set_option(sc.SC_OPT_TIME_FIELD, 1)
            ctx.reset_counters()
            for _ in range(reps):
                ctx.eval(mir, inc, om, pts)
            c = ctx.counters()
            ctx.set_option(sc.SC_OPT_TIME_FIELD, 0)
            evals = reps * len(w["points"]) * m["n_r"] * m["n_theta"] * n
            rate[n] = evals / (c["field_ms"] * 1e-3)
        return rate
    finally:
        ctx.close()


def first_chunks(rate: dict, penalty: float = 0.02) -> list:
    """First chunk of the cheapest split of every n (index n; 0 unused)."""
    n_max = max(rate)
    cost = {c: c / rate[c] for c in rate}
    extra = penalty * cost[32]
    best = np.zeros(n_max + 1)
    first = [0] * (n_max + 1)
    for n in range(1, n_max + 1):
        opts = [(cost[c] + best[n - c] + (extra if c < n else 0.0), c) for c in range(1, n + 1)]
        best[n], first[n] = min(opts)  # ties: the smaller first chunk
    return first


def main():
    rate = measure()
    first = first_chunks(rate)
    for n in sorted(rate):
        print("%3d omegas: %.3e evals/s" % (n, rate[n]))
    print("constexpr unsigned char kFirstChunk[65] = {")
    print("    0, " + ", ".join(str(v) for v in first[1:]) + "};")


if __name__ == "__main__":
    main()
