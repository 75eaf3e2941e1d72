"""Re-measure the omega-chunk tables of the FP32 path on this GPU.

The FP32 path cuts a request's uniform omega grid into chunks, each one pass
of a field kernel over the node tables.  It chooses the cut that minimises
the summed field time of the chunks, from the field throughput of one chunk
of n omegas.  This tool measures that throughput with chunk planning off, on
the broadband mirror and beam at 256 x 256 nodes and 4160 focal points:

* for every n = 1..64;
* for full grouped chunks of 64, 128, ..., 2048 omegas.  A grouped chunk of
  n > 64 omegas takes as long as a full one of its capacity, the next power
  of two >= n.

It prints both tables in the form of csrc/sc_batch.cpp (kRateSmall,
kRateFull), in units of 1e11 evaluations per second.  `first_chunks` is the
same split search as the library's, written again here for the tests.

With --layouts it instead times both tile shapes (threads per point x omegas
per thread) of the omega counts that have two, pinned with
SC_OPT_TILE_LAYOUT, and the shape the autotuner takes, at 4160 and 1040
points: one JSON line per (points, n).

    python -m paper_1609_08146_gb300.tune_chunks
    python -m paper_1609_08146_gb300.tune_chunks --layouts
"""
from __future__ import annotations

MAX_CHUNK = 2048
FULL = (64, 128, 256, 512, 1024, 2048)


def measure(reps: int = 3):
    """(small, full): field throughput in 1e11 evals/s of one chunk of n
    omegas, n = 1..64, and of full chunks of 64 .. 2048 omegas."""
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

        def rate(n):
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
            return evals / (c["field_ms"] * 1e-3) * 1e-11

        small = [0.0] + [rate(n) for n in range(1, 65)]
        full = [rate(n) for n in FULL]
        return small, full
    finally:
        ctx.close()


LAYOUT_COUNTS = (8, 11, 12, 15, 16, 40, 48, 57, 64, 100, 128)


def measure_layouts(counts=LAYOUT_COUNTS, n_points=(4160, 1040), reps: int = 5):
    """For each point count and omega count: {layout: (1e11 evals/s, kernel
    class, splits)} for SC_OPT_TILE_LAYOUT 0 (default shape), 1 (alternative)
    and -1 (autotuned)."""
    import torch

    import paper_1609_08146_gb300 as sc
    from paper_1609_08146_gb300 import workloads as wl

    w = wl.broadband(256, 8)
    ctx = sc.Context(0)
    rows = []
    try:
        m = w["mirror"]
        mir = ctx.mirror(m["f"], m["r_min"], m["r_max"], m["n_r"], m["n_theta"], rim=m["rim"])
        b = w["beam"]
        inc = ctx.incident(profile=b["profile"], w0=b["w0"], pol=b["pol"], spectrum=w["spectrum"])
        allp = torch.tensor(w["points"], device="cuda")
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
        for P in n_points:
            pts = allp[:P].contiguous()
            for n in counts:
                om = wl.uniform_omegas(n)
                row = dict(points=P, n_omega=n)
                for lay in (0, 1, -1):
                    ctx.set_option(sc.SC_OPT_TILE_LAYOUT, lay)
                    for _ in range(2):
                        _, _, st = ctx.eval(mir, inc, om, pts, stats=True)
                    ctx.set_option(sc.SC_OPT_TIME_FIELD, 1)
                    ctx.reset_counters()
                    for _ in range(reps):
                        ctx.eval(mir, inc, om, pts)
                    c = ctx.counters()
                    ctx.set_option(sc.SC_OPT_TIME_FIELD, 0)
                    evals = reps * P * m["n_r"] * m["n_theta"] * n
                    row[str(lay)] = (round(evals / (c["field_ms"] * 1e-3) * 1e-11, 3),
                                     st["kernel_class"], st["splits"])
                rows.append(row)
        return rows
    finally:
        ctx.set_option(sc.SC_OPT_TILE_LAYOUT, -1)
        ctx.close()


def chunk_cost(c: int, small, full) -> float:
    """Relative field time of one chunk of c omegas."""
    if c <= 64:
        return c / small[c]
    cap, i = 128, 1
    while cap < c:
        cap, i = cap * 2, i + 1
    return cap / full[i]


def first_chunks(small, full, small_cuts: bool = True, penalty: float = 0.02) -> list:
    """First chunk of the cheapest split of every n <= 2048 (index n): splits
    at any count up to 64 when small_cuts, else only at full grouped
    capacities; each extra chunk costs `penalty` of a 32-omega chunk."""
    extra = penalty * chunk_cost(32, small, full)
    best = [0.0] * (MAX_CHUNK + 1)
    first = [0] * (MAX_CHUNK + 1)
    for m in range(1, MAX_CHUNK + 1):
        b, f = chunk_cost(m, small, full), m
        cands = list(range(1, min(m - 1, 64) + 1)) if small_cuts else ([64] if m > 64 else [])
        c = 128
        while c < m:
            cands.append(c)
            c *= 2
        for c in cands:
            v = chunk_cost(c, small, full) + best[m - c] + extra
            if v < b:
                b, f = v, c
        best[m], first[m] = b, f
    return first


def plan(n_omega: int, first: list) -> list:
    """Chunk sizes of a request of n_omega omegas under a first-chunk table."""
    out = []
    while n_omega > 0:
        c = first[min(n_omega, MAX_CHUNK)]
        out.append(c)
        n_omega -= c
    return out


def main():
    import sys
    if "--layouts" in sys.argv[1:]:
        import json
        for row in measure_layouts():
            print(json.dumps(row), flush=True)
        return
    small, full = measure()
    print("constexpr double kRateSmall[65] = {\n    0.0,")
    for i in range(1, 65, 8):
        print("    " + ", ".join("%.3f" % v for v in small[i:i + 8]) + ",  // %d..%d" % (i, i + 7))
    print("};")
    print("constexpr double kRateFull[6] = {" + ", ".join("%.3f" % v for v in full) + "};  // 64 .. 2048")


if __name__ == "__main__":
    main()
