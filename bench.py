"""Benchmark of the Stratton-Chu focal-field hot path on GB300.

One step = one pass of the whole path over the broadband workload
(512 x 512 mirror nodes, 256 uniform omegas, 4160 focal points, 10 fs pulse
at f = 62,500 lambda0, NA = 1): spectrum a_n (Eqs. 16-18), per-pair geometry
with the compensated phase, the 24-op field-sum inner loop with the
three-term omega recurrence of the phasor (Eq. 11), the FP64 cross-split reduction and epilogue,
and the inverse transform to 512 time samples (Eq. 13).

Metric: obs x node x omega evaluations per second (surface nodes), whole job.
  value   device-resident inputs and outputs, CUDA events on the library's
          stream around each step; an L2 flush (256 MB memset) runs between
          steps outside the events.
  e2e     the same step through the C-ABI with host buffers: points from
          pinned host memory in, time-domain E(t), B(t) back to pinned host
          memory, copies inside the timed region.
  roofline  the dominant kernel (FP32 field sum) against the FP32-pipe peak
          SMs x 128 lanes x clock, counting the algorithmic work of one
          evaluation of the factorised summand as 28 FP32 instructions (a
          complex rotation and 12 real coefficients times a complex phasor);
          the kernel's own form needs 24, and the line reports that
          fraction too.
  cpu_baseline  the FP64 oracle on the host cores over a bounded sample of
          the same workload.
--impl reference times that oracle as the reference arm.
Multi-GPU (torchrun): every rank evaluates its own copy of the workload
(weak scaling), or with --scaling strong its shard of the points; no data-path
collective either way; timing is max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OPS_PER_EVAL = 28     # algorithmic FP32 instructions per (point, node, omega) of the factorised summand
KERNEL_OPS_PER_EVAL = 24  # what the kernel issues: three-term phasor recurrence, packed FMAs
FIELD_KERNEL = "field_direct_kernel<8, 32>"  # 256 omegas: 32 threads of 8 omegas per point
PROFILE_JSON = os.path.join(ROOT, "profiles", "field_direct_broadband.json")
CSRC = os.path.join(ROOT, "paper_1609_08146_gb300", "csrc")
FIELD_SRCS = [os.path.join(CSRC, f) for f in ("sc_field_direct.cu", "sc_field_common.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and serving legs")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="broadband",
                    choices=["broadband", "profile", "small_omega", "largest", "batched", "tiny", "sweep"],
                    help="broadband: the benchmark workload; profile: the same kernel "
                         "configuration at 128 x 128 nodes, for ncu captures; small_omega: the "
                         "broadband mirror, pulse and points at 256 x 256 nodes and 8 omegas (the "
                         "direct kernel of small requests); largest: the largest "
                         "serving request (1024^2 nodes, GRID^3 points over +-3, 512 omegas, "
                         "512 times) through the fused time-domain path, timed once; batched: the "
                         "batched leg at its full size (64 requests); tiny: 512 small requests "
                         "batched against one by one; sweep: the precision "
                         "sweep over f and node counts (per-component errors)")
    ap.add_argument("--grid", type=int, default=128, help="points per axis of the largest workload")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = every rank evaluates the whole workload (replicas); strong = the "
                         "points are sharded across ranks (sharding.py, no data-path collective) and the "
                         "end-to-end leg gathers E(t) to rank 0 by host copy")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][1]),
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median([num(r[2]) for r in rows if num(r[2]) is not None] or [0])}


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")  # barrier and timing only: no data-path collective
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def oracle_sample_rate(w, seconds: float, amp=True):
    """FP64 oracle on the host cores over a bounded sample of the workload:
    all nodes and omegas at a seeded subset of points, sized to ~seconds.
    Returns (evals/s, point indices, seconds, cores, E, B)."""
    import oracle
    from paper_1609_08146_gb300 import workloads as wl

    m, b = wl.oracle_args(w)
    om = w["omegas"]
    nodes = m["n_r"] * m["n_theta"]
    rng = np.random.Generator(np.random.PCG64(7))
    pts = w["points"]
    a = oracle.spectrum(w["spectrum"], om, b) if amp else None
    # calibrate on one point
    t0 = time.perf_counter()
    oracle.field(m, b, om, pts[:1], amp=a)
    dt1 = time.perf_counter() - t0
    n = int(max(1, min(len(pts), seconds / max(dt1, 1e-6))))
    idx = np.sort(rng.choice(len(pts), size=n, replace=False))
    t0 = time.perf_counter()
    E0, B0 = oracle.field(m, b, om, pts[idx], amp=a)
    dt = time.perf_counter() - t0
    evals = n * nodes * len(om)
    return evals / dt, idx, dt, os.cpu_count(), E0, B0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def oracle_single_core_rate(w, n_omega: int = 32):
    """The same oracle on one thread: one point x all nodes x the first
    n_omega omegas.  Returns (evals/s, seconds)."""
    import oracle
    from paper_1609_08146_gb300 import workloads as wl

    m, b = wl.oracle_args(w)
    om = w["omegas"][:n_omega]
    t0 = time.perf_counter()
    oracle.field(m, b, om, w["points"][:1], threads=1)
    dt = time.perf_counter() - t0
    oracle.field(m, b, om[:1], w["points"][:1], threads=os.cpu_count())  # restore the thread count
    return m["n_r"] * m["n_theta"] * len(om) / dt, dt


def rel_l2(F, R):
    """max over omega of sqrt(mean_points sum_c |F - R|^2) / max_points |R|."""
    F = np.asarray(F, dtype=np.complex128)
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def profile_traffic():
    """DRAM bytes per launch of the field kernel from the committed ncu
    summary, only while the kernel's sources are unchanged since the capture."""
    try:
        prof = json.load(open(PROFILE_JSON))
        sha = hashlib.sha256(b"".join(open(f, "rb").read() for f in FIELD_SRCS)).hexdigest()
        if prof.get("source_sha256") == sha:
            return prof.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def make_config_handles(ctx, configs):
    out = []
    for c in configs:
        mc, b = c["mirror"], c["beam"]
        m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"], rim=mc["rim"])
        inc = ctx.incident(profile=b["profile"], w0=b["w0"], sg_order=b["sg_order"], pol=b["pol"],
                           zernike=b["zernike"], spectrum=c["spectrum"])
        out.append((m, inc, mc["n_r"] * mc["n_theta"]))
    return out


def sampled_oracle_error(configs, reqs, outs, n_points=4, n_omega=16):
    """Max over requests of the R11 error (relative L2 over the sampled points,
    normalised by their largest |F|, max over omega) of the GPU outputs against
    the FP64 oracle at the first n_points points and up to n_omega omegas."""
    import oracle
    from paper_1609_08146_gb300 import workloads as wl

    worst = 0.0
    for r, (E, B) in zip(reqs, outs):
        m, b = wl.oracle_args(configs[r["config"]])
        om = r["omegas"]
        so = np.unique(np.round(np.linspace(0, len(om) - 1, min(n_omega, len(om)))).astype(int))
        a = oracle.spectrum(configs[r["config"]]["spectrum"], om[so], b)
        E0, B0 = oracle.field(m, b, om[so], r["points"][:n_points], amp=a)
        import torch

        ti = torch.as_tensor(so, device=E.device)
        Eg = E.index_select(0, ti)[:, :n_points].cpu().numpy()
        Bg = B.index_select(0, ti)[:, :n_points].cpu().numpy()
        worst = max(worst, rel_l2(Eg, E0), rel_l2(Bg, B0))
    return worst


def full_range_workload_name(n, seed):
    return ("%d seeded uneven requests (seed %d), each its own mirror and beam: f 1e3-1e5 lambda0 "
            "log-uniform, 128^2-1024^2 nodes, 1k-262k points, 1-512 omegas, Gaussian/super-Gaussian, "
            "linear/radial/azimuthal, Zernike j=2..15 N(0, 0.1) waves" % (n, seed))


def batch_leg(sc, torch, dev, n_req=16, seed=1609, check=True, tiny=False):
    """The uneven batch at the batched workload's full ranges: one
    sc_eval_batch against the same requests one by one (both timed after a
    warm-up pass that builds the tables and tunes the shapes); the batch
    must equal the one-by-one results bitwise.  tiny: a mix of small
    requests instead (64^2-128^2 nodes, 256-2048 points, 1-16 omegas), the
    regime where one scheduled pass pays over a call per request."""
    from paper_1609_08146_gb300 import workloads as wl

    if tiny:
        configs, reqs = wl.uneven_requests(n_req, seed, max_nodes=128, max_points=2048, max_omega=16)
    else:
        configs, reqs = wl.full_range_requests(n_req, seed=seed)
    stream = torch.cuda.Stream(device=dev)
    ctx = sc.Context(dev.index or 0, stream=stream)
    hs = make_config_handles(ctx, configs)
    batch = [(hs[r["config"]][0], hs[r["config"]][1], r["omegas"],
              torch.tensor(r["points"], device=dev)) for r in reqs]
    evals = sum(len(r["points"]) * hs[r["config"]][2] * len(r["omegas"]) for r in reqs)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for (m, inc, om, P) in batch:  # tables resident, shapes tuned
            ctx.eval(m, inc, om, P)
        stream.synchronize()
        warm_s = time.perf_counter() - t0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        outs_b = ctx.eval_batch(batch)
        ev[1].record(stream)
        outs_s = [ctx.eval(m, inc, om, P) for (m, inc, om, P) in batch]
        ev[2].record(stream)
        stream.synchronize()
    t_batch = ev[0].elapsed_time(ev[1]) / 1000.0
    t_seq = ev[1].elapsed_time(ev[2]) / 1000.0
    same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(outs_b, outs_s))
    err = sampled_oracle_error(configs, reqs, outs_b) if check else None
    ctx.close()
    return {"requests": n_req, "evals": evals, "value": evals / t_batch, "unit": "evals/s",
            "sequential_value": evals / t_seq, "batch_ms": 1000 * t_batch, "sequential_ms": 1000 * t_seq,
            "bitwise_equal_alone": bool(same), "oracle_rel_l2_err": err,
            "oracle_sample": "first 4 points x up to 16 omegas of every request, FP64 oracle",
            "warmup_s": warm_s,
            "workload": (("%d seeded small requests (seed %d) over 8 mirror/beam configurations: f 1e3-1e5 "
                          "lambda0, 64^2-128^2 nodes, 256-2048 points, 1-16 omegas, Gaussian/super-Gaussian, "
                          "linear/radial/azimuthal, Zernike" % (n_req, seed)) if tiny
                         else full_range_workload_name(n_req, seed))}


def serving_leg(sc, torch, dev, n_req=16, seed=2016, loads=(0.5, 0.8, 0.95), budget=150 << 30):
    """Poisson arrivals of the batched workload's requests (full ranges) at
    fractions of the saturated rate, HBM admission budget 150 GB, node tables
    resident; the same requests serve saturation and every load.  Latency =
    observed completion - submission (library clock), host points copied in
    by the server."""
    from paper_1609_08146_gb300 import workloads as wl

    configs, reqs = wl.full_range_requests(n_req, seed=seed)
    ctx = sc.Context(dev.index or 0, budget_bytes=budget)
    ctx.set_option(sc.SC_OPT_AUTOTUNE, 0)  # no timing runs on the serving path
    hs = make_config_handles(ctx, configs)
    for (m, inc, _) in hs:  # node tables resident before the first arrival
        ctx.eval(m, inc, [1.0], np.zeros((1, 3)))

    def evals(r):
        return len(r["points"]) * hs[r["config"]][2] * len(r["omegas"])

    total = sum(evals(r) for r in reqs)

    def run(arrivals, keep=()):
        t0 = time.perf_counter()
        pending, lat, kept = [], [], {}
        i = 0
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and arrivals[i] <= now:
                r = reqs[i]
                m, inc, _ = hs[r["config"]]
                pending.append((i, ctx.submit(m, inc, r["omegas"], r["points"])))
                i += 1
            still = []
            for k, t in pending:
                if ctx.poll(t):
                    s0, s1, s2 = ctx.ticket_times(t)
                    lat.append(s2 - s0)
                    if k in keep:
                        kept[k] = ctx.fetch(t)
                    ctx.release(t)
                else:
                    still.append((k, t))
            pending = still
            time.sleep(0.0002)
        return lat, time.perf_counter() - t0, kept

    # saturated: everything submitted at once; two small requests kept for the error check
    order = sorted(range(len(reqs)), key=lambda k: evals(reqs[k]))
    keep = tuple(order[:2])
    lat, wall, kept = run([0.0] * len(reqs), keep=keep)
    sat_rate = len(reqs) / wall
    err = sampled_oracle_error(configs, [reqs[k] for k in keep], [kept[k] for k in keep])
    out = {"saturated_req_per_s": sat_rate, "saturated_evals_per_s": total / wall,
           "requests": n_req, "evals": total, "budget_bytes": budget,
           "oracle_rel_l2_err": err,
           "oracle_sample": "the two smallest requests as served: first 4 points x up to 16 omegas",
           "workload": full_range_workload_name(n_req, seed) + ", Poisson arrivals, same requests at every load",
           "rates": []}
    rng = np.random.Generator(np.random.PCG64(5))
    draws = [(load, load * sat_rate) for load in loads]
    draws = [(load, rate, np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))) for load, rate in draws]

    def point(load, rate, arrivals):
        lat, wall, _ = run(arrivals)
        lat_ms = 1000.0 * np.array(lat)
        return {"load": load, "rate_req_per_s": rate, "requests": len(reqs),
                "p50_ms": float(np.percentile(lat_ms, 50)),
                "p99_ms": float(np.percentile(lat_ms, 99)),
                "throughput_evals_per_s": total / wall}

    for d in draws:
        out["rates"].append(point(*d))
    # the same arrivals, first come first served (SC_OPT_SERVE_PRIORITY = 0)
    ctx.set_option(sc.SC_OPT_SERVE_PRIORITY, 0)
    out["fifo_rates"] = [point(*d) for d in draws]
    out["policy"] = ("short requests (<= 1e11 evals) first on two high-priority lanes; long ones on two "
                     "low-priority lanes in launches of about 6e10 evals; fifo_rates: the same arrivals first "
                     "come first served on two lanes")
    ctx.close()
    return out


def run_reference(args, rank, world, pg):
    from paper_1609_08146_gb300 import workloads as wl

    w = wl.broadband()
    if rank != 0:
        return
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps))
    rates = []
    for i in range(args.warmup + args.steps):
        r, idx, dt, cores, _, _ = oracle_sample_rate(w, per_step)
        if i >= args.warmup:
            rates.append((r, len(idx), dt, cores))
    value = statistics.median([r[0] for r in rates])
    cores = rates[0][3]
    sample = "%d of %d points x all %d nodes x %d omegas per step (FP64 oracle, OpenMP)" % (
        rates[0][1], len(w["points"]), w["mirror"]["n_r"] * w["mirror"]["n_theta"], len(w["omegas"]))
    line = {
        "impl": "reference", "metric": "Stratton-Chu obs*node*omega evals/s", "value": value,
        "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.median([r[2] for r in rates]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "sampled": True},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def component_errors(F, R):
    """Per component c: max over omega of sqrt(mean_points |F_c - R_c|^2) /
    max_points |R| (the R11 metric split by component)."""
    F = np.asarray(F, dtype=np.complex128)
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    num = np.sqrt(np.mean(np.abs(F - R) ** 2, axis=1))  # [omega, c]
    return [float(np.max(num[:, c] / np.maximum(den, 1e-300))) for c in range(3)]


def run_sweep(args, ctx, sc, torch, dev, stream, wl):
    """Precision sweep: the broadband pulse's 256 omegas (unit amplitudes: the
    errors are those of the spatial sums) at f in {1e2, 1e3, 1e4, 1e5} lambda0
    and 256^2, 512^2, 1024^2 nodes, 4096 seeded points in the +-2 cube.
    FP32-compensated on every point, the FP64 GPU form on every 16th point,
    the FP64 oracle on every 512th; per-component error of E and B for each
    pair, and the field time of each form."""
    import oracle

    rows = []
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    clk.start()
    for n_nodes in (256, 512, 1024):
        for f in (1e2, 1e3, 1e4, 1e5):
            w = wl.sweep(f, n_nodes, n_points=4096)
            mc, b = w["mirror"], w["beam"]
            om = w["omegas"]
            m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"], rim=mc["rim"])
            inc = ctx.incident(profile=b["profile"], w0=b["w0"], pol=b["pol"],
                               spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
            with torch.cuda.stream(stream):
                P = torch.tensor(w["points"], device=dev)
                ctx.eval(m, inc, om, P[:8])  # table resident
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                e[0].record(stream)
                E32, B32 = ctx.eval(m, inc, om, P)
                e[1].record(stream)
                E64, B64 = ctx.eval(m, inc, om, P[::16], precision="fp64")
                e[2].record(stream)
                stream.synchronize()
            sel = np.arange(0, 4096, 512)
            mo, bo = wl.oracle_args(w)
            t0 = time.perf_counter()
            E0, B0 = oracle.field(mo, bo, om, w["points"][sel])
            t_or = time.perf_counter() - t0
            e32 = E32.cpu().numpy()
            b32 = B32.cpu().numpy()
            e64 = E64.cpu().numpy()
            b64 = B64.cpu().numpy()
            rows.append({
                "f_lambda0": f, "nodes": n_nodes * n_nodes,
                "fp32_vs_oracle": {"E": component_errors(e32[:, sel], E0), "B": component_errors(b32[:, sel], B0)},
                "fp64_vs_oracle": {"E": component_errors(e64[:, sel // 16], E0),
                                   "B": component_errors(b64[:, sel // 16], B0)},
                "fp32_vs_fp64_gpu": {"E": component_errors(e32[:, ::16], e64),
                                     "B": component_errors(b32[:, ::16], b64)},
                "fp32_vs_fp64_gpu_at_oracle_points": {"E": component_errors(e32[:, sel], e64[:, sel // 16]),
                                                      "B": component_errors(b32[:, sel], b64[:, sel // 16])},
                "fp32_ms": e[0].elapsed_time(e[1]), "fp64_ms_256_points": e[1].elapsed_time(e[2]),
                "oracle_s_8_points": t_or})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    clocks = clk.stop()
    line = {"metric": "precision sweep: per-component relative L2 error (R11 metric by component)",
            "config": {"workload": "broadband pulse, 256 omegas, f 1e2-1e5 lambda0, 256^2-1024^2 nodes, "
                                   "4096 seeded points in +-2 lambda0",
                       "samples": "FP32 all 4096 points; FP64 GPU every 16th (256); oracle every 512th (8); "
                                  "each error is normalised by the largest |F| over its own point set, so "
                                  "the 8-point errors read higher than the 256-point ones"},
            "rows": rows, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_largest(args, ctx, sc, torch, dev, stream, wl):
    """The largest serving request: the broadband mirror and pulse at 1024^2
    nodes and 512 omegas, a GRID^3 point grid over +-3 lambda0 and 512 time
    samples, straight to E(t), B(t) through sc_eval_time_domain (device
    buffers, one timed call after the node table is resident)."""
    w = wl.broadband(n_nodes=1024, n_omega=512)
    mc = w["mirror"]
    m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"], rim=mc["rim"])
    inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"], pol="linear", spectrum=w["spectrum"])
    x = np.linspace(-3.0, 3.0, args.grid)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    pts = torch.tensor(np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), device=dev)
    om, times = w["omegas"], w["times"]
    ctx.set_option(sc.SC_OPT_AUTOTUNE, 0)  # heuristic splits: no timing runs at this size
    with torch.cuda.stream(stream):
        ctx.eval(m, inc, om[:8], pts[:64])  # builds the 1024^2 node table
        stream.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        clk = ClockSampler(dev.index if dev.index is not None else 0)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Et, Bt, st = ctx.eval_time_domain(m, inc, om, pts, times, stats=True)
        e1.record(stream)
        stream.synchronize()
        clocks = clk.stop()
        free1 = torch.cuda.mem_get_info(dev)[0]
    ms = e0.elapsed_time(e1)
    evals = float(pts.shape[0]) * mc["n_r"] * mc["n_theta"] * len(om)
    line = {"metric": "Stratton-Chu obs*node*omega evals/s", "value": evals / (ms / 1000.0),
            "unit": "evals/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "largest serving request: broadband mirror and pulse, 1024^2 nodes, "
                                   "%d^3 points over +-3, 512 omegas, 512 times, fused time domain"
                                   % args.grid, "points": int(pts.shape[0]), "evals": evals},
            "field_ms": st["field_ms"], "launches": st["launches"],
            "device_bytes_allocated_during_call": int(free0 - free1), "clocks": clocks,
            "output_bytes": int(2 * Et.numel() * 4),
            "note": "one timed call; the node table is built before the timed region; the "
                    "allocated bytes include the E(t), B(t) outputs"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world, pg)
        return
    import torch

    import paper_1609_08146_gb300 as sc
    from paper_1609_08146_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    ctx = sc.Context(local, stream=stream)
    if args.workload == "largest":
        run_largest(args, ctx, sc, torch, dev, stream, wl)
        return
    if args.workload == "sweep":
        run_sweep(args, ctx, sc, torch, dev, stream, wl)
        return
    if args.workload in ("batched", "tiny"):
        clk = ClockSampler(local)
        clk.start()
        if args.workload == "batched":
            res = batch_leg(sc, torch, dev, n_req=64, seed=1609)
        else:
            res = batch_leg(sc, torch, dev, n_req=512, seed=7, tiny=True)
        res["clocks"] = clk.stop()
        res["metric"] = "Stratton-Chu obs*node*omega evals/s (batched)"
        print(json.dumps(res), flush=True)
        return
    if args.workload == "broadband":
        w = wl.broadband()
    elif args.workload == "small_omega":
        w = wl.broadband(n_nodes=256, n_omega=8)
    else:
        w = wl.broadband(n_nodes=128)
    mc = w["mirror"]
    m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"], rim=mc["rim"])
    inc = ctx.incident(profile=w["beam"]["profile"], w0=w["beam"]["w0"], pol=w["beam"]["pol"],
                       spectrum=w["spectrum"])
    om, times = w["omegas"], w["times"]
    n_nodes = mc["n_r"] * mc["n_theta"]
    strong = args.scaling == "strong" and world > 1
    n_total = len(w["points"])
    if strong:  # this rank's contiguous shard of the points
        from paper_1609_08146_gb300.sharding import shard_range

        lo, hi = shard_range(n_total, rank, world)
        w = dict(w, points=w["points"][lo:hi])
    npts = len(w["points"])
    evals_per_step = float(npts) * n_nodes * len(om)

    with torch.cuda.stream(stream):
        P = torch.tensor(w["points"], device=dev)
        E = torch.empty((len(om), npts, 3), dtype=torch.complex64, device=dev)
        B = torch.empty_like(E)
        Et = torch.empty((len(times), npts, 3), dtype=torch.float32, device=dev)
        Bt = torch.empty_like(Et)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        ctx.eval(m, inc, om, P, out=(E, B))
        ctx.time_domain(E, B, om, times, out=(Et, Bt))

    # warm-up (builds and uploads the node table on the first call)
    for _ in range(args.warmup):
        step()
    stream.synchronize()

    # ---- device-resident timed region
    ctx.reset_counters()
    ctx.set_option(sc.SC_OPT_TIME_FIELD, 1)
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between steps, outside the events
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ctr = ctx.counters()
    ctx.set_option(sc.SC_OPT_TIME_FIELD, 0)
    total_ms = max_over_ranks(pg, sum(step_ms))
    value = sum_over_ranks(pg, evals_per_step * args.steps) / (total_ms / 1000.0)
    launches_per_step = ctr["launches"] / args.steps
    field_ms = ctr["field_ms"] / max(1, ctr["field_launches"])
    field_evals = evals_per_step * args.steps / max(1, ctr["field_launches"])

    # ---- end to end through the C-ABI with host buffers
    Ph = torch.tensor(w["points"]).pin_memory()
    Eth = torch.empty((len(times), npts, 3), dtype=torch.float32).pin_memory()
    Bth = torch.empty_like(Eth).pin_memory()
    ctx.eval(m, inc, om, Ph.to(dev), out=(E, B))  # keep the table resident
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.eval(m, inc, om, Ph, out=(E, B))          # points: pinned host -> device
        ctx.time_domain(E, B, om, times, out=(Eth, Bth))  # E(t), B(t): device -> pinned host
        if strong:  # the whole E(t) on rank 0, by host copy over the process group
            from paper_1609_08146_gb300.sharding import gather_points

            gather_points(Eth, n_total, dim=1)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
    e2e_value = sum_over_ranks(pg, evals_per_step * args.steps) / e2e_s
    h2d = int(Ph.numel() * 8 + om.size * 8)
    d2h = int(Eth.numel() * 4 + Bth.numel() * 4)

    # ---- roofline of the dominant kernel
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak = sms * 128 * max_mhz * 1e6 * 1e-12  # TOP/s of FP32 lane-ops at the maximum SM clock
    achieved = field_evals * OPS_PER_EVAL / (field_ms / 1000.0) * 1e-12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
            "frac": achieved / peak,
            "traffic": profile_traffic() if args.workload != "small_omega" else None,
            "kernel": FIELD_KERNEL if args.workload != "small_omega" else "field_direct_kernel<4, 2>",
            "ops_per_eval": OPS_PER_EVAL,
            "ops_basis": "algorithmic work per evaluation: complex rotation (4) + 12 real coefficients "
                         "x complex phasor (24)",
            "kernel_ops_per_eval": KERNEL_OPS_PER_EVAL,
            "frac_at_kernel_ops": achieved / peak * KERNEL_OPS_PER_EVAL / OPS_PER_EVAL,
            "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (max SM clock)" % (sms, max_mhz),
            "kernel_ms": field_ms}
    if clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (sms * 128 * clk["sm_mhz"] * 1e6 * 1e-12)
    # what the FMA and MUFU pipes sustain on pure instruction streams (after the timed region)
    probes = ctx.measure_alu_peaks()
    fma_t = probes["fp32_lane_ops_per_s"] * 1e-12
    fma2_t = probes["fp32x2_lane_ops_per_s"] * 1e-12
    roof["measured_pipes"] = {
        "fp32_fma_TOPs": fma_t, "fp32_ffma2_TOPs": fma2_t,
        "mufu_Tops": probes["mufu_ops_per_s"] * 1e-12,
        "fma_frac_of_peak": max(fma_t, fma2_t) / peak,
        "basis": "sc_measure_alu_peaks: independent FFMA, FFMA2 and MUFU rsqrt streams on every SM, "
                 "best of 3 launches, clocks not pinned"}
    roof["frac_of_measured_fma"] = achieved / max(fma_t, fma2_t)

    # ---- plain FP64 GPU form of the same sum, on a point subsample
    sub = torch.tensor(w["points"][::65], device=dev)  # 64 points
    ctx.eval(m, inc, om, sub[:2], precision="fp64")
    e64 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        e64[0].record(stream)
        E64, B64 = ctx.eval(m, inc, om, sub, precision="fp64")
        e64[1].record(stream)
    stream.synchronize()
    fp64_rate = float(sub.shape[0]) * n_nodes * len(om) / (e64[0].elapsed_time(e64[1]) / 1000.0)
    fp64 = {"value": fp64_rate, "unit": "evals/s", "sample": "%d points x all nodes x all omegas"
            % sub.shape[0], "fp32_speedup": (value / world) / fp64_rate}

    # ---- batched uneven requests and serving (single GPU, rank 0)
    batched = serving = None
    if rank == 0 and world == 1 and not args.no_extras:
        batched = batch_leg(sc, torch, dev)
        serving = serving_leg(sc, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, idx, dt, cores, E0, B0 = oracle_sample_rate(w, args.cpu_seconds)
        r1, dt1 = oracle_single_core_rate(w)
        cpu = {"value": r, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "%d of %d points x all %d nodes x %d omegas (%.1f s, FP64 OpenMP)"
               % (len(idx), npts, n_nodes, len(om), dt),
               "cpu_model": cpu_model(), "single_core_value": r1,
               "single_core_sample": "1 point x all nodes x 32 omegas on one thread (%.1f s)" % dt1}
        # the oracle's sampled outputs also give the error of both GPU forms
        ti = torch.tensor(idx, device=dev)
        Eg = E.index_select(1, ti).cpu().numpy()
        Bg = B.index_select(1, ti).cpu().numpy()
        E6, B6 = ctx.eval(m, inc, om, P.index_select(0, ti), precision="fp64")
        torch.cuda.synchronize()
        cpu["fp32_rel_l2_err"] = max(rel_l2(Eg, E0), rel_l2(Bg, B0))
        cpu["fp64_rel_l2_err"] = max(rel_l2(E6.cpu().numpy(), E0), rel_l2(B6.cpu().numpy(), B0))
        fp64["fp32_rel_l2_err"] = cpu["fp32_rel_l2_err"]
        fp64["fp64_rel_l2_err"] = cpu["fp64_rel_l2_err"]

    if rank == 0:
        line = {
            "metric": "Stratton-Chu obs*node*omega evals/s", "value": value, "unit": "evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if strong else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "mirror_nodes": n_nodes, "points": npts,
                       "omegas": len(om), "time_samples": len(times), "f_lambda0": mc["f"],
                       "precision": "FP32 compensated phase, FP64 cross-split reduction",
                       "l2": "256 MB memset between steps, outside the timed events",
                       "parallelism": ("points sharded over %d GPUs" % world if strong else
                                       "replicas" if world > 1 else "single GPU")},
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(ctr["launches"]),
            "gpu_launches_per_step": launches_per_step,
            "roofline": roof,
            "fp64_gpu": fp64,
            "batched": batched,
            "serving": serving,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
