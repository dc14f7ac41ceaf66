"""Benchmark of the pairwise force loop on GB300.

Workload (default): the 2^20-particle all-pairs Newton set, half a Plummer
sphere and half a uniform cube of side 4, log-uniform masses, eps = 1e-3,
FP64 positions with FP32 offsets from FP64 tile centres and compensated
accumulation. One step = one force evaluation of every particle from every
particle (i staging and ordering, pair loop, reduction and output), 2^40
pair evaluations. Metric: interactions per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload instead.
Under torchrun (N > 1) the i-range is split across ranks (strong scaling, no
data-path collective: every rank generates the same seeded inputs).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

N_PART = 1 << 20
EPS = 1e-3
NEWTON_OPS = 13          # FP32-pipe lane-ops per Newton interaction (f32x2 counts 2)
FP32_LANES_PER_SM = 128
PAPER_FLOPS_PER_INT = 38
TREE_NCRIT = 256         # group size bound of the tree rows
HEADLINE_TRAFFIC = 96.95e6   # DRAM bytes of one 2^20 headline force launch (ncu, read 75.95 + write 21.00 MB)


def tree_model(model, n):
    """The tree runs' particle sets (Section 5.1): a Plummer sphere or a King
    model with W0 = 9, equal masses."""
    if model == "king":
        return gen.king(n, gen.CONFIG_SEEDS[2], W0=9.0)
    return gen.plummer(n, gen.CONFIG_SEEDS[2])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pg", choices=["pg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true")
    ap.add_argument("--n", type=int, default=N_PART,
                    help="particle count (default: the 2^20 workload; smaller for profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only: no e2e, extra rows or CPU baseline")
    ap.add_argument("--shape", default=None,
                    help="np,packed launch shape of the force kernel (default: the library's)")
    ap.add_argument("--workload", default="newton",
                    choices=["newton", "table", "cells", "groups", "backward", "narrow", "tree", "pm",
                             "small"],
                    help="newton: the headline; the others time one row of the path alone "
                         "(for profiling) and print its measurements")
    ap.add_argument("--model", default="plummer", choices=["plummer", "king"],
                    help="tree workload: the particle set")
    ap.add_argument("--quadrupole", action="store_true",
                    help="tree workload: quadrupole pseudo-particles")
    ap.add_argument("--level-walk", action="store_true",
                    help="tree workload: the level walk instead of the group walk")
    ap.add_argument("--ncrit", type=int, default=TREE_NCRIT, help="tree workload: group size bound")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(x, m, target_s=12.0):
    """The FP64 oracle as it stands, timed on this host's cores on a bounded
    sample of i against all j (interactions/s)."""
    import oracle
    oracle.build()
    nth = oracle.nthreads()
    # calibrate on a small sample, then size the timed sample
    idx = gen.sample_indices(len(x), 64, 4242)
    t0 = time.perf_counter()
    oracle.newton_subset(x, m, EPS, idx, nthreads_=nth)
    dt = max(time.perf_counter() - t0, 1e-3)
    k = int(min(len(x), max(64, 64 * target_s / dt)))
    idx = gen.sample_indices(len(x), k, 4243)
    t0 = time.perf_counter()
    oracle.newton_subset(x, m, EPS, idx, nthreads_=nth)
    dt = time.perf_counter() - t0
    pairs = len(idx) * len(x)
    return {"value": pairs / dt, "unit": "interactions/s", "cores": nth, "kind": "oracle",
            "sample": f"{len(idx)} i-particles x {len(x)} j-particles of the same set "
                      f"({pairs:.3e} FP64 pairs, {dt:.1f} s)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    x, m = gen.plummer_cube_mix(N_PART, gen.CONFIG_SEEDS[2])
    import oracle
    oracle.build()
    nth = oracle.nthreads()
    # size each step so that warm-up plus timed steps end within a few minutes
    idx = gen.sample_indices(N_PART, 32, 77)
    t0 = time.perf_counter()
    oracle.newton_subset(x, m, EPS, idx, nthreads_=nth)
    per32 = max(time.perf_counter() - t0, 1e-3)
    k = int(max(32, min(N_PART, 32 * 8.0 / per32)))
    idx = gen.sample_indices(N_PART, k, 78)
    for _ in range(args.warmup):
        oracle.newton_subset(x, m, EPS, idx[:32], nthreads_=nth)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        oracle.newton_subset(x, m, EPS, idx, nthreads_=nth)
        times.append(time.perf_counter() - t0)
    pairs = len(idx) * N_PART
    value = pairs * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "interactions/s", "value": value, "unit": "interactions/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "newton-allpairs-2^20-plummer+cube", "n": N_PART, "eps": EPS,
                   "sample_i_per_step": len(idx)},
        "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": nth, "kind": "oracle",
                         "sample": f"{len(idx)} i x {N_PART} j per step"},
        "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gauss_split(r, rs, eps):
    """Short-range part of the TreePM Gaussian split, softened: f(r)/r."""
    u = r / (2 * rs)
    w = math.erfc(u) + r / (rs * math.sqrt(math.pi)) * math.exp(-u * u)
    return w / (r * r + eps * eps) ** 1.5


def _time_kernel(ctx, fn, reps=5, warm=2):
    for _ in range(warm):
        fn()
    ks = []
    for _ in range(reps):
        fn()
        ks.append(ctx.kernel_time())
    return statistics.median(ks)


def _time_call(torch, fn, reps, warm=3):
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


# Oracle comparisons of every result, deferred to the oracle leg of the run
# (after all GPU timing, with the CPU baseline): each entry is (row name,
# function of the oracle module returning the row's "error" block). Only
# sampled GPU outputs are kept; the oracle recomputes from the same inputs.
CHECKS = []

ERR_NOTE = ("per-particle relative |da|/|a| (and |dphi|/|phi|) against the FP64 oracle of the "
            "same inputs; Newton tolerance: median 2e-6, max 1e-4")


def err_stats(a, ao, p=None, po=None, sample=None):
    ea = np.linalg.norm(np.asarray(a) - ao, axis=1) / np.linalg.norm(ao, axis=1)
    out = {"a_median": float(np.median(ea)), "a_max": float(np.max(ea))}
    if p is not None and po is not None:
        ep = np.abs(np.asarray(p) - po) / np.abs(po)
        out.update(phi_median=float(np.median(ep)), phi_max=float(np.max(ep)))
    if sample:
        out["sample"] = sample
    return out


def err_ref(a, p, ref, sample=None):
    """err_stats against an oracle result ref = (acc, pot)."""
    return err_stats(a, ref[0], p, ref[1], sample)


def table_err(orc, a, x, idx, m, E, F, r_cut, par, box=0.0):
    """Tabulated forces at x[idx] against the table semantics (O-T2: the
    paper's interpolant, per-particle relative, after the cutoff allowance
    of pairs within 1e-6 of s_max) and the closed form (O-T1: error over the
    sum of the pair terms' magnitudes, the per-pair bound of Section 4.2)."""
    v = orc.table_values(E, F, r_cut, orc.SHAPE_GAUSS_SPLIT, par)
    G0, G1 = orc.table_from_values(E, F, v)
    ao, amb = orc.table_forces(x[idx], x, m, E, F, r_cut, G0, G1, box=box, skip=idx, window=1e-6)
    norm = np.linalg.norm(ao, axis=1)
    ok = norm > 0
    rel = np.maximum(np.linalg.norm(a - ao, axis=1) - amb, 0)[ok] / norm[ok]
    ac, ambc, absum = orc.shape_forces(x[idx], x, m, orc.SHAPE_GAUSS_SPLIT, par, r_cut, box=box,
                                       skip=idx, window=1e-6, with_absum=True)
    okc = absum > 0
    relc = np.maximum(np.linalg.norm(a - ac, axis=1) - ambc, 0)[okc] / absum[okc]
    return {"vs_table_semantics_median": float(np.median(rel)),
            "vs_table_semantics_max": float(np.max(rel)),
            "vs_closed_form_over_abs_sum_median": float(np.median(relc)),
            "vs_closed_form_over_abs_sum_max": float(np.max(relc)),
            "sample": f"{len(idx)} i against all {len(x)} j"}, ao


def extra_rows(pg, torch, dev, peak_newton, headline_rate):
    """The other rows of the path, each timed on its own workload (not the
    headline): the 4096-body Plummer call (latency-bound, CUDA graph), the
    tabulated all-pairs kernel, the periodic cell-list cutoff force on the
    2^21-particle clustered box, the 20000 tree-style groups, and the
    backward pass on 65536 Plummer particles."""
    rows = {}
    st = torch.cuda.current_stream()
    peak_table = peak_newton * 13 / 11
    idx = dev.index or 0

    # 4096-body Plummer sphere, eps = 1/64, graph replay per call
    x, m = gen.plummer(4096, gen.CONFIG_SEEDS[1])
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    a, p = torch.empty_like(xd), torch.empty_like(md)
    with pg.Context(idx) as c:
        c.set_stream(st.cuda_stream)
        c.set_eps(1 / 64)
        c.set_self(True)
        c.set_graph(True)
        c.set_j_dev(xd, md)
        c.set_i_dev(xd)
        ms = _time_call(torch, lambda: c.run_dev(a, p), 200, warm=20)
        rate4 = 4096 * 4096 / (ms * 1e-3)
        # double-float differences: 19 FP32-pipe operations per interaction
        rows["newton_plummer_4096"] = {"interactions_per_s": rate4, "us_per_call": ms * 1e3,
                                       "graph": True, "launches": c.info()["launches"],
                                       "frac_fp32_peak_19_ops": rate4 / (peak_newton * 13 / 19)}
        # single-call latency: one call at a time, the stream idle before it;
        # CUDA events around the call, and the host's clock from the call to
        # the end of a synchronize
        for graph in (True, False):
            c.set_graph(graph)
            ev, host = [], []
            for k in range(25):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                e0.record(st)
                c.run_dev(a, p)
                e1.record(st)
                e1.synchronize()
                t1 = time.perf_counter()
                if k >= 5:
                    ev.append(e0.elapsed_time(e1) * 1e3)
                    host.append((t1 - t0) * 1e6)
            key = "single_call_graph" if graph else "single_call"
            rows["newton_plummer_4096"][key] = {"us_events": statistics.median(ev),
                                                "us_host": statistics.median(host)}
        a4, p4 = a.cpu().numpy(), p.cpu().numpy()
        CHECKS.append(("newton_plummer_4096",
                       lambda orc, x=x, m=m, a4=a4, p4=p4: err_ref(
                           a4, p4, orc.newton_allpairs(x, m, 1 / 64), "all 4096")))

    # individual time steps: the i-set is the n_i densest-core particles of the
    # 2^20 mixed set (those with the shortest steps), j = all 2^20; per call
    # through the device API with the path chosen automatically (narrow)
    n = N_PART
    x, m = gen.plummer_cube_mix(n, gen.CONFIG_SEEDS[2])
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    order = np.argsort(np.linalg.norm(x, axis=1))
    steps = {}
    for ni in (16, 64, 256, 1024):
        xi = torch.tensor(x[order[:ni]], device=dev)
        a = torch.empty_like(xi)
        with pg.Context(idx) as c:
            c.set_stream(st.cuda_stream)
            c.set_eps(1e-3)
            c.set_timing(True)
            c.set_j_dev(xd, md)
            c.set_i_dev(xi)
            ms = _time_call(torch, lambda: c.run_dev(a), 50, warm=5)
            kms = c.kernel_time()
            slots = c.info()["slots"]
            c.set_graph(True)       # the same call replayed as a CUDA graph
            ms_graph = _time_call(torch, lambda: c.run_dev(a), 50, warm=5)
            steps[str(ni)] = {"us_per_call": ms * 1e3, "kernel_us": kms * 1e3,
                              "interactions_per_s": ni * n / (ms * 1e-3),
                              "us_per_call_graph": ms_graph * 1e3,
                              "j_chunks": slots}
            ai = a.cpu().numpy()
            CHECKS.append((f"individual_steps_ni_vs_2e20/{ni}",
                           lambda orc, xi=x[order[:ni]], ai=ai, x=x, m=m: err_stats(
                               ai, orc.newton(xi, x, m, 1e-3)[0], sample=f"all {len(xi)} i")))
    rows["individual_steps_ni_vs_2e20"] = steps
    del xd, md

    # tree front end (Section 5.1's tree usage): 2^20-particle Plummer and
    # King (W0 = 9) models, theta = 0.75, monopole and quadrupole
    # pseudo-particles, groups of at most 256, leaves of at most 8,
    # eps = 1e-3; per call (tree build, walk, lists, forces) and the force
    # kernel alone
    n = N_PART
    for model in ("plummer", "king"):
        x, m = tree_model(model, n)
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        a, p = torch.empty_like(xd), torch.empty_like(md)
        for quad in (False, True):
            with pg.Context(idx) as c:
                c.set_stream(st.cuda_stream)
                c.set_eps(EPS)
                c.set_self(True)
                c.set_timing(True)
                c.set_tree(0.75, TREE_NCRIT, 8, quadrupole=quad)
                c.set_j_dev(xd, md)
                c.set_i_dev(xd)
                ms = _time_call(torch, lambda: c.run_dev(a, p), 5, warm=2)
                kms = c.kernel_time()
                info = c.info()
                t = c.get_tree()
                key = f"tree_{model}_2e20_theta075_{'quadrupole' if quad else 'monopole'}"
                tidx = gen.sample_indices(n, 1024, 61)
                at, pt = a[torch.tensor(tidx, device=dev)].cpu().numpy(), p[torch.tensor(tidx, device=dev)].cpu().numpy()
                CHECKS.append((key, lambda orc, x=x, m=m, tidx=tidx, at=at, pt=pt: dict(
                    err_ref(at, pt, orc.newton_subset(x, m, EPS, tidx),
                            f"{len(tidx)} particles against the direct sum"),
                    note="the tree method's own error against the direct sum (its lists are "
                         "bit-identical to the oracle tree's, checked in the tests)")))
                rows[key] = {
                    "ms_per_call": ms, "force_kernel_ms": kms, "pairs": info["pairs"],
                    "interactions_per_s_kernel": info["pairs"] / (kms * 1e-3),
                    "nodes": t["nnodes"], "groups": t["ngroups"], "list_entries": t["nlist"],
                    "ncrit": TREE_NCRIT,
                    "direct_sum_equivalent_speedup": (n * n / headline_rate) / (ms * 1e-3)}
        del xd, md, a, p

    # tabulated all-pairs: 65536 Plummer, Gaussian split, r_cut = 0.1, E=3, F=5
    n = 65536
    x, m = gen.plummer(n, gen.CONFIG_SEEDS[5])
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    a = torch.empty_like(xd)
    r_cut = 0.1
    with pg.Context(idx) as c:
        c.set_stream(st.cuda_stream)
        c.set_mode(pg.PG_TABLE)
        c.set_table(lambda r: gauss_split(r, r_cut / 4.5, 1 / 64), r_cut, 3, 5)
        c.set_self(True)
        c.set_timing(True)
        c.set_j_dev(xd, md)
        c.set_i_dev(xd)
        kms = _time_kernel(c, lambda: c.run_dev(a))
        rate = n * n / (kms * 1e-3)
        tidx = gen.sample_indices(n, 1024, 62)
        at = a[torch.tensor(tidx, device=dev)].cpu().numpy()
        CHECKS.append(("table_allpairs_65536_E3F5",
                       lambda orc, x=x, m=m, tidx=tidx, at=at: table_err(
                           orc, at, x, tidx, m, 3, 5, r_cut, [r_cut / 4.5, 1 / 64])[0]))
        # the same with the potential table (psi = -(r^2 + eps^2)^(-1/2))
        c.set_table_pot(lambda r: -1.0 / math.sqrt(r * r + (1 / 64) ** 2))
        kms_p = _time_kernel(c, lambda: c.run_dev(a))
        rows["table_allpairs_65536_E3F5"] = {"interactions_per_s": rate, "kernel_ms": kms,
                                             "frac_fp32_peak": rate / peak_table,
                                             "with_potential_kernel_ms": kms_p,
                                             "with_potential_interactions_per_s": n * n / (kms_p * 1e-3)}
        # Newton with a softening per particle (log-uniform in [1/256, 1/16])
        c.set_mode(pg.PG_NEWTON)
        c.set_table_pot(None)
        e = np.exp(np.random.default_rng(9).uniform(np.log(1 / 256), np.log(1 / 16), n))
        c.set_eps_i(e)
        kms_e = _time_kernel(c, lambda: c.run_dev(a))
        ae = a[torch.tensor(tidx, device=dev)].cpu().numpy()
        CHECKS.append(("newton_per_i_softening_65536",
                       lambda orc, x=x, m=m, e=e, tidx=tidx, ae=ae: err_stats(
                           ae, orc.newton_epsi(x[tidx], e[tidx], x, m, skip=tidx)[0],
                           sample=f"{len(tidx)} i against all {len(x)} j")))
        c.set_eps_i(None)
        c.set_eps(1 / 64)
        kms_g = _time_kernel(c, lambda: c.run_dev(a))
        rows["newton_per_i_softening_65536"] = {"kernel_ms": kms_e,
                                                "interactions_per_s": n * n / (kms_e * 1e-3),
                                                "global_eps_kernel_ms": kms_g}

    # backward on the same set: Newton (eps = 1/64) and the table
    from paper_1203_4037_gb300 import autograd  # noqa: F401  (binding used by users)
    w = torch.tensor(gen.unit_vectors(n, gen.CONFIG_SEEDS[5] + 1), device=dev)
    dx, dm = torch.empty_like(xd), torch.empty_like(md)
    with pg.Context(idx) as c:
        c.set_stream(st.cuda_stream)
        c.set_self(True)
        c.set_timing(True)
        c.set_eps(1 / 64)
        c.set_j_dev(xd, md)
        c.set_i_dev(xd)
        fwd = _time_kernel(c, lambda: c.run_dev(a))
        bwd = _time_kernel(c, lambda: c.backward_dev(w, dx, dm))
        c.set_mode(pg.PG_TABLE)
        c.set_table(lambda r: gauss_split(r, r_cut / 4.5, 1 / 64), r_cut, 3, 5)
        dv = torch.empty(256, dtype=torch.float32, device=dev)
        bwd_t = _time_kernel(c, lambda: c.backward_dev(w, dx, dm, dv))
        gidx = gen.sample_indices(n, 64, 63)
        gsel = torch.tensor(gidx, device=dev)
        wn = w.cpu().numpy()
        # the Newton gradients of the last Newton backward, recomputed here
        c.set_mode(pg.PG_NEWTON)
        c.backward_dev(w, dx, dm)
        gdx_n, gdm_n = dx[gsel].cpu().numpy(), dm[gsel].cpu().numpy()
        c.set_mode(pg.PG_TABLE)
        c.backward_dev(w, dx, dm, dv)
        gdx_t, gdm_t, gdv = dx[gsel].cpu().numpy(), dm[gsel].cpu().numpy(), dv.cpu().numpy()

        def grad_err(orc, x=x, m=m, wn=wn, gidx=gidx, gdx_n=gdx_n, gdm_n=gdm_n, gdx_t=gdx_t,
                     gdm_t=gdm_t, gdv=gdv):
            ox, om = orc.grad_newton_at(x, m, wn, 1 / 64, gidx)
            v = orc.table_values(3, 5, r_cut, orc.SHAPE_GAUSS_SPLIT, [r_cut / 4.5, 1 / 64])
            tx, tm = orc.grad_table_at(x, m, wn, 3, 5, r_cut, v, gidx)
            tv = orc.grad_table_v(x, m, wn, 3, 5, r_cut, v)
            nz = tv != 0

            def nrm(g, o):
                return float(np.linalg.norm(np.ravel(g) - np.ravel(o)) / np.linalg.norm(np.ravel(o)))
            return {"newton_dx": nrm(gdx_n, ox), "newton_dm": nrm(gdm_n, om),
                    "table_dx": nrm(gdx_t, tx), "table_dm": nrm(gdm_t, tm),
                    "table_dv": nrm(gdv[nz], tv[nz]),
                    "sample": f"norm-wise relative against the oracle's analytic FP64 gradient "
                              f"at {len(gidx)} particles (all knots with pairs for dv); "
                              f"tolerance 1e-4"}
        CHECKS.append(("backward_65536", grad_err))
        rows["backward_65536"] = {
            "newton_forward_kernel_ms": fwd, "newton_backward_kernel_ms": bwd,
            "newton_backward_interactions_per_s": n * n / (bwd * 1e-3),
            # 26 FP32-pipe lane operations per pair (the packed backward)
            "newton_backward_frac_fp32_peak_26_ops": n * n / (bwd * 1e-3) / (peak_newton * 13 / 26),
            "newton_backward_over_forward": bwd / fwd,
            "table_backward_kernel_ms": bwd_t,
            "table_backward_interactions_per_s": n * n / (bwd_t * 1e-3)}
    del xd, md, a, w, dx, dm

    # periodic cell list: 2^21 clustered box, Gaussian split r_s = 1/256
    n = 1 << 21
    x, m = gen.clustered_box(n, gen.CONFIG_SEEDS[3])
    xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
    a = torch.empty_like(xd)
    rs = 1 / 256
    with pg.Context(idx) as c:
        c.set_stream(st.cuda_stream)
        c.set_mode(pg.PG_TABLE)
        c.set_table(lambda r: gauss_split(r, rs, rs / 16), 4.5 * rs, 4, 8)
        c.set_self(True)
        c.set_periodic(1.0)
        c.set_timing(True)
        c.set_j_dev(xd, md)
        c.set_i_dev(xd)
        kms = _time_kernel(c, lambda: c.run_dev(a))
        pairs = c.info()["pairs"]
        call = _time_call(torch, lambda: c.run_dev(a), 5, warm=1)
        rate = pairs / (kms * 1e-3)
        rows["cells_2e21_E4F8"] = {"pairs_evaluated": pairs, "kernel_ms": kms,
                                   "interactions_per_s": rate, "frac_fp32_peak": rate / peak_table,
                                   "call_ms_with_cell_build": call,
                                   "interactions_per_s_with_build": pairs / (call * 1e-3)}
        try:
            # ordered pairs i != j closer than r_cut: the useful part of the
            # evaluated pairs (a k-d tree count with the periodic box)
            from scipy.spatial import cKDTree
            useful = int(cKDTree(x, boxsize=1.0).query_ball_point(
                x, 4.5 * rs, return_length=True, workers=-1).sum()) - n
            rows["cells_2e21_E4F8"].update(pairs_useful=useful,
                                           useful_per_s=useful / (kms * 1e-3),
                                           useful_fraction=useful / pairs)
        except Exception as exc:  # report, do not hide
            rows["cells_2e21_E4F8"]["pairs_useful_error"] = repr(exc)
        try:
            # the table lookup's own ceiling: random 8-byte gathers per SM per
            # clock from one shared table (the kernels' placement), four
            # interleaved shared copies, and the read-only global path
            sm_clk = peak_newton * 13 / 128          # SMs x basis clock
            g = {k: pg.pg_microbench(kind)[0] for k, kind in
                 (("shared", 4), ("shared_4_copies", 5), ("global_readonly", 6))}
            rows["cells_2e21_E4F8"].update(
                pairs_per_sm_clk=rate / sm_clk, gather_lane_per_sm_clk=g,
                frac_of_gather_ceiling=rate / sm_clk / g["shared"])
        except Exception as exc:  # report, do not hide
            rows["cells_2e21_E4F8"]["gather_ceiling_error"] = repr(exc)
        cidx = gen.sample_indices(n, 1024, 64)
        csel = torch.tensor(cidx, device=dev)
        ac = a[csel].cpu().numpy()
        cells_ref = {}

        def cells_err(orc, x=x, m=m, cidx=cidx, ac=ac):
            e, ao = table_err(orc, ac, x, cidx, m, 4, 8, 4.5 * rs, [rs, rs / 16], box=1.0)
            cells_ref["pp"] = ao
            return e
        CHECKS.append(("cells_2e21_E4F8", cells_err))
        # PPPM / TreePM: the same split's long range on a 256^3 mesh (r_s = h),
        # alone and added to the cell-list PP in one run
        p = torch.empty_like(md)
        c.set_pm(256, pg.PG_SPLIT_GAUSS, rs)
        call_pp_pm = _time_call(torch, lambda: c.run_dev(a), 5, warm=2)
        app = a[csel].cpu().numpy()
        pm_ms = _time_call(torch, lambda: c.pm_forces_dev(xd, md, a, p), 5, warm=2)
        pm_fft = c.pm_fft()
        # the same call with cuFFT's transforms instead of the hand-written ones
        c.set_pm_fft(pg.PG_FFT_LIBRARY)
        pm_lib_ms = _time_call(torch, lambda: c.pm_forces_dev(xd, md, a, p), 5, warm=2)
        c.set_pm_fft(pg.PG_FFT_AUTO)
        c.pm_forces_dev(xd, md, a, p)
        apm, ppm = a[csel].cpu().numpy(), p[csel].cpu().numpy()

        def pm_err(orc, x=x, m=m, cidx=cidx, apm=apm, ppm=ppm, app=app):
            from oracle import pm as opm
            rho = opm.deposit(x, m, 1.0, 256)
            ao, po = opm.solve(rho, x[cidx], 1.0, 256, "gauss", rs)
            cells_ref["pm"] = ao
            rms = float(np.sqrt(np.mean(np.sum(ao ** 2, axis=1))))
            prms = float(np.sqrt(np.mean(po ** 2)))
            ea = np.linalg.norm(apm - ao, axis=1) / rms
            out = {"a_over_rms_median": float(np.median(ea)), "a_over_rms_max": float(ea.max()),
                   "phi_over_rms_max": float(np.max(np.abs(ppm - po)) / prms),
                   "sample": f"{len(cidx)} particles; tolerance median 1e-5, max 1e-4 of the RMS"}
            return out

        def pppm_err(orc, cidx=cidx, app=app):
            ref = cells_ref["pp"] + cells_ref["pm"]
            e = np.linalg.norm(app - ref, axis=1) / np.linalg.norm(ref, axis=1)
            return {"a_median": float(np.median(e)), "a_max": float(np.max(e)),
                    "sample": f"{len(cidx)} particles against the table-semantics PP plus the "
                              "oracle mesh"}
        CHECKS.append(("pm_2e21_mesh256_gauss", pm_err))
        CHECKS.append(("pp_plus_pm_2e21_E4F8_mesh256", pppm_err))
        rows["pm_2e21_mesh256_gauss"] = {"ms_per_call": pm_ms, "particles_per_s": n / (pm_ms * 1e-3),
                                         "mesh": 256, "r_s_over_h": 1.0,
                                         "fft": {1: "hand-written", 2: "cuFFT"}.get(pm_fft, "none"),
                                         "ms_per_call_with_cufft": pm_lib_ms}
        rows["pp_plus_pm_2e21_E4F8_mesh256"] = {"ms_per_call": call_pp_pm,
                                                "particles_per_s": n / (call_pp_pm * 1e-3)}
    del xd, md, a

    # 20000 tree-style groups on the clustered 2^22 set, eps = 1e-3
    d = gen.tree_groups(gen.CONFIG_SEEDS[4])
    with pg.Context(idx) as c:
        c.set_stream(st.cuda_stream)
        c.set_eps(1e-3)
        c.set_timing(True)
        xj = torch.tensor(d["xj"], device=dev)
        mj = torch.tensor(d["mj"], device=dev)
        xi = torch.tensor(d["xi"], device=dev)
        a = torch.empty_like(xi)
        p = torch.empty(len(xi), dtype=torch.float64, device=dev)
        c.set_j_dev(xj, mj)
        c.set_i_dev(xi)
        c.set_groups(d["i_off"], d["j_off"], d["jlist"])
        pairs = int(((d["i_off"][1:] - d["i_off"][:-1]) * (d["j_off"][1:] - d["j_off"][:-1])).sum())
        c.tune()          # the launch shape picked by the autotuner (outside the timing)
        kms = _time_kernel(c, lambda: c.run_dev(a, p))
        info = c.info()
        c.set_graph(True)
        call = _time_call(torch, lambda: c.run_dev(a, p), 5, warm=2)
        rate = pairs / (kms * 1e-3)
        # 400 groups of the 20000, their lists and i-particles, for the oracle
        gsel = gen.sample_indices(len(d["i_off"]) - 1, 400, 65)
        io, jo = d["i_off"], d["j_off"]
        ii = np.concatenate([np.arange(io[g], io[g + 1]) for g in gsel])
        s_ioff = np.concatenate([[0], np.cumsum(io[gsel + 1] - io[gsel])])
        s_joff = np.concatenate([[0], np.cumsum(jo[gsel + 1] - jo[gsel])])
        s_jl = np.concatenate([d["jlist"][jo[g]:jo[g + 1]] for g in gsel])
        ag = a[torch.tensor(ii, device=dev)].cpu().numpy()
        pgv = p[torch.tensor(ii, device=dev)].cpu().numpy()
        CHECKS.append(("groups_20000",
                       lambda orc, d=d, ii=ii, s_ioff=s_ioff, s_joff=s_joff, s_jl=s_jl, ag=ag, pgv=pgv:
                       err_ref(ag, pgv, orc.newton_groups(s_ioff, s_joff, s_jl, d["xi"][ii], d["xj"],
                                                          d["mj"], 1e-3),
                               f"400 groups ({len(ii)} i) with their lists")))
        rows["groups_20000"] = {"pairs": pairs, "kernel_ms": kms, "interactions_per_s": rate,
                                "frac_fp32_peak": rate / peak_newton,
                                "call_ms_graph": call,
                                "ratio_to_allpairs": rate / headline_rate,
                                "tuned_shape": {"i_per_thread": info["i_per_thread"],
                                                "j_tile": info.get("j_tile"),
                                                "block_threads": info.get("block_threads"),
                                                "grid": info["grid"]}}
    return rows


def run_row(args):
    """Time one non-headline row alone (profiling aid): prints one JSON line."""
    import torch
    import paper_1203_4037_gb300 as pg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    pg.build()
    st = torch.cuda.current_stream()
    out = {"workload": args.workload}
    if args.workload in ("table", "backward"):
        n = min(args.n, 65536) if args.n != N_PART else 65536
        x, m = gen.plummer(n, gen.CONFIG_SEEDS[5])
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        a = torch.empty_like(xd)
        r_cut = 0.1
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_self(True)
            c.set_timing(True)
            c.set_j_dev(xd, md)
            c.set_i_dev(xd)
            if args.workload == "table":
                c.set_mode(pg.PG_TABLE)
                c.set_table(lambda r: gauss_split(r, r_cut / 4.5, 1 / 64), r_cut, 3, 5)
                kms = _time_kernel(c, lambda: c.run_dev(a), reps=args.steps, warm=args.warmup)
            else:
                c.set_eps(1 / 64)
                w = torch.tensor(gen.unit_vectors(n, gen.CONFIG_SEEDS[5] + 1), device=dev)
                dx, dm = torch.empty_like(xd), torch.empty_like(md)
                kms = _time_kernel(c, lambda: c.backward_dev(w, dx, dm), reps=args.steps,
                                   warm=args.warmup)
        out.update(n=n, kernel_ms=kms, interactions_per_s=n * n / (kms * 1e-3))
    elif args.workload == "tree":
        # the tree front end on --n particles (default 2^20) of --model
        n = args.n
        x, m = tree_model(args.model, n)
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        a = torch.empty_like(xd)
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_eps(EPS)
            c.set_self(True)
            c.set_timing(True)
            c.set_tree(0.75, args.ncrit, 8, quadrupole=args.quadrupole)
            if args.level_walk:
                c.set_tree_walk(pg.PG_TREE_WALK_LEVEL)
            c.set_j_dev(xd, md)
            c.set_i_dev(xd)
            kms = _time_kernel(c, lambda: c.run_dev(a), reps=args.steps, warm=args.warmup)
            ms = _time_call(torch, lambda: c.run_dev(a), args.steps, warm=args.warmup)
            info = c.info()
            stats = c.tree_stats()
        out.update(n=n, model=args.model, quadrupole=args.quadrupole, ncrit=args.ncrit,
                   pairs=info["pairs"], kernel_ms=kms, ms_per_call=ms,
                   interactions_per_s=info["pairs"] / (kms * 1e-3), walk=stats)
    elif args.workload == "narrow":
        # individual time steps: --n core particles of the 2^20 mixed set
        # against all 2^20 (default 16), path chosen automatically
        x, m = gen.plummer_cube_mix(N_PART, gen.CONFIG_SEEDS[2])
        ni = 16 if args.n == N_PART else args.n
        xi = x[np.argsort(np.linalg.norm(x, axis=1))[:ni]]
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        xid = torch.tensor(xi, device=dev)
        a = torch.empty_like(xid)
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_eps(EPS)
            c.set_timing(True)
            c.set_j_dev(xd, md)
            c.set_i_dev(xid)
            kms = _time_kernel(c, lambda: c.run_dev(a), reps=args.steps, warm=args.warmup)
            call = _time_call(torch, lambda: c.run_dev(a), args.steps, warm=args.warmup)
            info = c.info()
        out.update(ni=ni, nj=N_PART, kernel_ms=kms, us_per_call=call * 1e3,
                   interactions_per_s=ni * N_PART / (kms * 1e-3), j_chunks=info["slots"])
    elif args.workload == "small":
        # the 4096-body Plummer call (eps = 1/64) in one launch, graph-replayed
        n = args.n if args.n != N_PART else 4096
        x, m = gen.plummer(n, gen.CONFIG_SEEDS[1])
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        a, p = torch.empty_like(xd), torch.empty_like(md)
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_eps(1 / 64)
            c.set_self(True)
            c.set_graph(True)
            c.set_j_dev(xd, md)
            c.set_i_dev(xd)
            ms = _time_call(torch, lambda: c.run_dev(a, p), max(args.steps, 1), warm=args.warmup)
            info = c.info()
        out.update(n=n, us_per_call=ms * 1e3, interactions_per_s=n * n / (ms * 1e-3),
                   launches=info["launches"], grid=info["grid"])
    elif args.workload == "pm":
        # the particle-mesh long range alone on the 2^21 clustered box (or
        # --n particles), Gaussian split r_s = 1/256 on a 256^3 mesh
        n = args.n if args.n != N_PART else 1 << 21
        x, m = gen.clustered_box(n, gen.CONFIG_SEEDS[3])
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        a, p = torch.empty_like(xd), torch.empty_like(md)
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_periodic(1.0)
            c.set_pm(256, pg.PG_SPLIT_GAUSS, 1 / 256)
            ms = _time_call(torch, lambda: c.pm_forces_dev(xd, md, a, p), args.steps, warm=args.warmup)
            fft = c.pm_fft()
            c.set_pm_fft(pg.PG_FFT_LIBRARY)
            ms_lib = _time_call(torch, lambda: c.pm_forces_dev(xd, md, a, p), args.steps, warm=args.warmup)
        out.update(n=n, mesh=256, ms_per_call=ms, particles_per_s=n / (ms * 1e-3),
                   fft={1: "hand-written", 2: "cuFFT"}.get(fft, "none"), ms_per_call_with_cufft=ms_lib)
    elif args.workload == "cells":
        n = args.n if args.n != N_PART else 1 << 21
        x, m = gen.clustered_box(n, gen.CONFIG_SEEDS[3])
        xd, md = torch.tensor(x, device=dev), torch.tensor(m, device=dev)
        a = torch.empty_like(xd)
        rs = 1 / 256
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_mode(pg.PG_TABLE)
            c.set_table(lambda r: gauss_split(r, rs, rs / 16), 4.5 * rs, 4, 8)
            c.set_self(True)
            c.set_periodic(1.0)
            c.set_timing(True)
            c.set_j_dev(xd, md)
            c.set_i_dev(xd)
            kms = _time_kernel(c, lambda: c.run_dev(a), reps=args.steps, warm=args.warmup)
            pairs = c.info()["pairs"]
        out.update(n=n, pairs=pairs, kernel_ms=kms, interactions_per_s=pairs / (kms * 1e-3))
    else:
        ng = 20000 if args.n == N_PART else max(100, args.n // 200)
        npart = 1 << 22 if args.n == N_PART else args.n
        d = gen.tree_groups(gen.CONFIG_SEEDS[4], n=npart, ngroups=ng,
                            n_monopoles=max(1024, npart // 4))
        with pg.Context(0) as c:
            c.set_stream(st.cuda_stream)
            c.set_eps(1e-3)
            c.set_timing(True)
            xj, mj = torch.tensor(d["xj"], device=dev), torch.tensor(d["mj"], device=dev)
            xi = torch.tensor(d["xi"], device=dev)
            a = torch.empty_like(xi)
            c.set_j_dev(xj, mj)
            c.set_i_dev(xi)
            c.set_groups(d["i_off"], d["j_off"], d["jlist"])
            kms = _time_kernel(c, lambda: c.run_dev(a), reps=args.steps, warm=args.warmup)
            pairs = c.info()["pairs"]
        out.update(groups=ng, pairs=pairs, kernel_ms=kms, interactions_per_s=pairs / (kms * 1e-3))
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "newton":
        run_row(args)
        return
    import torch
    import torch.distributed as dist
    import paper_1203_4037_gb300 as pg
    from paper_1203_4037_gb300.multirank import ShardedAllPairs, max_over_ranks, shard

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # one non-default stream for the library, the timing events and graphs
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    pg.build()

    npart = args.n
    if args.quick:
        args.no_rows = args.no_cpu_baseline = True
    x, m = gen.plummer_cube_mix(npart, gen.CONFIG_SEEDS[2])
    if world > 1:
        # domain decomposition: each rank owns a Morton-contiguous run of the
        # particles, so its i-tiles are as compact as on one GPU
        order = gen.morton_order(x)
        x, m = x[order], m[order]
    lo, hi = shard(npart, rank, world)
    ni = hi - lo
    st = torch.cuda.current_stream()
    xi = torch.tensor(x[lo:hi], device=dev)      # this rank's particles
    mi = torch.tensor(m[lo:hi], device=dev)
    acc = torch.empty((ni, 3), dtype=torch.float64, device=dev)
    pot = torch.empty(ni, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    ctx = pg.Context(local)
    ctx.set_stream(st.cuda_stream)
    ctx.set_eps(EPS)
    ctx.set_timing(True)
    if args.shape:
        np_, packed = (int(v) for v in args.shape.split(","))
        ctx.set_shape(np_, 0, packed)
    # every step: this rank's records all-gathered from every rank (NCCL; a
    # copy on one GPU), then its slice against all of them, own pairs left
    # out through the self mode with the slice's offset
    gather = (dist.all_gather_into_tensor if world > 1
              else (lambda out, inp: out.copy_(inp)))
    sharded = ShardedAllPairs(ctx, npart, rank, world, gather, device=dev)

    def step():
        sharded.forces(xi, mi, acc, pot)

    warmup_done = max(args.warmup, 3)   # at least 3 untimed steps
    for _ in range(warmup_done):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 255)         # evict L2 between timed steps (not timed)
        ev[k][0].record(st)
        step()
        ev[k][1].record(st)
        kern_ms.append(ctx.kernel_time())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), device=dev)
    info = ctx.info()
    # the timed step's outputs at a fixed 4096-particle sample, kept for the
    # oracle comparison (made after all GPU timing)
    hidx = gen.sample_indices(ni, min(4096, ni), 4244)
    hsel = torch.tensor(hidx, device=dev)
    h_a, h_p = acc[hsel].cpu().numpy(), pot[hsel].cpu().numpy()
    pairs_job = npart * npart                      # all ranks together, one step
    value = pairs_job * args.steps / (total_ms * 1e-3)

    # end to end through the public host API: pinned-host inputs in, results out
    e2e = None
    if world > 1 and not args.quick:
        # every rank: its slice from pinned host memory, the exchange and the
        # force evaluation, its results back to the host
        xh = torch.tensor(x[lo:hi]).pin_memory()
        mh = torch.tensor(m[lo:hi]).pin_memory()
        ah = torch.empty((ni, 3), dtype=torch.float64).pin_memory()
        ph = torch.empty(ni, dtype=torch.float64).pin_memory()

        def e2e_step():
            xi.copy_(xh, non_blocking=True)
            mi.copy_(mh, non_blocking=True)
            sharded.forces(xi, mi, acc, pot)
            ah.copy_(acc, non_blocking=True)
            ph.copy_(pot, non_blocking=True)
            st.synchronize()
        e2e_step()
        ne = max(2, min(args.steps, 3))
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ne):
            e2e_step()
        dt = max_over_ranks(time.perf_counter() - t0, device=dev)
        e2e = {"value": npart * npart * ne / dt, "unit": "interactions/s",
               "h2d_bytes_per_step": npart * 32, "d2h_bytes_per_step": npart * 32, "steps": ne}
    elif rank == 0 and not args.quick:
        # inputs and results in page-locked host memory, as a caller that
        # streams particles each step would hold them
        def pinned(arr):
            return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory().numpy()
        xh, mh, xh_i = pinned(x), pinned(m), pinned(x[lo:hi])
        ah, ph = pinned(np.zeros((ni, 3))), pinned(np.zeros(ni))
        ctx2 = pg.Context(local)
        ctx2.set_eps(EPS)
        ctx2.set_self(True)
        for _ in range(2):
            ctx2.set_j(xh, mh)
            ctx2.set_i(xh_i)
            ctx2.run()
            ctx2.get_force(ni, out=(ah, ph))
        t0 = time.perf_counter()
        ne = max(2, min(args.steps, 3))
        for _ in range(ne):
            ctx2.set_j(xh, mh)
            ctx2.set_i(xh_i)
            ctx2.run()
            ctx2.get_force(ni, out=(ah, ph))
        dt = time.perf_counter() - t0
        ctx2.close()
        e2e = {"value": pairs_job * ne / dt, "unit": "interactions/s",
               "h2d_bytes_per_step": npart * 32 + ni * 24, "d2h_bytes_per_step": ni * 32,
               "steps": ne}

    rows = None
    if rank == 0 and not args.no_rows:
        sms_ = torch.cuda.get_device_properties(dev).multi_processor_count
        f_ = float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6
        kern_rate = ni * npart / (statistics.median(kern_ms) * 1e-3)
        try:
            rows = extra_rows(pg, torch, dev, sms_ * f_ * FP32_LANES_PER_SM / NEWTON_OPS, kern_rate)
        except Exception as exc:  # report, do not hide
            rows = {"error": repr(exc)}

    if rank != 0:
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_int = sms * f_max * FP32_LANES_PER_SM / NEWTON_OPS
    kms = statistics.median(kern_ms)
    pairs_rank = ni * npart
    achieved = pairs_rank / (kms * 1e-3)
    # DRAM bytes of one headline launch of this kernel build, from one ncu
    # pass (dram__bytes_read.sum + dram__bytes_write.sum); null for other
    # sizes or shapes, and until measured for this build
    traffic = HEADLINE_TRAFFIC if (npart == N_PART and world == 1 and info["i_per_thread"] == 8) else None
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_int / 1e9,
            "unit": "Ginteractions/s", "frac": achieved / peak_int, "traffic": traffic,
            "kernel": f"k_allpairs<np={info['i_per_thread'] // 2}, packed={info['packed']}>",
            "kernel_ms": kms,
            "peak_basis": f"{sms} SMs x {f_max / 1e6:.0f} MHz x 128 FP32 lanes / 13 ops per "
                          "interaction (FP32 pipe; MUFU allows 16 per SM-clock)"}
    if clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (sms * clk["sm_mhz"] * 1e6 * FP32_LANES_PER_SM /
                                                    NEWTON_OPS)
    try:
        # measured ceilings: FP32x2 lane rate and the pair term with register operands
        ffma2 = pg.pg_microbench(1)[1]
        mix = pg.pg_microbench(3)[1]
        roof["measured_fp32x2_lane_ops_per_s"] = ffma2
        roof["measured_pair_term_ceiling"] = mix / 1e9
        roof["frac_of_pair_term_ceiling"] = achieved / mix
    except Exception as exc:  # report, do not hide
        roof["microbench_error"] = repr(exc)
    cpu = None
    error = None
    if not args.no_cpu_baseline:
        # the oracle leg: the CPU baseline, then every result against the oracle
        cpu = cpu_baseline(x, m)
        import oracle
        try:
            error = err_ref(h_a, h_p, oracle.newton_subset(x, m, EPS, lo + hidx),
                            f"{len(hidx)} i (fixed sample) against all {npart} j")
            error["note"] = ERR_NOTE
        except Exception as exc:  # report, do not hide
            error = {"error": repr(exc)}
        if rows and "error" not in rows:
            for key, fn in CHECKS:
                parts = key.split("/")
                dst = rows
                for k in parts:
                    dst = dst.setdefault(k, {})
                try:
                    dst["error"] = fn(oracle)
                except Exception as exc:  # report, do not hide
                    dst["error"] = {"error": repr(exc)}
    line = {
        "metric": "interactions/s", "value": value, "unit": "interactions/s", "n_gpus": world,
        "steps": args.steps, "warmup": warmup_done, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "exchange": ("one all-gather of the 32-byte j records per step (NCCL), inside the timed "
                     "step" if world > 1 else "none (one GPU: the records are copied in place)"),
        "data": "synthetic",
        "config": {"workload": "newton-allpairs-2^20-plummer+cube" if npart == N_PART else
                   f"newton-allpairs-{npart}-plummer+cube", "n": npart, "eps": EPS,
                   "positions": "fp64 in, fp32 offsets from fp64 tile centres",
                   "accumulation": "fp32 per 256-j sub-tile, TwoSum across, fp64 combine",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": (f"particles split over {world} GPUs (Morton-contiguous slices), "
                                   "j records all-gathered every step" if world > 1 else "1 GPU")},
        "gflops_at_38": value * PAPER_FLOPS_PER_INT / 1e9,
        "error": error,
        "roofline": roof,
        "clocks": clk,
        "e2e": e2e,
        # per step: the i pack kernel plus the run's sort, tile, force and combine kernels
        "gpu_launches": (int(info["launches"]) + 1) * args.steps,
        "cpu_baseline": cpu,
        "rows": rows,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
