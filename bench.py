"""Benchmark: matrix-free Helmholtz apply throughput (GDOF/s) on one GB300.

Default workload: 32^3 curved hexahedra (periodic sine map), P = 4, Q = 6,
FP64 fused Helmholtz apply (lambda = 1), coefficients uniform[-1,1] seed 0.
A step is one Helmholtz apply over all elements (BwdTrans, collocation
gradient, metric, transposed gradient and IProductWRTBase fused in one
launch).  Throughput = elements x modes / time (the paper's DOF/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nir|reference]
                    [--workload NAME] [--prec f64|f32|bf16]

Under torchrun each rank applies the operator to its own copy of the
workload (element-parallel, no data-path collective: weak scaling); rank 0
prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
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

import workloads as W  # noqa: E402

L2_BYTES = 129 * 2 ** 20


def helm_flops_per_elem(shape: str, N: int, Q: int) -> int:
    """Algorithmic flops of one sum-factorised Helmholtz apply: the BwdTrans
    contraction stages and their transposes (2 flops per multiply-add, each
    stage's count = outputs x summed modes), the collocation gradient and its
    transpose (2 Q^(d+1) flops per direction each way) and the per-point
    metric (20 flops in 3-D, 10 in 2-D).  Collapsed shapes contract their
    ragged mode ranges in the order of Eq. bwdsumfactet: tet M Q + N(N+1)/2 Q^2
    + N Q^3, prism and pyramid M Q + N^2 Q^2 + N Q^3, triangle M Q + N Q^2."""
    if shape == "hex":
        stages = N * N * N * Q + N * N * Q * Q + N * Q ** 3
    elif shape == "tet":
        stages = (N * (N + 1) * (N + 2) // 6) * Q + (N * (N + 1) // 2) * Q * Q + N * Q ** 3
    elif shape == "prism":
        stages = (N * N * (N + 1) // 2) * Q + N * N * Q * Q + N * Q ** 3
    elif shape == "pyr":
        stages = (N * (N + 1) * (2 * N + 1) // 6) * Q + N * N * Q * Q + N * Q ** 3
    elif shape == "quad":
        return 4 * (N * N * Q + N * Q * Q) + 8 * Q ** 3 + 10 * Q ** 2
    elif shape == "tri":
        return 4 * ((N * (N + 1) // 2) * Q + N * Q * Q) + 8 * Q ** 3 + 10 * Q ** 2
    else:
        raise ValueError(shape)
    return 4 * stages + 12 * Q ** 4 + 20 * Q ** 3


def op_work_per_elem(op: str, N: int, Q: int, wb: int, deformed: bool):
    """(algorithmic flops, algorithmic bytes) per hexahedron for each operator.

    Flops are the plain sum-factorised counts: one psiA contraction sweep is
    2N(N^2 Q + N Q^2 + Q^3), a collocation derivative 2 Q^4 per direction,
    a physical-derivative chain rule 2 d^2 Q^3.  Bytes are the arrays read
    and written once (coefficients M, point fields Q^3, per-point factors:
    W alone, 9 + 1 for d eta/d x with W)."""
    M, P3 = N ** 3, Q ** 3
    sweep = 2 * N * (N * N * Q + N * Q * Q + Q ** 3)
    fac = 1 if deformed else 0
    if op == "bwd":
        return sweep, (M + P3) * wb
    if op == "iprod":
        return sweep + P3, (P3 + M + fac * P3) * wb
    if op == "physderiv":
        return 3 * 2 * Q ** 4 + 18 * P3, (P3 + 3 * P3 + fac * 10 * P3) * wb
    if op == "iprod_deriv":
        return 3 * 2 * Q ** 4 + 19 * P3 + sweep, (3 * P3 + M + fac * 10 * P3) * wb
    if op == "mass":
        return 2 * sweep + P3, (2 * M + fac * P3) * wb
    raise KeyError(op)


def num_modes(shape: str, N: int) -> int:
    return {"quad": N * N, "tri": N * (N + 1) // 2, "hex": N ** 3, "prism": N * N * (N + 1) // 2,
            "tet": N * (N + 1) * (N + 2) // 6, "pyr": N * (N + 1) * (2 * N + 1) // 6}[shape]


def helm_bytes_per_elem(shape: str, N: int, Q: int, wb: int, deformed: bool) -> int:
    """Coefficients in and out, plus the metric: per point (deformed quad/hex and
    every collapsed shape, whose factors vary across the element) or once per
    element (undeformed quad/hex)."""
    d = 2 if shape in ("quad", "tri") else 3
    ng = 4 if d == 2 else 7
    per_point = deformed or shape in ("tri", "tet", "prism", "pyr")
    geo = ng * Q ** d if per_point else ng
    return 2 * num_modes(shape, N) * wb + geo * wb


KERNEL_SOURCES = ("paper_2606_20917_gb300/csrc/nir_kernels.cuh", "paper_2606_20917_gb300/csrc/nir_inst.cu",
                  "paper_2606_20917_gb300/csrc/nir_layout.h")


# the threading-over-elements Helmholtz kernel (tuning variant 4)
TOE_SOURCES = ("paper_2606_20917_gb300/csrc/nir_toe.cuh", "paper_2606_20917_gb300/csrc/nir_toe.cu",
               "paper_2606_20917_gb300/csrc/nir_layout.h")


def kernel_sources_sha256(sources=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(name: str, sources=KERNEL_SOURCES):
    """DRAM bytes per launch from the committed ncu summary profiles/<name>.md,
    or None when the kernel sources changed since that capture."""
    import re
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", txt)
    h = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", txt)
    if not t or not h or h.group(1) != kernel_sources_sha256(sources):
        return None
    return int(t.group(1))


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "nir" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float, device=None) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, v: float, device=None) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def run_reference(args, ws, rank):
    """The FP64 oracle on a bounded sample of the workload, on the host cores."""
    import oracle
    if rank != 0:
        return
    wl = W.workload(args.workload)
    shape, P, Q, g = wl["shape"], wl["P"], wl["Q"], wl["gorder"]
    M = oracle.num_modes(shape, P)
    k = args.sample
    ids = W.sample_elements(wl["nodes"].shape[0], k, seed=0)
    nodes = np.ascontiguousarray(wl["nodes"][ids])
    u = W.coefficients(wl["nodes"].shape[0], M, seed=0)[ids]
    for _ in range(args.warmup):
        oracle.helmholtz(shape, P, Q, g, nodes, 1.0, u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.helmholtz(shape, P, Q, g, nodes, 1.0, u)
    dt = (time.perf_counter() - t0) / args.steps
    v = k * M / dt / 1e9
    cores = oracle.threads()
    line = {"impl": "reference", "metric": "Helmholtz apply GDOF/s", "value": v, "unit": "GDOF/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, wl),
            "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                             "sample": f"{k} seeded elements of {wl['nodes'].shape[0]} per step"},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, wl):
    E = wl["nodes"].shape[0]
    cfg = {"workload": args.workload, "shape": wl["shape"], "nelem": E, "P": wl["P"], "Q": wl["Q"],
           "geometry": "curved (per-point factors)" if wl["deformed"] else "affine",
           "lambda": 1.0, "precision": args.prec}
    if getattr(args, "basis", "modified") != "modified":
        cfg["basis"] = "GLL-Lagrange (nodal)"
    return cfg


def cpu_baseline(args, wl, budget_s: float = 15.0, y_gpu=None):
    """Oracle timed on a bounded seeded sample (rank 0, N = 1 only).  With the
    GPU result y_gpu [E][M] (FP64), also its error against the oracle on that
    sample."""
    import oracle
    shape, P, Q, g = wl["shape"], wl["P"], wl["Q"], wl["gorder"]
    M = oracle.num_modes(shape, P)
    E = wl["nodes"].shape[0]
    k = 64
    u_all = W.coefficients(E, M, seed=0)
    while True:
        ids = W.sample_elements(E, k, seed=0)
        t0 = time.perf_counter()
        y_or = oracle.helmholtz(shape, P, Q, g, np.ascontiguousarray(wl["nodes"][ids]), 1.0, u_all[ids])
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or k >= E:
            break
        k = min(E, int(k * max(2.0, budget_s / 4 / max(dt, 1e-3))))
    out = {"value": k * M / dt / 1e9, "unit": "GDOF/s", "cores": oracle.threads(), "kind": "oracle",
           "sample": f"{k} seeded elements of {E}, one dense-matrix Helmholtz apply each"}
    if y_gpu is not None:
        out["gpu_rel_error_on_sample"] = rel_err(y_gpu[ids], y_or)
    return out


_FLUSH = {}


def needs_flush(nbytes: int) -> bool:
    """A step streaming less than twice the L2 could find part of its data
    still in L2 from the previous step: such timings flush L2 in between."""
    return nbytes < 2 * L2_BYTES


def l2_flush(stream):
    """Write a buffer of twice the L2 size on `stream` and read it back: what
    the previous launch left in L2 is evicted, and the write-back of the
    buffer's own dirty lines happens here rather than inside the next timed
    launch (L2 then holds only clean lines of the buffer)."""
    import torch
    dev = torch.cuda.current_device()
    if dev not in _FLUSH:
        _FLUSH[dev] = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    with torch.cuda.stream(stream):
        _FLUSH[dev].fill_(1.0)
        _FLUSH[dev].sum()


def l2_note(nbytes: int) -> str:
    mib = nbytes / 2 ** 20
    if needs_flush(nbytes):
        return (f"flushed: {2 * L2_BYTES / 2**20:.0f} MiB written and read back before each timed launch "
                f"({mib:.0f} MiB per step)")
    return f"no flush: {mib:.0f} MiB streamed per step > 2 x 129 MiB L2"


def time_calls(fn, stream, reps: int, nbytes: int = 0) -> float:
    """Seconds per call: CUDA events on the launching stream, after 3 untimed
    calls; around all `reps` calls, or, when the call streams less than twice
    the L2 (`nbytes`), around each call with L2 flushed before it."""
    import torch
    for _ in range(3):
        fn()
    if nbytes and needs_flush(nbytes):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for a, b in ev:
            l2_flush(stream)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / reps * 1e-3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps * 1e-3


def roofline_entry(prec, flops, nbytes, sec, fp64_peak, peaks):
    """FP64: FP64-pipe bound (flops / measured DFMA peak); FP32/BF16: HBM bound
    (algorithmic bytes / measured copy bandwidth)."""
    if prec == "f64":
        ach = flops / sec / 1e12
        return {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak}
    ach = nbytes / sec / 1e9
    pk = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk}


# the other configurations, plus the pyramid mesh (the shape the paper leaves
# to future work; not one of the measured configurations)
CONFIG_WORKLOADS = ("quad8x8_p4", "tet20_kuhn_p4", "prism40x40x20_p4", "pyr20_split_p4")


def config_table(nir, ctx, dev, stream, peaks, fp64_peak, args):
    """FP64 and FP32 Helmholtz apply rates, roofline fractions and sampled
    errors against the oracle on the other workloads: the 8x8 quad mesh, the
    Kuhn-split tet mesh, the prism mesh and the ~150k-element hybrid mesh (one
    graph launch per apply).  Each is tuned first (set-up, untimed)."""
    import torch
    import oracle
    out = {}
    for name in CONFIG_WORKLOADS:
        wl = W.workload(name)
        shape, P, Q, g = wl["shape"], wl["P"], wl["Q"], wl["gorder"]
        E = wl["nodes"].shape[0]
        blk = nir.Block(ctx, shape, E, P, deformed=wl["deformed"])
        blk.set_geometry(g, torch.from_numpy(wl["nodes"]).to(dev))
        if not args.no_tune:
            nir.Mesh(ctx, [blk]).tune(args.tune_cache)
        u64 = W.coefficients(E, blk.M, seed=0)
        ids = W.sample_elements(E, 16, seed=5)
        y_or = oracle.helmholtz(shape, P, Q, g, np.ascontiguousarray(wl["nodes"][ids]), 1.0, u64[ids])
        rec = {"shape": shape, "nelem": E, "P": P, "Q": Q, "dof": E * blk.M}
        reps = max(20, min(500, int(4e8 / (E * blk.M))))
        for prec in ("f64", "f32"):
            u = torch.from_numpy(u64).to(dev, nir.DTYPE[prec])
            y = torch.empty_like(u)
            wb = u.element_size()
            nb = E * helm_bytes_per_elem(shape, P + 1, Q, wb, wl["deformed"])
            sec = time_calls(lambda: blk.helmholtz(u, prec=prec, out=y), stream, reps, nb)
            rec[prec] = {"gdofs": E * blk.M / sec / 1e9, "ms_per_apply": sec * 1e3, "l2": l2_note(nb),
                         "roofline": roofline_entry(prec, E * helm_flops_per_elem(shape, P + 1, Q), nb,
                                                    sec, fp64_peak, peaks),
                         "rel_error_vs_oracle": rel_err(y.double().cpu().numpy()[ids], y_or)}
        out[name] = rec
        del blk, u, y
    parts = W.hybrid_mesh(seed=0)
    blocks = []
    for p in parts:
        b = nir.Block(ctx, p["shape"], p["nodes"].shape[0], p["P"], deformed=p["deformed"])
        b.set_geometry(p["gorder"], torch.from_numpy(p["nodes"]).to(dev))
        blocks.append(b)
    mesh = nir.Mesh(ctx, blocks)
    if not args.no_tune:
        mesh.tune(args.tune_cache)
    x64 = W.coefficients(1, mesh.ndof, seed=0)[0]
    samples = []
    for b, o, p in zip(blocks, mesh.offsets, parts):
        ids = W.sample_elements(b.nelem, 2, seed=p["P"])
        ref = oracle.helmholtz(p["shape"], p["P"], p["Q"], p["gorder"], np.ascontiguousarray(p["nodes"][ids]), 1.0,
                               x64[o:o + b.nelem * b.M].reshape(b.nelem, b.M)[ids])
        samples.append((o, b, ids, ref))
    rec = {"nelem": sum(b.nelem for b in blocks), "dof": mesh.ndof, "blocks": len(blocks)}
    for prec in ("f64", "f32"):
        x = torch.from_numpy(x64).to(dev, nir.DTYPE[prec])
        y = torch.empty_like(x)
        wb = x.element_size()
        flops = sum(p["nodes"].shape[0] * helm_flops_per_elem(p["shape"], p["P"] + 1, p["Q"]) for p in parts)
        nbytes = sum(p["nodes"].shape[0] * helm_bytes_per_elem(p["shape"], p["P"] + 1, p["Q"], wb, p["deformed"])
                     for p in parts)
        sec = time_calls(lambda: mesh.helmholtz(x, prec=prec, out=y), stream, 20, nbytes)
        yh = y.double().cpu().numpy()
        got = np.concatenate([yh[o:o + b.nelem * b.M].reshape(b.nelem, b.M)[ids].ravel() for o, b, ids, _ in samples])
        want = np.concatenate([r.ravel() for *_, r in samples])
        rec[prec] = {"gdofs": mesh.ndof / sec / 1e9, "ms_per_apply": sec * 1e3, "launch": mesh.get_launch(prec),
                     "l2": l2_note(nbytes),
                     "roofline": roofline_entry(prec, flops, nbytes, sec, fp64_peak, peaks),
                     "rel_error_vs_oracle": rel_err(got, want)}
    out["hybrid150k_p2to8"] = rec
    return out


def solve_section(nir, ctx, dev, args, local):
    """The P = 6 48^3 curved-hex solve: every solver variant, with wall time,
    iterations, residual, forward error against the oracle and speed-up over
    plain FP64 CG."""
    import torch
    wl = W.workload("hex48_curved_p6")
    E = wl["nodes"].shape[0]
    blk = nir.Block(ctx, wl["shape"], E, wl["P"], deformed=wl["deformed"])
    blk.set_geometry(wl["gorder"], torch.from_numpy(wl["nodes"]).to(dev))
    mesh = nir.Mesh(ctx, [blk])
    if not args.no_tune:
        mesh.tune(args.tune_cache)
    results, ndof = solve_compare(nir, mesh, blk, wl, dev, args, 1, local, args.solve_precs.split(","))
    best = max((k for k, r in results.items() if k != "f64" and r["rc"] == 0), key=lambda k: results[k]["gdofs"],
               default=None)
    return {"workload": "hex48_curved_p6", "nelem": E, "P": wl["P"], "Q": wl["Q"], "dof": ndof,
            "tol": args.tol, "fwd_tol": args.fwd_tol, "inner_tol": args.inner_tol,
            "solve": "CG on the broken operator, Jacobi preconditioner; rhs B^T W f, "
                     "f = (3 pi^2 + 1) sin(pi x) sin(pi y) sin(pi z)",
            "variants": results, "fastest": best,
            "speedup_vs_fp64_cg": results[best]["speedup_vs_fp64_cg"] if best else None}


def run_nir(args, ws, rank, local):
    import torch
    import paper_2606_20917_gb300 as nir

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = nir.Context(local, stream)
    wl = W.workload(args.workload)
    shape, P, Q, g = wl["shape"], wl["P"], wl["Q"], wl["gorder"]
    E = wl["nodes"].shape[0]
    blk = nir.Block(ctx, shape, E, P, deformed=wl["deformed"], basis=args.basis)
    blk.set_geometry(g, torch.from_numpy(wl["nodes"]).to(dev))
    if not args.no_tune:
        # set-up, untimed: the library's autotuner picks elements per CTA, grid
        # size and metric-prefetch policy for this block on this GPU (a cache
        # file, when given, is read back instead of re-timing)
        nir.Mesh(ctx, [blk]).tune(args.tune_cache)
    toe = args.strategy == "elements"
    if toe:  # the paper's other GPU strategy: one thread per element (tuning variant 4)
        blk.set_tuning(args.prec, 4, 0, 0)
    prof = (f"helm_toe_{args.workload}_{args.prec}", TOE_SOURCES) if toe else \
        (f"helm_{args.workload}_{args.prec}", KERNEL_SOURCES)
    M = blk.M
    dt_t = nir.DTYPE[args.prec]
    u = torch.from_numpy(W.coefficients(E, M, seed=0)).to(dev, dt_t)
    y = torch.empty_like(u)
    wb = u.element_size()
    work_bytes = E * helm_bytes_per_elem(shape, P + 1, Q, wb, wl["deformed"])

    for _ in range(args.warmup):
        blk.helmholtz(u, lam=1.0, prec=args.prec, out=y)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    flush = needs_flush(work_bytes)   # then L2 is flushed before each launch, outside its events
    with ClockSampler(local) as clk:
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for k in range(args.steps):
            if flush:
                l2_flush(stream)
            ev[k][0].record(stream)
            blk.helmholtz(u, lam=1.0, prec=args.prec, out=y)
            ev[k][1].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    per_launch = [a.elapsed_time(b) for a, b in ev]
    ms_total = sum(per_launch) if flush else t_all0.elapsed_time(t_all1)
    ms_total = max_over_ranks(ws, ms_total, dev)
    ms_step = ms_total / args.steps
    dof = E * M
    value = ws * dof * args.steps / (ms_total * 1e-3) / 1e9

    # e2e: the same apply through the host-buffer C-ABI call (H2D + apply + D2H)
    uh = u.cpu().pin_memory()
    yh = torch.empty_like(uh).pin_memory()
    for _ in range(2):
        blk.helmholtz_host(uh, yh, lam=1.0, prec=args.prec)
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        blk.helmholtz_host(uh, yh, lam=1.0, prec=args.prec)
    e2e_s = max_over_ranks(ws, (time.perf_counter() - t0) / args.steps, dev)
    e2e = {"value": ws * dof / e2e_s / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": uh.numel() * wb,
           "d2h_bytes_per_step": yh.numel() * wb}

    if rank != 0:
        return
    peaks = measured_peaks()
    avg_launch_s = statistics.mean(per_launch) * 1e-3
    flops = helm_flops_per_elem(shape, P + 1, Q) * E
    if args.prec == "f64":
        with ClockSampler(local) as pclk:   # probes repeated so the clock sampler sees them
            probes = [ctx.probe_fp64_peak() for _ in range(5)]
            mma = max(ctx.probe_fp64_mma_peak() for _ in range(3))
        fp64 = max(probes)
        roof = {"bound": "alu", "achieved": flops / avg_launch_s / 1e12, "peak": fp64, "unit": "TFLOP/s",
                "frac": flops / avg_launch_s / 1e12 / fp64,
                "traffic": profiled_traffic(*prof),
                "peak_source": "FP64 FMA throughput measured in this run by nir_probe_fp64_peak "
                               "(register-resident DFMA chains); nominal GB300 FP64 is 1.25 TFLOP/s",
                "flops_per_elem": flops // E,
                "hbm_gbs_at_this_rate": work_bytes / avg_launch_s / 1e9,
                "peak_probe": {"dfma_tflops": probes, "dmma_tflops": mma, "clocks": pclk.summary(),
                               "note": "FP64 tensor-core (mma.sync m8n8k4 f64) rate; below DFMA, so no "
                                       "FP64 kernel uses the tensor pipe"}}
    else:
        gbs = work_bytes / avg_launch_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "traffic": profiled_traffic(*prof),
                "bytes_per_elem": work_bytes // E,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "_fallback" not in peaks else "fallback 6.8 TB/s"}
    # three fields sharing the operator in one launch (after the timed region)
    fields = None
    if ws == 1 and not args.no_operators:
        us = [u, u.clone(), u.clone()]
        ys = [torch.empty_like(u) for _ in range(3)]
        nb3 = work_bytes + 4 * E * M * wb   # two more fields in and out; the metric once
        fms = time_calls(lambda: blk.helmholtz_fields(us, lam=1.0, prec=args.prec, outs=ys), stream, args.steps,
                         nb3) * 1e3
        fields = {"fields": 3, "ms_per_launch": fms, "gdofs": 3 * dof / (fms * 1e-3) / 1e9, "l2": l2_note(nb3),
                  "speedup_per_field_vs_single": (3 * dof / (fms * 1e-3)) / (dof / avg_launch_s)}
        del us, ys
    operators = {}
    if shape == "hex" and ws == 1 and not args.no_operators:
        operators = operator_table(blk, args.prec, dev, stream, wl, ctx if args.prec == "f64" else None, peaks,
                                   roof["peak"] if (roof and args.prec == "f64") else None)
    extras = {}
    if args.extras and ws == 1:
        for p in ("f32", "bf16"):
            if p == args.prec:
                continue
            up = u.to(nir.DTYPE[p])
            yp = torch.empty_like(up)
            nb = E * helm_bytes_per_elem(shape, P + 1, Q, up.element_size(), wl["deformed"])
            sec = time_calls(lambda: blk.helmholtz(up, prec=p, out=yp), stream, 10, nb)
            extras[f"{p}_apply_gdofs"] = dof / sec / 1e9
    line = {"metric": "Helmholtz apply GDOF/s", "value": value, "unit": "GDOF/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": dict(workload_config(args, wl), tuned=not args.no_tune,
                           strategy="threading over elements" if toe else "element groups per CTA",
                           l2=l2_note(work_bytes)),
            "roofline": roof, "e2e": e2e, "gpu_launches": args.steps, "clocks": clk.summary(),
            "multi_field": fields,
            "kernel_ms_per_launch": statistics.mean(per_launch)}
    if operators:
        line["operators"] = operators
    if extras:
        line["extras"] = extras
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, wl, y_gpu=y.double().cpu().numpy() if args.prec == "f64" else None)
    if ws == 1 and not args.no_configs:
        fp64_pk = roof["peak"] if args.prec == "f64" else ctx.probe_fp64_peak()
        line["configs"] = config_table(nir, ctx, dev, stream, peaks, fp64_pk, args)
    if ws == 1 and not args.no_solve:
        line["solve"] = solve_section(nir, ctx, dev, args, local)
    print(json.dumps(line), flush=True)


def operator_table(blk, prec, dev, stream, wl, ctx, peaks, fp64_peak):
    """Throughput and roofline fraction of every elemental operator (not only
    the fused Helmholtz) on the same block, timed with CUDA events."""
    import torch
    import paper_2606_20917_gb300 as nir
    E, M, NQ = blk.nelem, blk.M, blk.NQ
    dt = nir.DTYPE[prec]
    wb = torch.empty((), dtype=dt).element_size()
    N, Q = wl["P"] + 1, wl["Q"]
    u = torch.from_numpy(W.coefficients(E, M, seed=0)).to(dev, dt)
    f = torch.from_numpy(W.phys_samples(E, NQ, seed=1)).to(dev, dt)
    fs = [torch.from_numpy(W.phys_samples(E, NQ, seed=2 + i)).to(dev, dt) for i in range(3)]
    outs = {"bwd": torch.empty((E, NQ), dtype=dt, device=dev), "m": torch.empty((E, M), dtype=dt, device=dev),
            "d": [torch.empty((E, NQ), dtype=dt, device=dev) for _ in range(3)]}
    calls = {
        "bwd": lambda: blk.bwd_trans(u, prec=prec, out=outs["bwd"]),
        "iprod": lambda: blk.iproduct_wrt_base(f, prec=prec, out=outs["m"]),
        "physderiv": lambda: blk.phys_deriv(f, prec=prec, outs=outs["d"]),
        "iprod_deriv": lambda: blk.iproduct_wrt_deriv_base(fs, prec=prec, out=outs["m"]),
        "mass": lambda: blk.mass(u, prec=prec, out=outs["m"]),
    }
    res = {}
    for op, fn in calls.items():
        flops, byts = op_work_per_elem(op, N, Q, wb, wl["deformed"])
        sec = time_calls(fn, stream, 10, byts * E)
        r = {"gdofs": E * M / sec / 1e9, "ms": sec * 1e3, "flops_per_elem": flops, "bytes_per_elem": byts,
             "l2": l2_note(byts * E)}
        if prec == "f64" and fp64_peak:
            # FP64 on GB300: the ridge is ~0.19 flop/B, so every operator is FP64-pipe bound
            ach = flops * E / sec / 1e12
            r["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": ach / fp64_peak}
        else:
            gbs = byts * E / sec / 1e9
            pk = peaks.get("hbm_gbs", 6800.0)
            r["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": pk, "unit": "GB/s", "frac": gbs / pk}
        res[op] = r
    return res


# Solver variants compared on the P = 6 workload: name -> (operator precision
# inside CG, inner-solver vector precision).  "f64" is plain FP64 CG.
SOLVE_VARIANTS = {
    "f64": ("f64", "f64"),
    "f32": ("f32", "f64"),        # FP32 operator, FP64 inner vectors and dots
    "f32_vec32": ("f32", "f32"),  # FP32 operator, FP32 inner vectors, compensated dots
    "bf16": ("bf16", "f64"),      # BF16 storage operator, FP64 inner vectors
}


def rel_err(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_solve_sample(wl, ids, lam):
    """The oracle's own solution on sampled elements: right-hand side
    b = B^T W f with f = (3 pi^2 + lam) sin(pi x) sin(pi y) sin(pi z) at the
    oracle's quadrature points (its own geometry), then the per-element dense
    Cholesky solve of the broken operator."""
    import oracle
    shape, P, Q, g = wl["shape"], wl["P"], wl["Q"], wl["gorder"]
    nodes = np.ascontiguousarray(wl["nodes"][ids])
    _, _, X = oracle.geom_factors(shape, Q, g, nodes, with_x=True)
    s = np.sin(np.pi * X)
    f = (3 * np.pi ** 2 + lam) * s[..., 0] * s[..., 1] * s[..., 2]
    bs = oracle.iprod(shape, P, Q, g, nodes, f)
    return oracle.helmholtz_solve(shape, P, Q, g, nodes, lam, bs)


def dist_allreduce(ws, dev):
    """Host-array sum over the torchrun ranks for a sharded solve (None at N = 1)."""
    if ws == 1:
        return None
    import torch
    import torch.distributed as dist
    on_gpu = dist.get_backend() == "nccl"

    def f(v):
        t = torch.from_numpy(v.copy())
        if on_gpu:
            t = t.to(dev)
        dist.all_reduce(t)
        v[:] = t.cpu().numpy()
    return f


def solve_compare(nir, mesh, blk, wl, dev, args, ws, local, variants, sample=8, allreduce=None):
    """Time each solver variant once (after a loose warm-up solve that captures
    its iteration graphs and builds the preconditioner) on the manufactured
    right-hand side, to relative residual args.tol and forward tolerance
    args.fwd_tol; report its error against the oracle's per-element Cholesky
    solution on a seeded sample of elements.  With `allreduce` the mesh is this
    rank's part of a sharded mesh (wl holds its elements) and the solve sums
    its scalars over the ranks."""
    import torch
    lam = 1.0
    E, M = blk.nelem, blk.M
    eta, xi = blk.points()
    f = manufactured_rhs_points(wl, xi, lam, dev)
    b = blk.iproduct_wrt_base(f).reshape(-1).contiguous()
    del f
    ids = W.sample_elements(E, sample, seed=11)
    x_or = oracle_solve_sample(wl, ids, lam) if ws == 1 or int(os.environ.get("RANK", "0")) == 0 else None
    results, xs = {}, {}
    for name in variants:
        inner, vec = SOLVE_VARIANTS[name]
        kw = dict(lam=lam, inner_prec=inner, inner_vectors=vec, tol=args.tol, fwd_tol=args.fwd_tol, max_outer=60,
                  max_inner=args.max_inner if inner != "bf16" else min(args.max_inner, 3000),
                  inner_tol=args.inner_tol)
        if allreduce is not None:
            kw["allreduce"] = allreduce
        mesh.cg_solve(b, torch.zeros_like(b), **dict(kw, tol=1e-2, fwd_tol=0.0))
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        barrier(ws)
        with ClockSampler(local) as clk, ProfileRegion(args.profile_region):
            t0 = time.perf_counter()
            rc, st = mesh.cg_solve(b, x, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        dt = max_over_ranks(ws, dt, dev)
        # replicas: N copies of the problem; sharded: one problem split over the ranks
        ndof_all = ws * b.numel() if allreduce is None else int(sum_over_ranks(ws, float(b.numel()), dev))
        r = dict(rc=rc, operator=inner, inner_vectors=vec if inner != "f64" else "f64", wall_seconds=dt,
                 gdofs=ndof_all / dt / 1e9, outer=st["outer"], inner_total=st["inner_total"],
                 rel_residual=st["rel_residual"], rel_correction=st["rel_correction"], clocks=clk.summary())
        if x_or is not None:
            r["fwd_error_vs_oracle"] = rel_err(x.view(E, M)[torch.from_numpy(ids).to(dev)].cpu().numpy(), x_or)
            r["oracle_sample"] = f"{len(ids)} seeded elements of {E}: oracle b = B^T W f and dense Cholesky"
        results[name] = r
        xs[name] = x
    if "f64" in xs:
        ref = xs["f64"]
        for name, x in xs.items():
            if name != "f64":
                results[name]["rel_diff_vs_fp64_cg"] = float(torch.linalg.norm(x - ref) / torch.linalg.norm(ref))
    base = results.get("f64")
    ok = base is not None and base["rc"] == 0
    for name, r in results.items():
        if name != "f64":
            r["speedup_vs_fp64_cg"] = (base["wall_seconds"] / r["wall_seconds"]) if (ok and r["rc"] == 0) else None
    return results, b.numel()


def run_solve(args, ws, rank, local):
    """Helmholtz solve on the P = 6 curved-hex workload: plain FP64 CG versus CG
    with the operator in FP32 / BF16 inside FP64 iterative refinement.  Under
    torchrun (N > 1) the mesh is sharded: each rank takes its cost-balanced
    contiguous element range (nir_partition_elements) and the solve sums its
    FP64 scalars over the ranks (strong scaling: one problem, N GPUs)."""
    import torch
    import paper_2606_20917_gb300 as nir

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = nir.Context(local, torch.cuda.current_stream())
    wl = W.workload(args.workload)
    if ws > 1:
        first = nir.partition_elements([(wl["shape"], wl["P"], wl["nodes"].shape[0])], ws)
        wl = dict(wl, nodes=np.ascontiguousarray(wl["nodes"][first[rank]:first[rank + 1]]))
    E = wl["nodes"].shape[0]
    blk = nir.Block(ctx, wl["shape"], E, wl["P"], deformed=wl["deformed"])
    blk.set_geometry(wl["gorder"], torch.from_numpy(wl["nodes"]).to(dev))
    mesh = nir.Mesh(ctx, [blk])
    if not args.no_tune:
        mesh.tune(args.tune_cache)  # set-up, untimed
    results, ndof = solve_compare(nir, mesh, blk, wl, dev, args, ws, local, args.solve_precs.split(","),
                                  allreduce=dist_allreduce(ws, dev))
    if rank != 0:
        return
    best = max((r for k, r in results.items() if k != "f64" and r["rc"] == 0), key=lambda r: r["gdofs"],
               default=None)
    line = {"metric": "Helmholtz solve GDOF/s to relative residual %g, forward tolerance %g" % (args.tol, args.fwd_tol),
            "value": best["gdofs"] if best else None, "unit": "GDOF/s", "n_gpus": ws, "steps": 1,
            "warmup": 1, "ms_per_step": best["wall_seconds"] * 1e3 if best else None, "higher_is_better": True,
            "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None,
            "dtype": "f32 operator / f64 refinement", "data": "synthetic",
            "config": dict(workload_config(args, wl), solve="CG on the broken operator, Jacobi preconditioner",
                           rhs="B^T W f, f = (3 pi^2 + 1) sin(pi x) sin(pi y) sin(pi z)",
                           sharding=(f"{ws} ranks, contiguous cost-balanced element ranges, CG scalars summed "
                                     f"over the ranks") if ws > 1 else "none"),
            "solves": results,
            "speedup_vs_fp64_cg": best.get("speedup_vs_fp64_cg") if best else None}
    print(json.dumps(line), flush=True)


def manufactured_rhs_points(wl, xi, lam, dev):
    """f at the quadrature points of every element (input generation: the
    element map is evaluated from the lattice nodes by tensor Lagrange
    interpolation, with torch on the device)."""
    import torch
    g = wl["gorder"]
    t = np.linspace(-1.0, 1.0, g + 1)

    def lag(x):
        L = np.ones((x.size, g + 1))
        for a in range(g + 1):
            for c in range(g + 1):
                if c != a:
                    L[:, a] *= (x - t[c]) / (t[a] - t[c])
        return L

    L1, L2, L3 = lag(xi[:, 0]), lag(xi[:, 1]), lag(xi[:, 2])
    Lt = np.einsum("na,nb,nc->ncba", L1, L2, L3).reshape(xi.shape[0], -1)  # node a fastest
    Lt = torch.from_numpy(Lt).to(dev)
    nodes = torch.from_numpy(wl["nodes"]).to(dev)
    X = torch.einsum("nv,evd->end", Lt, nodes)
    s = torch.sin(np.pi * X)
    return ((3 * np.pi ** 2 + lam) * s[..., 0] * s[..., 1] * s[..., 2]).contiguous()


class ProfileRegion:
    """cudaProfilerStart/Stop around a timed region when --profile-region is set."""

    def __init__(self, on: bool):
        self.on = on

    def __enter__(self):
        if self.on:
            import torch
            torch.cuda.cudart().cudaProfilerStart()
        return self

    def __exit__(self, *a):
        if self.on:
            import torch
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()


def run_gsolve(args, ws, rank, local):
    """Global C0 Helmholtz solve with Dirichlet data on the P = 6 curved-hex
    workload: the elements are assembled into the continuous space, the
    boundary values are the L2 projection of the exact solution (an assembled
    mass-matrix CG, set-up), and CG solves for the interior dofs -- plain FP64
    versus the FP32 / BF16 operator inside FP64 iterative refinement."""
    import torch
    import paper_2606_20917_gb300 as nir

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = nir.Context(local, torch.cuda.current_stream())
    wl = W.workload(args.workload)
    E = wl["nodes"].shape[0]
    n = int(round(E ** (1.0 / 3.0)))
    blk = nir.Block(ctx, wl["shape"], E, wl["P"], deformed=wl["deformed"])
    blk.set_geometry(wl["gorder"], torch.from_numpy(wl["nodes"]).to(dev))
    mesh = nir.Mesh(ctx, [blk])
    if not args.no_tune:
        mesh.tune(args.tune_cache)  # set-up, untimed
    t0 = time.perf_counter()
    asm = nir.Assembly(ctx, [blk], [W.grid_vertices(n, 3)])
    t_number = time.perf_counter() - t0
    eta, xi = blk.points()
    lam = 1.0
    f = manufactured_rhs_points(wl, xi, lam, dev)
    u = f / (3 * np.pi ** 2 + lam)
    # Dirichlet data: L2 projection of u onto the conforming space (set-up)
    bu = asm.assemble(blk.iproduct_wrt_base(u).reshape(-1))
    up = torch.zeros_like(bu)
    t0 = time.perf_counter()
    rc_p, st_p = asm.cg_solve(bu, up, op="mass", fix_boundary=False, inner_prec="f32", tol=1e-12,
                              max_outer=60, max_inner=args.max_inner, inner_tol=args.inner_tol)
    torch.cuda.synchronize()
    t_proj = time.perf_counter() - t0
    b = asm.assemble(blk.iproduct_wrt_base(f).reshape(-1))
    umax = float(u.abs().max())
    results = {}
    for name in args.solve_precs.split(","):
        inner, vec = SOLVE_VARIANTS[name]
        kw = dict(lam=lam, inner_prec=inner, inner_vectors=vec, tol=args.tol, max_outer=60,
                  max_inner=args.max_inner, inner_tol=args.inner_tol)
        x = up.clone()
        x[:asm.n_free] = 0.0
        xw = x.clone()
        asm.cg_solve(b, xw, **dict(kw, tol=1e-2))  # warm-up: graph capture, preconditioner
        del xw
        torch.cuda.synchronize()
        barrier(ws)
        with ClockSampler(local) as clk, ProfileRegion(args.profile_region):
            t0 = time.perf_counter()
            rc, st = asm.cg_solve(b, x, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        dt = max_over_ranks(ws, dt, dev)
        uq = blk.bwd_trans(asm.gather(x).view(E, blk.M))
        err = float((uq - u).abs().max()) / umax
        results[name] = dict(rc=rc, operator=inner, inner_vectors=vec, wall_seconds=dt,
                              gdofs=ws * asm.n_free / dt / 1e9,
                              gdofs_local=ws * E * blk.M / dt / 1e9, clocks=clk.summary(), outer=st["outer"],
                              inner_total=st["inner_total"], rel_residual=st["rel_residual"],
                              max_rel_error_vs_exact=err)
    if rank != 0:
        return
    best = max((r for k, r in results.items() if k != "f64" and r["rc"] == 0), key=lambda r: r["gdofs"],
               default=None)
    base = results.get("f64")
    line = {"metric": "Assembled C0 Helmholtz solve GDOF/s (Dirichlet) to relative residual %g" % args.tol,
            "value": best["gdofs"] if best else None, "unit": "GDOF/s", "n_gpus": ws, "steps": 1,
            "warmup": 1, "ms_per_step": best["wall_seconds"] * 1e3 if best else None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 operator / f64 refinement", "data": "synthetic",
            "config": dict(workload_config(args, wl), solve="CG on A^T H A over the free dofs, Jacobi",
                           dofs_global=asm.n_global, dofs_free=asm.n_free, dofs_local=E * blk.M,
                           exact="u = sin(pi x) sin(pi y) sin(pi z); f = (3 pi^2 + 1) u",
                           dirichlet="L2 projection of u (assembled mass CG, FP32 inner / FP64 refinement, to 1e-12)"),
            "setup": dict(numbering_seconds=t_number, projection_seconds=t_proj, projection_rc=rc_p,
                          projection_iters=st_p["inner_total"], projection_sweeps=st_p["outer"]),
            "solves": results,
            "speedup_vs_fp64_cg": (best["gdofs"] / base["gdofs"]) if (best and base and base["rc"] == 0) else None}
    print(json.dumps(line), flush=True)


def run_sweep(args, ws, rank, local):
    """Helmholtz throughput against problem size for P = 1..9 on hexahedra and
    tetrahedra (the paper's GPU throughput study, Sec. 4.2): one block per
    (shape, P, size), throughput = DOF / device time of one apply (CUDA events
    over repeated applies, the faster of the two code generations of the
    default group), with the kernel's registers per thread; and the same for
    the paper's other strategy, threading over elements (key "toe")."""
    import torch
    import paper_2606_20917_gb300 as nir

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = nir.Context(local, stream)
    fp64_peak = ctx.probe_fp64_peak()
    peaks = measured_peaks()
    prec = args.prec
    wb = {"f64": 8, "f32": 4, "bf16": 2}[prec]
    targets = [float(t) for t in args.sweep_dofs.split(",")]
    recs = []
    for shape in args.sweep_shapes.split(","):
        for P in [int(v) for v in args.sweep_orders.split(",")]:
            N, Q = P + 1, P + 2
            M = num_modes(shape, N)
            for target in targets:
                E = max(1, int(round(target / M)))
                if shape == "hex":
                    n = max(1, int(round(E ** (1.0 / 3.0))))
                    nodes, gorder, deformed = W.hex_grid(n, 2), 2, True
                else:   # 6 tets or 6 pyramids per cell
                    n = max(1, int(round((E / 6.0) ** (1.0 / 3.0))))
                    nodes = W.tet_kuhn(n) if shape == "tet" else W.pyramid_split(n, n, n)
                    gorder, deformed = 1, False
                E = nodes.shape[0]
                blk = nir.Block(ctx, shape, E, P, deformed=deformed)
                blk.set_geometry(gorder, torch.from_numpy(nodes).to(dev))
                x = torch.from_numpy(W.coefficients(E, M, seed=0)).to(dev, nir.DTYPE[prec])
                y = torch.empty_like(x)
                reps = max(3, min(50, int(2e8 / (E * M))))
                # the two code generations of the default group (variants 0 and 3), L2
                # metric prefetch on in FP32/BF16; the faster is reported
                def time_apply():
                    for _ in range(3):
                        blk.helmholtz(x, prec=prec, out=y)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    a.record(stream)
                    for _ in range(reps):
                        blk.helmholtz(x, prec=prec, out=y)
                    b.record(stream)
                    torch.cuda.synchronize()
                    return a.elapsed_time(b) / reps * 1e-3

                best = None
                for variant in (0, 3):
                    blk.set_tuning(prec, variant, 0, 0 if prec == "f64" else 1)
                    tv = time_apply()
                    if best is None or tv < best[0]:
                        best = (tv, variant, blk.kernel_info(prec, "helm"))
                t = best[0]
                rec = {"shape": shape, "P": P, "nelem": E, "dof": E * M, "gdofs": E * M / t / 1e9,
                       "ms": t * 1e3, "variant": best[1], **best[2]}

                def frac(tt):
                    if prec == "f64":
                        return {"frac_fp64": E * helm_flops_per_elem(shape, N, Q) / tt / 1e12 / fp64_peak}
                    return {"frac_hbm": E * helm_bytes_per_elem(shape, N, Q, wb, deformed) / tt / 1e9
                            / peaks["hbm_gbs"]}
                rec.update(frac(t))
                if not args.sweep_no_toe and shape != "pyr":
                    # the other strategy: threading over elements (one thread per element)
                    blk.set_tuning(prec, 4, 0, 0)
                    tt = time_apply()
                    rec["toe"] = {"gdofs": E * M / tt / 1e9, "ms": tt * 1e3, **blk.kernel_info(prec, "helm"),
                                  **frac(tt)}
                recs.append(rec)
                del blk, x, y
                torch.cuda.empty_cache()
    if rank != 0:
        return
    line = {"metric": "Helmholtz apply GDOF/s vs DOF and P (sweep)", "value": None, "unit": "GDOF/s",
            "n_gpus": ws, "higher_is_better": True, "dtype": prec, "data": "synthetic",
            "config": {"workload": "hex (32-cell-style curved grids, lattice g = 2) and Kuhn-split tet meshes, "
                                   "P = 1..9, Q = P + 2", "dof_targets": targets, "fp64_peak_tflops": fp64_peak},
            "sweep": recs}
    print(json.dumps(line), flush=True)


def run_hybrid(args, ws, rank, local):
    """Hybrid mesh (~150k hex/prism/tet, P = 2..8) in one persistent launch."""
    import torch
    import paper_2606_20917_gb300 as nir

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = nir.Context(local, stream)
    parts = W.hybrid_mesh(seed=0)
    blocks = []
    for p in parts:
        b = nir.Block(ctx, p["shape"], p["nodes"].shape[0], p["P"], deformed=p["deformed"])
        b.set_geometry(p["gorder"], torch.from_numpy(p["nodes"]).to(dev))
        blocks.append(b)
    mesh = nir.Mesh(ctx, blocks)
    if not args.no_tune:
        mesh.tune(args.tune_cache)  # set-up, untimed
    res = {}
    nel = sum(b.nelem for b in blocks)
    peaks = measured_peaks()
    fp64_peak = ctx.probe_fp64_peak()
    for prec in ("f64", "f32"):
        x = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=0)[0]).to(dev, nir.DTYPE[prec])
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            mesh.helmholtz(x, prec=prec, out=y)
        torch.cuda.synchronize()
        barrier(ws)
        a, bev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            a.record(stream)
            for _ in range(args.steps):
                mesh.helmholtz(x, prec=prec, out=y)
            bev.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(ws, a.elapsed_time(bev) / args.steps, dev)
        res[prec] = {"gdofs": ws * mesh.ndof / (ms * 1e-3) / 1e9, "ms_per_apply": ms, "clocks": clk.summary(),
                     "launch": mesh.get_launch(prec)}
        # the other launch form, for comparison (the tuner picked the one above)
        chosen = mesh.get_launch(prec)
        other = "blocks" if chosen == "persistent" else "persistent"
        mesh.set_launch(prec, other)
        for _ in range(args.warmup):
            mesh.helmholtz(x, prec=prec, out=y)
        a.record(stream)
        for _ in range(args.steps):
            mesh.helmholtz(x, prec=prec, out=y)
        bev.record(stream)
        torch.cuda.synchronize()
        res[prec]["ms_per_apply_" + other] = a.elapsed_time(bev) / args.steps
        mesh.set_launch(prec, chosen)
        wb = {"f64": 8, "f32": 4}[prec]
        flops = sum(p["nodes"].shape[0] * helm_flops_per_elem(p["shape"], p["P"] + 1, p["Q"]) for p in parts)
        nbytes = sum(p["nodes"].shape[0] * helm_bytes_per_elem(p["shape"], p["P"] + 1, p["Q"], wb, p["deformed"])
                     for p in parts)
        t = ms * 1e-3
        if prec == "f64":
            ach = flops / t / 1e12
            res[prec]["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                     "frac": ach / fp64_peak, "flops_per_apply": flops,
                                     "peak_source": "FP64 FMA throughput measured in this run"}
        else:
            ach = nbytes / t / 1e9
            res[prec]["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                     "frac": ach / peaks["hbm_gbs"], "bytes_per_apply": nbytes,
                                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    if rank != 0:
        return
    line = {"metric": "Helmholtz apply GDOF/s (hybrid mesh, one graph launch)", "value": res["f64"]["gdofs"],
            "unit": "GDOF/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["f64"]["ms_per_apply"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "hybrid mesh: 50000 curved hex + 25000 prism + 75000 tet, P ~ U{2..8}, Q = P+2",
                       "launch": "one CUDA graph per apply: the persistent queue or the block kernels in "
                                 "sequence, whichever the tuner measured faster (per precision)",
                       "nelem": nel, "ndof": mesh.ndof, "blocks": len(blocks), "tuned": not args.no_tune},
            "precisions": res,
            "gpu_launches": args.steps * (1 if res["f64"]["launch"] == "persistent" else len(blocks))}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)  # ~0.9 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["nir", "reference"], default="nir")
    ap.add_argument("--workload", default="hex32_curved_p4")
    ap.add_argument("--prec", choices=["f64", "f32", "bf16"], default="f64")
    ap.add_argument("--sample", type=int, default=256, help="reference arm: elements per step")
    ap.add_argument("--extras", action="store_true", help="also time the FP32/BF16 applies")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-operators", action="store_true", help="skip the per-operator table")
    ap.add_argument("--no-configs", action="store_true",
                    help="apply mode: skip the quad/tet/prism/hybrid apply table")
    ap.add_argument("--no-solve", action="store_true",
                    help="apply mode: skip the P = 6 solve comparison")
    ap.add_argument("--mode", choices=["apply", "solve", "gsolve", "hybrid", "sweep"], default="apply")
    ap.add_argument("--basis", choices=["modified", "nodal"], default="modified",
                    help="apply mode: expansion basis (nodal = GLL-Lagrange, quad/hex)")
    ap.add_argument("--sweep-shapes", default="hex,tet", help="sweep: shapes among hex, tet, pyr")
    ap.add_argument("--sweep-dofs", default="1e5,1e6,1e7,3e7")
    ap.add_argument("--sweep-orders", default="1,2,3,4,5,6,7,8,9", help="sweep: polynomial degrees P")
    ap.add_argument("--sweep-no-toe", action="store_true", help="sweep the default strategy only")
    ap.add_argument("--strategy", choices=["groups", "elements"], default="groups",
                    help="apply mode: the default kernels (element groups per CTA) or threading over elements")
    ap.add_argument("--solve-precs", default="f64,f32,f32_vec32,bf16",
                    help="solver variants: " + ",".join(SOLVE_VARIANTS))
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--fwd-tol", type=float, default=1e-10,
                    help="solves: also stop only when the last correction |dx| <= fwd_tol |x|")
    ap.add_argument("--inner-tol", type=float, default=1e-3)
    ap.add_argument("--max-inner", type=int, default=20000)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner set-up")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (read if present, else written)")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed region with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup(args)
    if args.mode in ("solve", "gsolve") and args.workload == "hex32_curved_p4":
        args.workload = "hex48_curved_p6"
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.mode == "solve":
        run_solve(args, ws, rank, local)
    elif args.mode == "gsolve":
        run_gsolve(args, ws, rank, local)
    elif args.mode == "hybrid":
        run_hybrid(args, ws, rank, local)
    elif args.mode == "sweep":
        run_sweep(args, ws, rank, local)
    else:
        run_nir(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
