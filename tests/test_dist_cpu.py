"""Multi-process host logic on CPU (gloo, world size 2).

The operators are element-local, so N GPUs run N independent copies of the
workload (weak scaling) with no data-path collective; only the timing uses a
barrier and a max over ranks.  A solve sharded across ranks splits the mesh
into contiguous cost-balanced element ranges (the library's partitioner) and
sums the CG's FP64 scalars over the ranks.  These tests exercise that logic
without a GPU.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.max_over_ranks(world, float(rank + 1) * 0.25)
    out[rank] = m
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 0.5


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29519", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--sample", "4"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"


# ---------------------------------------------------------------------------
# Sharded solve: the library's partitioner (host code, no GPU) and the CG
# recurrence with its FP64 scalars summed over gloo ranks.

def _nir():
    sys.path.insert(0, ROOT)
    import paper_2606_20917_gb300 as nir
    return nir


def _flops(shape, P):
    """Independent restatement of the per-element Helmholtz flop counts."""
    sys.path.insert(0, ROOT)
    import bench
    return bench.helm_flops_per_elem(shape, P + 1, P + 2)


def test_partition_closed_forms():
    nir = _nir()
    assert nir.partition_elements([("hex", 3, 10)], 2) == [0, 5, 10]
    assert nir.partition_elements([("hex", 3, 10)], 3) == [0, 3, 7, 10]
    assert nir.partition_elements([("tet", 2, 7)], 1) == [0, 7]
    # more ranks than elements: empty ranges, still covering everything in order
    f = nir.partition_elements([("quad", 1, 2)], 5)
    assert f[0] == 0 and f[-1] == 2 and all(a <= b for a, b in zip(f, f[1:]))
    with pytest.raises(nir.NirError):
        nir.partition_elements([("hex", 0, 10)], 2)
    with pytest.raises(nir.NirError):
        nir.partition_elements([("hex", 3, 10)], 0)


@pytest.mark.parametrize("nranks", [2, 3, 4, 7, 8])
def test_partition_balances_flops(nranks):
    """Ranges over a mixed mesh cover every element once, in order, and each
    rank's flops differ from the even share by at most one element's cost."""
    nir = _nir()
    rng = np.random.default_rng(nranks)
    blocks = [(s, int(rng.integers(1, 9)), int(rng.integers(0, 3000))) for s in
              ("hex", "prism", "tet", "hex", "tri", "quad", "tet")]
    first = nir.partition_elements(blocks, nranks)
    assert first[0] == 0 and first[-1] == sum(b[2] for b in blocks)
    assert all(a <= b for a, b in zip(first, first[1:]))
    cost = np.concatenate([np.full(n, _flops(s, P), dtype=np.float64) for s, P, n in blocks])
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    share = cum[-1] / nranks
    worst = cost.max()
    for r in range(nranks):
        assert abs(cum[first[r + 1]] - cum[first[r]] - share) <= worst + 1e-6 * share, r


def _mesh_parts():
    sys.path.insert(0, ROOT)
    import workloads as W
    return [dict(shape="hex", P=2, Q=4, gorder=2, nodes=W.hex_grid(3, 2, amp=0.05), deformed=True),
            dict(shape="tet", P=3, Q=5, gorder=1, nodes=W.perturb_vertices(W.tet_kuhn(2), 0.1, 0), deformed=False),
            dict(shape="prism", P=2, Q=4, gorder=1, nodes=W.perturb_vertices(W.prism_split(2, 2, 2), 0.1, 1),
                 deformed=False)]


def _pcg(Hblocks, b, dinv, reduce, iters_out, tol=1e-12, max_iter=4000):
    """Jacobi-preconditioned CG in the library's order of operations and
    reductions: start (r.z, r.r); per iteration (p.Ap), then (r.z, r.r) --
    each a partial sum passed through `reduce`.  Records x after every
    iteration in iters_out."""
    def H(v):
        out, o = [], 0
        for h in Hblocks:
            n = h.shape[0] * h.shape[1]
            out.append(np.einsum("eij,ej->ei", h, v[o:o + n].reshape(h.shape[0], h.shape[1])).ravel())
            o += n
        return np.concatenate(out) if out else np.zeros(0)
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz, rr = reduce(np.array([r @ z, r @ r]))
    bb = rr
    it = 0
    while rr > tol * tol * bb and it < max_iter:
        Ap = H(p)
        (pAp,) = reduce(np.array([p @ Ap]))
        a = rz / pAp
        x = x + a * p
        r = r - a * Ap
        z = dinv * r
        rzn, rr = reduce(np.array([r @ z, r @ r]))
        beta = rzn / rz
        rz = rzn
        it += 1
        iters_out.append(x.copy())
        p = z + beta * p
    return x


def _cg_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import oracle
    import workloads as W
    nir = _nir()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = _mesh_parts()
    M = [oracle.num_modes(p["shape"], p["P"]) for p in parts]
    ndof = sum(p["nodes"].shape[0] * m for p, m in zip(parts, M))
    b_full = W.coefficients(1, ndof, seed=5)[0]
    first = nir.partition_elements([(p["shape"], p["P"], p["nodes"].shape[0]) for p in parts], world)
    mine = W.shard_parts(parts, first, rank)
    # this rank's element matrices and dof range (blocks are concatenated in order)
    dof_of_elem = np.concatenate([[0], np.cumsum(np.concatenate([np.full(p["nodes"].shape[0], m)
                                                                 for p, m in zip(parts, M)]))])
    lo, hi = dof_of_elem[first[rank]], dof_of_elem[first[rank + 1]]
    Hb = [oracle.helmholtz_matrix(q["shape"], q["P"], q["Q"], q["gorder"], q["nodes"], 1.0) for q in mine]
    dinv = np.concatenate([1.0 / np.einsum("eii->ei", h).ravel() for h in Hb]) if Hb else np.zeros(0)

    def reduce(v):
        t = torch.from_numpy(v.copy())
        dist.all_reduce(t)
        return t.numpy()

    its = []
    x = _pcg(Hb, b_full[lo:hi], dinv, reduce, its)
    full = np.zeros(ndof)
    full[lo:hi] = x
    t = torch.from_numpy(full)
    dist.all_reduce(t)
    trace = np.zeros((len(its), ndof))
    for k, xi in enumerate(its):
        trace[k, lo:hi] = xi
    tt = torch.from_numpy(trace)
    dist.all_reduce(tt)
    if rank == 0:
        out["x"] = t.numpy().tolist()
        at = [0, 4, 9, 19]
        out["trace"] = tt.numpy()[at].tolist()
        out["trace_at"] = at
        out["iters"] = len(its)
        out["first"] = first
    dist.destroy_process_group()


def test_sharded_cg_recurrence_matches_single_rank():
    """Two gloo ranks, each holding its partitioned element range, run CG with
    the scalars summed over the ranks; the iterates equal the single-rank ones
    up to the rounding of the reduction order, and the solution equals the
    oracle's per-element Cholesky solve."""
    import oracle
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = 29523
    procs = [ctx.Process(target=_cg_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    parts = _mesh_parts()
    Hb = [oracle.helmholtz_matrix(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"], 1.0) for p in parts]
    M = [h.shape[1] for h in Hb]
    sys.path.insert(0, ROOT)
    import workloads as W
    b = W.coefficients(1, sum(h.shape[0] * h.shape[1] for h in Hb), seed=5)[0]
    dinv = np.concatenate([1.0 / np.einsum("eii->ei", h).ravel() for h in Hb])
    its = []
    x1 = _pcg(Hb, b, dinv, lambda v: v, its)
    # rounding differences reach the stopping test: counts may differ slightly
    assert abs(out["iters"] - len(its)) <= max(2, len(its) // 50), (out["iters"], len(its))
    assert 0 < out["first"][1] < out["first"][2]
    for k, got in zip(out["trace_at"], out["trace"]):
        want = its[k]
        # the reduction order changes the rounding of every dot product; CG
        # carries such differences along, and after many iterations (loss of
        # orthogonality) amplifies them, so only early iterates are compared
        # this tightly; the converged solutions are compared below
        assert np.linalg.norm(np.array(got) - want) <= 1e-11 * np.linalg.norm(want), k
    xs = np.array(out["x"])
    assert np.linalg.norm(xs - x1) <= 1e-10 * np.linalg.norm(x1)
    xc, o = [], 0
    for p, h, m in zip(parts, Hb, M):
        n = h.shape[0] * m
        xc.append(oracle.helmholtz_solve(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"], 1.0,
                                         b[o:o + n].reshape(h.shape[0], m)).ravel())
        o += n
    xc = np.concatenate(xc)
    assert np.linalg.norm(xs - xc) <= 1e-10 * np.linalg.norm(xc)
