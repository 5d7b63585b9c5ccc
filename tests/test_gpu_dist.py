"""GPU tests of the sharded solve (nir_cg_solve_dist): a mesh split into
contiguous cost-balanced element ranges (nir_partition_elements), each rank
solving on its own elements with the CG's FP64 scalars summed over the ranks
by a caller-given reduction.

On one GPU the ranks are host threads, each with its own context, stream and
blocks; their kernels never wait on one another (only the host reduction
joins them, with a timeout).  Results must equal the single-rank solve up to
the rounding of the reduction order and the oracle's per-element Cholesky
solution to 1e-10."""
import threading

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
FWD = 1e-10


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


def parts_small():
    return [dict(shape="hex", P=3, Q=5, gorder=2, nodes=W.hex_grid(5, 2, amp=0.05), deformed=True),
            dict(shape="prism", P=2, Q=4, gorder=1, nodes=W.perturb_vertices(W.prism_split(4, 4, 3), 0.1, 1),
                 deformed=False),
            dict(shape="tet", P=4, Q=6, gorder=1, nodes=W.perturb_vertices(W.tet_kuhn(3), 0.1, 0), deformed=False)]


def make_mesh(nir, ctx, parts):
    blocks = []
    for p in parts:
        b = nir.Block(ctx, p["shape"], p["nodes"].shape[0], p["P"], deformed=p["deformed"])
        b.set_geometry(p["gorder"], torch.from_numpy(np.ascontiguousarray(p["nodes"])).cuda())
        blocks.append(b)
    return nir.Mesh(ctx, blocks), blocks


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_solution(parts, b):
    out, o = [], 0
    for p in parts:
        M = oracle.num_modes(p["shape"], p["P"])
        n = p["nodes"].shape[0] * M
        out.append(oracle.helmholtz_solve(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"], 1.0,
                                          b[o:o + n].reshape(-1, M)).ravel())
        o += n
    return np.concatenate(out)


KW = dict(tol=1e-10, fwd_tol=FWD, max_outer=60, max_inner=20000, inner_tol=1e-3)


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_one_rank_reduction_matches_plain_solve(nir, inner):
    """With one rank (an identity reduction) the deferred-scalar iterations
    compute exactly what the captured iterations do."""
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    parts = parts_small()
    mesh, _ = make_mesh(nir, ctx, parts)
    b = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=3)[0]).cuda()
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    calls = []
    rc0, s0 = mesh.cg_solve(b, x0, inner_prec=inner, **KW)
    rc1, s1 = mesh.cg_solve(b, x1, inner_prec=inner, allreduce=lambda v: calls.append(len(v)), **KW)
    assert rc0 == 0 and rc1 == 0, (s0, s1)
    assert s1["inner_total"] == s0["inner_total"] and s1["outer"] == s0["outer"]
    assert rel(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-13
    assert calls.count(1) >= s1["inner_total"]       # one p.Ap reduction per iteration
    assert rel(x1.cpu().numpy(), oracle_solution(parts, b.cpu().numpy())) <= FWD


class ThreadSum:
    """Sum over `n` host threads in rank order (the same bits on every rank);
    a broken or timed-out barrier raises, which the library reports as COMM."""

    def __init__(self, n):
        self.bar = threading.Barrier(n, timeout=120)
        self.buf = [None] * n

    def rank(self, r):
        def f(v):
            self.buf[r] = v.copy()
            self.bar.wait()
            tot = self.buf[0].copy()
            for k in range(1, len(self.buf)):
                tot += self.buf[k]
            self.bar.wait()
            v[:] = tot
        return f


@pytest.mark.parametrize("nranks,inner", [(2, "f32"), (3, "f64")])
def test_sharded_solve_matches_single_rank_and_oracle(nir, nranks, inner):
    torch.cuda.set_device(0)
    parts = parts_small()
    ndof_of = [p["nodes"].shape[0] * oracle.num_modes(p["shape"], p["P"]) for p in parts]
    b = W.coefficients(1, sum(ndof_of), seed=8)[0]
    first = nir.partition_elements([(p["shape"], p["P"], p["nodes"].shape[0]) for p in parts], nranks)
    # global dof offset of every element
    M_of = np.concatenate([np.full(p["nodes"].shape[0], oracle.num_modes(p["shape"], p["P"])) for p in parts])
    dof0 = np.concatenate([[0], np.cumsum(M_of)])
    red = ThreadSum(nranks)
    res = [None] * nranks

    def rank_main(r):
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        ctx = nir.Context(0, st)
        mine = W.shard_parts(parts, first, r)
        mesh, _ = make_mesh(nir, ctx, mine)
        lo, hi = dof0[first[r]], dof0[first[r + 1]]
        with torch.cuda.stream(st):
            bl = torch.from_numpy(b[lo:hi].copy()).cuda()
            x = torch.zeros_like(bl)
        rc, s = mesh.cg_solve(bl, x, inner_prec=inner, allreduce=red.rank(r), **KW)
        st.synchronize()
        res[r] = (rc, s, x.cpu().numpy())

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(nranks)]
    for t in th:
        t.start()
    for t in th:
        t.join(600)
    assert all(r is not None for r in res)
    for rc, s, _ in res:
        assert rc == 0, s
    # every rank ran the same sweeps and iterations (same reduced scalars)
    assert len({(s["outer"], s["inner_total"]) for _, s, _ in res}) == 1
    xs = np.concatenate([x for _, _, x in res])
    ctx = nir.Context(0)
    mesh, _ = make_mesh(nir, ctx, parts)
    bt = torch.from_numpy(b).cuda()
    x1 = torch.zeros_like(bt)
    rc, s1 = mesh.cg_solve(bt, x1, inner_prec=inner, **KW)
    assert rc == 0
    assert rel(xs, x1.cpu().numpy()) <= 1e-9
    assert rel(xs, oracle_solution(parts, b)) <= FWD


def test_failing_reduction_is_reported(nir):
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    mesh, _ = make_mesh(nir, ctx, parts_small()[:1])
    b = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=1)[0]).cuda()

    def bad(v):
        raise RuntimeError("peer lost")
    rc, _ = mesh.cg_solve(b, torch.zeros_like(b), inner_prec="f32", allreduce=bad, **KW)
    assert rc == -10
    # the mesh still solves afterwards
    rc, s = mesh.cg_solve(b, torch.zeros_like(b), inner_prec="f32", **KW)
    assert rc == 0, s
