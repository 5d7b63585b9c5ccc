"""GPU tests of the hybrid mesh (one persistent launch, CUDA graphs,
autotuner) and of the conjugate-gradient Helmholtz solve with FP64 iterative
refinement, against the FP64 oracle (per-element operator and dense Cholesky)."""
import ctypes as C
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def build_mesh(nir, ctx, parts):
    blocks = []
    for p in parts:
        b = nir.Block(ctx, p["shape"], p["nodes"].shape[0], p["P"], deformed=p["deformed"])
        b.set_geometry(p["gorder"], torch.from_numpy(np.ascontiguousarray(p["nodes"])).cuda())
        blocks.append(b)
    return nir.Mesh(ctx, blocks), blocks


def small_hybrid():
    return W.hybrid_mesh(seed=0, scale=20)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_mesh_apply_matches_blocks_and_oracle(nir, ctx, prec, tol):
    parts = small_hybrid()
    mesh, blocks = build_mesh(nir, ctx, parts)
    x64 = W.coefficients(1, mesh.ndof, seed=4)[0]
    x = torch.from_numpy(x64).cuda().to(nir.DTYPE[prec])
    y = mesh.helmholtz(x, lam=1.0, prec=prec).double().cpu().numpy()
    for b, o, p in zip(blocks, mesh.offsets, parts):
        n = b.nelem * b.M
        xb = x[o:o + n].view(b.nelem, b.M).contiguous()
        yb = b.helmholtz(xb, lam=1.0, prec=prec).double().cpu().numpy().ravel()
        # the persistent kernel runs the same element-group code as the block kernel
        assert np.array_equal(y[o:o + n], yb), (p["shape"], p["P"])
        ids = W.sample_elements(b.nelem, 8, seed=p["P"])
        ref = oracle.helmholtz(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"][ids], 1.0,
                               x64[o:o + n].reshape(b.nelem, b.M)[ids])
        assert rel(y[o:o + n].reshape(b.nelem, b.M)[ids], ref) <= tol, (p["shape"], p["P"])


def test_mesh_graph_replay_and_buffers(nir, ctx):
    parts = small_hybrid()
    mesh, blocks = build_mesh(nir, ctx, parts)
    out = torch.empty(mesh.ndof, dtype=torch.float64, device="cuda")
    xa = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=1)[0]).cuda()
    xb = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=2)[0]).cuda()
    ya = mesh.helmholtz(xa, out=out).clone()
    xa.copy_(xb)  # same buffer, new data: the replayed graph must read it
    yb = mesh.helmholtz(xa, out=out).clone()
    yc = mesh.helmholtz(xb)  # different buffers: another graph
    assert not torch.equal(ya, yb)
    assert torch.equal(yb, yc)


def test_tune_and_cache(nir, ctx, tmp_path):
    parts = small_hybrid()
    mesh, blocks = build_mesh(nir, ctx, parts)
    x = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=3)[0]).cuda()
    before = mesh.helmholtz(x).clone()
    cache = str(tmp_path / "tune.json")
    mesh.tune(cache)
    after = mesh.helmholtz(x)
    assert torch.equal(before, after)
    kv = json.load(open(cache))
    assert any("|mesh|" in k for k in kv) and any("|block|" in k for k in kv)
    mesh.tune(cache)  # second call reads the cache
    assert torch.equal(mesh.helmholtz(x), before)


def test_tune_cache_named_by_environment(nir, ctx, tmp_path, monkeypatch):
    """With no cache path given, the tuner uses the file NIR_TUNE_CACHE names."""
    mesh, _ = build_mesh(nir, ctx, small_hybrid())
    cache = tmp_path / "env_tune.json"
    monkeypatch.setenv("NIR_TUNE_CACHE", str(cache))
    mesh.tune(None)
    kv = json.load(open(cache))
    assert any("|mesh|" in k for k in kv)
    stamp = cache.stat().st_mtime_ns
    mesh.tune("")                      # an empty path falls back to the environment too
    assert json.load(open(cache)) == kv and cache.stat().st_mtime_ns >= stamp


def hex_problem(nir, ctx, n=4, P=3, amp=0.05):
    nodes = W.hex_grid(n, 2, amp=amp)
    parts = [dict(shape="hex", P=P, Q=P + 2, gorder=2, nodes=nodes, deformed=True)]
    mesh, blocks = build_mesh(nir, ctx, parts)
    b = W.coefficients(nodes.shape[0], blocks[0].M, seed=7)
    x_ref = oracle.helmholtz_solve("hex", P, P + 2, 2, nodes, 1.0, b)
    return mesh, nodes, b, x_ref


# The solve's accuracy target: 1e-10 relative error of the final solution
# against the oracle's (per-element dense Cholesky of the broken operator).
FWD = 1e-10


@pytest.mark.parametrize("jacobi", [True, False])
def test_fp64_cg_matches_dense_cholesky(nir, ctx, jacobi):
    mesh, nodes, b, x_ref = hex_problem(nir, ctx)
    bt = torch.from_numpy(b.ravel()).cuda()
    x = torch.zeros_like(bt)
    rc, st = mesh.cg_solve(bt, x, inner_prec="f64", tol=1e-10, fwd_tol=FWD, max_inner=20000, jacobi=jacobi)
    assert rc == 0, st
    assert st["rel_residual"] <= 1e-10 and st["rel_correction"] <= FWD, st
    assert rel(x.cpu().numpy(), x_ref.ravel()) <= FWD


@pytest.mark.parametrize("vectors", ["f64", "f32"])
@pytest.mark.parametrize("inner", ["f32", "bf16"])
def test_mixed_refinement_reaches_fp64_accuracy(nir, ctx, inner, vectors):
    mesh, nodes, b, x_ref = hex_problem(nir, ctx)
    bt = torch.from_numpy(b.ravel()).cuda()
    x = torch.zeros_like(bt)
    rc, st = mesh.cg_solve(bt, x, inner_prec=inner, inner_vectors=vectors, tol=1e-10, fwd_tol=FWD, max_outer=60,
                           max_inner=5000, inner_tol=1e-3)
    if inner == "f32":
        assert rc == 0, st
    if rc == 0:
        assert st["rel_residual"] <= 1e-10 and st["rel_correction"] <= FWD, st
        assert rel(x.cpu().numpy(), x_ref.ravel()) <= FWD, (rel(x.cpu().numpy(), x_ref.ravel()), st)
    else:
        assert rc == -4, (rc, st)   # refinement stalls: reported, not hidden


def test_forward_criterion_adds_sweeps(nir, ctx):
    """The residual alone can stop refinement while the correction is still
    large; fwd_tol keeps refining until the correction meets it."""
    mesh, nodes, b, x_ref = hex_problem(nir, ctx)
    bt = torch.from_numpy(b.ravel()).cuda()
    x1, x2 = torch.zeros_like(bt), torch.zeros_like(bt)
    rc1, st1 = mesh.cg_solve(bt, x1, inner_prec="f32", tol=1e-6, max_outer=60, max_inner=5000, inner_tol=1e-3)
    rc2, st2 = mesh.cg_solve(bt, x2, inner_prec="f32", tol=1e-6, fwd_tol=FWD, max_outer=60, max_inner=5000,
                             inner_tol=1e-3)
    assert rc1 == 0 and rc2 == 0, (st1, st2)
    assert st2["outer"] > st1["outer"] and st2["rel_correction"] <= FWD
    assert rel(x2.cpu().numpy(), x_ref.ravel()) <= FWD < rel(x1.cpu().numpy(), x_ref.ravel())


def test_cg_options_rejected(nir, ctx):
    mesh, nodes, b, x_ref = hex_problem(nir, ctx, n=2, P=2)
    bt = torch.from_numpy(b.ravel()).cuda()
    x = torch.zeros_like(bt)
    L = nir.lib()
    for kw in (dict(inner_vectors="bf16"), dict(fwd_tol=-1.0), dict(fwd_tol=float("nan"))):
        o = nir._cg_opts(**{**dict(inner_prec="f32", tol=1e-10, max_outer=10, max_inner=100, inner_tol=1e-3,
                                   jacobi=1, inner_vectors="f64", fwd_tol=0.0), **kw})
        s = nir.CGStats()
        assert L.nir_cg_solve(mesh.h, 1.0, C.c_void_p(bt.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(o),
                              C.byref(s)) == -1, kw


def test_cg_on_hybrid_mesh(nir, ctx):
    parts = small_hybrid()
    mesh, blocks = build_mesh(nir, ctx, parts)
    b = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=9)[0]).cuda()
    x = torch.zeros_like(b)
    rc, st = mesh.cg_solve(b, x, inner_prec="f32", tol=1e-10, fwd_tol=FWD, max_outer=60, max_inner=5000,
                           inner_tol=1e-3)
    assert rc == 0 and st["rel_residual"] <= 1e-10, st
    # check against the per-element dense solve on a few elements of every block
    xh = x.cpu().numpy()
    bh = b.cpu().numpy()
    for blk, o, p in zip(blocks, mesh.offsets, parts):
        ids = W.sample_elements(blk.nelem, 3, seed=1)
        n = blk.nelem * blk.M
        xr = oracle.helmholtz_solve(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"][ids], 1.0,
                                    bh[o:o + n].reshape(blk.nelem, blk.M)[ids])
        assert rel(xh[o:o + n].reshape(blk.nelem, blk.M)[ids], xr) <= FWD, (p["shape"], p["P"])


def test_cg_failure_reporting(nir, ctx):
    mesh, nodes, b, x_ref = hex_problem(nir, ctx, n=2, P=2)
    bt = torch.from_numpy(b.ravel()).cuda()
    x = torch.zeros_like(bt)
    rc, st = mesh.cg_solve(bt, x, inner_prec="f64", tol=1e-12, max_inner=3)
    assert rc == -4 and st["inner_total"] <= 25  # iteration cap -> NOT_CONVERGED
    bad = bt.clone()
    bad[5] = float("nan")
    rc, st = mesh.cg_solve(bad, torch.zeros_like(bt), inner_prec="f32")
    assert rc == -5  # NaN input -> NONFINITE
    with pytest.raises(ValueError):
        mesh.cg_solve(bt.float(), x)
    rc, _ = mesh.cg_solve(bt, x, lam=-1.0)
    assert rc == -1


def test_graphs_follow_retuning_and_new_geometry(nir, ctx):
    """Captured graphs (mesh applies and CG chunks) are rebuilt when the work
    list is re-tuned or a block's geometry is set again."""
    mesh, nodes, b, x_ref = hex_problem(nir, ctx, n=3, P=2)
    bt = torch.from_numpy(b.ravel()).cuda()
    x1 = torch.zeros_like(bt)
    rc, _ = mesh.cg_solve(bt, x1, inner_prec="f32", tol=1e-10, max_outer=60, max_inner=5000)
    assert rc == 0
    mesh.tune(None)
    x2 = torch.zeros_like(bt)
    rc, _ = mesh.cg_solve(bt, x2, inner_prec="f32", tol=1e-10, max_outer=60, max_inner=5000)
    assert rc == 0
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-8
    # move the geometry: the next apply must use the new factors
    blk = mesh.blocks[0]
    y_old = mesh.helmholtz(bt).cpu().numpy()
    moved = W.hex_grid(3, 2, amp=0.02)
    blk.set_geometry(2, torch.from_numpy(moved).cuda())
    y_new = mesh.helmholtz(bt).cpu().numpy()
    ref = oracle.helmholtz("hex", 2, 4, 2, moved, 1.0, b)
    assert rel(y_new, ref.ravel()) <= 1e-12
    assert rel(y_old, ref.ravel()) > 1e-6


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_launch_forms_agree(nir, ctx, prec):
    """The persistent queue and the sequence of block kernels run the same
    per-element code: identical results, also inside CG."""
    parts = small_hybrid()
    mesh, blocks = build_mesh(nir, ctx, parts)
    assert mesh.get_launch(prec) == "persistent"
    x = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=6)[0]).cuda().to(nir.DTYPE[prec])
    y0 = mesh.helmholtz(x, prec=prec).clone()
    mesh.set_launch(prec, "blocks")
    assert mesh.get_launch(prec) == "blocks"
    y1 = mesh.helmholtz(x, prec=prec)
    assert torch.equal(y0, y1)
    if prec == "f32":
        b = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=7)[0]).cuda()
        xs = []
        for form in ("persistent", "blocks"):
            mesh.set_launch("f32", form)
            mesh.set_launch("f64", form)
            xx = torch.zeros_like(b)
            rc, st = mesh.cg_solve(b, xx, inner_prec="f32", tol=1e-10, max_outer=60, max_inner=5000)
            assert rc == 0, st
            xs.append(xx)
        assert torch.equal(xs[0], xs[1])
    assert nir.lib().nir_mesh_set_launch(mesh.h, nir.PREC[prec], 7) == -1  # INVALID_ARG


def test_full_hybrid_mesh_sampled(nir, ctx):
    """The ~150k-element hybrid mesh in one persistent launch (tuned, as the
    benchmark runs it); the oracle recomputes two elements of every block."""
    parts = W.hybrid_mesh(seed=0)
    mesh, blocks = build_mesh(nir, ctx, parts)
    mesh.tune(None)
    x64 = W.coefficients(1, mesh.ndof, seed=0)[0]
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        y = mesh.helmholtz(torch.from_numpy(x64).cuda().to(nir.DTYPE[prec]), prec=prec).double().cpu().numpy()
        for b, o, p in zip(blocks, mesh.offsets, parts):
            n = b.nelem * b.M
            ids = W.sample_elements(b.nelem, 2, seed=p["P"])
            ref = oracle.helmholtz(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"][ids], 1.0,
                                   x64[o:o + n].reshape(b.nelem, b.M)[ids])
            assert rel(y[o:o + n].reshape(b.nelem, b.M)[ids], ref) <= tol, (prec, p["shape"], p["P"])


@pytest.mark.parametrize("inner,vectors", [("f32", "f64"), ("f32", "f32"), ("f64", "f64")])
def test_full_p6_solve_sampled(nir, ctx, inner, vectors):
    """Solve of the full 48^3 P6 curved mesh (110 592 elements, 37.9 M DOF) to
    relative residual 1e-10 and forward tolerance 1e-10: FP32 operator inside FP64
    refinement with FP64 or FP32 inner vectors, and plain FP64 CG.  The broken
    operator is block diagonal, so each element's exact solution is the
    oracle's dense per-element Cholesky solve; the sampled elements must match
    it to 1e-10."""
    wl = W.workload("hex48_curved_p6")
    nodes = wl["nodes"]
    E = nodes.shape[0]
    blk = nir.Block(ctx, "hex", E, 6, deformed=True)
    blk.set_geometry(6, torch.from_numpy(nodes).cuda())
    mesh = nir.Mesh(ctx, [blk])
    b = W.coefficients(E, blk.M, seed=3)
    bt = torch.from_numpy(b.ravel()).cuda()
    x = torch.zeros_like(bt)
    rc, st = mesh.cg_solve(bt, x, inner_prec=inner, inner_vectors=vectors, tol=1e-10, fwd_tol=FWD, max_outer=60,
                           max_inner=20000, inner_tol=1e-3)
    assert rc == 0 and st["rel_residual"] <= 1e-10 and st["rel_correction"] <= FWD, st
    ids = W.sample_elements(E, 6, seed=4)
    xr = oracle.helmholtz_solve("hex", 6, 8, 6, nodes[ids], 1.0, b[ids])
    xs = x.cpu().numpy().reshape(E, blk.M)[ids]
    assert rel(xs, xr) <= FWD, (rel(xs, xr), st)
    for i in range(len(ids)):
        assert rel(xs[i], xr[i]) <= FWD, (i, rel(xs[i], xr[i]))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_mesh_with_p9_blocks(nir, ctx, prec, tol):
    """P = 9 (the top order of the paper's GPU study) in the persistent mesh
    kernel and in the block-kernel launch form: the same bits, and the oracle."""
    parts = [dict(shape="hex", P=9, Q=11, gorder=2, nodes=W.hex_grid(2, 2, amp=0.05)[:7], deformed=True),
             dict(shape="prism", P=9, Q=11, gorder=1, nodes=W.perturb_vertices(W.prism_split(2, 2, 2), 0.1, 3)[:5],
                  deformed=False),
             dict(shape="tet", P=9, Q=11, gorder=1, nodes=W.perturb_vertices(W.tet_kuhn(2), 0.1, 4)[:13],
                  deformed=False),
             dict(shape="hex", P=2, Q=4, gorder=2, nodes=W.hex_grid(3, 2, amp=0.05)[:20], deformed=True)]
    mesh, blocks = build_mesh(nir, ctx, parts)
    x64 = W.coefficients(1, mesh.ndof, seed=9)[0]
    x = torch.from_numpy(x64).cuda().to(nir.DTYPE[prec])
    mesh.set_launch(prec, "persistent")
    y0 = mesh.helmholtz(x, prec=prec).clone()
    mesh.set_launch(prec, "blocks")
    y1 = mesh.helmholtz(x, prec=prec)
    assert torch.equal(y0, y1)
    y = y0.double().cpu().numpy()
    for b, o, p in zip(blocks, mesh.offsets, parts):
        n = b.nelem * b.M
        ref = oracle.helmholtz(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"], 1.0,
                               x64[o:o + n].reshape(b.nelem, b.M))
        assert rel(y[o:o + n].reshape(b.nelem, b.M), ref) <= tol, (p["shape"], p["P"])
