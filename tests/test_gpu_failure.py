"""Failure detection on the GPU without a fault: the bounded mbarrier wait
that every staged kernel uses runs out on purpose (a barrier nothing arrives
on, no copy in flight, a short cycle limit); the kernel must set the device
error word and return, nir_ctx_check must report NIR_ERR_CUDA once and clear
the word, and the context must stay usable."""
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


def test_bounded_wait_runs_out_and_is_reported(nir):
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    ctx.check()                      # clean to start with
    ctx.selftest_wait(1 << 20)       # ~0.5 ms at 2 GHz
    with pytest.raises(nir.NirError) as ei:
        ctx.check()
    assert ei.value.code == -3       # NIR_ERR_CUDA
    ctx.check()                      # the word was cleared
    # the context still works: a staged FP32 Helmholtz apply after the timeout
    E, P = 64, 3
    nodes = W.hex_grid(4, 2, amp=0.05)[:E]
    blk = nir.Block(ctx, "hex", E, P, deformed=True)
    blk.set_geometry(2, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    x = W.coefficients(E, blk.M, seed=0)
    y = blk.helmholtz(torch.from_numpy(x).cuda().float(), prec="f32").double().cpu().numpy()
    ctx.check()
    ref = oracle.helmholtz("hex", P, P + 2, 2, nodes, 1.0, x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5


def test_selftest_argument_checks(nir):
    ctx = nir.Context(0)
    L = nir.lib()
    assert L.nir_ctx_selftest_wait(ctx.h, 0) == -1
    assert L.nir_ctx_selftest_wait(ctx.h, (1 << 31) + 1) == -1
    assert L.nir_ctx_selftest_wait(None, 100) == -1


def test_fp64_tensor_core_probe(nir):
    """The DMMA probe returns a finite positive rate next to the DFMA one (the
    comparison is recorded by the benchmark, not asserted here)."""
    ctx = nir.Context(0)
    dmma, dfma = ctx.probe_fp64_mma_peak(), ctx.probe_fp64_peak()
    assert np.isfinite(dmma) and dmma > 0 and np.isfinite(dfma) and dfma > 0


def small_hex_block(nir, ctx, E=64, P=3):
    nodes = W.hex_grid(4, 2, amp=0.05)[:E]
    blk = nir.Block(ctx, "hex", E, P, deformed=True)
    blk.set_geometry(2, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    return nodes, blk


def test_debug_mode_reports_at_the_failing_call(nir):
    """With debug mode on, the operator call after the timed-out wait raises
    NIR_ERR_CUDA itself (the word is read and cleared there); the next call
    succeeds and matches the oracle; off, the same call returns normally and
    only the later check() reports."""
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    ctx.debug = True
    assert ctx.debug
    nodes, blk = small_hex_block(nir, ctx)
    x = W.coefficients(blk.nelem, blk.M, seed=1)
    xt = torch.from_numpy(x).cuda()
    ctx.selftest_wait(1 << 20)
    with pytest.raises(nir.NirError) as ei:
        blk.helmholtz(xt, prec="f64")
    assert ei.value.code == -3
    y = blk.helmholtz(xt, prec="f64").cpu().numpy()
    ctx.check()
    ref = oracle.helmholtz("hex", 3, 5, 2, nodes, 1.0, x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-12
    ctx.debug = False
    ctx.selftest_wait(1 << 20)
    blk.helmholtz(xt, prec="f64")          # returns: the failure is not looked for here
    with pytest.raises(nir.NirError):
        ctx.check()
    ctx.check()


def test_debug_mode_does_not_change_results(nir):
    """Every operator and the mesh apply (graph-replayed) give the same bits
    with debug mode on and off; a CG solve the same solution."""
    import tests.test_gpu_ops as T
    ctx = nir.Context(0)
    nodes, blk = small_hex_block(nir, ctx)
    tet_nodes = np.ascontiguousarray(W.perturb_vertices(W.tet_kuhn(2), 0.1, 2))
    tet = nir.Block(ctx, "tet", tet_nodes.shape[0], 4)
    tet.set_geometry(1, torch.from_numpy(tet_nodes).cuda())
    mesh = nir.Mesh(ctx, [blk, tet])
    xm = torch.from_numpy(W.coefficients(1, mesh.ndof, seed=2)[0]).cuda()
    res = {}
    for dbg in (False, True):
        ctx.debug = dbg
        outs = [T.run_op(blk, op, prec, T.inputs(blk, op, seed=3), 0.7) for op in T.OPS for prec in ("f64", "f32")]
        ym = mesh.helmholtz(xm).clone()
        x = torch.zeros_like(xm)
        rc, st = mesh.cg_solve(xm, x, inner_prec="f32", tol=1e-10, max_outer=40, max_inner=5000, inner_tol=1e-3)
        assert rc == 0, st
        res[dbg] = (outs, ym, x)
    for a, b in zip(res[False][0], res[True][0]):
        assert np.array_equal(a, b)
    assert torch.equal(res[False][1], res[True][1])
    xf, xt = res[False][2], res[True][2]
    assert float((xf - xt).norm() / xf.norm()) <= 1e-12


def test_debug_mode_from_environment(nir, monkeypatch):
    monkeypatch.setenv("NIR_DEBUG", "1")
    assert nir.Context(0).debug
    monkeypatch.setenv("NIR_DEBUG", "0")
    assert not nir.Context(0).debug
    monkeypatch.delenv("NIR_DEBUG")
    assert not nir.Context(0).debug
    ctx = nir.Context(0)
    L = nir.lib()
    assert L.nir_ctx_set_debug(ctx.h, 2) == -1
    assert L.nir_ctx_set_debug(None, 1) == -1
    assert L.nir_ctx_get_debug(ctx.h, None) == -1
