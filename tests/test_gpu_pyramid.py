"""GPU parity of the pyramid (the shape the paper motivates for hybrid meshes
and leaves to future work) against the pinned FP64 oracle.

  * every operator x P = 1..9 in FP64 on affine pyramids (affinely distorted
    cells of a split grid) and on non-affine ones (base vertex moved off the
    parallelogram: the rational vertex map), element counts spanning several
    CTAs plus a ragged tail, E = 1;
  * FP32 / BF16 within their tolerances; every Helmholtz launch variant; the
    threading-over-elements variant refused (UNSUPPORTED);
  * a mixed hex / tet / pyramid mesh in both launch forms; a CG solve on a
    pyramid mesh to 1e-10 against the oracle's Cholesky; geometry given as
    geometric factors; a 48 000-element mesh sampled.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_ops import OPS, TOL, inputs, oracle_op, per_elem_rel, rel, run_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def pyr_mesh(E, affine=True, seed=0):
    n = int(np.ceil((E / 6) ** (1 / 3))) + 1
    nodes = W.perturb_vertices(W.pyramid_split(n, n, n)[:E], 0.1, seed)
    if not affine:   # move each base's third vertex off the parallelogram
        rng = np.random.default_rng(seed + 100)
        h = 1.0 / n
        nodes = nodes.copy()
        nodes[:, 2, :] += 0.08 * h * rng.uniform(-1, 1, (E, 3))
    return np.ascontiguousarray(nodes)


def block(nir, ctx, E, P, affine=True, seed=0):
    nodes = pyr_mesh(E, affine, seed)
    blk = nir.Block(ctx, "pyr", E, P)
    blk.set_geometry(1, torch.from_numpy(nodes).cuda())
    assert blk.M == oracle.num_modes("pyr", P) and blk.NQ == oracle.num_points("pyr", P + 2)
    return nodes, blk


@pytest.mark.parametrize("affine", [True, False])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_fp64_all_ops(nir, ctx, P, affine):
    E = 37 if P <= 4 else 13
    nodes, blk = block(nir, ctx, E, P, affine, seed=P)
    for op in OPS:
        x = inputs(blk, op, seed=P)
        got = run_op(blk, op, "f64", x, 1.3)
        ref = oracle_op("pyr", P, 1, nodes, op, x, 1.3)
        assert got.shape == ref.shape, op
        assert rel(got, ref) <= TOL["f64"], (op, rel(got, ref))
        assert per_elem_rel(got, ref) <= 1e-11, (op, per_elem_rel(got, ref))


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("P", [1, 4, 8, 9])
def test_low_precision_all_ops(nir, ctx, prec, P):
    nodes, blk = block(nir, ctx, 41, P, affine=(P % 2 == 0), seed=3)
    for op in OPS:
        x = inputs(blk, op, seed=5)
        got = run_op(blk, op, prec, x, 0.9)
        ref = oracle_op("pyr", P, 1, nodes, op, x, 0.9)
        assert rel(got, ref) <= TOL[prec], (op, prec, rel(got, ref))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("P", [2, 4, 6])
def test_helmholtz_launch_variants_and_single_element(nir, ctx, prec, P):
    nodes, blk = block(nir, ctx, 70, P, seed=7)
    x = W.coefficients(70, blk.M, seed=2)
    ref = oracle_op("pyr", P, 1, nodes, "helm", x, 1.0)
    outs = []
    for v in (0, 1, 2, 3):
        blk.set_tuning(prec, v, 0, 0)
        y = run_op(blk, "helm", prec, x, 1.0)
        assert rel(y, ref) <= TOL[prec], (v, rel(y, ref))
        outs.append(y)
    if prec == "f64":
        for y in outs[1:]:
            assert np.array_equal(y, outs[0])   # every variant runs the same arithmetic
    with pytest.raises(nir.NirError) as ei:     # no threading-over-elements kernel for pyramids
        blk.set_tuning(prec, 4, 0, 0)
    assert ei.value.code == -2
    one_nodes, one = block(nir, ctx, 1, P, affine=False, seed=9)
    x1 = W.coefficients(1, one.M, seed=4)
    assert rel(run_op(one, "helm", prec, x1, 1.0), oracle_op("pyr", P, 1, one_nodes, "helm", x1, 1.0)) <= TOL[prec]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_mixed_mesh_with_pyramids(nir, ctx, prec, tol):
    parts = [dict(shape="pyr", P=3, Q=5, gorder=1, nodes=pyr_mesh(60, seed=1), deformed=False),
             dict(shape="hex", P=3, Q=5, gorder=2, nodes=W.hex_grid(3, 2, amp=0.05)[:20], deformed=True),
             dict(shape="tet", P=4, Q=6, gorder=1, nodes=W.perturb_vertices(W.tet_kuhn(2), 0.1, 2), deformed=False),
             dict(shape="pyr", P=6, Q=8, gorder=1, nodes=pyr_mesh(17, affine=False, seed=2), deformed=False)]
    blocks = []
    for p in parts:
        b = nir.Block(ctx, p["shape"], p["nodes"].shape[0], p["P"], deformed=p["deformed"])
        b.set_geometry(p["gorder"], torch.from_numpy(np.ascontiguousarray(p["nodes"])).cuda())
        blocks.append(b)
    mesh = nir.Mesh(ctx, blocks)
    x64 = W.coefficients(1, mesh.ndof, seed=6)[0]
    x = torch.from_numpy(x64).cuda().to(nir.DTYPE[prec])
    mesh.set_launch(prec, "persistent")
    y0 = mesh.helmholtz(x, prec=prec).clone()
    mesh.set_launch(prec, "blocks")
    assert torch.equal(y0, mesh.helmholtz(x, prec=prec))
    y = y0.double().cpu().numpy()
    for b, o, p in zip(blocks, mesh.offsets, parts):
        n = b.nelem * b.M
        ref = oracle.helmholtz(p["shape"], p["P"], p["Q"], p["gorder"], p["nodes"], 1.0,
                               x64[o:o + n].reshape(b.nelem, b.M))
        assert rel(y[o:o + n].reshape(b.nelem, b.M), ref) <= tol, (p["shape"], p["P"])


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_cg_solve_on_pyramids(nir, ctx, inner):
    nodes, blk = block(nir, ctx, 48, 4, affine=False, seed=11)
    mesh = nir.Mesh(ctx, [blk])
    b = W.coefficients(48, blk.M, seed=12)
    bt = torch.from_numpy(b.ravel()).cuda()
    x = torch.zeros_like(bt)
    rc, st = mesh.cg_solve(bt, x, inner_prec=inner, tol=1e-10, fwd_tol=1e-10, max_outer=60, max_inner=20000,
                           inner_tol=1e-3)
    assert rc == 0, st
    xr = oracle.helmholtz_solve("pyr", 4, 6, 1, nodes, 1.0, b)
    assert rel(x.cpu().numpy(), xr.ravel()) <= 1e-10


def test_geometric_factor_input(nir, ctx):
    P = 3
    nodes = pyr_mesh(30, affine=False, seed=13)
    Wq, Lam, _ = oracle.geom_factors("pyr", P + 2, 1, nodes)
    _, _, w = oracle.ref_points("pyr", P + 2)
    blk = nir.Block(ctx, "pyr", 30, P)
    blk.set_geometric_factors(torch.from_numpy(Lam).cuda(), torch.from_numpy(Wq / w[None]).cuda())
    for op in OPS:
        x = inputs(blk, op, seed=1)
        got = run_op(blk, op, "f64", x, 1.0)
        assert rel(got, oracle_op("pyr", P, 1, nodes, op, x, 1.0)) <= TOL["f64"], op


def test_full_pyramid_mesh_sampled(nir, ctx):
    """20^3 cells split into 6 pyramids each (48 000 elements, P = 4), tuned;
    the oracle recomputes a seeded sample of elements."""
    nodes = W.pyramid_split(20, 20, 20)
    E = nodes.shape[0]
    blk = nir.Block(ctx, "pyr", E, 4)
    blk.set_geometry(1, torch.from_numpy(nodes).cuda())
    nir.Mesh(ctx, [blk]).tune(None)
    x64 = W.coefficients(E, blk.M, seed=0)
    ids = W.sample_elements(E, 24, seed=3)
    ref = oracle.helmholtz("pyr", 4, 6, 1, nodes[ids], 1.0, x64[ids])
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        y = blk.helmholtz(torch.from_numpy(x64).cuda().to(nir.DTYPE[prec]), prec=prec).double().cpu().numpy()
        assert rel(y[ids], ref) <= tol, prec
