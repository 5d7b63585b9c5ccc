"""GPU tests of nir_block_set_geometric_factors: geometry given as the
geometric factors of the problem statement (Sec. 2.1: d xi/d x and |J| per
point, or per element for affine maps) instead of element maps.

The factors fed in are the oracle's own (orc_geom_factors: Lambda = d xi/d x
and W = w |J|, so |J| = W / w), so every operator must match the oracle as
tightly as with the library's own geometry path, and match that path."""
import numpy as np
import pytest
import torch

import oracle
from tests.test_gpu_ops import OPS, TOL, inputs, make_mesh, oracle_op, per_elem_rel, rel, run_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def oracle_factors(shape, P, g, nodes):
    """(dxi_dx [E][Nq][d][d], |J| [E][Nq]) from the oracle."""
    Q = P + 2
    Wq, Lam, _ = oracle.geom_factors(shape, Q, g, nodes)
    _, _, w = oracle.ref_points(shape, Q)
    return Lam, Wq / w[None, :]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape", ["quad", "tri", "hex", "prism", "tet"])
@pytest.mark.parametrize("P", [2, 5])
def test_factors_per_point_match_oracle_and_map_path(nir, ctx, shape, P):
    deformed = shape in ("hex", "quad")
    E = 150 if shape in ("quad", "tri") else 37
    g, nodes = make_mesh(shape, E, deformed)
    Lam, jac = oracle_factors(shape, P, g, nodes)
    blk_f = nir.Block(ctx, shape, E, P, deformed=deformed)
    blk_f.set_geometric_factors(dev(Lam), dev(jac))
    blk_m = nir.Block(ctx, shape, E, P, deformed=deformed)
    blk_m.set_geometry(g, dev(nodes))
    for op in OPS:
        x = inputs(blk_f, op, seed=2)
        got = run_op(blk_f, op, "f64", x, 1.1)
        ref = oracle_op(shape, P, g, nodes, op, x, 1.1)
        assert rel(got, ref) <= TOL["f64"], (op, rel(got, ref))
        assert per_elem_rel(got, ref) <= 1e-11, (op, per_elem_rel(got, ref))
        via_map = run_op(blk_m, op, "f64", x, 1.1)
        assert rel(got, via_map) <= 1e-13, (op, rel(got, via_map))
    # the derived FP32 factors serve a single FP32 apply within its tolerance
    x = inputs(blk_f, "helm", seed=4)
    got = run_op(blk_f, "helm", "f32", x, 1.1)
    assert rel(got, oracle_op(shape, P, g, nodes, "helm", x, 1.1)) <= TOL["f32"]


@pytest.mark.parametrize("shape,deformed", [("quad", False), ("hex", False), ("tri", False), ("tet", False),
                                            ("prism", False), ("hex", True)])
def test_factors_per_element_for_affine_maps(nir, ctx, shape, deformed):
    """Affine elements: one d xi/d x and |J| per element (any shape; an
    undeformed quad/hex block stores exactly these)."""
    P, E = 4, 41
    g, nodes = make_mesh(shape, E, deformed=False)   # straight cells, each affinely distorted
    Lam, jac = oracle_factors(shape, P, g, nodes)
    assert np.allclose(Lam, Lam[:, :1], rtol=1e-12, atol=1e-12)   # the maps are affine
    blk = nir.Block(ctx, shape, E, P, deformed=deformed)
    blk.set_geometric_factors(dev(Lam[:, 0]), dev(jac[:, 0]), per_element=True)
    for op in OPS:
        x = inputs(blk, op, seed=5)
        got = run_op(blk, op, "f64", x, 0.8)
        ref = oracle_op(shape, P, g, nodes, op, x, 0.8)
        assert rel(got, ref) <= TOL["f64"], (op, rel(got, ref))


def test_factor_errors(nir, ctx):
    P, E = 3, 8
    g, nodes = make_mesh("hex", E, deformed=False)
    Lam, jac = oracle_factors("hex", P, g, nodes)
    blk = nir.Block(ctx, "hex", E, P, deformed=False)
    with pytest.raises(nir.NirError) as ei:   # undeformed block: per-element factors only
        blk.set_geometric_factors(dev(Lam), dev(jac))
    assert ei.value.code == -1
    bad = jac[:, 0].copy()
    bad[3] = -bad[3]
    with pytest.raises(nir.NirError) as ei:   # inverted element
        blk.set_geometric_factors(dev(Lam[:, 0]), dev(bad), per_element=True)
    assert ei.value.code == -7
    nan = jac[:, 0].copy()
    nan[1] = np.nan
    with pytest.raises(nir.NirError) as ei:
        blk.set_geometric_factors(dev(Lam[:, 0]), dev(nan), per_element=True)
    assert ei.value.code == -7
    with pytest.raises(nir.NirError):         # no geometry after a failed call
        blk.helmholtz(torch.zeros(E, blk.M, dtype=torch.float64, device="cuda"))
    t = dev(jac[:, 0])
    assert nir.lib().nir_block_set_geometric_factors(blk.h, 1, t.data_ptr(), t.data_ptr()) == -1
    assert nir.lib().nir_block_set_geometric_factors(blk.h, 2, dev(Lam[:, 0]).data_ptr(), t.data_ptr()) == -1
    blk.set_geometric_factors(dev(Lam[:, 0]), t, per_element=True)   # a valid call restores the block
    x = np.random.default_rng(0).uniform(-1, 1, (E, blk.M))
    y = blk.helmholtz(dev(x)).cpu().numpy()
    assert rel(y, oracle.helmholtz("hex", P, P + 2, g, nodes, 1.0, x)) <= 1e-12
