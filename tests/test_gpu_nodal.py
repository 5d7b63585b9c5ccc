"""GPU parity of the nodal (GLL-Lagrange) quad/hex expansions against the
nodal oracle (``oracle/nodal.py``, itself pinned to the modified-basis oracle
by the change of basis): every modal operator in FP64 at P = 1..8, the FP32
and BF16 Helmholtz (fused kernel with bulk-copy staging), several launch
variants, multi-field calls, the hybrid mesh in both launch forms, the full
benchmark mesh on sampled elements, the conforming C0 assembly and Dirichlet
solve against the numbering-free oracle of ``oracle/conforming.py`` in the
nodal basis, and the unsupported combinations."""
import numpy as np
import pytest
import torch

import oracle as orc
import workloads as W
from oracle import conforming as cf
from oracle import nodal as nd

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-2}


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def mesh(shape, E, seed=0):
    if shape == "quad":
        n = int(np.ceil(E ** 0.5)) + 1
        return 1, W.perturb_vertices(W.quad_grid(n, n)[:E], 0.1, seed)
    n = int(np.ceil(E ** (1 / 3))) + 1
    return 2, W.hex_grid(n, 2, amp=0.05)[:E]


def block(nir, ctx, shape, P, E):
    g, nodes = mesh(shape, E)
    blk = nir.Block(ctx, shape, E, P, deformed=True, basis="nodal")
    blk.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    return g, nodes, blk


def dev(x, prec, nir):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", nir.DTYPE[prec])


@pytest.mark.parametrize("shape", ["quad", "hex"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8, 9])
def test_fp64_modal_operators(nir, ctx, shape, P):
    E = 70 if shape == "quad" else (40 if P <= 4 else 12)
    g, nodes, blk = block(nir, ctx, shape, P, E)
    Q = P + 2
    rng = np.random.default_rng(P)
    u = rng.uniform(-1, 1, (E, blk.M))
    f = rng.uniform(-1, 1, (E, blk.NQ))
    fs = rng.uniform(-1, 1, (blk.dim, E, blk.NQ))
    got = blk.bwd_trans(dev(u, "f64", nir)).cpu().numpy()
    assert rel(got, nd.bwd(shape, P, Q, u)) <= TOL["f64"]
    got = blk.iproduct_wrt_base(dev(f, "f64", nir)).cpu().numpy()
    assert rel(got, nd.iprod(shape, P, Q, g, nodes, f)) <= TOL["f64"]
    got = blk.iproduct_wrt_deriv_base([dev(x, "f64", nir) for x in fs]).cpu().numpy()
    assert rel(got, nd.iprod_deriv(shape, P, Q, g, nodes, fs)) <= TOL["f64"]
    got = blk.mass(dev(u, "f64", nir)).cpu().numpy()
    assert rel(got, nd.mass(shape, P, Q, g, nodes, u)) <= TOL["f64"]
    got = blk.helmholtz(dev(u, "f64", nir), lam=1.7).cpu().numpy()
    assert rel(got, nd.helmholtz(shape, P, Q, g, nodes, 1.7, u)) <= TOL["f64"]


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("shape,P", [("quad", 4), ("quad", 7), ("hex", 3), ("hex", 4), ("hex", 6)])
def test_low_precision_helmholtz_variants(nir, ctx, prec, shape, P):
    E = 300 if shape == "quad" else (150 if P <= 4 else 101)
    g, nodes, blk = block(nir, ctx, shape, P, E)
    u = np.random.default_rng(2).uniform(-1, 1, (E, blk.M))
    ref = nd.helmholtz(shape, P, P + 2, g, nodes, 1.0, u)
    for variant in (0, 1, 2, 3, 5):
        blk.set_tuning(prec, variant, 0, 1)
        got = blk.helmholtz(dev(u, prec, nir), prec=prec).double().cpu().numpy()
        assert rel(got, ref) <= TOL[prec], (variant, rel(got, ref))
    outs = blk.helmholtz_fields([dev(u, prec, nir), dev(2 * u, prec, nir)], prec=prec)
    assert torch.equal(outs[0], blk.helmholtz(dev(u, prec, nir), prec=prec))


def test_mesh_with_nodal_and_modified_blocks(nir, ctx):
    P, E = 3, 40
    g, nodes = mesh("hex", E)
    blocks = []
    for basis in ("nodal", "modified"):
        b = nir.Block(ctx, "hex", E, P, deformed=True, basis=basis)
        b.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
        blocks.append(b)
    m = nir.Mesh(ctx, blocks)
    x = np.random.default_rng(4).uniform(-1, 1, m.ndof)
    for prec in ("f64", "f32"):
        xt = dev(x, prec, nir)
        m.set_launch(prec, "persistent")
        y0 = m.helmholtz(xt, prec=prec)
        m.set_launch(prec, "blocks")
        y1 = m.helmholtz(xt, prec=prec)
        assert torch.equal(y0, y1)
        M = blocks[0].M
        yn = y0[:E * M].double().cpu().numpy().reshape(E, M)
        assert rel(yn, nd.helmholtz("hex", P, P + 2, g, nodes, 1.0, x[:E * M].reshape(E, M))) <= TOL[prec]
        ym = y0[E * M:].double().cpu().numpy().reshape(E, M)
        assert rel(ym, orc.helmholtz("hex", P, P + 2, g, nodes, 1.0, x[E * M:].reshape(E, M))) <= TOL[prec]


def test_full_benchmark_mesh_nodal_sampled(nir, ctx):
    wl = W.workload("hex32_curved_p4")
    E = wl["nodes"].shape[0]
    blk = nir.Block(ctx, "hex", E, 4, deformed=True, basis="nodal")
    blk.set_geometry(4, torch.from_numpy(wl["nodes"]).cuda())
    u = W.coefficients(E, blk.M, seed=0)
    ids = W.sample_elements(E, 8, seed=5)
    for prec in ("f64", "f32"):
        y = blk.helmholtz(dev(u, prec, nir), prec=prec).double().cpu().numpy()
        ref = nd.helmholtz("hex", 4, 6, 4, wl["nodes"][ids], 1.0, u[ids])
        assert rel(y[ids], ref) <= TOL[prec]


@pytest.mark.parametrize("shape,n,P,g", [("quad", 3, 4, 1), ("hex", 2, 4, 2), ("hex", 2, 5, 2)])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_nodal_assembly_and_dirichlet_solve(nir, ctx, shape, n, P, g, inner):
    """Rotated local frames (every edge and face orientation): the gathered
    space is the oracle's conforming nodal space, and the Dirichlet Helmholtz
    solve through the nodal kernels equals the oracle's global solution."""
    d = 2 if shape == "quad" else 3
    lam = 1.5
    nodes = W.quad_grid(n, n) if d == 2 else W.hex_grid(n, g, amp=0.05)
    nodes, verts, _ = W.rotate_elements(nodes, W.grid_vertices(n, d), g, seed=7 * P)
    nodes = np.ascontiguousarray(nodes)
    E, Q = nodes.shape[0], P + 2
    cut = E // 2
    blocks = []
    for a, b in ((0, cut), (cut, E)):
        blk = nir.Block(ctx, shape, b - a, P, deformed=True, basis="nodal")
        blk.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes[a:b])).cuda())
        blocks.append(blk)
    asm = nir.Assembly(ctx, blocks, [verts[:cut], verts[cut:]])
    assert (asm.n_global, asm.n_free) == ((n * P + 1) ** d, (n * P - 1) ** d)
    assert (asm.local_map() > 0).all()
    Z = cf.conforming_basis(shape, P, verts, dirichlet=False, basis="nodal")
    xl = asm.gather(torch.from_numpy(W.coefficients(1, asm.n_global, seed=3)[0]).cuda()).cpu().numpy()
    assert np.linalg.norm(xl - Z @ (Z.T @ xl)) <= 1e-12 * np.linalg.norm(xl)
    X = orc.geom_factors(shape, Q, g, nodes, with_x=True)[2]
    u = np.prod(np.sin(np.pi * X), axis=-1)
    f = (d * np.pi ** 2 + lam) * u
    sol, lift = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, f, u, basis="nodal")
    parts = [blocks[0].iproduct_wrt_base(torch.from_numpy(np.ascontiguousarray(f[:cut])).cuda()),
             blocks[1].iproduct_wrt_base(torch.from_numpy(np.ascontiguousarray(f[cut:])).cuda())]
    b = asm.assemble(torch.cat([p.view(-1) for p in parts]))
    x = asm.pick(torch.from_numpy(lift.ravel()).cuda())
    xb = x[asm.n_free:].clone()
    x[:asm.n_free] = 0.0
    rc, st = asm.cg_solve(b, x, lam=lam, inner_prec=inner, tol=1e-12, max_inner=5000)
    assert rc == 0, st
    assert torch.equal(x[asm.n_free:], xb)
    got = asm.gather(x).cpu().numpy().reshape(sol.shape)
    assert np.linalg.norm(got - sol) <= 1e-9 * np.linalg.norm(sol)


def test_unsupported_combinations(nir, ctx):
    with pytest.raises(nir.NirError) as e:
        nir.Block(ctx, "tet", 4, 3, basis="nodal")
    assert e.value.code == -2
    g, nodes, blk = block(nir, ctx, "hex", 2, 8)
    mod = nir.Block(ctx, "hex", 8, 2, deformed=True)
    mod.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    verts = W.grid_vertices(2, 3)
    with pytest.raises(nir.NirError) as e:           # one assembly, two bases
        nir.Assembly(ctx, [blk, mod], [verts, verts + 100])
    assert e.value.code == -2
