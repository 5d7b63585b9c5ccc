"""GPU tests of the conforming C0 assembly (nir_asm_*) against the numbering-
free oracle of ``oracle/conforming.py``: the global space has the closed-form
dimension, gathered vectors are continuous (they lie in the oracle's
conforming space), the assembled operator has the oracle's bilinear form, and
the Dirichlet Helmholtz solve reproduces the oracle's global solution.
Meshes are described in randomly rotated local frames, so shared edges and
faces are met in every orientation."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import conforming as cf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def mesh(shape, n, P, g, amp, rotate, seed=0):
    d = 2 if shape == "quad" else 3
    nodes = W.quad_grid(n, n) if d == 2 else W.hex_grid(n, g, amp=amp)
    if d == 2:
        g = 1
    verts = W.grid_vertices(n, d)
    if rotate:
        nodes, verts, _ = W.rotate_elements(nodes, verts, g, seed=seed)
    return dict(shape=shape, P=P, Q=P + 2, gorder=g, nodes=np.ascontiguousarray(nodes), verts=verts, n=n, d=d)


def build(nir, ctx, m, split=1):
    """Blocks (optionally the elements split over several blocks) + assembly."""
    E = m["nodes"].shape[0]
    cuts = np.linspace(0, E, split + 1).astype(int)
    blocks = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        blk = nir.Block(ctx, m["shape"], b - a, m["P"], deformed=m["d"] == 3)
        blk.set_geometry(m["gorder"], torch.from_numpy(np.ascontiguousarray(m["nodes"][a:b])).cuda())
        blocks.append(blk)
    asm = nir.Assembly(ctx, blocks, [m["verts"][a:b] for a, b in zip(cuts[:-1], cuts[1:])])
    return asm, blocks


CASES = [("quad", 3, 3, False), ("quad", 3, 4, True), ("hex", 2, 2, False), ("hex", 2, 3, True),
         ("hex", 3, 2, True)]


@pytest.mark.parametrize("shape,n,P,rotate", CASES)
def test_dimensions_and_continuity(nir, ctx, shape, n, P, rotate):
    m = mesh(shape, n, P, 1, 0.0, rotate, seed=P + n)
    asm, _ = build(nir, ctx, m, split=2)
    d = m["d"]
    assert asm.n_global == (n * P + 1) ** d
    assert asm.n_free == (n * P - 1) ** d
    Z = cf.conforming_basis(shape, P, m["verts"], dirichlet=False)
    Z0 = cf.conforming_basis(shape, P, m["verts"], dirichlet=True)
    x = torch.from_numpy(W.coefficients(1, asm.n_global, seed=5)[0]).cuda()
    xl = asm.gather(x).cpu().numpy()
    # continuous: no component outside the oracle's conforming space
    assert np.linalg.norm(xl - Z @ (Z.T @ xl)) <= 1e-12 * np.linalg.norm(xl)
    x0 = x.clone()
    x0[asm.n_free:] = 0.0
    xl0 = asm.gather(x0).cpu().numpy()
    assert np.linalg.norm(xl0 - Z0 @ (Z0.T @ xl0)) <= 1e-12 * np.linalg.norm(xl0)
    # every global dof is reached; signs are +-1
    mp = asm.local_map()
    assert np.array_equal(np.unique(np.abs(mp)), np.arange(1, asm.n_global + 1))


def test_gather_assemble_pick_are_consistent(nir, ctx):
    m = mesh("hex", 2, 4, 2, 0.05, True, seed=9)
    asm, _ = build(nir, ctx, m)
    x = torch.from_numpy(W.coefficients(1, asm.n_global, seed=1)[0]).cuda()
    yl = torch.from_numpy(W.coefficients(1, asm.n_local, seed=2)[0]).cuda()
    # adjointness <A x, y> = <x, A^T y>
    lhs = float(torch.dot(asm.gather(x), yl))
    rhs = float(torch.dot(x, asm.assemble(yl)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) * 10 + 1e-13
    # pick inverts gather exactly
    assert torch.equal(asm.pick(asm.gather(x)), x)
    # low-precision gather/assemble are the FP64 ones rounded
    for prec, tol in (("f32", 1e-6), ("bf16", 1e-2)):
        xl = asm.gather(x.to(nir.DTYPE[prec]), prec=prec).double()
        assert torch.allclose(xl, asm.gather(x), rtol=tol, atol=tol)
        yg = asm.assemble(yl.to(nir.DTYPE[prec]), prec=prec).double()
        ref = asm.assemble(yl.to(nir.DTYPE[prec]).double())
        assert torch.allclose(yg, ref, rtol=tol, atol=tol)


@pytest.mark.parametrize("shape,n,P,rotate", [("quad", 3, 3, True), ("hex", 2, 3, True)])
@pytest.mark.parametrize("op", ["helmholtz", "mass"])
def test_assembled_bilinear_form_matches_oracle(nir, ctx, shape, n, P, rotate, op):
    lam = 1.25
    m = mesh(shape, n, P, 2 if shape == "hex" else 1, 0.05, rotate, seed=3)
    asm, _ = build(nir, ctx, m)
    E = m["nodes"].shape[0]
    Z = cf.conforming_basis(shape, P, m["verts"], dirichlet=False)
    if op == "helmholtz":
        K = cf.block_matrix(oracle.helmholtz_matrix(shape, P, m["Q"], m["gorder"], m["nodes"], lam))
    else:
        K = cf.block_matrix(cf.mass_matrices(shape, P, m["Q"], m["gorder"], m["nodes"]))
    rng = np.random.default_rng(0)
    U = Z @ rng.uniform(-1, 1, size=(Z.shape[1], 3))      # continuous local vectors (oracle)
    V = Z @ rng.uniform(-1, 1, size=(Z.shape[1], 3))
    ref = V.T @ K @ U
    got = np.zeros((3, 3))
    for j in range(3):
        ug = asm.pick(torch.from_numpy(np.ascontiguousarray(U[:, j])).cuda())
        yg = asm.apply(ug, op=op, lam=lam)
        for i in range(3):
            vg = asm.pick(torch.from_numpy(np.ascontiguousarray(V[:, i])).cuda())
            got[i, j] = float(torch.dot(vg, yg))
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def _dirichlet_problem(m, lam):
    X = oracle.geom_factors(m["shape"], m["Q"], m["gorder"], m["nodes"], with_x=True)[2]
    u = np.prod(np.sin(np.pi * X), axis=-1)
    f = (m["d"] * np.pi ** 2 + lam) * u
    return u, f


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_dirichlet_solve_matches_oracle(nir, ctx, inner):
    lam = 1.0
    m = mesh("hex", 2, 4, 4, 0.05, True, seed=21)
    asm, blocks = build(nir, ctx, m)
    u, f = _dirichlet_problem(m, lam)
    sol, lift = cf.dirichlet_solve("hex", 4, m["Q"], m["gorder"], m["nodes"], m["verts"], lam, f, u)
    blk = blocks[0]
    b = asm.assemble(blk.iproduct_wrt_base(torch.from_numpy(f).cuda()).view(-1))
    x = asm.pick(torch.from_numpy(lift.ravel()).cuda())
    xb = x[asm.n_free:].clone()
    x[:asm.n_free] = 0.0
    rc, st = asm.cg_solve(b, x, lam=lam, inner_prec=inner, tol=1e-12, max_inner=5000)
    assert rc == 0, st
    assert torch.equal(x[asm.n_free:], xb)          # Dirichlet values held
    got = asm.gather(x).cpu().numpy().reshape(sol.shape)
    assert np.linalg.norm(got - sol) <= 1e-9 * np.linalg.norm(sol)


def test_projection_and_dirichlet_solve_on_gpu_alone(nir, ctx):
    """The GPU builds its own lift (mass-matrix CG with all dofs free) and
    solves; the result equals the oracle's solution (same discrete problem)."""
    lam = 2.0
    m = mesh("hex", 2, 3, 3, 0.05, True, seed=4)
    asm, blocks = build(nir, ctx, m, split=2)
    u, f = _dirichlet_problem(m, lam)
    sol, _ = cf.dirichlet_solve("hex", 3, m["Q"], m["gorder"], m["nodes"], m["verts"], lam, f, u)
    E1 = blocks[0].nelem

    def assembled_rhs(vals):
        parts = [blocks[0].iproduct_wrt_base(torch.from_numpy(np.ascontiguousarray(vals[:E1])).cuda()),
                 blocks[1].iproduct_wrt_base(torch.from_numpy(np.ascontiguousarray(vals[E1:])).cuda())]
        return asm.assemble(torch.cat([p.view(-1) for p in parts]))

    bu = assembled_rhs(u)
    up = torch.zeros(asm.n_global, dtype=torch.float64, device="cuda")
    rc, st = asm.cg_solve(bu, up, op="mass", fix_boundary=False, inner_prec="f64", tol=1e-13, max_inner=5000)
    assert rc == 0, st
    b = assembled_rhs(f)
    x = up.clone()
    x[:asm.n_free] = 0.0
    rc, st = asm.cg_solve(b, x, lam=lam, inner_prec="f32", tol=1e-12)
    assert rc == 0, st
    got = asm.gather(x).cpu().numpy().reshape(sol.shape)
    assert np.linalg.norm(got - sol) <= 1e-8 * np.linalg.norm(sol)


def test_invalid_arguments(nir, ctx):
    m = mesh("hex", 2, 2, 1, 0.0, False)
    blk = nir.Block(ctx, "hex", 8, 2)
    blk.set_geometry(1, torch.from_numpy(m["nodes"]).cuda())
    bad = m["verts"].copy()
    bad[1] = bad[0]                      # two elements on the same cell: faces held 4 times...
    bad[2] = bad[0]
    with pytest.raises(nir.NirError):
        nir.Assembly(ctx, [blk], [bad])
    tet = nir.Block(ctx, "tet", 6, 2)
    with pytest.raises(nir.NirError) as e:
        nir.Assembly(ctx, [tet], [np.zeros((6, 8), np.int64)])
    assert e.value.code == -2


def _face_trace_mismatch(P, c1, c2, verts1, verts2):
    """Largest trace difference of two elements' expansions (coefficients c1,
    c2) over their shared face, evaluated by the oracle at Gauss points."""
    shared = set(verts1.tolist()) & set(verts2.tolist())
    assert len(shared) == 4
    s = cf._face_samples(3, P)
    f1 = next(f for f in cf._face_list(3) if {int(verts1[v]) for v in cf._face_corners(3, *f)} == shared)
    f2 = next(f for f in cf._face_list(3) if {int(verts2[v]) for v in cf._face_corners(3, *f)} == shared)
    k1 = cf._face_corners(3, *f1)
    pos2 = {int(verts2[v]): v for v in cf._face_corners(3, *f2)}
    xi1 = cf._bilinear(s, np.stack([cf._vertex_xi(3, v) for v in k1]))
    xi2 = cf._bilinear(s, np.stack([cf._vertex_xi(3, pos2[int(verts1[v])]) for v in k1]))
    B1, _ = oracle.eval_basis("hex", P, xi1)
    B2, _ = oracle.eval_basis("hex", P, xi2)
    return np.abs(B1 @ c1 - B2 @ c2).max(), np.abs(B1 @ c1).max()


def test_full_size_dirichlet_solve_properties(nir, ctx):
    """48^3 curved hexes, P = 6 (the solve workload): the mixed-precision
    solve converges, holds the Dirichlet values, matches the exact solution to
    the discretisation error, and its traces agree across sampled shared faces
    (oracle evaluation, element pair by element pair)."""
    wl = W.workload("hex48_curved_p6")
    n, P, E = 48, 6, wl["nodes"].shape[0]
    verts = W.grid_vertices(n, 3)
    blk = nir.Block(ctx, "hex", E, P, deformed=True)
    blk.set_geometry(wl["gorder"], torch.from_numpy(wl["nodes"]).cuda())
    asm = nir.Assembly(ctx, [blk], [verts])
    assert asm.n_global == (n * P + 1) ** 3 and asm.n_free == (n * P - 1) ** 3
    lam = 1.0
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(E, 24, replace=False))
    X = oracle.geom_factors("hex", P + 2, wl["gorder"], wl["nodes"][ids], with_x=True)[2]
    # exact solution at all points (input generation on the device)
    eta, xi = blk.points()
    import bench
    f = bench.manufactured_rhs_points(wl, xi, lam, torch.device("cuda"))
    u = f / (3 * np.pi ** 2 + lam)
    assert np.allclose(u[ids].cpu().numpy(), np.prod(np.sin(np.pi * X), axis=-1), atol=1e-13)
    bu = asm.assemble(blk.iproduct_wrt_base(u).reshape(-1))
    up = torch.zeros_like(bu)
    rc, st = asm.cg_solve(bu, up, op="mass", fix_boundary=False, inner_prec="f32", tol=1e-12, max_outer=60)
    assert rc == 0, st
    b = asm.assemble(blk.iproduct_wrt_base(f).reshape(-1))
    x = up.clone()
    x[:asm.n_free] = 0.0
    rc, st = asm.cg_solve(b, x, lam=lam, inner_prec="f32", tol=1e-10, max_outer=60)
    assert rc == 0 and st["rel_residual"] <= 1e-10, st
    assert torch.equal(x[asm.n_free:], up[asm.n_free:])
    # the FP64 residual recomputed through the assembled FP64 operator
    r = (b - asm.apply(x, lam=lam))[:asm.n_free]
    assert float(r.norm() / b[:asm.n_free].norm()) <= 1.5e-10
    ul = asm.gather(x).view(E, blk.M)
    err = float((blk.bwd_trans(ul) - u).abs().max() / u.abs().max())
    # discretisation error at P = 6, h = 1/48 with the lift projected to 1e-12:
    # measured 5e-11; a wrong sign, index or boundary value gives O(1)
    assert err < 1e-8, err
    # traces across sampled interior faces (x-neighbours) agree
    cl = ul.cpu().numpy()
    worst = 0.0
    for e1 in ids[:12]:
        i = e1 % n
        e2 = e1 + 1 if i < n - 1 else e1 - 1
        d, s = _face_trace_mismatch(P, cl[e1], cl[e2], verts[e1], verts[e2])
        worst = max(worst, d / max(s, 1e-300))
    assert worst < 1e-12, worst


@pytest.mark.parametrize("P,nfree", [(1, 0), (2, 1), (3, 8)])
def test_single_element_edge_cases(nir, ctx, P, nfree):
    """One hexahedron: every vertex, edge and face dof is on the boundary; the
    free dofs are the (P-1)^3 interior modes (none at P = 1: nothing to solve)."""
    nodes = W.hex_grid(1, 1, amp=0.0)
    blk = nir.Block(ctx, "hex", 1, P)
    blk.set_geometry(1, torch.from_numpy(nodes).cuda())
    asm = nir.Assembly(ctx, [blk], [W.grid_vertices(1, 3)])
    assert asm.n_global == (P + 1) ** 3 and asm.n_free == nfree
    x = torch.from_numpy(W.coefficients(1, asm.n_global, seed=3)[0]).cuda()
    # a single element: the gather is a signed permutation of the modes
    assert np.array_equal(np.sort(np.abs(asm.local_map())), np.arange(1, asm.n_global + 1))
    b = asm.apply(x, lam=1.0)
    x0 = x.clone()
    x[:nfree] = 0.0
    rc, st = asm.cg_solve(b, x, lam=1.0, inner_prec="f64", tol=1e-13)
    assert rc == 0, st
    assert torch.allclose(x, x0, rtol=0, atol=1e-10)
