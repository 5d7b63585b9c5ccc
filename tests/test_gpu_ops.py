"""GPU parity of every elemental operator against the FP64 oracle.

Through the C ABI (Python binding over libnir.so) on seeded synthetic meshes:
  * every operator x every shape x P in {1..9} in FP64, element by element
    (norm-wise relative error <= 1e-12 per block, <= 1e-11 per element);
  * FP32 single apply <= 1e-5, BF16 (bf16 storage, FP32 arithmetic) <= 3e-2;
  * element counts chosen to span several CTAs plus a ragged tail, E = 1, and
    the full-size workloads on sampled elements in the benchmark's launch
    configuration;
  * error paths: in-place calls, missing geometry, inverted elements.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

DIM = {"quad": 2, "tri": 2, "hex": 3, "prism": 3, "tet": 3}
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-2}
TDT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def curved_quads(n, g, amp=0.04):
    off = W.lattice_offsets(g, 2)
    h = 1.0 / n
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    org = np.stack([ii.ravel(), jj.ravel()], axis=1) * h
    X = org[:, None, :] + off[None] * h
    x, y = X[..., 0].copy(), X[..., 1].copy()
    X[..., 0] = x + amp * np.sin(2 * np.pi * y)
    X[..., 1] = y + amp * np.sin(2 * np.pi * x)
    return X


def make_mesh(shape, E, deformed, seed=0):
    """(gorder, nodes[E]) for a test mesh of E elements."""
    if shape == "hex":
        if deformed:
            n = int(np.ceil(E ** (1 / 3))) + 1
            return 2, W.hex_grid(n, 2, amp=0.05)[:E]
        n = int(np.ceil(E ** (1 / 3))) + 1
        return 1, W.perturb_vertices(W.hex_grid(n, 1, amp=0.0)[:E], 0.15, seed)
    if shape == "quad":
        n = int(np.ceil(E ** 0.5)) + 1
        if deformed:
            return 3, curved_quads(n, 3)[:E]
        return 1, W.perturb_vertices(W.quad_grid(n, n)[:E], 0.15, seed)
    if shape == "tri":
        n = int(np.ceil((E / 2) ** 0.5)) + 1
        return 1, W.perturb_vertices(W.tri_grid(n, n)[:E], 0.15, seed)
    if shape == "tet":
        n = int(np.ceil((E / 6) ** (1 / 3))) + 1
        return 1, W.perturb_vertices(W.tet_kuhn(n)[:E], 0.1, seed)
    if shape == "prism":
        n = int(np.ceil((E / 2) ** (1 / 3))) + 1
        return 1, W.perturb_vertices(W.prism_split(n, n, n)[:E], 0.1, seed)
    raise KeyError(shape)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def per_elem_rel(a, b):
    a = a.reshape(a.shape[0], -1) if a.ndim == 2 else np.moveaxis(a, 1, 0).reshape(a.shape[1], -1)
    b = b.reshape(b.shape[0], -1) if b.ndim == 2 else np.moveaxis(b, 1, 0).reshape(b.shape[1], -1)
    return (np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)).max()


def nelem_for(shape, P):
    if DIM[shape] == 2:
        return 150
    return 37 if P <= 4 else 11


def setup(nir, ctx, shape, P, E, deformed, seed=0):
    g, nodes = make_mesh(shape, E, deformed, seed)
    blk = nir.Block(ctx, shape, E, P, deformed=deformed)
    blk.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    assert blk.M == oracle.num_modes(shape, P) and blk.NQ == oracle.num_points(shape, P + 2)
    return g, nodes, blk


def run_op(blk, op, prec, x, lam):
    t = [torch.from_numpy(np.ascontiguousarray(v)).to("cuda", TDT[prec]) for v in x] if op in (
        "iprod_deriv",) else torch.from_numpy(np.ascontiguousarray(x)).to("cuda", TDT[prec])
    if op == "bwd":
        out = blk.bwd_trans(t, prec=prec)
    elif op == "iprod":
        out = blk.iproduct_wrt_base(t, prec=prec)
    elif op == "physderiv":
        out = torch.stack(blk.phys_deriv(t, prec=prec))
    elif op == "iprod_deriv":
        out = blk.iproduct_wrt_deriv_base(t, prec=prec)
    elif op == "mass":
        out = blk.mass(t, prec=prec)
    else:
        out = blk.helmholtz(t, lam=lam, prec=prec)
    torch.cuda.synchronize()
    return out.to(torch.float64).cpu().numpy()


def oracle_op(shape, P, g, nodes, op, x, lam):
    Q = P + 2
    if op == "bwd":
        return oracle.bwd(shape, P, Q, x)
    if op == "iprod":
        return oracle.iprod(shape, P, Q, g, nodes, x)
    if op == "physderiv":
        return oracle.physderiv(shape, Q, g, nodes, x)
    if op == "iprod_deriv":
        return oracle.iprod_deriv(shape, P, Q, g, nodes, x)
    if op == "mass":
        return oracle.mass(shape, P, Q, g, nodes, x)
    return oracle.helmholtz(shape, P, Q, g, nodes, lam, x)


def inputs(blk, op, seed=0):
    if op in ("bwd", "mass", "helm"):
        return W.coefficients(blk.nelem, blk.M, seed)
    if op == "iprod_deriv":
        return W.phys_samples(blk.nelem, blk.NQ, seed + 1, ncomp=blk.dim)
    return W.phys_samples(blk.nelem, blk.NQ, seed + 1)


OPS = ["bwd", "iprod", "physderiv", "iprod_deriv", "mass", "helm"]


@pytest.mark.parametrize("shape", ["quad", "tri", "hex", "prism", "tet"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_fp64_all_ops(nir, ctx, shape, P):
    deformed = shape in ("hex", "quad")
    E = nelem_for(shape, P)
    g, nodes, blk = setup(nir, ctx, shape, P, E, deformed)
    lam = 1.3
    for op in OPS:
        x = inputs(blk, op)
        got = run_op(blk, op, "f64", x, lam)
        ref = oracle_op(shape, P, g, nodes, op, x, lam)
        assert got.shape == ref.shape, op
        assert rel(got, ref) <= TOL["f64"], (op, rel(got, ref))
        assert per_elem_rel(got, ref) <= 1e-11, (op, per_elem_rel(got, ref))


@pytest.mark.parametrize("shape", ["quad", "hex"])
@pytest.mark.parametrize("P", [2, 4, 6])
def test_fp64_affine_tensor_blocks(nir, ctx, shape, P):
    """Undeformed quad/hex blocks keep one set of factors per element."""
    E = nelem_for(shape, P)
    g, nodes, blk = setup(nir, ctx, shape, P, E, deformed=False)
    for op in OPS:
        x = inputs(blk, op, seed=3)
        got = run_op(blk, op, "f64", x, 0.7)
        ref = oracle_op(shape, P, g, nodes, op, x, 0.7)
        assert rel(got, ref) <= TOL["f64"], (op, rel(got, ref))


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("shape", ["quad", "tri", "hex", "prism", "tet"])
@pytest.mark.parametrize("P", [1, 4, 8, 9])
def test_low_precision_all_ops(nir, ctx, prec, shape, P):
    deformed = shape in ("hex", "quad")
    E = nelem_for(shape, P)
    g, nodes, blk = setup(nir, ctx, shape, P, E, deformed)
    for op in OPS:
        x = inputs(blk, op)
        got = run_op(blk, op, prec, x, 1.0)
        ref = oracle_op(shape, P, g, nodes, op, x, 1.0)
        assert rel(got, ref) <= TOL[prec], (op, prec, rel(got, ref))


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape,P", [("hex", 4), ("hex", 6), ("tet", 4), ("prism", 6), ("quad", 4), ("tri", 7),
                                     ("hex", 9), ("tet", 9)])
def test_helmholtz_every_launch_variant(nir, ctx, prec, shape, P):
    """Every elements-per-CTA variant the tuner may pick (default, half, double;
    for FP32/BF16 at P = 6 the double group runs without its staging buffer;
    FP32/BF16 quad/hex also two elements per thread), under every L2 metric
    prefetch policy and at two grid sizes."""
    deformed = shape in ("hex", "quad")
    E = 300 if DIM[shape] == 2 else (150 if P <= 4 else 101)   # several groups of every variant + a ragged tail
    g, nodes, blk = setup(nir, ctx, shape, P, E, deformed)
    x = inputs(blk, "helm")
    ref = oracle_op(shape, P, g, nodes, "helm", x, 1.0)
    paired = prec != "f64" and shape in ("hex", "quad")   # variant 5: two elements per thread
    variants = (0, 1, 2, 3) + ((5,) if paired else ())
    for variant in variants:
        for pf in (0, 1, 2):
            for grid in (0, 152):
                blk.set_tuning(prec, variant, grid, pf)
                got = run_op(blk, "helm", prec, x, 1.0)
                assert rel(got, ref) <= TOL[prec], (variant, pf, grid, rel(got, ref))
    assert blk.get_tuning(prec) == (variants[-1], 152, 2)
    blk.set_tuning(prec, 0, 0, 0)
    y0 = run_op(blk, "helm", prec, x, 1.0)
    blk.set_tuning(prec, 3, 0, 0)
    assert np.array_equal(run_op(blk, "helm", prec, x, 1.0), y0)   # same arithmetic, other allocation
    if not paired:
        with pytest.raises(nir.NirError) as ei:
            blk.set_tuning(prec, 5)
        assert ei.value.code == -2
    for bad in (dict(variant=6), dict(variant=0, pf=3), dict(variant=0, pf=-1)):
        with pytest.raises(nir.NirError) as ei:
            blk.set_tuning(prec, **bad)
        assert ei.value.code == -1


@pytest.mark.parametrize("shape", ["quad", "tri", "hex", "prism", "tet"])
def test_single_element_and_exact_group(nir, ctx, shape):
    P = 3
    for E in (1, 32, 64):
        g, nodes, blk = setup(nir, ctx, shape, P, E, shape in ("hex", "quad"))
        x = inputs(blk, "helm")
        got = run_op(blk, "helm", "f64", x, 2.0)
        ref = oracle_op(shape, P, g, nodes, "helm", x, 2.0)
        assert rel(got, ref) <= TOL["f64"]


def test_laplacian_of_constant_vanishes_on_full_mesh(nir, ctx):
    """Property check at the benchmark's full size: L 1 = 0 for every element."""
    wl = W.workload("hex32_curved_p4")
    E = wl["nodes"].shape[0]
    blk = nir.Block(ctx, "hex", E, wl["P"], deformed=True)
    blk.set_geometry(wl["gorder"], torch.from_numpy(wl["nodes"]).cuda())
    one = torch.zeros((E, blk.M), dtype=torch.float64, device="cuda")
    # vertex modes (p, q, r in {0, 1}) of the packed hex ordering m = (p N + q) N + r
    N = wl["P"] + 1
    for p in (0, 1):
        for q in (0, 1):
            for r in (0, 1):
                one[:, (p * N + q) * N + r] = 1.0
    y = blk.helmholtz(one, lam=0.0)
    mass = blk.helmholtz(one, lam=1.0)
    torch.cuda.synchronize()
    assert y.abs().max().item() < 1e-13
    # 1^T M 1 summed over the mesh = volume of the periodically mapped unit cube
    vol = (mass * one).sum().item()
    assert abs(vol - 1.0) < 1e-12


@pytest.mark.parametrize("name", ["hex32_curved_p4", "tet20_kuhn_p4", "prism40x40x20_p4", "quad8x8_p4"])
def test_full_workloads_sampled(nir, ctx, name):
    """Full-size blocks in the benchmark's launch configuration; the oracle
    recomputes a seeded sample of elements one by one."""
    wl = W.workload(name)
    nodes, shape, P, Q, g = wl["nodes"], wl["shape"], wl["P"], wl["Q"], wl["gorder"]
    E = nodes.shape[0]
    blk = nir.Block(ctx, shape, E, P, deformed=wl["deformed"])
    blk.set_geometry(g, torch.from_numpy(nodes).cuda())
    u = W.coefficients(E, blk.M, seed=0)
    ut = torch.from_numpy(u).cuda()
    y = blk.helmholtz(ut, lam=1.0).cpu().numpy()
    b = blk.bwd_trans(ut).cpu().numpy()
    ids = W.sample_elements(E, 64, seed=1)
    y_o = oracle.helmholtz(shape, P, Q, g, nodes[ids], 1.0, u[ids])
    b_o = oracle.bwd(shape, P, Q, u[ids])
    assert rel(y[ids], y_o) <= 1e-12 and rel(b[ids], b_o) <= 1e-12
    # FP32 apply on the same sample
    y32 = blk.helmholtz(ut.float(), lam=1.0, prec="f32").double().cpu().numpy()
    assert rel(y32[ids], y_o) <= 1e-5


def test_full_p6_workload_sampled(nir, ctx):
    wl = W.workload("hex48_curved_p6")
    nodes, P, Q, g = wl["nodes"], wl["P"], wl["Q"], wl["gorder"]
    E = nodes.shape[0]
    blk = nir.Block(ctx, "hex", E, P, deformed=True)
    blk.set_geometry(g, torch.from_numpy(nodes).cuda())
    u = W.coefficients(E, blk.M, seed=0)
    y = blk.helmholtz(torch.from_numpy(u).cuda(), lam=1.0).cpu().numpy()
    ids = W.sample_elements(E, 24, seed=2)
    y_o = oracle.helmholtz("hex", P, Q, g, nodes[ids], 1.0, u[ids])
    assert rel(y[ids], y_o) <= 1e-12


def test_error_paths(nir, ctx):
    g, nodes, blk = setup(nir, ctx, "tet", 2, 10, False)
    u = torch.zeros((10, blk.M), dtype=torch.float64, device="cuda")
    # in-place (aliased) call is rejected before any GPU work
    assert nir.lib().nir_helmholtz(blk.h, 0, 1.0, nir._ptr(u), nir._ptr(u)) == -1
    fresh = nir.Block(ctx, "tet", 10, 2)
    with pytest.raises(nir.NirError) as ei:
        fresh.helmholtz(u)
    assert ei.value.code == -8
    bad = nodes.copy()
    bad[:, [1, 2]] = bad[:, [2, 1]]  # swap two vertices: negative Jacobian
    with pytest.raises(nir.NirError) as ei:
        fresh.set_geometry(1, torch.from_numpy(bad).cuda())
    assert ei.value.code == -7
    with pytest.raises(nir.NirError) as ei:
        nir.Block(ctx, "hex", 10, 10)   # P = 9 is the highest order compiled
    assert ei.value.code == -2


def test_host_buffer_entry_point(nir, ctx):
    g, nodes, blk = setup(nir, ctx, "hex", 4, 37, True)
    u = torch.from_numpy(W.coefficients(37, blk.M, 5)).pin_memory()
    out = torch.empty_like(u).pin_memory()
    blk.helmholtz_host(u, out, lam=1.0)
    ref = blk.helmholtz(u.cuda(), lam=1.0).cpu()
    assert torch.equal(out, ref)


def test_host_buffer_pipeline_chunks(nir, ctx):
    """The host-buffer entry point splits large blocks into chunks whose
    copies overlap the applies; results equal the device apply bit for bit."""
    for prec in ("f64", "f32"):
        g, nodes, blk = setup(nir, ctx, "hex", 3, 3001, True)
        u = torch.from_numpy(W.coefficients(3001, blk.M, 6)).to(nir.DTYPE[prec]).pin_memory()
        out = torch.empty_like(u).pin_memory()
        blk.helmholtz_host(u, out, lam=1.0, prec=prec)
        ref = blk.helmholtz(u.cuda(), lam=1.0, prec=prec).cpu()
        assert torch.equal(out, ref), prec


def test_host_buffer_graph_replay(nir, ctx):
    """Pinned host buffers replay a captured pipeline: new host contents, a new
    lambda, new geometry and new tuning are all honoured; pageable buffers take
    the direct path.  Every result equals the device apply bit for bit."""
    g, nodes, blk = setup(nir, ctx, "hex", 3, 3001, True)
    for prec in ("f64", "f32"):
        u = torch.from_numpy(W.coefficients(3001, blk.M, 7)).to(nir.DTYPE[prec]).pin_memory()
        out = torch.empty_like(u).pin_memory()
        for it in range(4):
            lam = 1.0 if it < 3 else 2.5
            u.add_(0.125 * (it + 1))                      # new host contents each call
            blk.helmholtz_host(u, out, lam=lam, prec=prec)
            ref = blk.helmholtz(u.cuda(), lam=lam, prec=prec).cpu()
            assert torch.equal(out, ref), (prec, it)
    u = torch.from_numpy(W.coefficients(3001, blk.M, 8)).pin_memory()
    out = torch.empty_like(u).pin_memory()
    blk.helmholtz_host(u, out)
    blk.helmholtz_host(u, out)                            # replayed
    moved = nodes.copy()
    moved[..., 0] += 0.01 * np.sin(3.0 * nodes[..., 1])
    blk.set_geometry(g, torch.from_numpy(np.ascontiguousarray(moved)).cuda())
    blk.helmholtz_host(u, out)
    assert torch.equal(out, blk.helmholtz(u.cuda()).cpu())
    blk.set_tuning("f64", 1, 0, 0)
    blk.helmholtz_host(u, out)
    blk.helmholtz_host(u, out)
    assert torch.equal(out, blk.helmholtz(u.cuda()).cpu())
    up = torch.from_numpy(W.coefficients(3001, blk.M, 9))  # pageable
    op = torch.empty_like(up)
    blk.helmholtz_host(up, op)
    assert torch.equal(op, blk.helmholtz(up.cuda()).cpu())


def test_kernel_info_reports_the_launched_kernel(nir, ctx):
    g, nodes, blk = setup(nir, ctx, "hex", 4, 40, True)
    for prec in ("f64", "f32"):
        for op in ("bwd", "helm"):
            ki = blk.kernel_info(prec, op)
            # whole warps; the fused FP32/BF16 CTA is sized to run its heaviest stages in whole rounds
            assert 0 < ki["registers"] <= 255 and ki["threads"] % 32 == 0 and 32 <= ki["threads"] <= 1024
            assert ki["smem_bytes"] > 0 and ki["elems_per_cta"] >= 1
    blk.set_tuning("f32", 1, 0, 0)
    half = blk.kernel_info("f32", "helm")["elems_per_cta"]
    blk.set_tuning("f32", 0, 0, 0)
    assert blk.kernel_info("f32", "helm")["elems_per_cta"] == 2 * half


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape,P", [("hex", 4), ("tet", 3), ("quad", 5), ("prism", 6)])
def test_multi_field_helmholtz(nir, ctx, prec, shape, P):
    """1..3 fields in one launch equal the single-field applies exactly (the
    same per-element code), and the oracle."""
    deformed = shape in ("hex", "quad")
    E = 75 if P <= 4 else 37
    g, nodes, blk = setup(nir, ctx, shape, P, E, deformed)
    xs = [W.coefficients(E, blk.M, seed=10 + f) for f in range(3)]
    ts = [torch.from_numpy(x).to("cuda", TDT[prec]) for x in xs]
    for nf in (1, 2, 3):
        outs = blk.helmholtz_fields(ts[:nf], lam=1.5, prec=prec)
        for f in range(nf):
            single = blk.helmholtz(ts[f], lam=1.5, prec=prec)
            assert torch.equal(outs[f], single), (nf, f)
    ref = oracle.helmholtz(shape, P, P + 2, g, nodes, 1.5, xs[2])
    assert rel(outs[2].double().cpu().numpy(), ref) <= TOL[prec]
    with pytest.raises(nir.NirError):
        blk.helmholtz_fields(ts[:2], prec=prec, outs=[ts[2], ts[2]])  # aliased outputs
    with pytest.raises(ValueError):
        blk.helmholtz_fields([], prec=prec)
