"""Pins of the FP64 oracle against what mathematics fixes independently of it.

Each test checks the oracle against closed forms, textbook matrices, library
quadrature routines or invariants (nothing here retypes the oracle's own
formulas):
  * quadrature nodes vs numpy/scipy; exactness on monomials vs closed-form moments
  * mode counts vs the dimension of the polynomial space; every mode is a
    polynomial (least-squares fit in xi) and the modes span the space (rank)
  * analytic basis gradients vs the derivative of that polynomial fit
  * mass of monomials vs Dirichlet-type closed forms on affine elements
  * exact physical derivatives of polynomials; Green's identity for L
  * Q1 hexahedron and P1 tetrahedron textbook stiffness/mass matrices
  * Helmholtz symmetry, SPD, L 1 = 0 (also on curved elements), 1^T H 1 = lambda vol
  * manufactured-solution residual vanishes on interior (bubble) modes
  * affine simplex operators do not depend on the quadrature order
  * cube = 6 tets = 2 prisms
"""
import numpy as np
import pytest

import workloads as W
from tests import polyexact as PX

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

DIM = {"quad": 2, "tri": 2, "hex": 3, "prism": 3, "tet": 3}
KIND = {"quad": "cube", "hex": "cube", "tri": "simplex", "tet": "simplex", "prism": "prism"}


def unit_nodes(shape):
    """Nodes of the unit reference-shaped element in x space ([1][nv][d])."""
    if shape == "quad":
        return W.lattice_offsets(1, 2)[None]
    if shape == "hex":
        return W.lattice_offsets(1, 3)[None]
    if shape == "tri":
        return np.array([[[0, 0], [1, 0], [0, 1]]], float)
    if shape == "tet":
        return np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], float)
    if shape == "prism":
        return np.array([[[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [0, 1, 1]]], float)
    raise KeyError(shape)


AFF = {2: (np.array([[1.3, 0.4], [-0.2, 0.9]]), np.array([0.3, -0.7])),
       3: (np.array([[1.2, 0.3, -0.1], [0.2, 0.8, 0.25], [-0.15, 0.1, 1.1]]), np.array([0.5, -0.2, 0.1]))}


def affine_nodes(shape):
    A, b = AFF[DIM[shape]]
    return np.einsum("ij,evj->evi", A, unit_nodes(shape)) + b


def integrate_affine(shape, poly):
    """Exact integral of poly over the affinely mapped unit element."""
    A, b = AFF[DIM[shape]]
    return np.linalg.det(A) * PX.integrate(PX.compose_affine(poly, A, b), KIND[shape])


def packed_modes(shape, P):
    """(p, q, r) of each packed mode: p outermost, then q, then r."""
    N, out = P + 1, []
    for p in range(N):
        if shape == "quad":
            out += [(p, q, 0) for q in range(N)]
        elif shape == "tri":
            out += [(p, q, 0) for q in range(N - p)]
        elif shape == "hex":
            out += [(p, q, r) for q in range(N) for r in range(N)]
        elif shape == "prism":
            out += [(p, q, r) for q in range(N) for r in range(N - p)]
        else:
            out += [(p, q, r) for q in range(N - p) for r in range(N - p - q)]
    return out


def vertex_modes(shape, P):
    want = {"quad": {(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)},
            "tri": {(0, 0, 0), (1, 0, 0), (0, 1, 0)},
            "hex": {(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)},
            "prism": {(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1) if not (a == 1 and c == 1)},
            "tet": {(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)}}[shape]
    return [m for m, t in enumerate(packed_modes(shape, P)) if t in want]


def space_monomials(shape, P):
    d = DIM[shape]
    if shape in ("quad", "hex"):
        return PX.monomials(d, P, total=False)
    if shape in ("tri", "tet"):
        return PX.monomials(d, P, total=True)
    # prism: total degree <= P in (xi1, xi3), degree <= P in xi2
    return [k for k in PX.monomials(3, P, total=False) if k[0] + k[2] <= P]


def random_ref_points(shape, n, rng):
    d = DIM[shape]
    pts = []
    while len(pts) < n:
        x = rng.uniform(-1, 1, size=d)
        if shape == "tri" and x[0] + x[1] > -1e-3:
            continue
        if shape == "tet" and x.sum() > -1 - 1e-3:
            continue
        if shape == "prism" and x[0] + x[2] > -1e-3:
            continue
        pts.append(x)
    return np.array(pts)


def mass_matrix(orc, shape, P, Q, g, nodes):
    return orc.helmholtz_matrix(shape, P, Q, g, nodes, 1.0) - orc.helmholtz_matrix(shape, P, Q, g, nodes, 0.0)


def project(orc, shape, P, Q, g, nodes, u_pts):
    """Galerkin projection: solve M u_hat = B^T W u."""
    M = mass_matrix(orc, shape, P, Q, g, nodes)[0]
    rhs = orc.iprod(shape, P, Q, g, nodes, u_pts)[0]
    return np.linalg.solve(M, rhs)


# ----------------------------------------------------------------------------- quadrature

@pytest.mark.parametrize("Q", [2, 3, 6, 9])
def test_gauss_legendre_matches_numpy(orc, Q):
    z, w = orc.quad_rule("gj0", Q)
    z0, w0 = np.polynomial.legendre.leggauss(Q)
    assert np.allclose(z, z0, atol=1e-14) and np.allclose(w, w0, atol=1e-14)


@pytest.mark.parametrize("alpha", [1, 2])
@pytest.mark.parametrize("Q", [2, 5, 8])
def test_gauss_jacobi_matches_scipy(orc, alpha, Q):
    sp = pytest.importorskip("scipy.special")
    z, w = orc.quad_rule(f"gj{alpha}", Q)
    z0, w0 = sp.roots_jacobi(Q, alpha, 0)
    assert np.allclose(z, z0, atol=1e-13) and np.allclose(w, w0, rtol=1e-12)


@pytest.mark.parametrize("Q", [2, 3, 4, 6, 8, 10])
def test_gll_exactness(orc, Q):
    z, w = orc.quad_rule("gll", Q)
    assert z[0] == -1.0 and z[-1] == 1.0
    for k in range(2 * Q - 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, z ** k) - exact) < 1e-13
    # one degree beyond the exactness limit must fail (the rule is not overfitted)
    k = 2 * Q - 2
    assert abs(np.dot(w, z ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("alpha", [0, 1, 2])
@pytest.mark.parametrize("Q", [3, 6, 9])
def test_gauss_jacobi_exactness(orc, alpha, Q):
    from fractions import Fraction
    from math import comb
    z, w = orc.quad_rule(f"gj{alpha}", Q)
    assert np.all(np.abs(z) < 1)
    for k in range(2 * Q):
        # int_{-1}^{1} (1-x)^alpha x^k dx by binomial expansion
        ex = sum(Fraction(comb(alpha, j) * (-1) ** j) * Fraction(1 - (-1) ** (k + j + 1), k + j + 1)
                 for j in range(alpha + 1))
        assert abs(np.dot(w, z ** k) - float(ex)) < 1e-13


def test_collocation_1d_exact(orc):
    rng = np.random.default_rng(3)
    for kind in ("gll", "gj1", "gj2"):
        z, _ = orc.quad_rule(kind, 7)
        D = orc.colloc_1d(z)
        c = rng.uniform(-1, 1, 7)
        p = np.polynomial.Polynomial(c)
        assert np.allclose(D @ p(z), p.deriv()(z), atol=1e-11)


# ----------------------------------------------------------------------------- basis

@pytest.mark.parametrize("shape", W.SHAPES)
@pytest.mark.parametrize("P", [1, 2, 4, 6, 8])
def test_mode_count_is_space_dimension(orc, shape, P):
    assert orc.num_modes(shape, P) == len(space_monomials(shape, P))
    assert len(packed_modes(shape, P)) == orc.num_modes(shape, P)


@pytest.mark.parametrize("shape", W.SHAPES)
@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_modes_are_polynomials_spanning_the_space(orc, shape, P):
    rng = np.random.default_rng(P)
    d = DIM[shape]
    mons = space_monomials(shape, P)
    pts = random_ref_points(shape, 3 * len(mons) + 20, rng)
    # include points close to the collapsed vertex / edge
    if shape == "tri":
        pts = np.vstack([pts, [[-1 + 1e-4, 1 - 2e-4], [-0.9999, 0.9998]]])
    if shape == "tet":
        pts = np.vstack([pts, [[-1 + 1e-4, -1 + 1e-4, 1 - 3e-4], [-0.9999, 0.99, -0.99995]]])
    if shape == "prism":
        pts = np.vstack([pts, [[-1 + 1e-4, 0.3, 1 - 2e-4], [-0.9999, -0.7, 0.9998]]])
    B, dB = orc.eval_basis(shape, P, pts)
    V = np.stack([np.prod([pts[:, i] ** k[i] for i in range(d)], axis=0) for k in mons], axis=1)
    coef, *_ = np.linalg.lstsq(V, B, rcond=None)
    assert np.abs(V @ coef - B).max() < 1e-10 * max(1.0, np.abs(B).max())
    assert np.linalg.matrix_rank(B, tol=1e-9) == len(mons)
    # gradients equal the derivative of the fitted polynomials
    for i in range(d):
        Vd = np.stack([k[i] * np.prod([pts[:, j] ** (k[j] - (j == i)) if (k[j] - (j == i)) >= 0 else 0 * pts[:, j]
                                        for j in range(d)], axis=0) for k in mons], axis=1)
        assert np.abs(Vd @ coef - dB[i]).max() < 1e-8 * max(1.0, np.abs(dB[i]).max())


@pytest.mark.parametrize("shape", W.SHAPES)
def test_vertex_modes_partition_unity(orc, shape):
    P = 4
    rng = np.random.default_rng(7)
    pts = random_ref_points(shape, 50, rng)
    B, _ = orc.eval_basis(shape, P, pts)
    assert np.allclose(B[:, vertex_modes(shape, P)].sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("shape", W.SHAPES)
def test_basis_rank_at_quadrature_points(orc, shape):
    for P in (2, 4, 6):
        B, _ = orc.ref_basis(shape, P, P + 2)
        assert np.linalg.matrix_rank(B) == orc.num_modes(shape, P)


# ----------------------------------------------------------------------------- integration

@pytest.mark.parametrize("shape", W.SHAPES)
@pytest.mark.parametrize("P", [2, 4])
def test_mass_of_monomials(orc, shape, P):
    Q, d = P + 2, DIM[shape]
    nodes = affine_nodes(shape)
    _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    one = np.zeros(orc.num_modes(shape, P))
    one[vertex_modes(shape, P)] = 1.0
    # an affine map turns total degree D in x into degree D per reference
    # direction; GLL with Q = P+2 is exact to 2P+1 per direction
    for k in PX.monomials(d, 2 * P, total=True):
        f = PX.mono(k)
        got = one @ orc.iprod(shape, P, Q, 1, nodes, PX.evaluate(f, X[0])[None])[0]
        assert abs(got - integrate_affine(shape, f)) < 1e-13, k


def test_cube_is_six_tets_and_two_prisms(orc):
    tets = W.tet_kuhn(1)
    prisms = W.prism_split(1, 1, 1)
    hexes = W.hex_grid(1, 1, amp=0.0)
    for shape, nodes in (("tet", tets), ("prism", prisms), ("hex", hexes)):
        Wt, _, X = orc.geom_factors(shape, 6, 1, nodes, with_x=True)
        assert abs(Wt.sum() - 1.0) < 1e-14
        f = {(2, 1, 3): 1.0, (0, 4, 1): -0.5}
        got = sum(float(np.dot(Wt[e], PX.evaluate(f, X[e]))) for e in range(nodes.shape[0]))
        assert abs(got - PX.integrate(f, "cube")) < 1e-14


def test_curved_hex_jacobian(orc):
    # x1 = X1 (1 + 0.3 X2): det J = 1 + 0.3 X2, volume 1.15; quadratic lattice
    off = W.lattice_offsets(2, 3)
    nodes = off.copy()
    nodes[:, 0] = off[:, 0] * (1 + 0.3 * off[:, 1])
    Wt, L, X = orc.geom_factors("hex", 4, 2, nodes[None], with_x=True)
    assert abs(Wt.sum() - 1.15) < 1e-14
    # the coordinate functions differentiate to the identity
    for l in range(3):
        g = orc.physderiv("hex", 4, 2, nodes[None], X[:, :, l])
        for i in range(3):
            assert np.allclose(g[i], float(i == l), atol=1e-13)


# ----------------------------------------------------------------------------- derivatives

@pytest.mark.parametrize("shape", W.SHAPES)
def test_physderiv_of_polynomial_is_exact(orc, shape):
    P, Q, d = 4, 6, DIM[shape]
    rng = np.random.default_rng(11)
    nodes = affine_nodes(shape)
    _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    u = PX.random_poly(d, P, rng, total=True)   # total degree P survives an affine map
    g = orc.physderiv(shape, Q, 1, nodes, PX.evaluate(u, X[0])[None])
    for l in range(d):
        assert np.allclose(g[l, 0], PX.evaluate(PX.deriv(u, l), X[0]), atol=1e-11)


@pytest.mark.parametrize("shape", W.SHAPES)
def test_projection_reproduces_polynomials(orc, shape):
    P, Q, d = 3, 5, DIM[shape]
    rng = np.random.default_rng(5)
    nodes = affine_nodes(shape)
    _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    u = PX.random_poly(d, P, rng, total=shape in ("tri", "tet"))
    if shape == "prism":
        u = {k: v for k, v in PX.random_poly(3, P, rng, total=False).items() if k[0] + k[2] <= P}
        # an affine map mixes the prism's variables; use the unit prism for this case
        nodes = unit_nodes(shape)
        _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    if shape in ("quad", "hex"):
        nodes = unit_nodes(shape)
        _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    uh = project(orc, shape, P, Q, 1, nodes, PX.evaluate(u, X[0])[None])
    assert np.allclose(orc.bwd(shape, P, Q, uh[None])[0], PX.evaluate(u, X[0]), atol=1e-12)


@pytest.mark.parametrize("shape", W.SHAPES)
def test_green_identity_and_iprod_deriv(orc, shape):
    P, Q, d = 3, 5, DIM[shape]
    rng = np.random.default_rng(13)
    nodes = affine_nodes(shape) if shape in ("tri", "tet") else unit_nodes(shape)
    _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    total = shape in ("tri", "tet")

    def rp():
        p = PX.random_poly(d, P, rng, total=total)
        if shape == "prism":
            p = {k: v for k, v in p.items() if k[0] + k[2] <= P}
        return p

    u, v = rp(), rp()
    uh = project(orc, shape, P, Q, 1, nodes, PX.evaluate(u, X[0])[None])
    vh = project(orc, shape, P, Q, 1, nodes, PX.evaluate(v, X[0])[None])
    L = orc.helmholtz_matrix(shape, P, Q, 1, nodes, 0.0)[0]
    gg = {}
    for l in range(d):
        gg = PX.add(gg, PX.mul(PX.deriv(u, l), PX.deriv(v, l)))
    exact = integrate_affine(shape, gg) if shape in ("tri", "tet") else PX.integrate(gg, KIND[shape])
    assert abs(uh @ L @ vh - exact) < 1e-11 * max(1, abs(exact))
    # IProductWRTDerivBase: u_hat . sum_l (d phi/d x_l, f_l) = int grad u . f
    f = [rp() for _ in range(d)]
    F = np.stack([PX.evaluate(fl, X[0])[None] for fl in f])
    out = orc.iprod_deriv(shape, P, Q, 1, nodes, F)[0]
    gf = {}
    for l in range(d):
        gf = PX.add(gf, PX.mul(PX.deriv(u, l), f[l]))
    exact = integrate_affine(shape, gf) if shape in ("tri", "tet") else PX.integrate(gf, KIND[shape])
    assert abs(uh @ out - exact) < 1e-11 * max(1, abs(exact))


# ----------------------------------------------------------------------------- textbook matrices

def test_q1_hex_textbook_matrices(orc):
    nodes = unit_nodes("hex")
    K = orc.helmholtz_matrix("hex", 1, 3, 1, nodes, 0.0)[0]
    Mm = mass_matrix(orc, "hex", 1, 3, 1, nodes)[0]
    modes = packed_modes("hex", 1)
    kval = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}
    mval = {0: 8 / 216, 1: 4 / 216, 2: 2 / 216, 3: 1 / 216}
    for a, ta in enumerate(modes):
        for b, tb in enumerate(modes):
            dist = sum(x != y for x, y in zip(ta, tb))
            assert abs(K[a, b] - kval[dist]) < 1e-14
            assert abs(Mm[a, b] - mval[dist]) < 1e-15


def test_p1_tet_textbook_matrices(orc):
    nodes = unit_nodes("tet")
    K = orc.helmholtz_matrix("tet", 1, 3, 1, nodes, 0.0)[0]
    Mm = mass_matrix(orc, "tet", 1, 3, 1, nodes)[0]
    # packed P=1 modes: (0,0,0)->V0, (0,0,1)->V3, (0,1,0)->V2, (1,0,0)->V1
    perm = [0, 3, 2, 1]
    K_tb = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    M_tb = (np.ones((4, 4)) + np.eye(4)) / 120.0
    assert np.allclose(K, K_tb[np.ix_(perm, perm)], atol=1e-14)
    assert np.allclose(Mm, M_tb[np.ix_(perm, perm)], atol=1e-15)


# ----------------------------------------------------------------------------- Helmholtz

@pytest.mark.parametrize("shape", W.SHAPES)
def test_helmholtz_invariants(orc, shape):
    P, Q, lam = 3, 5, 1.7
    nodes = affine_nodes(shape)
    H = orc.helmholtz_matrix(shape, P, Q, 1, nodes, lam)[0]
    assert np.abs(H - H.T).max() < 1e-14 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() > 0
    one = np.zeros(H.shape[0])
    one[vertex_modes(shape, P)] = 1.0
    L = orc.helmholtz_matrix(shape, P, Q, 1, nodes, 0.0)[0]
    assert np.abs(L @ one).max() < 1e-13
    Wt, _, _ = orc.geom_factors(shape, Q, 1, nodes)
    assert abs(one @ H @ one - lam * Wt.sum()) < 1e-13
    # matrix-free apply agrees with the assembled matrix
    u = np.random.default_rng(1).uniform(-1, 1, H.shape[0])
    assert np.allclose(orc.helmholtz(shape, P, Q, 1, nodes, lam, u[None])[0], H @ u, atol=1e-13)


def test_laplacian_kills_constants_on_curved_hexes(orc):
    nodes = W.hex_grid(4, 4, amp=0.05)[:5]
    P, Q = 4, 6
    one = np.zeros((5, orc.num_modes("hex", P)))
    one[:, vertex_modes("hex", P)] = 1.0
    assert np.abs(orc.helmholtz("hex", P, Q, 4, nodes, 0.0, one)).max() < 1e-13
    H = orc.helmholtz_matrix("hex", P, Q, 4, nodes, 1.0)
    for e in range(5):
        assert np.abs(H[e] - H[e].T).max() < 1e-14 * np.abs(H[e]).max()


def interior_modes(orc, shape, P):
    """Modes vanishing on the whole element boundary (found numerically)."""
    rng = np.random.default_rng(0)
    d = DIM[shape]
    faces = []
    for _ in range(200):
        x = random_ref_points(shape, 1, rng)[0]
        c = rng.integers(d)
        y = x.copy()
        y[c] = -1.0
        faces.append(y)
        # slanted faces of the collapsed shapes and the +1 faces of tensor shapes
        if shape in ("quad", "hex") or (shape == "prism" and c == 1):
            z = x.copy()
            z[c] = 1.0
            faces.append(z)
    for _ in range(100):
        x = random_ref_points(shape, 1, rng)[0]
        if shape == "tri":
            faces.append(np.array([x[0], -x[0]]))
        if shape == "tet":
            s = -1.0 - x[0] - x[1]
            if s >= -1:
                faces.append(np.array([x[0], x[1], s]))
        if shape == "prism":
            faces.append(np.array([x[0], x[1], -x[0]]))
    B, _ = orc.eval_basis(shape, P, np.array(faces))
    return np.nonzero(np.abs(B).max(axis=0) < 1e-12)[0]


@pytest.mark.parametrize("shape", W.SHAPES)
def test_manufactured_solution_bubble_residual(orc, shape):
    P, Q, lam, d = 4, 6, 2.0, DIM[shape]
    rng = np.random.default_rng(21)
    nodes = affine_nodes(shape) if shape in ("tri", "tet") else unit_nodes(shape)
    _, _, X = orc.geom_factors(shape, Q, 1, nodes, with_x=True)
    u = PX.random_poly(d, P, rng, total=shape in ("tri", "tet"))
    if shape == "prism":
        u = {k: v for k, v in u.items() if k[0] + k[2] <= P}
    lap = {}
    for l in range(d):
        lap = PX.add(lap, PX.deriv(PX.deriv(u, l), l))
    f = PX.add(PX.scale(u, lam), lap, -1.0)
    uh = project(orc, shape, P, Q, 1, nodes, PX.evaluate(u, X[0])[None])
    res = orc.helmholtz(shape, P, Q, 1, nodes, lam, uh[None])[0] - orc.iprod(
        shape, P, Q, 1, nodes, PX.evaluate(f, X[0])[None])[0]
    inner = interior_modes(orc, shape, P)
    assert inner.size > 0
    assert np.abs(res[inner]).max() < 1e-11
    # boundary modes carry the Neumann flux, so the residual there is not zero
    assert np.abs(res).max() > 1e-6


@pytest.mark.parametrize("shape", ["tri", "tet", "prism"])
def test_affine_simplex_quadrature_independence(orc, shape):
    P = 3
    nodes = affine_nodes(shape)
    H1 = orc.helmholtz_matrix(shape, P, P + 2, 1, nodes, 1.0)[0]
    H2 = orc.helmholtz_matrix(shape, P, P + 4, 1, nodes, 1.0)[0]
    assert np.abs(H1 - H2).max() < 1e-13 * np.abs(H1).max()


def test_dense_solve_matches_numpy(orc):
    nodes = W.hex_grid(3, 2, amp=0.05)[:3]
    P, Q = 3, 5
    H = orc.helmholtz_matrix("hex", P, Q, 2, nodes, 1.0)
    b = np.random.default_rng(2).uniform(-1, 1, (3, H.shape[1]))
    x = orc.helmholtz_solve("hex", P, Q, 2, nodes, 1.0, b)
    for e in range(3):
        assert np.allclose(x[e], np.linalg.solve(H[e], b[e]), rtol=1e-10, atol=1e-12)
