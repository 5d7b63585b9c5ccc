"""Pins of the oracle's pyramid against what mathematics fixes independently.

The pyramid is a shape the paper motivates (hybrid meshes joining hexahedra
and tetrahedra) and leaves to future work.  Reference pyramid: square base
xi3 = -1, apex (-1,-1,1); collapsed coordinates eta1 = 2(1+xi1)/(1-xi3) - 1,
eta2 = 2(1+xi2)/(1-xi3) - 1, eta3 = xi3.  The expansion is rational in xi
(as pyramid spaces are), so the pins check what it must contain and what its
traces must be, not polynomiality:
  * mode count N(N+1)(2N+1)/6, the packed order, partition of unity
  * volume 8/3 and monomial integrals against the closed form
    int_{unit pyramid} x^a y^b z^c = c! (a+b+2)! / ((a+b+c+3)! (a+1)(b+1))
  * every polynomial of total degree <= P reproduced exactly (projection),
    the basis of full rank, analytic gradients against finite differences
  * traces: on the square base they span Q_P (conforming with hexahedra), on
    a triangular face P_P (conforming with tetrahedra)
  * continuity at the apex (the collapsed vertex)
  * Helmholtz symmetry, SPD, L 1 = 0, 1^T H 1 = lambda vol, Green's identity,
    bubble residual of a manufactured solution, quadrature independence
  * a cube is 3 pyramids (apex at a corner) and 6 pyramids (apex at the
    centre); a pyramid over a trapezoid has volume base area x height / 3
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

from tests import polyexact as PX

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

UNIT = np.array([[[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1]]], float)
A3 = np.array([[1.2, 0.3, -0.1], [0.2, 0.8, 0.25], [-0.15, 0.1, 1.1]])
B3 = np.array([0.5, -0.2, 0.1])
AFFINE = np.einsum("ij,evj->evi", A3, UNIT) + B3


def pyr_moment(a, b, c):
    """Exact integral of x^a y^b z^c over the unit pyramid (base [0,1]^2 at
    z = 0, apex (0,0,1)): for fixed z the section is [0,1-z]^2."""
    return Fraction(factorial(c) * factorial(a + b + 2), factorial(a + b + c + 3) * (a + 1) * (b + 1))


def integrate_unit(poly):
    return sum(v * float(pyr_moment(*k)) for k, v in poly.items())


def integrate_affine(poly):
    return np.linalg.det(A3) * integrate_unit(PX.compose_affine(poly, A3, B3))


def packed(P):
    N = P + 1
    return [(p, q, r) for p in range(N) for q in range(N) for r in range(N - max(p, q))]


def vertex_modes(P):
    want = {(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1)}
    return [m for m, t in enumerate(packed(P)) if t in want]


def random_ref_points(n, rng):
    pts = []
    while len(pts) < n:
        x = rng.uniform(-1, 1, 3)
        if x[0] + x[2] < -1e-3 and x[1] + x[2] < -1e-3:
            pts.append(x)
    return np.array(pts)


def mass_matrix(orc, P, Q, nodes):
    return orc.helmholtz_matrix("pyr", P, Q, 1, nodes, 1.0) - orc.helmholtz_matrix("pyr", P, Q, 1, nodes, 0.0)


def project(orc, P, Q, nodes, u_pts):
    M = mass_matrix(orc, P, Q, nodes)[0]
    return np.linalg.solve(M, orc.iprod("pyr", P, Q, 1, nodes, u_pts)[0])


# ----------------------------------------------------------------------------- counting, quadrature

@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 9])
def test_mode_count(orc, P):
    N = P + 1
    assert orc.num_modes("pyr", P) == N * (N + 1) * (2 * N + 1) // 6 == len(packed(P))
    assert orc.num_points("pyr", P + 2) == (P + 2) ** 3


def test_closed_form_moment_pin():
    # the closed form itself against two elementary integrals
    assert pyr_moment(0, 0, 0) == Fraction(1, 3)          # base 1 x height 1 / 3
    assert pyr_moment(0, 0, 1) == Fraction(1, 12)         # centroid height 1/4
    assert pyr_moment(1, 0, 0) == Fraction(1, 8)          # centroid x 3/8


@pytest.mark.parametrize("Q", [3, 5, 8])
def test_reference_weights_and_points(orc, Q):
    eta, xi, w = orc.ref_points("pyr", Q)
    assert abs(w.sum() - 8.0 / 3.0) < 1e-14
    assert np.all(w > 0)
    # every point lies inside the reference pyramid, none at the apex
    assert np.all(xi[:, 0] + xi[:, 2] <= 1e-14) and np.all(xi[:, 1] + xi[:, 2] <= 1e-14)
    assert np.all(xi[:, 2] < 1.0)


@pytest.mark.parametrize("P", [2, 4])
def test_mass_of_monomials(orc, P):
    Q = P + 2
    for nodes, integ in ((UNIT, integrate_unit), (AFFINE, integrate_affine)):
        _, _, X = orc.geom_factors("pyr", Q, 1, nodes, with_x=True)
        one = np.zeros(orc.num_modes("pyr", P))
        one[vertex_modes(P)] = 1.0
        for k in PX.monomials(3, 2 * P, total=True):
            f = PX.mono(k)
            got = one @ orc.iprod("pyr", P, Q, 1, nodes, PX.evaluate(f, X[0])[None])[0]
            assert abs(got - integ(f)) < 1e-13, k


# ----------------------------------------------------------------------------- basis

@pytest.mark.parametrize("P", [1, 3, 5])
def test_partition_of_unity_and_rank(orc, P):
    rng = np.random.default_rng(P)
    pts = random_ref_points(80 + 3 * orc.num_modes("pyr", P), rng)
    B, _ = orc.eval_basis("pyr", P, pts)
    assert np.allclose(B[:, vertex_modes(P)].sum(axis=1), 1.0, atol=1e-14)
    assert np.linalg.matrix_rank(B, tol=1e-10) == orc.num_modes("pyr", P)
    Bq, _ = orc.ref_basis("pyr", P, P + 2)
    assert np.linalg.matrix_rank(Bq) == orc.num_modes("pyr", P)


@pytest.mark.parametrize("P", [2, 4])
def test_gradients_match_finite_differences(orc, P):
    rng = np.random.default_rng(3)
    pts = random_ref_points(25, rng) * 0.9 - 0.05
    pts = pts[(pts[:, 0] + pts[:, 2] < -0.02) & (pts[:, 1] + pts[:, 2] < -0.02)]
    _, dB = orc.eval_basis("pyr", P, pts)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        Bp, _ = orc.eval_basis("pyr", P, pts + e)
        Bm, _ = orc.eval_basis("pyr", P, pts - e)
        fd = (Bp - Bm) / (2 * h)
        assert np.abs(fd - dB[i]).max() < 1e-6 * max(1.0, np.abs(dB[i]).max()), i


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_projection_reproduces_total_degree_polynomials(orc, P):
    rng = np.random.default_rng(40 + P)
    Q = P + 2
    _, _, X = orc.geom_factors("pyr", Q, 1, AFFINE, with_x=True)
    u = PX.random_poly(3, P, rng, total=True)       # total degree P survives the affine map
    uh = project(orc, P, Q, AFFINE, PX.evaluate(u, X[0])[None])
    assert np.allclose(orc.bwd("pyr", P, Q, uh[None])[0], PX.evaluate(u, X[0]), atol=1e-12)
    # and at points off the quadrature grid
    pts = random_ref_points(30, rng)
    B, _ = orc.eval_basis("pyr", P, pts)
    x = ((pts + 1) / 2) @ A3.T + B3
    assert np.allclose(B @ uh, PX.evaluate(u, x), atol=1e-11)


def test_traces_on_base_span_tensor_space(orc):
    """On the square base (xi3 = -1) the expansion's traces span exactly Q_P,
    the space of the neighbouring hexahedron's face."""
    P = 4
    rng = np.random.default_rng(5)
    pts = np.column_stack([rng.uniform(-1, 1, 120), rng.uniform(-1, 1, 120), -np.ones(120)])
    B, _ = orc.eval_basis("pyr", P, pts)
    V = np.stack([pts[:, 0] ** a * pts[:, 1] ** b for a in range(P + 1) for b in range(P + 1)], axis=1)
    coef, *_ = np.linalg.lstsq(V, B, rcond=None)
    assert np.abs(V @ coef - B).max() < 1e-11
    assert np.linalg.matrix_rank(B, tol=1e-10) == (P + 1) ** 2


def test_traces_on_triangular_face_span_total_degree(orc):
    """On the face xi2 = -1 (a triangle in (xi1, xi3)) the traces span exactly
    P_P, the space of the neighbouring tetrahedron's face."""
    P = 4
    rng = np.random.default_rng(6)
    pts = []
    while len(pts) < 150:
        a, c = rng.uniform(-1, 1, 2)
        if a + c < -1e-3:
            pts.append([a, -1.0, c])
    pts = np.array(pts)
    B, _ = orc.eval_basis("pyr", P, pts)
    V = np.stack([pts[:, 0] ** a * pts[:, 2] ** c for a in range(P + 1) for c in range(P + 1 - a)], axis=1)
    coef, *_ = np.linalg.lstsq(V, B, rcond=None)
    assert np.abs(V @ coef - B).max() < 1e-10
    assert np.linalg.matrix_rank(B, tol=1e-10) == (P + 1) * (P + 2) // 2


def test_continuous_at_the_apex(orc):
    """Every mode has one limit at the collapsed vertex whatever the direction
    of approach: 1 for the apex vertex mode, 0 for all others."""
    P = 5
    apex_mode = packed(P).index((0, 0, 1))
    for t in (1e-4, 1e-6):
        pts = np.array([[-1 + t * a, -1 + t * b, 1 - t * c] for a, b, c in
                        ((0.1, 0.2, 1.0), (0.9, 0.05, 1.0), (0.5, 0.5, 0.6), (0.01, 0.95, 1.0))])
        B, _ = orc.eval_basis("pyr", P, pts)
        want = np.zeros(B.shape[1])
        want[apex_mode] = 1.0
        assert np.abs(B - want).max() < 20 * t


# ----------------------------------------------------------------------------- operators

def test_helmholtz_invariants(orc):
    P, Q, lam = 3, 5, 1.7
    H = orc.helmholtz_matrix("pyr", P, Q, 1, AFFINE, lam)[0]
    assert np.abs(H - H.T).max() < 1e-14 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() > 0
    one = np.zeros(H.shape[0])
    one[vertex_modes(P)] = 1.0
    L = orc.helmholtz_matrix("pyr", P, Q, 1, AFFINE, 0.0)[0]
    assert np.abs(L @ one).max() < 1e-13
    Wt, _, _ = orc.geom_factors("pyr", Q, 1, AFFINE)
    assert abs(Wt.sum() - np.linalg.det(A3) / 3.0) < 1e-14
    assert abs(one @ H @ one - lam * Wt.sum()) < 1e-13
    u = np.random.default_rng(1).uniform(-1, 1, H.shape[0])
    assert np.allclose(orc.helmholtz("pyr", P, Q, 1, AFFINE, lam, u[None])[0], H @ u, atol=1e-13)


def test_green_identity_and_iprod_deriv(orc):
    P, Q = 3, 5
    rng = np.random.default_rng(13)
    _, _, X = orc.geom_factors("pyr", Q, 1, AFFINE, with_x=True)
    u, v = PX.random_poly(3, P, rng, total=True), PX.random_poly(3, P, rng, total=True)
    uh = project(orc, P, Q, AFFINE, PX.evaluate(u, X[0])[None])
    vh = project(orc, P, Q, AFFINE, PX.evaluate(v, X[0])[None])
    L = orc.helmholtz_matrix("pyr", P, Q, 1, AFFINE, 0.0)[0]
    gg = {}
    for l in range(3):
        gg = PX.add(gg, PX.mul(PX.deriv(u, l), PX.deriv(v, l)))
    exact = integrate_affine(gg)
    assert abs(uh @ L @ vh - exact) < 1e-11 * max(1, abs(exact))
    f = [PX.random_poly(3, P, rng, total=True) for _ in range(3)]
    F = np.stack([PX.evaluate(fl, X[0])[None] for fl in f])
    out = orc.iprod_deriv("pyr", P, Q, 1, AFFINE, F)[0]
    gf = {}
    for l in range(3):
        gf = PX.add(gf, PX.mul(PX.deriv(u, l), f[l]))
    exact = integrate_affine(gf)
    assert abs(uh @ out - exact) < 1e-11 * max(1, abs(exact))
    # exact physical derivatives of a total-degree-P polynomial
    g = orc.physderiv("pyr", Q, 1, AFFINE, PX.evaluate(u, X[0])[None])
    for l in range(3):
        assert np.allclose(g[l, 0], PX.evaluate(PX.deriv(u, l), X[0]), atol=1e-10)


def test_manufactured_solution_bubble_residual(orc):
    P, Q, lam = 4, 6, 2.0
    rng = np.random.default_rng(21)
    _, _, X = orc.geom_factors("pyr", Q, 1, AFFINE, with_x=True)
    u = PX.random_poly(3, P, rng, total=True)
    lap = {}
    for l in range(3):
        lap = PX.add(lap, PX.deriv(PX.deriv(u, l), l))
    f = PX.add(PX.scale(u, lam), lap, -1.0)
    uh = project(orc, P, Q, AFFINE, PX.evaluate(u, X[0])[None])
    res = orc.helmholtz("pyr", P, Q, 1, AFFINE, lam, uh[None])[0] - orc.iprod(
        "pyr", P, Q, 1, AFFINE, PX.evaluate(f, X[0])[None])[0]
    # interior modes: those vanishing on all five faces (found numerically)
    fp = []
    for _ in range(300):
        a, b, c = rng.uniform(-1, 1, 3)
        fp += [[a, b, -1.0]]
        if a + c < 0:
            fp += [[a, -1.0, c], [-1.0, a, c]]
        if b + c < 0:
            fp += [[-c, b, c], [b, -c, c]]
    B, _ = orc.eval_basis("pyr", P, np.array(fp))
    inner = np.nonzero(np.abs(B).max(axis=0) < 1e-12)[0]
    assert inner.size > 0
    assert np.abs(res[inner]).max() < 1e-11
    assert np.abs(res).max() > 1e-6


def test_quadrature_independence_on_affine_pyramids(orc):
    P = 3
    H1 = orc.helmholtz_matrix("pyr", P, P + 2, 1, AFFINE, 1.0)[0]
    H2 = orc.helmholtz_matrix("pyr", P, P + 4, 1, AFFINE, 1.0)[0]
    assert np.abs(H1 - H2).max() < 1e-13 * np.abs(H1).max()


# ----------------------------------------------------------------------------- meshes of pyramids

def oriented(base, apex):
    """Pyramid nodes with the base ordered like the reference one: counter-
    clockwise seen from the apex, i.e. det[v1 - v0, v3 - v0, apex - v0] > 0."""
    v = np.array(base, float)
    a = np.array(apex, float)
    if np.linalg.det(np.stack([v[1] - v[0], v[3] - v[0], a - v[0]])) < 0:
        v = v[[0, 3, 2, 1]]
    return np.vstack([v, a])


def cube_corner_pyramids():
    """The unit cube as 3 pyramids with apex (0,0,0), one per far face."""
    faces = [[[1, 0, 0], [1, 1, 0], [1, 1, 1], [1, 0, 1]],
             [[0, 1, 0], [0, 1, 1], [1, 1, 1], [1, 1, 0]],
             [[0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]]]
    return np.array([oriented(f, [0, 0, 0]) for f in faces])


def cube_centre_pyramids():
    """The unit cube as 6 pyramids with apex at its centre, one per face."""
    out = []
    for axis in range(3):
        for side in (0, 1):
            quad = []
            for (a, b) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                v = [0.0, 0.0, 0.0]
                v[axis] = side
                v[(axis + 1) % 3] = a
                v[(axis + 2) % 3] = b
                quad.append(v)
            out.append(oriented(quad, [0.5, 0.5, 0.5]))
    return np.array(out)


@pytest.mark.parametrize("build", [cube_corner_pyramids, cube_centre_pyramids])
def test_cube_is_a_union_of_pyramids(orc, build):
    nodes = build()
    Wt, _, X = orc.geom_factors("pyr", 6, 1, nodes, with_x=True)
    assert abs(Wt.sum() - 1.0) < 1e-14
    f = {(2, 1, 3): 1.0, (0, 4, 1): -0.5, (1, 1, 1): 0.25}
    got = sum(float(np.dot(Wt[e], PX.evaluate(f, X[e]))) for e in range(nodes.shape[0]))
    assert abs(got - PX.integrate(f, "cube")) < 1e-14


def test_pyramid_split_mesh_fills_the_cube(orc):
    import workloads as W
    nodes = W.pyramid_split(2, 3, 2)
    Wt, _, X = orc.geom_factors("pyr", 5, 1, nodes, with_x=True)
    assert nodes.shape == (72, 5, 3) and np.all(Wt > 0)
    f = {(1, 2, 0): 1.0, (0, 0, 3): 0.5}
    got = sum(float(np.dot(Wt[e], PX.evaluate(f, X[e]))) for e in range(nodes.shape[0]))
    assert abs(got - PX.integrate(f, "cube")) < 1e-13


def test_pyramid_over_a_trapezoid(orc):
    """A non-affine element (trapezoid base): the rational vertex map still
    fills the straight-sided pyramid, whose volume is area x height / 3, and
    its Jacobian determinant stays positive."""
    base = np.array([[0, 0, 0], [2.0, 0, 0], [1.5, 1.0, 0], [0.5, 1.0, 0]])
    nodes = np.vstack([base, [[0.7, 0.4, 1.3]]])[None]
    Wt, L, _ = orc.geom_factors("pyr", 7, 1, nodes)
    assert np.all(Wt > 0)
    area = 0.5 * (2.0 + 1.0) * 1.0
    assert abs(Wt.sum() - area * 1.3 / 3.0) < 1e-13
    # the coordinate functions differentiate to the identity
    _, _, X = orc.geom_factors("pyr", 7, 1, nodes, with_x=True)
    for l in range(3):
        g = orc.physderiv("pyr", 7, 1, nodes, X[:, :, l])
        for i in range(3):
            assert np.allclose(g[i], float(i == l), atol=1e-11)
