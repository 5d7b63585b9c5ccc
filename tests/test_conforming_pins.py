"""Pins of the conforming-space oracle (``oracle/conforming.py``) against facts
fixed by the mathematics, not by the oracle itself:

* the dimension of the C0 space of degree P on an n^d grid is (nP+1)^d, and
  (nP-1)^d with homogeneous Dirichlet conditions (closed form);
* functions in the space are reproduced exactly by the L2 projection: the
  constant, and the physical coordinates on an isoparametric curved mesh;
* a quadratic manufactured solution of (-lap + lambda) u = f with its own
  Dirichlet data is recovered exactly (to roundoff) when P >= 2;
* for a smooth solution the error decreases geometrically with P (spectral
  convergence).
Meshes are described in randomly rotated local frames so shared faces are met
in every orientation.
"""
import numpy as np
import pytest

import oracle as orc
import workloads as W
from oracle import conforming as cf


def _mesh(shape, n, g, amp, rotate, seed=0):
    d = 2 if shape == "quad" else 3
    if d == 2:
        nodes = W.quad_grid(n, n)
        g = 1
    else:
        nodes = W.hex_grid(n, g, amp=amp)
    verts = W.grid_vertices(n, d)
    if rotate:
        nodes, verts, _ = W.rotate_elements(nodes, verts, g, seed=seed)
    return nodes, verts, g


def _xq(shape, Q, g, nodes):
    return orc.geom_factors(shape, Q, g, nodes, with_x=True)[2]


@pytest.mark.parametrize("shape,n,P", [("quad", 3, 3), ("quad", 2, 4), ("hex", 2, 2), ("hex", 2, 3)])
@pytest.mark.parametrize("rotate", [False, True])
def test_dimension_closed_form(shape, n, P, rotate):
    d = 2 if shape == "quad" else 3
    nodes, verts, g = _mesh(shape, n, 1, 0.0, rotate, seed=P)
    Z = cf.conforming_basis(shape, P, verts, dirichlet=False)
    Z0 = cf.conforming_basis(shape, P, verts, dirichlet=True)
    assert Z.shape[1] == (n * P + 1) ** d
    assert Z0.shape[1] == (n * P - 1) ** d


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_projection_reproduces_constant_and_coordinates(shape):
    P, Q, n = 3, 5, 2
    g = 1 if shape == "quad" else 2          # isoparametric curved hexes (g <= P)
    nodes, verts, g = _mesh(shape, n, g, 0.05, rotate=True, seed=7)
    X = _xq(shape, Q, g, nodes)
    one = np.ones(X.shape[:2])
    u = cf.project(shape, P, Q, g, nodes, verts, one)
    assert np.abs(orc.bwd(shape, P, Q, u) - 1.0).max() < 1e-10
    for k in range(X.shape[2]):
        u = cf.project(shape, P, Q, g, nodes, verts, X[:, :, k])
        assert np.abs(orc.bwd(shape, P, Q, u) - X[:, :, k]).max() < 1e-10


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_quadratic_dirichlet_solution_is_exact(shape):
    P, Q, n, lam = 3, 5, 2, 1.5
    nodes, verts, g = _mesh(shape, n, 1, 0.0, rotate=True, seed=11)
    X = _xq(shape, Q, g, nodes)
    if shape == "quad":
        x, y = X[..., 0], X[..., 1]
        u = x * x - x * y + 2.0 * y * y + y
        lap = 2.0 + 4.0
    else:
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        u = x * x - x * y + 2.0 * z * z + y + 0.5 * y * z
        lap = 2.0 + 4.0
    f = -lap + lam * u
    sol, lift = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, f, u)
    assert np.abs(orc.bwd(shape, P, Q, sol) - u).max() < 1e-10
    # the lift alone is already the exact function (u is in the space)
    assert np.abs(orc.bwd(shape, P, Q, lift) - u).max() < 1e-10


def test_wrong_data_is_detected():
    """A dropped lambda term or a lift from the wrong data breaks exactness."""
    shape, P, Q, n, lam = "quad", 3, 5, 2, 1.5
    nodes, verts, g = _mesh(shape, n, 1, 0.0, rotate=True, seed=3)
    X = _xq(shape, Q, g, nodes)
    x, y = X[..., 0], X[..., 1]
    u = x * x + y
    sol, _ = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, -2.0 + 0.0 * u, u)  # lambda u dropped in f
    assert np.abs(orc.bwd(shape, P, Q, sol) - u).max() > 1e-3
    sol, _ = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, -2.0 + lam * u, u + 0.01)
    assert np.abs(orc.bwd(shape, P, Q, sol) - u).max() > 1e-3


def test_spectral_convergence_curved_hex():
    n, lam = 2, 1.0
    errs = []
    for P in (2, 3, 4, 5):
        Q = P + 2
        nodes, verts, g = _mesh("hex", n, P, 0.05, rotate=True, seed=P)
        X = _xq("hex", Q, g, nodes)
        u = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
        f = (3.0 * np.pi ** 2 + lam) * u
        sol, _ = cf.dirichlet_solve("hex", P, Q, g, nodes, verts, lam, f, u)
        errs.append(np.abs(orc.bwd("hex", P, Q, sol) - u).max())
    # geometric decrease (measured here: factors 4.5, 3.0, 4.9 on this 2^3 mesh);
    # a wrong lift or a broken face match stalls the error instead
    for a, b in zip(errs, errs[1:]):
        assert b < a / 2.0, errs
    assert errs[-1] < errs[0] / 30.0, errs


@pytest.mark.parametrize("shape,n,P", [("quad", 3, 3), ("hex", 2, 3)])
def test_nodal_space_dimension_and_quadratic_solve(shape, n, P):
    """The same closed-form dimensions and exact quadratic recovery in the
    nodal (GLL-Lagrange) basis."""
    d = 2 if shape == "quad" else 3
    nodes, verts, g = _mesh(shape, n, 1, 0.0, rotate=True, seed=5)
    assert cf.conforming_basis(shape, P, verts, False, "nodal").shape[1] == (n * P + 1) ** d
    assert cf.conforming_basis(shape, P, verts, True, "nodal").shape[1] == (n * P - 1) ** d
    from oracle import nodal as nd
    Q, lam = P + 2, 0.75
    X = _xq(shape, Q, g, nodes)
    u = X[..., 0] ** 2 + X[..., 0] * X[..., 1] - 0.5 * X[..., 1] + (X[..., 2] ** 2 if d == 3 else 0.0)
    lap = 2.0 + (2.0 if d == 3 else 0.0)
    sol, _ = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, -lap + lam * u, u, basis="nodal")
    assert np.abs(nd.bwd(shape, P, Q, sol) - u).max() < 1e-10


@pytest.mark.parametrize("shape,n,P,g", [("quad", 3, 4, 1), ("hex", 2, 3, 2)])
def test_nodal_and_modified_solutions_coincide(shape, n, P, g):
    """Both bases span the same conforming space, so the Galerkin solutions of
    one Dirichlet problem are the same function: equal at every quadrature
    point, on a curved mesh in rotated frames."""
    from oracle import nodal as nd
    d = 2 if shape == "quad" else 3
    nodes = W.quad_grid(n, n) if d == 2 else W.hex_grid(n, g, amp=0.05)
    nodes, verts, _ = W.rotate_elements(nodes, W.grid_vertices(n, d), g, seed=11)
    Q, lam = P + 2, 1.5
    X = _xq(shape, Q, g, nodes)
    u = np.prod(np.sin(np.pi * X), axis=-1)
    f = (d * np.pi ** 2 + lam) * u
    sn, _ = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, f, u, basis="nodal")
    sm, _ = cf.dirichlet_solve(shape, P, Q, g, nodes, verts, lam, f, u)
    vn, vm = nd.bwd(shape, P, Q, sn), orc.bwd(shape, P, Q, sm)
    assert np.abs(vn - vm).max() <= 1e-10 * np.abs(vm).max()
