"""Conforming (C0) spaces and global solves on quadrilateral / hexahedral meshes.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): used by ``tests/``,
never by the library.

Definition followed.  The paper's operators act on one element at a time and
its solve is stated without assembly (Sec. 2.1, Neumann boundaries); a global
C0 space is the standard spectral/hp construction the paper's elemental
operators are assembled into.  It is defined here WITHOUT any dof numbering or
orientation signs: a broken expansion (element-local coefficients x[e][m]) is
conforming when its traces agree on every face shared by two elements, i.e.
when

    sum_m phi_m(xi_1(s)) x[e1][m] = sum_m phi_m(xi_2(s)) x[e2][m]

at enough points s of the shared face to determine a polynomial of degree P
per direction; xi_1(s) and xi_2(s) are the two elements' reference coordinates
of the same face point, related by matching the face's corners through their
global vertex ids (the map between the two reference faces is one of the
symmetries of the square or segment, so bilinear interpolation of the corner
coordinates is exact).  The homogeneous-Dirichlet subspace additionally
vanishes at the points of every boundary face (a face owned by one element).
Both spaces are the null spaces of these point constraints, computed by SVD.

The global Helmholtz problem (L + lambda M) u = f with u = g on the boundary
is then solved in the affine space u_p + V_0, where u_p is the L2 projection of
g onto the conforming space (the Dirichlet lift):
    u = u_p + Z0 w,   Z0^T H Z0 w = Z0^T (b - H u_p),   b = B^T W f,
with H the block-diagonal matrix of the oracle's dense elemental matrices.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

import oracle as orc


def _face_list(d: int):
    """Reference faces (edges in 2-D) as (fixed axis, side, free axes)."""
    out = []
    for ax in range(d):
        for side in (0, 1):
            out.append((ax, side, [k for k in range(d) if k != ax]))
    return out


def _face_corners(d: int, ax: int, side: int, free):
    """Local vertex numbers of a reference face, indexed by the corner's bits
    along the free axes (first free axis fastest)."""
    out = []
    for t in range(2 ** (d - 1)):
        bits = [0] * d
        bits[ax] = side
        for k, fa in enumerate(free):
            bits[fa] = (t >> k) & 1
        out.append(sum(b << k for k, b in enumerate(bits)))
    return out


def _vertex_xi(d: int, v: int) -> np.ndarray:
    return np.array([-1.0 + 2.0 * ((v >> k) & 1) for k in range(d)])


def _face_samples(d: int, P: int) -> np.ndarray:
    """Sample points on [-1,1]^(d-1): P+2 Gauss-Legendre points per direction
    (more than the P+1 a degree-P polynomial needs)."""
    z, _ = np.polynomial.legendre.leggauss(P + 2)
    if d == 2:
        return z[:, None]
    b, a = np.meshgrid(z, z, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


def _bilinear(s: np.ndarray, corners: np.ndarray) -> np.ndarray:
    """Interpolate corner coordinates [2^(d-1)][d] at face parameters s [n][d-1]."""
    n, k = s.shape
    out = np.zeros((n, corners.shape[1]))
    for t in range(2 ** k):
        w = np.ones(n)
        for j in range(k):
            bj = (t >> j) & 1
            w = w * (0.5 * (1.0 + s[:, j]) if bj else 0.5 * (1.0 - s[:, j]))
        out += w[:, None] * corners[t][None, :]
    return out


def faces_of(verts: np.ndarray):
    """Map frozenset(global corner ids) -> list of (element, face tuple)."""
    d = int(round(np.log2(verts.shape[1])))
    table = {}
    for e in range(verts.shape[0]):
        for f in _face_list(d):
            key = frozenset(int(verts[e, v]) for v in _face_corners(d, *f))
            table.setdefault(key, []).append((e, f))
    return table


def _basis_at(shape, P, xi, basis):
    if basis == "nodal":
        from oracle import nodal
        return nodal.eval_basis(shape, P, xi)
    return orc.eval_basis(shape, P, xi)[0]


def constraints(shape: str, P: int, verts: np.ndarray, dirichlet: bool, basis: str = "modified") -> np.ndarray:
    """Rows C with C x = 0 exactly for the conforming (and, with ``dirichlet``,
    boundary-vanishing) broken expansions x (flattened [E][M]) in the modified
    or the nodal (GLL-Lagrange) basis."""
    d = orc.dim(shape)
    E, M = verts.shape[0], orc.num_modes(shape, P)
    s = _face_samples(d, P)
    rows = []
    for key, owners in faces_of(verts).items():
        if len(owners) > 2:
            raise ValueError("non-manifold face")
        e1, f1 = owners[0]
        c1 = _face_corners(d, *f1)
        xi1 = _bilinear(s, np.stack([_vertex_xi(d, v) for v in c1]))
        B1 = _basis_at(shape, P, xi1, basis)
        if len(owners) == 2:
            e2, f2 = owners[1]
            c2 = _face_corners(d, *f2)
            # element 2's reference corners listed in element 1's corner order
            pos2 = {int(verts[e2, v]): v for v in c2}
            xi2 = _bilinear(s, np.stack([_vertex_xi(d, pos2[int(verts[e1, v])]) for v in c1]))
            B2 = _basis_at(shape, P, xi2, basis)
            R = np.zeros((s.shape[0], E * M))
            R[:, e1 * M:(e1 + 1) * M] = B1
            R[:, e2 * M:(e2 + 1) * M] -= B2
            rows.append(R)
        elif dirichlet:
            R = np.zeros((s.shape[0], E * M))
            R[:, e1 * M:(e1 + 1) * M] = B1
            rows.append(R)
    if not rows:
        return np.zeros((0, E * M))
    return np.concatenate(rows, axis=0)


def conforming_basis(shape: str, P: int, verts: np.ndarray, dirichlet: bool, basis: str = "modified") -> np.ndarray:
    """Orthonormal basis Z [E*M][n] of the conforming (homogeneous-Dirichlet)
    space, as the numerical null space of ``constraints``."""
    C = constraints(shape, P, verts, dirichlet, basis)
    if C.shape[0] == 0:
        return np.eye(C.shape[1])
    return sla.null_space(C, rcond=1e-9)


def block_matrix(mats: np.ndarray) -> np.ndarray:
    """Block-diagonal matrix of [E][M][M] elemental matrices."""
    return sla.block_diag(*mats)


def _ops(basis):
    """(mass matrices, Helmholtz matrices, IProductWRTBase) of the chosen basis."""
    if basis == "nodal":
        from oracle import nodal
        return nodal.mass_matrices, nodal.helmholtz_matrices, nodal.iprod
    return _mass_modified, orc.helmholtz_matrix, orc.iprod


def _mass_modified(shape, P, Q, gorder, nodes) -> np.ndarray:
    B, _ = orc.ref_basis(shape, P, Q)
    W, _, _ = orc.geom_factors(shape, Q, gorder, nodes)
    return np.einsum("nm,en,nk->emk", B, W, B)


def mass_matrices(shape, P, Q, gorder, nodes, basis: str = "modified") -> np.ndarray:
    """Dense elemental mass matrices B^T diag(W_e) B, [E][M][M]."""
    return _ops(basis)[0](shape, P, Q, gorder, nodes)


def project(shape, P, Q, gorder, nodes, verts, g_phys, basis: str = "modified") -> np.ndarray:
    """L2 projection onto the conforming space of values g at the quadrature
    points [E][Nq]; returns the local coefficients [E][M]."""
    Z = conforming_basis(shape, P, verts, dirichlet=False, basis=basis)
    Mb = block_matrix(mass_matrices(shape, P, Q, gorder, nodes, basis))
    rhs = _ops(basis)[2](shape, P, Q, gorder, nodes, g_phys).ravel()
    y = np.linalg.solve(Z.T @ Mb @ Z, Z.T @ rhs)
    return (Z @ y).reshape(nodes.shape[0], -1)


def dirichlet_solve(shape, P, Q, gorder, nodes, verts, lam, f_phys, g_phys, basis: str = "modified"):
    """Global (L + lambda M) u = f, u = g on the boundary (g through its L2
    projection).  Returns (u, u_p): local coefficients [E][M] of the solution
    and of the lift."""
    E = nodes.shape[0]
    _, helm, iprod = _ops(basis)
    u_p = project(shape, P, Q, gorder, nodes, verts, g_phys, basis)
    H = block_matrix(helm(shape, P, Q, gorder, nodes, lam))
    b = iprod(shape, P, Q, gorder, nodes, f_phys).ravel()
    Z0 = conforming_basis(shape, P, verts, dirichlet=True, basis=basis)
    A = Z0.T @ H @ Z0
    w = sla.cho_solve(sla.cho_factor(A), Z0.T @ (b - H @ u_p.ravel()))
    return (u_p.ravel() + Z0 @ w).reshape(E, -1), u_p
