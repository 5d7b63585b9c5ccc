"""Seeded synthetic workloads for the spectral/hp operator benchmarks and tests.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA library (``paper_2606_20917_gb300``).  It produces *inputs* only: element
geometry (vertex or lattice-node coordinates), expansion coefficients and
physical-space samples.  It contains no quadrature, no basis functions and no
operator arithmetic; each side derives those from the node coordinates with its
own code.

Geometry conventions (the element maps both sides must implement):

* quad / hex: a tensor lattice of ``(g+1)**d`` equispaced nodes per element,
  node ``a + (g+1)*b (+ (g+1)**2*c)`` sitting at reference coordinate
  ``xi = -1 + 2*(a, b, c)/g``; the element map is the tensor Lagrange
  interpolant through these nodes (degree ``g`` per direction).
* tri: vertices V0=(-1,-1), V1=(1,-1), V2=(-1,1) (affine map).
* tet: vertices V0=(-1,-1,-1), V1=(1,-1,-1), V2=(-1,1,-1), V3=(-1,-1,1).
* prism: the triangle lives in the (xi1, xi3) plane and is extruded along xi2:
  V0=(-1,-1,-1), V1=(1,-1,-1), V2=(1,1,-1), V3=(-1,1,-1), V4=(-1,-1,1),
  V5=(-1,1,1); the map is linear in the triangle and in xi2.
* pyr: base V0=(-1,-1,-1), V1=(1,-1,-1), V2=(1,1,-1), V3=(-1,1,-1), apex
  V4=(-1,-1,1); the map is that of the five vertex functions (affine when
  the base is a parallelogram, as in ``pyramid_split``).

The curved hexahedral meshes use the periodic displacement
``x = X + a sin(2 pi Y) sin(2 pi Z)`` with the same formula permuted cyclically
for y and z, evaluated at the lattice nodes (a = 0.05 on the unit cube).
"""
from __future__ import annotations

import numpy as np

SHAPES = ("quad", "tri", "hex", "prism", "tet")
DIM = {"quad": 2, "tri": 2, "hex": 3, "prism": 3, "tet": 3}
NVERT = {"tri": 3, "tet": 4, "prism": 6, "pyr": 5}


def lattice_offsets(g: int, d: int) -> np.ndarray:
    """Unit-cube offsets (a/g, b/g, c/g) of the equispaced lattice, a fastest."""
    t = np.arange(g + 1, dtype=np.float64) / g
    if d == 2:
        b, a = np.meshgrid(t, t, indexing="ij")
        return np.stack([a.ravel(), b.ravel()], axis=1)
    c, b, a = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def sine_map(X: np.ndarray, amp: float) -> np.ndarray:
    """Periodic cyclic displacement of the unit cube (identity when amp == 0)."""
    if amp == 0.0:
        return X.copy()
    tp = 2.0 * np.pi
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    out = np.empty_like(X)
    out[..., 0] = x + amp * np.sin(tp * y) * np.sin(tp * z)
    out[..., 1] = y + amp * np.sin(tp * z) * np.sin(tp * x)
    out[..., 2] = z + amp * np.sin(tp * x) * np.sin(tp * y)
    return out


def quad_grid(nx: int, ny: int) -> np.ndarray:
    """Affine quads of a regular nx-by-ny grid on [0,1]^2; nodes [E][4][2] (g=1)."""
    off = lattice_offsets(1, 2)
    hx, hy = 1.0 / nx, 1.0 / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    org = np.stack([ii.ravel() * hx, jj.ravel() * hy], axis=1)
    return (org[:, None, :] + off[None, :, :] * np.array([hx, hy])).astype(np.float64)


def hex_grid(n: int, g: int, amp: float = 0.05, count: int | None = None) -> np.ndarray:
    """Hexahedra of an n^3 grid on [0,1]^3 mapped by ``sine_map``.

    Returns lattice nodes [E][(g+1)^3][3] (element index x fastest).  With
    ``count`` only the first ``count`` cells are returned.
    """
    off = lattice_offsets(g, 3)
    h = 1.0 / n
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    org = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1) * h
    if count is not None:
        org = org[:count]
    X = org[:, None, :] + off[None, :, :] * h
    return sine_map(X, amp)


def _cube_corners(nx, ny, nz):
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (np.stack([ii.ravel() / nx, jj.ravel() / ny, kk.ravel() / nz], axis=1),
            np.array([1.0 / nx, 1.0 / ny, 1.0 / nz]))


def tet_kuhn(nx: int, ny: int | None = None, nz: int | None = None) -> np.ndarray:
    """Each cube of an nx*ny*nz grid split into 6 tets along its main diagonal.

    Vertices [E][4][3], ordered so the affine map from the reference tet has a
    positive Jacobian determinant.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    org, h = _cube_corners(nx, ny, nz)
    e = np.eye(3)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for a, b, c in perms:
        v0 = np.zeros(3)
        v1 = e[a]
        v2 = e[a] + e[b]
        v3 = np.ones(3)
        vs = np.stack([v0, v1, v2, v3])
        if np.linalg.det(np.stack([v1 - v0, v2 - v0, v3 - v0], axis=1)) < 0:
            vs = vs[[0, 2, 1, 3]]
        tets.append(vs)
    ref = np.stack(tets)  # [6][4][3] in the unit cube
    V = org[:, None, None, :] + ref[None, :, :, :] * h
    return V.reshape(-1, 4, 3).astype(np.float64)


def prism_split(nx: int, ny: int, nz: int) -> np.ndarray:
    """Each cell of an nx*ny*nz grid split into 2 prisms across an x-z face diagonal.

    The prism's triangle lies in the x-z plane and is extruded along y.
    Vertices [E][6][3] in the reference order V0..V5, positively oriented.
    """
    org, h = _cube_corners(nx, ny, nz)
    tris = [np.array([[0, 0], [1, 0], [0, 1]], float),   # (x, z) corners
            np.array([[1, 1], [0, 1], [1, 0]], float)]
    def xyz(p, y):
        return np.array([p[0], y, p[1]])

    def corners(a, b, c):
        return np.stack([xyz(a, 0), xyz(b, 0), xyz(b, 1), xyz(a, 1), xyz(c, 0), xyz(c, 1)])

    ref = []
    for a, b, c in tris:
        v = corners(a, b, c)
        # Jacobian columns (up to 1/2): V1-V0, V3-V0, V4-V0
        if np.linalg.det(np.stack([v[1] - v[0], v[3] - v[0], v[4] - v[0]], axis=1)) < 0:
            v = corners(a, c, b)
        ref.append(v)
    ref = np.stack(ref)
    V = org[:, None, None, :] + ref[None] * h
    return V.reshape(-1, 6, 3).astype(np.float64)


def pyramid_split(nx: int, ny: int, nz: int) -> np.ndarray:
    """Each cell of an nx*ny*nz grid split into 6 pyramids, one per face, with
    their apex at the cell centre (each pyramid over a square: affine).

    Vertices [E][5][3]: the base (V0..V3) counter-clockwise seen from the apex
    (V4), the reference order, so every element is positively oriented.
    """
    org, h = _cube_corners(nx, ny, nz)
    pyrs = []
    for axis in range(3):
        for side in (0.0, 1.0):
            quad = []
            for a, b in ((0, 0), (1, 0), (1, 1), (0, 1)):
                v = [0.0, 0.0, 0.0]
                v[axis] = side
                v[(axis + 1) % 3] = a
                v[(axis + 2) % 3] = b
                quad.append(v)
            quad = np.array(quad)
            apex = np.array([0.5, 0.5, 0.5])
            if np.linalg.det(np.stack([quad[1] - quad[0], quad[3] - quad[0], apex - quad[0]])) < 0:
                quad = quad[[0, 3, 2, 1]]
            pyrs.append(np.vstack([quad, apex]))
    local = np.stack(pyrs)                                    # [6][5][3] in the unit cube
    return (org[:, None, None, :] + h * local[None]).reshape(-1, 5, 3)


def tri_grid(nx: int, ny: int) -> np.ndarray:
    """Each square of an nx-by-ny grid on [0,1]^2 split into 2 triangles."""
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    org = np.stack([ii.ravel() / nx, jj.ravel() / ny], axis=1)
    h = np.array([1.0 / nx, 1.0 / ny])
    ref = np.array([[[0, 0], [1, 0], [0, 1]], [[1, 1], [0, 1], [1, 0]]], float)
    V = org[:, None, None, :] + ref[None] * h
    return V.reshape(-1, 3, 2).astype(np.float64)


def perturb_vertices(V: np.ndarray, scale: float, seed: int) -> np.ndarray:
    """Random affine distortion of each element (keeps orientation for small scale)."""
    rng = np.random.default_rng(seed)
    d = V.shape[-1]
    A = np.eye(d)[None] + scale * rng.uniform(-1, 1, size=(V.shape[0], d, d))
    c = V.mean(axis=1, keepdims=True)
    return np.einsum("eij,evj->evi", A, V - c) + c


def coefficients(E: int, M: int, seed: int = 0) -> np.ndarray:
    """Expansion coefficients uniform on [-1, 1], element-major [E][M]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(E, M))


def phys_samples(E: int, Nq: int, seed: int = 1, ncomp: int = 1) -> np.ndarray:
    """Physical-space values uniform on [-1, 1]: [E][Nq] or [ncomp][E][Nq]."""
    rng = np.random.default_rng(seed)
    if ncomp == 1:
        return rng.uniform(-1.0, 1.0, size=(E, Nq))
    return rng.uniform(-1.0, 1.0, size=(ncomp, E, Nq))


def sample_elements(E: int, k: int, seed: int = 0) -> np.ndarray:
    """Sorted seeded sample of k distinct element ids (all ids if k >= E)."""
    if k >= E:
        return np.arange(E)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(E, size=k, replace=False))


# --- the named workloads -------------------------------------------------------

def workload(name: str) -> dict:
    """Geometry of a named workload: dict(shape, P, Q, gorder, nodes, deformed)."""
    if name == "quad8x8_p4":
        return dict(shape="quad", P=4, Q=6, gorder=1, nodes=quad_grid(8, 8), deformed=False)
    if name == "hex32_curved_p4":
        return dict(shape="hex", P=4, Q=6, gorder=4, nodes=hex_grid(32, 4), deformed=True)
    if name == "tet20_kuhn_p4":
        return dict(shape="tet", P=4, Q=6, gorder=1, nodes=tet_kuhn(20), deformed=False)
    if name == "prism40x40x20_p4":
        return dict(shape="prism", P=4, Q=6, gorder=1, nodes=prism_split(40, 40, 20), deformed=False)
    if name == "pyr20_split_p4":
        return dict(shape="pyr", P=4, Q=6, gorder=1, nodes=pyramid_split(20, 20, 20), deformed=False)
    if name == "hex48_curved_p6":
        return dict(shape="hex", P=6, Q=8, gorder=6, nodes=hex_grid(48, 6), deformed=True)
    if name == "tet12_kuhn_p8":   # high-order tets (the sweep's weakest FP32 point), for profiling
        return dict(shape="tet", P=8, Q=10, gorder=1, nodes=tet_kuhn(12), deformed=False)
    raise KeyError(name)


def hybrid_mesh(seed: int = 0, scale: int = 1) -> list[dict]:
    """Hybrid mesh of ~150k elements (hex:prism:tet = 2:1:3), P ~ U{2..8}, Q = P+2.

    Hexes are curved cells of a 37^3 grid (first 50000), prisms split 25x25x20
    cells, tets Kuhn-split 25x25x20 cells.  Elements are grouped into blocks of
    equal (shape, P).  ``scale`` > 1 divides every element count (small tests).
    Returns a list of dict(shape, P, Q, gorder, nodes, deformed).
    """
    rng = np.random.default_rng(seed)
    parts = [("hex", hex_grid(37, 2, count=50000 // scale), True),
             ("prism", prism_split(25, 25, 20 // scale if scale <= 20 else 1), False),
             ("tet", tet_kuhn(25, 25, 20 // scale if scale <= 20 else 1), False)]
    blocks = []
    for shape, nodes, deformed in parts:
        Ps = rng.integers(2, 9, size=nodes.shape[0])
        for P in range(2, 9):
            sel = np.nonzero(Ps == P)[0]
            if sel.size == 0:
                continue
            nd = nodes[sel]
            g = 2 if shape == "hex" else 1   # curved hexes carry a degree-2 lattice
            blocks.append(dict(shape=shape, P=int(P), Q=int(P) + 2, gorder=g,
                               nodes=np.ascontiguousarray(nd), deformed=deformed))
    return blocks


# --- conforming meshes (vertex connectivity) --------------------------------------

def grid_vertices(n: int, d: int, count: int | None = None) -> np.ndarray:
    """Global vertex ids of the cells of an n^d grid, in the cell order of
    ``quad_grid(n, n)`` / ``hex_grid(n, g)`` (x fastest).

    Local vertex v = a + 2b (+ 4c) sits at reference xi = (-1 + 2a, -1 + 2b(, -1 + 2c));
    global vertex (I, J(, K)) has id I + (n+1)(J + (n+1)K).  Returns int64 [E][2^d].
    """
    cells = np.arange(n ** d)
    ci = [(cells // n ** k) % n for k in range(d)]
    out = np.zeros((cells.size, 2 ** d), dtype=np.int64)
    for v in range(2 ** d):
        bits = [(v >> k) & 1 for k in range(d)]
        gid = np.zeros(cells.size, dtype=np.int64)
        for k in range(d - 1, -1, -1):
            gid = gid * (n + 1) + ci[k] + bits[k]
        out[:, v] = gid
    return out if count is None else out[:count]


def _rotations(d: int) -> list[np.ndarray]:
    """Signed permutation matrices of determinant +1 (the proper symmetries of
    the reference square or cube)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(d)):
        for signs in itertools.product((1, -1), repeat=d):
            R = np.zeros((d, d))
            for i in range(d):
                R[i, perm[i]] = signs[i]
            if np.linalg.det(R) > 0.5:
                out.append(R)
    return out


def rotate_elements(nodes: np.ndarray, verts: np.ndarray, g: int, seed: int = 0):
    """Re-describe every element in a randomly rotated local frame.

    Element e gets a proper symmetry R_e of the reference element; its new
    local point xi' is the old local point R_e xi'.  The lattice nodes [E][(g+1)^d][d]
    and the vertex ids [E][2^d] are permuted accordingly, so the physical
    elements are unchanged while neighbouring elements see their shared faces
    in different orientations.  Returns (nodes, verts, rotation index per element).
    """
    d = nodes.shape[-1]
    rots = _rotations(d)
    rng = np.random.default_rng(seed)
    which = rng.integers(0, len(rots), size=nodes.shape[0])

    def index_map(gg):
        t = np.arange(gg + 1)
        grids = np.meshgrid(*([t] * d), indexing="ij")  # grids[k][..] = index along axis k
        new_idx = np.stack([gr.ravel() for gr in grids], axis=1)  # rows: (a0, a1, ...) new indices
        maps = []
        for R in rots:
            xi_new = -1.0 + 2.0 * new_idx / gg
            xi_old = xi_new @ R.T
            old_idx = np.rint((xi_old + 1.0) * gg / 2.0).astype(np.int64)
            lin_new = sum(new_idx[:, k] * (gg + 1) ** k for k in range(d))
            lin_old = sum(old_idx[:, k] * (gg + 1) ** k for k in range(d))
            m = np.empty((gg + 1) ** d, dtype=np.int64)
            m[lin_new] = lin_old
            maps.append(m)
        return maps

    nmap, vmap = index_map(g), index_map(1)
    new_nodes = np.empty_like(nodes)
    new_verts = np.empty_like(verts)
    for r in range(len(rots)):
        sel = np.nonzero(which == r)[0]
        if sel.size:
            new_nodes[sel] = nodes[sel][:, nmap[r], :]
            new_verts[sel] = verts[sel][:, vmap[r]]
    return new_nodes, new_verts, which


def shard_parts(parts: list[dict], first: list[int], rank: int) -> list[dict]:
    """The blocks of rank `rank` of a mesh split into contiguous element ranges
    (first[r] .. first[r+1] over the concatenation of `parts` in block order):
    each part that overlaps the rank's range is cut to the overlap (its nodes
    sliced; every other key kept), empty overlaps dropped.  Also records the
    global element offset of each cut as "global_first"."""
    lo, hi = first[rank], first[rank + 1]
    out, off = [], 0
    for p in parts:
        n = p["nodes"].shape[0]
        a, b = max(lo, off), min(hi, off + n)
        if a < b:
            q = dict(p)
            q["nodes"] = np.ascontiguousarray(p["nodes"][a - off:b - off])
            q["global_first"] = a
            out.append(q)
        off += n
    return out
