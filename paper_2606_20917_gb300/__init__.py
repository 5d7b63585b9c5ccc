"""Python binding of the GB300 spectral/hp elemental-operator library (libnir.so).

Argument marshalling only: every operator runs in the library's CUDA kernels.
PyTorch provides device memory and the stream; tensors are passed by
``data_ptr()``.  There is no CPU fallback: importing this package without a
built ``libnir.so`` raises.

    ctx = Context()                                   # device 0, current torch stream
    blk = Block(ctx, "hex", nelem, P=4, deformed=True)
    blk.set_geometry(gorder, nodes_f64_cuda)          # [E][(g+1)^3][3]
    y = blk.helmholtz(u, lam=1.0)                     # u: [E][M] cuda tensor
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnir.so")
SHAPES = {"quad": 0, "tri": 1, "hex": 2, "prism": 3, "tet": 4, "pyr": 5}
DIM = {"quad": 2, "tri": 2, "hex": 3, "prism": 3, "tet": 3, "pyr": 3}
PREC = {"f64": 0, "f32": 1, "bf16": 2}
DTYPE = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run `python paper_2606_20917_gb300/build.py` "
                      "(the library has no CPU fallback)")

_lib = C.CDLL(LIB_PATH)
_vp, _i, _d, _i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64


class BlockDesc(C.Structure):
    _fields_ = [("shape", C.c_int), ("nelem", C.c_int64), ("P", C.c_int), ("Q", C.c_int),
                ("deformed", C.c_int), ("basis", C.c_int)]


BASIS = {"modified": 0, "nodal": 1}


class CGOpts(C.Structure):
    _fields_ = [("inner_prec", C.c_int), ("tol", C.c_double), ("max_outer", C.c_int),
                ("max_inner", C.c_int), ("inner_tol", C.c_double), ("jacobi", C.c_int),
                ("inner_vectors", C.c_int), ("fwd_tol", C.c_double)]


class CGStats(C.Structure):
    _fields_ = [("outer", C.c_int), ("inner_total", C.c_int), ("rel_residual", C.c_double),
                ("seconds", C.c_double), ("rel_correction", C.c_double)]


def _cg_opts(inner_prec, tol, max_outer, max_inner, inner_tol, jacobi, inner_vectors, fwd_tol):
    return CGOpts(PREC[inner_prec], float(tol), int(max_outer), int(max_inner), float(inner_tol), int(jacobi),
                  PREC[inner_vectors], float(fwd_tol))


def _cg_stats(s):
    return dict(outer=s.outer, inner_total=s.inner_total, rel_residual=s.rel_residual, seconds=s.seconds,
                rel_correction=s.rel_correction)


_SIGS = {
    "nir_ctx_create": [C.POINTER(_vp), _i, _vp],
    "nir_ctx_set_stream": [_vp, _vp],
    "nir_ctx_check": [_vp],
    "nir_block_create": [_vp, C.POINTER(BlockDesc), C.POINTER(_vp)],
    "nir_block_num_modes": [_vp, C.POINTER(_i64)],
    "nir_block_num_points": [_vp, C.POINTER(_i64)],
    "nir_block_points": [_vp, _vp, _vp],
    "nir_block_set_geometry": [_vp, _i, _vp],
    "nir_block_set_geometric_factors": [_vp, _i, _vp, _vp],
    "nir_bwd_trans": [_vp, _i, _vp, _vp],
    "nir_iproduct_wrt_base": [_vp, _i, _vp, _vp],
    "nir_phys_deriv": [_vp, _i, _vp, _vp, _vp, _vp],
    "nir_iproduct_wrt_deriv_base": [_vp, _i, _vp, _vp, _vp, _vp],
    "nir_mass": [_vp, _i, _vp, _vp],
    "nir_helmholtz": [_vp, _i, _d, _vp, _vp],
    "nir_helmholtz_host": [_vp, _i, _d, _vp, _vp],
    "nir_helmholtz_fields": [_vp, _i, _d, _i, C.POINTER(_vp), C.POINTER(_vp)],
    "nir_block_set_tuning": [_vp, _i, _i, _i, _i],
    "nir_block_kernel_info": [_vp, _i, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "nir_block_get_tuning": [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "nir_mesh_create": [_vp, C.POINTER(_vp), _i, C.POINTER(_vp)],
    "nir_mesh_num_dofs": [_vp, C.POINTER(_i64)],
    "nir_mesh_helmholtz": [_vp, _i, _d, _vp, _vp],
    "nir_tune": [_vp, C.c_char_p],
    "nir_mesh_set_launch": [_vp, _i, _i],
    "nir_mesh_get_launch": [_vp, _i, C.POINTER(_i)],
    "nir_cg_solve": [_vp, _d, _vp, _vp, C.POINTER(CGOpts), C.POINTER(CGStats)],
    "nir_probe_fp64_peak": [_vp, C.POINTER(_d)],
    "nir_probe_fp64_mma_peak": [_vp, C.POINTER(_d)],
    "nir_ctx_selftest_wait": [_vp, _i64],
    "nir_ctx_set_debug": [_vp, C.c_int],
    "nir_ctx_get_debug": [_vp, C.POINTER(C.c_int)],
    "nir_cg_solve_dist": [_vp, _d, _vp, _vp, C.POINTER(CGOpts), C.POINTER(CGStats), _vp, _vp],
    "nir_partition_elements": [_i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i64), _i, C.POINTER(_i64)],
    "nir_asm_create": [_vp, C.POINTER(_vp), C.POINTER(_vp), _i, C.POINTER(_vp)],
    "nir_asm_num_dofs": [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)],
    "nir_asm_local_map": [_vp, _vp],
    "nir_asm_gather": [_vp, _i, _vp, _vp],
    "nir_asm_assemble": [_vp, _i, _vp, _vp],
    "nir_asm_pick": [_vp, _vp, _vp],
    "nir_asm_apply": [_vp, _i, _d, _i, _vp, _vp],
    "nir_asm_cg_solve": [_vp, _i, _d, _i, _vp, _vp, C.POINTER(CGOpts), C.POINTER(CGStats)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _i
for _name in ("nir_ctx_destroy", "nir_block_destroy", "nir_mesh_destroy", "nir_asm_destroy"):
    getattr(_lib, _name).argtypes = [_vp]
    getattr(_lib, _name).restype = None
_lib.nir_strerror.argtypes = [_i]
_lib.nir_strerror.restype = C.c_char_p
_lib.nir_version.restype = C.c_char_p


# nir_allreduce_fn: int (*)(double *values, int n, void *user)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p)


def partition_elements(blocks, nranks: int) -> list[int]:
    """Contiguous cost-balanced element ranges (nir_partition_elements) of
    blocks given as (shape, P, nelem) in block order: returns first[nranks + 1];
    rank r owns global elements [first[r], first[r + 1]).  Host only."""
    nb = len(blocks)
    sh = (C.c_int * nb)(*[SHAPES[b[0]] for b in blocks])
    pp = (C.c_int * nb)(*[int(b[1]) for b in blocks])
    ne = (_i64 * nb)(*[int(b[2]) for b in blocks])
    out = (_i64 * (nranks + 1))()
    _chk(_lib.nir_partition_elements(nb, sh, pp, ne, int(nranks), out), "nir_partition_elements")
    return list(out)


def _allreduce_callback(fn):
    """Wrap fn(values: numpy float64 array) -> None (in-place sum over ranks)
    as a nir_allreduce_fn; an exception becomes a non-zero return."""
    import numpy as np

    def cb(values, n, user):
        try:
            arr = np.ctypeslib.as_array(values, shape=(n,))
            fn(arr)
            return 0
        except Exception:  # noqa: BLE001 -- reported to the library as a failed reduction
            return 1
    return ALLREDUCE_FN(cb)


class NirError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_lib.nir_strerror(code).decode()} ({code})")
        self.code = code


def _chk(rc: int, what: str):
    if rc != 0:
        raise NirError(rc, what)


def lib():
    return _lib


def version() -> str:
    return _lib.nir_version().decode()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """A device plus the CUDA stream every call is issued on."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = device
        with torch.cuda.device(device):
            h = _vp()
            _chk(_lib.nir_ctx_create(C.byref(h), device, _stream_handle(stream)), "nir_ctx_create")
        self.h = h

    def set_stream(self, stream: torch.cuda.Stream):
        _chk(_lib.nir_ctx_set_stream(self.h, _stream_handle(stream)), "nir_ctx_set_stream")

    def check(self):
        """Synchronise and raise if a kernel reported a device-side failure."""
        _chk(_lib.nir_ctx_check(self.h), "nir_ctx_check")

    def probe_fp64_peak(self) -> float:
        v = _d()
        _chk(_lib.nir_probe_fp64_peak(self.h, C.byref(v)), "nir_probe_fp64_peak")
        return v.value

    def probe_fp64_mma_peak(self) -> float:
        """FP64 tensor-core (DMMA) throughput in TFLOP/s."""
        v = _d()
        _chk(_lib.nir_probe_fp64_mma_peak(self.h, C.byref(v)), "nir_probe_fp64_mma_peak")
        return v.value

    @property
    def debug(self) -> bool:
        """Debug mode: every device-buffer operator call synchronises and
        raises at the call whose kernel (or earlier stream work) failed.
        Initially on when the environment variable NIR_DEBUG is set and not "0"."""
        v = C.c_int(0)
        _chk(_lib.nir_ctx_get_debug(self.h, C.byref(v)), "nir_ctx_get_debug")
        return bool(v.value)

    @debug.setter
    def debug(self, on: bool):
        _chk(_lib.nir_ctx_set_debug(self.h, 1 if on else 0), "nir_ctx_set_debug")

    def selftest_wait(self, limit_cycles: int):
        """Launch the bounded-wait self-test (see nir_ctx_selftest_wait); the
        next check() raises NIR_ERR_CUDA."""
        _chk(_lib.nir_ctx_selftest_wait(self.h, int(limit_cycles)), "nir_ctx_selftest_wait")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.nir_ctx_destroy(h)
            self.h = None


class Block:
    """A block of alike elements (shape, P, Q = P + 2, deformed flag)."""

    def __init__(self, ctx: Context, shape: str, nelem: int, P: int, Q: int | None = None,
                 deformed: bool = False, basis: str = "modified"):
        """basis: "modified" (every shape) or "nodal" (GLL-Lagrange, quad/hex)."""
        self.ctx, self.shape, self.nelem, self.P = ctx, shape, int(nelem), int(P)
        self.Q = int(P) + 2 if Q is None else int(Q)
        self.dim = DIM[shape]
        self.basis = basis
        d = BlockDesc(SHAPES[shape], self.nelem, self.P, self.Q, int(bool(deformed)), BASIS[basis])
        h = _vp()
        _chk(_lib.nir_block_create(ctx.h, C.byref(d), C.byref(h)), "nir_block_create")
        self.h = h
        m, n = _i64(), _i64()
        _chk(_lib.nir_block_num_modes(h, C.byref(m)), "num_modes")
        _chk(_lib.nir_block_num_points(h, C.byref(n)), "num_points")
        self.M, self.NQ = m.value, n.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.nir_block_destroy(h)
            self.h = None

    def set_tuning(self, prec: str, variant: int = 0, grid: int = 0, pf: int = 0):
        """Force the Helmholtz launch tuning in one precision (see nir_block_set_tuning;
        variant 4 = the threading-over-elements kernel, grid in CTAs of 128 threads)."""
        _chk(_lib.nir_block_set_tuning(self.h, PREC[prec], int(variant), int(grid), int(pf)), "set_tuning")

    def get_tuning(self, prec: str):
        v, g, p = _i(), _i(), _i()
        _chk(_lib.nir_block_get_tuning(self.h, PREC[prec], C.byref(v), C.byref(g), C.byref(p)), "get_tuning")
        return v.value, g.value, p.value

    OPS = {"bwd": 0, "iprod": 1, "physderiv": 2, "iprod_deriv": 3, "mass": 4, "helm": 5}

    def kernel_info(self, prec: str = "f64", op: str = "helm") -> dict:
        """Registers, shared memory, threads and elements per CTA of the kernel this
        block launches for `op` (with its current tuning)."""
        r, sm, t, e = _i(), _i(), _i(), _i()
        _chk(_lib.nir_block_kernel_info(self.h, PREC[prec], self.OPS[op], C.byref(r), C.byref(sm), C.byref(t),
                                        C.byref(e)), "nir_block_kernel_info")
        return {"registers": r.value, "smem_bytes": sm.value, "threads": t.value, "elems_per_cta": e.value}

    def points(self):
        import numpy as np
        eta = np.zeros((self.NQ, self.dim))
        xi = np.zeros((self.NQ, self.dim))
        _chk(_lib.nir_block_points(self.h, eta.ctypes.data_as(_vp), xi.ctypes.data_as(_vp)), "points")
        return eta, xi

    def set_geometry(self, gorder: int, nodes: torch.Tensor):
        nodes = self._dev(nodes, torch.float64, "nodes")
        if self.shape in ("quad", "hex"):
            npe = (int(gorder) + 1) ** self.dim
        else:
            npe = {"tri": 3, "tet": 4, "prism": 6, "pyr": 5}[self.shape]
        if nodes.numel() != self.nelem * npe * self.dim:
            raise ValueError(f"nodes must be [{self.nelem}][{npe}][{self.dim}]")
        _chk(_lib.nir_block_set_geometry(self.h, int(gorder), _ptr(nodes)), "nir_block_set_geometry")

    def set_geometric_factors(self, dxi_dx: torch.Tensor, jac: torch.Tensor, per_element: bool = False):
        """Geometry from d xi/d x and |J| (FP64 CUDA tensors): per point
        [E][Nq][d][d] and [E][Nq], or per element [E][d][d] and [E]."""
        dxi_dx = self._dev(dxi_dx, torch.float64, "dxi_dx")
        jac = self._dev(jac, torch.float64, "jac")
        units = self.nelem * (1 if per_element else self.NQ)
        if dxi_dx.numel() != units * self.dim * self.dim or jac.numel() != units:
            raise ValueError(f"dxi_dx must hold {units} x {self.dim} x {self.dim} values and jac {units}")
        _chk(_lib.nir_block_set_geometric_factors(self.h, int(bool(per_element)), _ptr(dxi_dx), _ptr(jac)),
             "nir_block_set_geometric_factors")

    # -- helpers
    def _dev(self, t, dtype, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _chk_shape(self, t, n, name):
        if t.numel() != self.nelem * n:
            raise ValueError(f"{name} must hold {self.nelem} x {n} values")

    def _out(self, n, prec, out):
        if out is None:
            return torch.empty((self.nelem, n), dtype=DTYPE[prec], device=f"cuda:{self.ctx.device}")
        self._dev(out, DTYPE[prec], "out")
        self._chk_shape(out, n, "out")
        return out

    # -- operators
    def bwd_trans(self, coeff, prec="f64", out=None):
        self._dev(coeff, DTYPE[prec], "coeff"); self._chk_shape(coeff, self.M, "coeff")
        out = self._out(self.NQ, prec, out)
        _chk(_lib.nir_bwd_trans(self.h, PREC[prec], _ptr(coeff), _ptr(out)), "nir_bwd_trans")
        return out

    def iproduct_wrt_base(self, phys, prec="f64", out=None):
        self._dev(phys, DTYPE[prec], "phys"); self._chk_shape(phys, self.NQ, "phys")
        out = self._out(self.M, prec, out)
        _chk(_lib.nir_iproduct_wrt_base(self.h, PREC[prec], _ptr(phys), _ptr(out)), "nir_iproduct_wrt_base")
        return out

    def phys_deriv(self, phys, prec="f64", outs=None):
        self._dev(phys, DTYPE[prec], "phys"); self._chk_shape(phys, self.NQ, "phys")
        outs = outs or [self._out(self.NQ, prec, None) for _ in range(self.dim)]
        for o in outs:
            self._dev(o, DTYPE[prec], "out"); self._chk_shape(o, self.NQ, "out")
        d2 = _ptr(outs[2]) if self.dim == 3 else None
        _chk(_lib.nir_phys_deriv(self.h, PREC[prec], _ptr(phys), _ptr(outs[0]), _ptr(outs[1]), d2),
             "nir_phys_deriv")
        return outs

    def iproduct_wrt_deriv_base(self, fields, prec="f64", out=None):
        if len(fields) != self.dim:
            raise ValueError(f"need {self.dim} fields")
        for f in fields:
            self._dev(f, DTYPE[prec], "field"); self._chk_shape(f, self.NQ, "field")
        out = self._out(self.M, prec, out)
        f2 = _ptr(fields[2]) if self.dim == 3 else None
        _chk(_lib.nir_iproduct_wrt_deriv_base(self.h, PREC[prec], _ptr(fields[0]), _ptr(fields[1]), f2,
                                              _ptr(out)), "nir_iproduct_wrt_deriv_base")
        return out

    def mass(self, coeff, prec="f64", out=None):
        self._dev(coeff, DTYPE[prec], "coeff"); self._chk_shape(coeff, self.M, "coeff")
        out = self._out(self.M, prec, out)
        _chk(_lib.nir_mass(self.h, PREC[prec], _ptr(coeff), _ptr(out)), "nir_mass")
        return out

    def helmholtz(self, coeff, lam=1.0, prec="f64", out=None):
        self._dev(coeff, DTYPE[prec], "coeff"); self._chk_shape(coeff, self.M, "coeff")
        out = self._out(self.M, prec, out)
        _chk(_lib.nir_helmholtz(self.h, PREC[prec], float(lam), _ptr(coeff), _ptr(out)), "nir_helmholtz")
        return out

    def helmholtz_fields(self, fields, lam=1.0, prec="f64", outs=None):
        """Helmholtz on 1..3 fields [E][M] in one launch; returns the outputs."""
        if not 1 <= len(fields) <= 3:
            raise ValueError("1 to 3 fields")
        for f in fields:
            self._dev(f, DTYPE[prec], "field"); self._chk_shape(f, self.M, "field")
        outs = outs or [self._out(self.M, prec, None) for _ in fields]
        for o in outs:
            self._dev(o, DTYPE[prec], "out"); self._chk_shape(o, self.M, "out")
        ins = (_vp * len(fields))(*[f.data_ptr() for f in fields])
        ous = (_vp * len(outs))(*[o.data_ptr() for o in outs])
        _chk(_lib.nir_helmholtz_fields(self.h, PREC[prec], float(lam), len(fields), ins, ous), "nir_helmholtz_fields")
        return outs

    def helmholtz_host(self, coeff_host, out_host, lam=1.0, prec="f64"):
        """Helmholtz on host tensors (pinned for full bandwidth); synchronous."""
        for t in (coeff_host, out_host):
            if t.is_cuda or t.dtype != DTYPE[prec] or not t.is_contiguous():
                raise TypeError("host tensors of the precision's dtype expected")
            self._chk_shape(t, self.M, "host tensor")
        _chk(_lib.nir_helmholtz_host(self.h, PREC[prec], float(lam), _ptr(coeff_host), _ptr(out_host)),
             "nir_helmholtz_host")
        return out_host


class Mesh:
    """Hybrid mesh over several blocks (concatenated coefficient vectors)."""

    def __init__(self, ctx: Context, blocks: list[Block]):
        self.ctx, self.blocks = ctx, list(blocks)
        arr = (_vp * len(blocks))(*[b.h for b in blocks])
        h = _vp()
        _chk(_lib.nir_mesh_create(ctx.h, arr, len(blocks), C.byref(h)), "nir_mesh_create")
        self.h = h
        n = _i64()
        _chk(_lib.nir_mesh_num_dofs(h, C.byref(n)), "nir_mesh_num_dofs")
        self.ndof = n.value
        self.offsets = []
        o = 0
        for b in blocks:
            self.offsets.append(o)
            o += b.nelem * b.M

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.nir_mesh_destroy(h)
            self.h = None

    def helmholtz(self, x, lam=1.0, prec="f64", out=None):
        if x.numel() != self.ndof or x.dtype != DTYPE[prec] or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA vector of the mesh's dofs")
        out = torch.empty_like(x) if out is None else out
        _chk(_lib.nir_mesh_helmholtz(self.h, PREC[prec], float(lam), _ptr(x), _ptr(out)), "nir_mesh_helmholtz")
        return out

    def tune(self, cache_path: str | None = None):
        _chk(_lib.nir_tune(self.h, None if cache_path is None else cache_path.encode()), "nir_tune")

    LAUNCH = {"persistent": 0, "blocks": 1}

    def set_launch(self, prec: str, form: str):
        """Force the launch form of applies in one precision ("persistent" or "blocks")."""
        _chk(_lib.nir_mesh_set_launch(self.h, PREC[prec], self.LAUNCH[form]), "nir_mesh_set_launch")

    def get_launch(self, prec: str) -> str:
        v = _i()
        _chk(_lib.nir_mesh_get_launch(self.h, PREC[prec], C.byref(v)), "nir_mesh_get_launch")
        return {0: "persistent", 1: "blocks"}[v.value]

    def cg_solve(self, b, x, lam=1.0, inner_prec="f32", tol=1e-10, max_outer=50, max_inner=2000,
                 inner_tol=1e-4, jacobi=True, inner_vectors="f64", fwd_tol=0.0, allreduce=None):
        """Returns (status code, stats dict); x is updated in place.  inner_vectors:
        "f64" (FP64 inner vectors and dots) or "f32"; fwd_tol > 0 also requires the
        last correction |dx| <= fwd_tol |x| (see nir_cg_opts).  allreduce: for a
        mesh that is one rank's part of a sharded mesh, a callable that sums a
        float64 numpy array in place over the ranks (nir_cg_solve_dist)."""
        for t in (b, x):
            if t.dtype != torch.float64 or not t.is_cuda or t.numel() != self.ndof:
                raise ValueError("b and x must be FP64 CUDA vectors of the mesh's dofs")
        o = _cg_opts(inner_prec, tol, max_outer, max_inner, inner_tol, jacobi, inner_vectors, fwd_tol)
        s = CGStats()
        if allreduce is None:
            rc = _lib.nir_cg_solve(self.h, float(lam), _ptr(b), _ptr(x), C.byref(o), C.byref(s))
        else:
            cb = _allreduce_callback(allreduce)   # kept alive for the call
            rc = _lib.nir_cg_solve_dist(self.h, float(lam), _ptr(b), _ptr(x), C.byref(o), C.byref(s),
                                        C.cast(cb, _vp), None)
        return rc, _cg_stats(s)


ASM_OPS = {"helmholtz": 0, "mass": 1}


class Assembly:
    """Conforming C0 assembly of quad or hex blocks of one order and one basis
    (modified or GLL-Lagrange; global vectors: free dofs
    first, then boundary dofs; local vectors: the blocks' [E][M] arrays
    concatenated)."""

    def __init__(self, ctx: Context, blocks: list[Block], vertex_ids: list):
        import numpy as np
        self.ctx, self.blocks = ctx, list(blocks)
        nv = 4 if blocks[0].dim == 2 else 8
        self._verts = []
        for b, v in zip(blocks, vertex_ids):
            v = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
            if v.shape != (b.nelem, nv):
                raise ValueError(f"vertex ids must be [{b.nelem}][{nv}]")
            self._verts.append(v)
        if len(self._verts) != len(blocks):
            raise ValueError("one vertex-id array per block")
        barr = (_vp * len(blocks))(*[b.h for b in blocks])
        varr = (_vp * len(blocks))(*[v.ctypes.data_as(_vp) for v in self._verts])
        h = _vp()
        _chk(_lib.nir_asm_create(ctx.h, barr, varr, len(blocks), C.byref(h)), "nir_asm_create")
        self.h = h
        ng, nf, nl = _i64(), _i64(), _i64()
        _chk(_lib.nir_asm_num_dofs(h, C.byref(ng), C.byref(nf), C.byref(nl)), "nir_asm_num_dofs")
        self.n_global, self.n_free, self.n_local = ng.value, nf.value, nl.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.nir_asm_destroy(h)
            self.h = None

    def _vec(self, t, n, prec, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != DTYPE[prec] or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA {DTYPE[prec]} tensor")
        if t.numel() != n:
            raise ValueError(f"{name} must hold {n} values")
        return t

    def _new(self, n, prec):
        return torch.empty(n, dtype=DTYPE[prec], device=f"cuda:{self.ctx.device}")

    def local_map(self):
        """Host int64 [n_local]: s * (g + 1) per local dof."""
        import numpy as np
        out = np.zeros(self.n_local, dtype=np.int64)
        _chk(_lib.nir_asm_local_map(self.h, out.ctypes.data_as(_vp)), "nir_asm_local_map")
        return out

    def gather(self, xg, prec="f64", out=None):
        self._vec(xg, self.n_global, prec, "x_global")
        out = self._new(self.n_local, prec) if out is None else self._vec(out, self.n_local, prec, "out")
        _chk(_lib.nir_asm_gather(self.h, PREC[prec], _ptr(xg), _ptr(out)), "nir_asm_gather")
        return out

    def assemble(self, yl, prec="f64", out=None):
        self._vec(yl, self.n_local, prec, "y_local")
        out = self._new(self.n_global, prec) if out is None else self._vec(out, self.n_global, prec, "out")
        _chk(_lib.nir_asm_assemble(self.h, PREC[prec], _ptr(yl), _ptr(out)), "nir_asm_assemble")
        return out

    def pick(self, xl, out=None):
        self._vec(xl, self.n_local, "f64", "x_local")
        out = self._new(self.n_global, "f64") if out is None else self._vec(out, self.n_global, "f64", "out")
        _chk(_lib.nir_asm_pick(self.h, _ptr(xl), _ptr(out)), "nir_asm_pick")
        return out

    def apply(self, xg, op="helmholtz", lam=1.0, prec="f64", out=None):
        self._vec(xg, self.n_global, prec, "x_global")
        out = self._new(self.n_global, prec) if out is None else self._vec(out, self.n_global, prec, "out")
        _chk(_lib.nir_asm_apply(self.h, ASM_OPS[op], float(lam), PREC[prec], _ptr(xg), _ptr(out)),
             "nir_asm_apply")
        return out

    def cg_solve(self, b, x, op="helmholtz", lam=1.0, fix_boundary=True, inner_prec="f32", tol=1e-10,
                 max_outer=50, max_inner=5000, inner_tol=1e-3, jacobi=True, inner_vectors="f64", fwd_tol=0.0):
        """Returns (status code, stats dict); x is updated in place (options as Mesh.cg_solve)."""
        self._vec(b, self.n_global, "f64", "b")
        self._vec(x, self.n_global, "f64", "x")
        o = _cg_opts(inner_prec, tol, max_outer, max_inner, inner_tol, jacobi, inner_vectors, fwd_tol)
        s = CGStats()
        rc = _lib.nir_asm_cg_solve(self.h, ASM_OPS[op], float(lam), int(bool(fix_boundary)), _ptr(b), _ptr(x),
                                   C.byref(o), C.byref(s))
        return rc, _cg_stats(s)
