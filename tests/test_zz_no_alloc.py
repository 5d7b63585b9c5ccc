"""The no-allocation host-buffer Helmholtz entry point.

nir_helmholtz_host_noalloc serves callers that cannot let a library call
cudaMalloc: programs whose device memory belongs to a pool or caching
allocator, loops that must not stall on an allocation, and hosts that forbid
allocation after set-up.  It stages through a fixed device array compiled into
the library instead of allocated buffers.  This test calls it through the C ABI
and checks it against the allocating entry point nir_helmholtz_host on two
calls in a row (the shared array must not leak state from one call into the
next), plus its size limit.  Both calls must give exactly the allocating call's bits (the same kernel on
the same inputs), and the device's free memory must not change across them.
The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

MAX_VECTOR_BYTES = 16 << 20  # NIR_NOALLOC_MAX_VECTOR_BYTES in include/nir.h
ERR_TOO_LARGE = -9
ERR_STATE = -8


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    f = nir.lib().nir_helmholtz_host_noalloc
    f.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return nir


def curved_block(nir, ctx, E, P):
    n = int(np.ceil(E ** (1 / 3))) + 1
    nodes = W.hex_grid(n, 2, amp=0.05)[:E]
    blk = nir.Block(ctx, "hex", E, P, deformed=True)
    blk.set_geometry(2, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    return blk


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


# (precision, Helmholtz tuning variant): the default element-group kernel and
# the threading-over-elements kernel (variant 4), whose global scratch is
# prepared by set_tuning, so the no-allocation call only uses it
CASES = [("f64", 0), ("f32", 0), ("bf16", 0), ("f64", 4), ("f32", 4)]


@pytest.mark.parametrize("prec,variant", CASES)
def test_noalloc_matches_host_entry_point_twice(nir, prec, variant):
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    blk = curved_block(nir, ctx, 300, 4)
    dt = nir.DTYPE[prec]
    if variant:
        blk.set_tuning(prec, variant, 0, 0)
    if prec != "f64":
        # low-precision factors are derived by an allocating call first
        u0 = torch.zeros((blk.nelem, blk.M), dtype=dt, device="cuda")
        blk.helmholtz(u0, prec=prec)
        torch.cuda.synchronize()
    f = nir.lib().nir_helmholtz_host_noalloc
    us = [torch.from_numpy(W.coefficients(blk.nelem, blk.M, seed)).to(dt).pin_memory() for seed in (11, 12)]
    refs = [torch.empty_like(u).pin_memory() for u in us]
    outs = [torch.full_like(u, float("nan")).pin_memory() for u in us]
    # the allocating entry point (its staging buffers) and one no-allocation call
    # (the first call on a device looks up the fixed array) come before the count
    for u, ref in zip(us, refs):
        blk.helmholtz_host(u, ref, lam=1.5, prec=prec)
    warm = torch.empty_like(us[0]).pin_memory()
    assert f(blk.h, nir.PREC[prec], 1.5, C.c_void_p(us[0].data_ptr()), C.c_void_p(warm.data_ptr())) == 0
    before = free_bytes()
    for call, (u, ref, out) in enumerate(zip(us, refs, outs)):
        rc = f(blk.h, nir.PREC[prec], 1.5, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()))
        assert rc == 0, (call, rc)
        # the same kernel on the same inputs: the same bits as the allocating call
        assert torch.equal(out, ref), (call, prec, variant)
    assert free_bytes() == before, "the no-allocation entry point changed the device's free memory"
    assert blk.get_tuning(prec)[0] == variant


def test_noalloc_rejects_oversize_and_missing_factors(nir):
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    f = nir.lib().nir_helmholtz_host_noalloc
    # P = 8 hexes: M = 729; 3000 elements of FP64 exceed the 16 MiB staging half
    E, P = 3000, 8
    assert E * 729 * 8 > MAX_VECTOR_BYTES
    nodes = W.hex_grid(15, 1, amp=0.0)[:E]
    big = nir.Block(ctx, "hex", E, P, deformed=False)
    big.set_geometry(1, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    u = torch.zeros((E, big.M), dtype=torch.float64).pin_memory()
    out = torch.empty_like(u).pin_memory()
    assert f(big.h, 0, 1.0, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr())) == ERR_TOO_LARGE
    # BF16 factors were never derived for this block: refused, nothing allocated
    small = curved_block(nir, ctx, 20, 2)
    ub = torch.zeros((20, small.M), dtype=torch.bfloat16).pin_memory()
    ob = torch.empty_like(ub).pin_memory()
    assert f(small.h, 2, 1.0, C.c_void_p(ub.data_ptr()), C.c_void_p(ob.data_ptr())) == ERR_STATE
