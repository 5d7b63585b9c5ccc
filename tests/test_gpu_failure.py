"""Failure detection on the GPU without a fault: the bounded mbarrier wait
that every staged kernel uses runs out on purpose (a barrier nothing arrives
on, no copy in flight, a short cycle limit); the kernel must set the device
error word and return, nir_ctx_check must report NIR_ERR_CUDA once and clear
the word, and the context must stay usable."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


def test_bounded_wait_runs_out_and_is_reported(nir):
    torch.cuda.set_device(0)
    ctx = nir.Context(0)
    ctx.check()                      # clean to start with
    ctx.selftest_wait(1 << 20)       # ~0.5 ms at 2 GHz
    with pytest.raises(nir.NirError) as ei:
        ctx.check()
    assert ei.value.code == -3       # NIR_ERR_CUDA
    ctx.check()                      # the word was cleared
    # the context still works: a staged FP32 Helmholtz apply after the timeout
    E, P = 64, 3
    nodes = W.hex_grid(4, 2, amp=0.05)[:E]
    blk = nir.Block(ctx, "hex", E, P, deformed=True)
    blk.set_geometry(2, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    x = W.coefficients(E, blk.M, seed=0)
    y = blk.helmholtz(torch.from_numpy(x).cuda().float(), prec="f32").double().cpu().numpy()
    ctx.check()
    ref = oracle.helmholtz("hex", P, P + 2, 2, nodes, 1.0, x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5


def test_selftest_argument_checks(nir):
    ctx = nir.Context(0)
    L = nir.lib()
    assert L.nir_ctx_selftest_wait(ctx.h, 0) == -1
    assert L.nir_ctx_selftest_wait(ctx.h, (1 << 31) + 1) == -1
    assert L.nir_ctx_selftest_wait(None, 100) == -1


def test_fp64_tensor_core_probe(nir):
    """The DMMA probe returns a finite positive rate next to the DFMA one (the
    comparison is recorded by the benchmark, not asserted here)."""
    ctx = nir.Context(0)
    dmma, dfma = ctx.probe_fp64_mma_peak(), ctx.probe_fp64_peak()
    assert np.isfinite(dmma) and dmma > 0 and np.isfinite(dfma) and dfma > 0
