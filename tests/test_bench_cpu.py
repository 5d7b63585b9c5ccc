"""The benchmark's accounting on CPU: algorithmic bytes and flops per element
against their closed forms, the L2-flush rule of the timed loops, and the
profile-hash guard on the reported DRAM traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import workloads as W  # noqa: E402


def test_hex_work_per_element_closed_forms():
    # P = 4 (N = 5, Q = 6): 4N(N^2 Q + N Q^2 + Q^3) + 12 Q^4 + 20 Q^3 flops; u, y and 7 metric values per point
    assert bench.helm_flops_per_elem("hex", 5, 6) == 4 * 5 * (25 * 6 + 5 * 36 + 216) + 12 * 6 ** 4 + 20 * 6 ** 3
    assert bench.helm_flops_per_elem("hex", 5, 6) == 30792
    assert bench.helm_bytes_per_elem("hex", 5, 6, 8, True) == (2 * 125 + 7 * 216) * 8
    assert bench.helm_bytes_per_elem("hex", 5, 6, 4, True) == 7048


def test_l2_flush_rule():
    """Steps streaming less than twice the 129 MiB L2 are timed with L2 flushed."""
    E = W.workload("hex32_curved_p4")["nodes"].shape[0]
    f64 = E * bench.helm_bytes_per_elem("hex", 5, 6, 8, True)
    f32 = E * bench.helm_bytes_per_elem("hex", 5, 6, 4, True)
    bf16 = E * bench.helm_bytes_per_elem("hex", 5, 6, 2, True)
    assert not bench.needs_flush(f64)            # 440 MiB
    assert bench.needs_flush(f32) and bench.needs_flush(bf16)   # 220 and 110 MiB
    assert bench.needs_flush(2 * bench.L2_BYTES - 1) and not bench.needs_flush(2 * bench.L2_BYTES)
    assert bench.l2_note(f64).startswith("no flush") and bench.l2_note(bf16).startswith("flushed")


def test_profile_traffic_follows_the_sources():
    """The committed summaries carry the hash of the kernel sources they were
    captured from; a summary for other sources reports no traffic."""
    import re
    for name in ("helm_hex32_curved_p4_f64", "helm_hex32_curved_p4_f32", "helm_hex32_curved_p4_bf16"):
        txt = open(os.path.join(ROOT, "profiles", name + ".md")).read()
        h = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", txt).group(1)
        t = bench.profiled_traffic(name)
        assert (t is not None) == (h == bench.kernel_sources_sha256())
    assert bench.profiled_traffic("no_such_profile") is None
