"""The ncu summaries under profiles/ that bench.py reads: when their recorded
source hashes match the kernel sources, the benchmark reports DRAM traffic
scaled from the capture (and it is consistent with the algorithmic bytes);
when the kernel has changed since the capture, it reports null."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_tensor_core_profile_matches_sources():
    import bench
    t = bench.tc_traffic(16384, 16384)
    fields = bench.profile_fields(bench.TC_PROFILE)
    if fields.get("kernel_sources_sha256_16") != bench.tc_source_hash():
        assert t is None      # stale capture: no traffic figure
        return
    assert t is not None
    # scaling is by m n: a 32768^2 launch moves four times the captured traffic
    assert bench.tc_traffic(32768, 32768) == pytest.approx(4 * t)
    # within a few percent of the algorithmic bytes of the captured launch
    alg = 2 * 16384 * 16384 + 2 * 16384 * 256 + 4 * 16384 * 256
    assert 1.0 <= t / alg < 1.1


def test_batched_profile_matches_sources():
    import bench
    import hashlib
    f = bench.profile_fields(bench.BATCH_PROFILE)
    t = bench.batched_traffic(float(f["capture_sum_mn"]))
    src = os.path.join(ROOT, "paper_1607_01649_gb300", "csrc", "k_batched.cu")
    if f.get("kernel_sources_sha256_16") != hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]:
        assert t is None
        return
    assert t is not None
    assert t == pytest.approx(float(f["dram_bytes_per_launch"]))
