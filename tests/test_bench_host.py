"""Host-side checks of bench.py's roofline record (CPU only).

The `traffic` field of the bench line comes from committed ncu summaries
(profiles/step_kernel_<storage>_traffic.txt), and only while they were taken on the current
step-kernel source. These tests keep that link from breaking silently: a change to the kernel
files without a new capture fails here, before a GPU run reports `traffic: null`.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

# Algorithmic bytes per node update: 9 FP32 populations read and written, or 8 16-bit
# deviations plus the FP32 rest population and anchor read and written.
ALGORITHMIC = {"f32": 72, "bf16_dev": 48, "f16_dev": 48}


@pytest.mark.parametrize("storage", sorted(ALGORITHMIC))
def test_traffic_record_matches_current_kernel(storage):
    b = bench.profiled_traffic(storage)
    assert b is not None, (f"profiles/step_kernel_{storage}_traffic.txt was not taken on the current "
                           f"step-kernel source (hash {bench.kernel_source_hash()})")
    # DRAM bytes within a few percent of the algorithmic bytes: no re-reads, and writes
    # only partly absorbed by L2 at the 4096^2 capture size.
    assert 0.9 * ALGORITHMIC[storage] <= b <= 1.05 * ALGORITHMIC[storage], b


def test_kernel_hash_covers_the_step_sources():
    for rel in bench.STEP_KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, rel)), rel
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
