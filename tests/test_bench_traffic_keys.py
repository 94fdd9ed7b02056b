"""bench.py reports the ncu DRAM traffic of the dominant kernel only while
the kernel's sources are the ones the counters were taken on.  Every entry of
its traffic table must still match the current sources: an entry left
behind by a kernel change reports nothing and means the capture is due."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_table_matches_current_kernel_sources():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    assert mod.NCU_TRAFFIC
    for (kernel, digest), traffic in mod.NCU_TRAFFIC.items():
        assert mod.kernel_source_hash(kernel) == digest, kernel
        assert traffic > 0
