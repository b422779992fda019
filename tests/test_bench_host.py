"""Host-side logic of bench.py (no GPU): the byte models of the step paths,
the launch count it reports, and the lookup of the stored ncu traffic."""
import pytest

import bench


def test_fp32_byte_models_add_up_by_path():
    # force phase: split (lane sums + epilogue) 120 B, fused 100 B; update phase
    # 104 B on its own, 80 B inside the persistent velocity update
    assert bench.fp32_bytes_per_node(2, False) == 120
    assert bench.fp32_bytes_per_node(0, False) == 100
    assert bench.fp32_bytes_per_node(1, True) == 100 + 80
    assert bench.fp32_bytes_per_node(3, True) == 120 + 80
    assert bench.fp32_bytes_per_node(0, True) == 100 + 104
    assert bench.fp32_bytes_per_node(2, True) == 120 + 104
    # the rebuild-every-step variants (modes 4 and 6) move the same bytes
    assert bench.fp32_bytes_per_node(6, True) == bench.fp32_bytes_per_node(2, True)
    assert bench.BYTES_PER_NODE_STEP_FP32_MAX == max(bench.fp32_bytes_per_node(m, True) for m in range(8))


def test_launch_count_per_path():
    steps, rebuilds = 10, 3
    assert bench._launches(1, steps, rebuilds) == steps                     # one persistent launch per step
    assert bench._launches(3, steps, rebuilds) == steps
    assert bench._launches(0, steps, rebuilds) == 2 * steps + 6 * rebuilds  # update + force, rebuild chain
    assert bench._launches(2, steps, rebuilds) == 3 * steps + 6 * rebuilds  # update + sums + epilogue
    assert bench._launches(6, steps, rebuilds) == 9 * steps                 # rebuild kernels every step


@pytest.mark.parametrize("workload,path", [
    ("ensemble64", {"mode": 1, "lanes": 1, "block": 256}),
    ("ensemble64", {"mode": 2, "lanes": 1, "block": 128}),
    ("compaction500", {"mode": 1, "lanes": 1, "block": 256}),
    ("compaction500", {"mode": 1, "lanes": 1, "block": 128}),
    ("compaction500", {"mode": 2, "lanes": 1, "block": 128}),
])
def test_stored_traffic_is_found_for_the_tuned_paths(workload, path):
    """The kernel names the bench looks up match those of the ncu captures, for
    the paths the autotuner picks on these workloads (FP32 split and FP64)."""
    if bench.kernel_digest() != bench.TRAFFIC_DIGEST:
        pytest.skip("kernel sources changed since the stored capture: the bench reports null")
    for fp32 in (True, False):
        t = bench.force_phase_traffic(path, fp32, workload)
        assert t is not None and t > 0
