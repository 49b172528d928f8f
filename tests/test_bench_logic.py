"""Host-side arithmetic of bench.py: the algorithmic bytes per fluid node of every workload and
storage mode (one read and one write of every stored population of the fluid lattices), and
the workloads' labels, which name the committed profile summaries."""
import pytest

import bench


@pytest.mark.parametrize("name,precision,bpn", [
    ("dissolution", "fp32", 2 * 4 * (19 + 7)),
    ("dissolution", "fp16", 2 * 2 * (19 + 7)),
    ("dissolution", "bf16", 2 * 2 * (19 + 7)),
    ("dissolution", "fp16s32", 2 * (2 * 19 + 4 * 7)),
    ("dissolution", "fp64", 2 * 8 * (19 + 7)),
    ("droplet", "fp32", 2 * 4 * (2 * 19)),
    ("channel", "fp64", 2 * 8 * (9 + 5)),
    ("combustion", "fp32", 2 * 4 * (9 + 3 * 5)),
])
def test_bytes_per_fluid_node(name, precision, bpn):
    cfg, geom, fields, label = bench.workload(name, 16 if name in ("dissolution", "droplet") else 0, precision)
    assert bench.bytes_per_fluid_node(cfg) == bpn
    assert label.endswith(precision)


def test_labels_name_the_profile_summaries():
    import os
    for name in ("dissolution", "droplet"):
        _, _, _, label = bench.workload(name, 16, "fp32")
        path = os.path.join(bench.PROFILES, f"k_step_{label.split('_')[0]}_{label.split('_')[-1]}.md")
        assert os.path.exists(path), path
