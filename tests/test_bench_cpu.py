"""bench.py's host logic (CPU).

- The kernel-source fingerprint that ties the committed ncu DRAM traffic to
  the kernels it was measured on ignores comments and whitespace, not code.
- The committed traffic table covers both kernels of the batched step on the
  four timed legs at the library's default tuning (include/april.h) for the
  current kernel sources, each entry citing a summary under profiles/.
- The step's launch count follows the tuning: the routing for partitioned
  sets, the triage or the binning kernel, the lane groups, and the kernel
  that finishes handed-over joins."""
import os
import shutil

import bench

DEFAULT_TUNE = {"cta_threshold": 0xFFFFFFFF, "group_lanes": 4, "group_window": 32, "cta_window": 128,
                "join_order": 2, "escalate_windows": 0, "triage_off": 0}


def test_source_fingerprint_ignores_comments_not_code(tmp_path, monkeypatch):
    base = bench.kernel_source_sha()
    d = tmp_path / "paper_2307_01716_gb300" / "csrc"
    d.mkdir(parents=True)
    for f in ("filter.cu", "join_device.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2307_01716_gb300", "csrc", f), d / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_sha() == base
    f = d / "filter.cu"
    src = f.read_text()
    f.write_text("// a comment line\n/* a block\n   comment */\n" + src.replace("\n", "\n\n", 40))
    assert bench.kernel_source_sha() == base
    knob = "#define APRIL_TRIAGE_GRID_PER_SM 64"
    assert knob in src
    f.write_text(src.replace(knob, "#define APRIL_TRIAGE_GRID_PER_SM 8", 1))
    assert bench.kernel_source_sha() != base


def test_committed_traffic_matches_the_current_kernels():
    legs = [("paper-scale-200k", "batched"), ("skewed-pareto-340k-10M", "batched"),
            ("partitioned-16x16-n14", "batched"), ("partitioned-16x16-n14", "packed")]
    for workload, mode in legs:
        for kernel in ("k_triage", "k_persistent"):
            b, src = bench.kernel_traffic(kernel, workload, mode, DEFAULT_TUNE)
            assert b is not None and b > 0, (kernel, workload, mode)
            assert os.path.exists(os.path.join(bench.ROOT, src)), src
    # another tuning has no entry: its traffic would be reported as unknown
    other = dict(DEFAULT_TUNE, group_lanes=8)
    assert bench.kernel_traffic("k_persistent", "paper-scale-200k", "batched", other) == (None, None)


def test_launches_per_step_follow_the_tuning():
    t = dict(DEFAULT_TUNE)
    assert bench.launches_per_step(t, 0, "batched") == 2  # triage, lane groups
    assert bench.launches_per_step(t, 16, "packed") == 3  # routing, triage, lane groups
    assert bench.launches_per_step(dict(t, triage_off=1), 0, "batched") == 1
    assert bench.launches_per_step(dict(t, cta_threshold=2048), 0, "batched") == 2  # binning, lane groups
    assert bench.launches_per_step(dict(t, cta_threshold=2048, escalate_windows=8), 16, "batched") == 4
    assert bench.launches_per_step(dict(t, group_lanes=32), 0, "batched") == 1
    assert bench.launches_per_step(t, 0, "warp") == 1
