"""Host logic of the benchmark's roofline bookkeeping (no GPU).

The DRAM traffic the bench reports for its dominant kernel comes from a single-pass
ncu capture recorded in `MEASURED_TRAFFIC`, keyed by a hash of the kernel's sources:
it is reported while the sources are the ones captured and turns null by itself as
soon as any of them changes (a record of another kernel revision is never used).
"""
import os
import shutil
import tempfile

import bench


def test_traffic_record_matches_the_current_sweep_sources():
    # the record in the repository belongs to the committed sources of the sweep kernel
    rec = bench.MEASURED_TRAFFIC["k_sweep_cols"]
    assert bench.source_hash("k_sweep_cols") == rec["sha"]
    assert bench.measured_traffic("k_sweep_cols") == rec["bytes"]
    assert bench.measured_traffic("no_such_kernel") is None


def test_traffic_record_turns_null_when_a_source_changes(monkeypatch):
    # a copy of the sources with one byte appended to one file: the hash moves and the
    # recorded traffic is no longer reported
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(bench.ROOT, "paper_1901_11371_gb300", "csrc")
        dst = os.path.join(d, "paper_1901_11371_gb300", "csrc")
        os.makedirs(dst)
        for name in bench.KERNEL_SOURCES["k_sweep_cols"]:
            shutil.copy(os.path.join(src, name), os.path.join(dst, name))
        monkeypatch.setattr(bench, "ROOT", d)
        assert bench.measured_traffic("k_sweep_cols") is not None
        with open(os.path.join(dst, bench.KERNEL_SOURCES["k_sweep_cols"][0]), "ab") as f:
            f.write(b"\n")
        assert bench.measured_traffic("k_sweep_cols") is None
