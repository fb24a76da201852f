"""Host-side logic of the benchmark that needs no GPU: the traffic figures are reported only
for the captured workload and only while the kernel's sources are unchanged."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _sha(files):
    m = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1907_04435_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:16]


def test_traffic_needs_matching_sources_and_workload(monkeypatch):
    import bench
    files = ("sa_sort.cu",)
    good = {"bytes": 123, "workload": "district", "sources": files, "sha256_16": _sha(files)}
    monkeypatch.setitem(bench.TRAFFIC, "k_test", good)
    assert bench.kernel_traffic("k_test", "district") == 123
    assert bench.kernel_traffic("k_test", "district_1k") is None
    monkeypatch.setitem(bench.TRAFFIC, "k_test", dict(good, sha256_16="0" * 16))
    assert bench.kernel_traffic("k_test", "district") is None
    assert bench.kernel_traffic("k_unknown", "district") is None


def test_launch_count_covers_both_maps(monkeypatch):
    """District: 9 blocks in one chunk for each map; 1M facade points at runs of 16 fit
    the facade map's 1 GiB chunk budget in one chunk, 40M do not."""
    import bench

    class _Sun:
        n_blocks = 9

    class _Fac:
        def __init__(self, R):
            self.R = R

    monkeypatch.setattr(bench, "B_option_run", lambda: 16)
    assert bench.count_launches(None, _Sun(), None, None) == 7
    assert bench.count_launches(None, _Sun(), None, _Fac(1_000_000)) == 7 + 15
    assert bench.count_launches(None, _Sun(), None, _Fac(40_000_000)) == 7 + 15 * 9
