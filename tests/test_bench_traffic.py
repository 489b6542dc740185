"""The bench's roofline traffic figures (CPU).

`roofline.traffic` is the DRAM traffic an ncu capture measured for one launch
of the dominant kernel.  bench.py keeps each figure with a digest of the
kernel sources it was captured from and reports it only while the sources
still have that digest, so a figure taken before a kernel change is never
printed for the changed kernel: it becomes null.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_digest_covers_the_kernel_sources():
    d = bench.kernel_source_digest()
    assert len(d) == 16 and int(d, 16) >= 0
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_2302_00850_gb300", "csrc", f)), f


def test_traffic_only_for_the_captured_sources(monkeypatch):
    for prec, (nbytes, digest) in bench.NCU_TRAFFIC.items():
        monkeypatch.setattr(bench, "kernel_source_digest", lambda d=digest: d)
        assert bench.ncu_traffic(prec) == nbytes
        monkeypatch.setattr(bench, "kernel_source_digest", lambda d=digest: "0" * 16 if d != "0" * 16 else "1" * 16)
        assert bench.ncu_traffic(prec) is None


def test_traffic_figures_are_per_launch_bytes():
    # FP16: about 300 MB per 32^3x64 parity launch (296 algorithmic bytes per site);
    # FP64: about 1.6 GB (1536 algorithmic bytes per site); both within 10 % of that
    vh = 32 ** 3 * 64 // 2
    assert abs(bench.NCU_TRAFFIC["f16"][0] / (296 * vh) - 1) < 0.1
    assert abs(bench.NCU_TRAFFIC["f64"][0] / (1536 * vh) - 1) < 0.1
