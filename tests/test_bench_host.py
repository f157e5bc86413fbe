"""Host logic of the benchmark line that needs no GPU: the ncu DRAM-traffic record is reported
only while the kernel sources it was captured with are unchanged (the reconstruction source for
every entry, the degree 4-6 source as well for those degrees), and the per-variant key format."""
import hashlib
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2312_17042_gb300", "csrc")


def _tree(tmp, recon_extra="", high_extra=""):
    """A copy of the two sources (optionally edited) with a traffic record taken on the originals."""
    src = os.path.join(str(tmp), "paper_2312_17042_gb300", "csrc")
    os.makedirs(src, exist_ok=True)
    os.makedirs(os.path.join(str(tmp), "profiles"), exist_ok=True)
    rec = {"bytes_per_launch": {"blast_3d_96:CTENO4_r3_mixed:5160": 111, "dmr_2d:CTENO5_r4_mixed:1664": 222}}
    for name, field, extra in (("recon.cuh", "recon_cuh_sha256", recon_extra),
                               ("recon_high.cuh", "recon_high_cuh_sha256", high_extra)):
        text = open(os.path.join(CSRC, name), "rb").read()
        rec[field] = hashlib.sha256(text).hexdigest()
        with open(os.path.join(src, name), "wb") as f:
            f.write(text + extra.encode())
    with open(os.path.join(str(tmp), "profiles", "ncu_traffic.json"), "w") as f:
        json.dump(rec, f)


def test_traffic_only_while_the_captured_sources_are_unchanged(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path)
    assert bench.ncu_traffic("blast_3d_96:CTENO4_r3_mixed:5160") == 111
    assert bench.ncu_traffic("dmr_2d:CTENO5_r4_mixed:1664") == 222
    assert bench.ncu_traffic("blast_3d_96:CTENO4_r3_mixed:5168") is None      # not captured
    shutil.rmtree(tmp_path / "paper_2312_17042_gb300")
    _tree(tmp_path, high_extra="// edited\n")          # the degree 4-6 kernels changed
    assert bench.ncu_traffic("blast_3d_96:CTENO4_r3_mixed:5160") == 111
    assert bench.ncu_traffic("dmr_2d:CTENO5_r4_mixed:1664") is None
    shutil.rmtree(tmp_path / "paper_2312_17042_gb300")
    _tree(tmp_path, recon_extra="// edited\n")         # every reconstruction kernel changed
    assert bench.ncu_traffic("blast_3d_96:CTENO4_r3_mixed:5160") is None
    assert bench.ncu_traffic("dmr_2d:CTENO5_r4_mixed:1664") is None


def test_variant_names():
    assert bench.variant_name(0, 3, 1) == "CTENO4_r3_mixed"
    assert bench.variant_name(1, 4, 0) == "CTENOZ5_r4_fp64"
    assert bench.variant_name(2, 6, 1) == "CWENO7_r6_mixed"
