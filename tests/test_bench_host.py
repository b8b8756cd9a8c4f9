"""Host logic of bench.py (no GPU): the byte accounting behind the roofline
fields and the rule that the committed DRAM record applies only to the
kernel sources it was taken on."""
import json
import os

import bench


def test_algorithmic_bytes_per_site():
    # one read and one write of 2 x 19 populations plus the 1-byte node mask
    assert bench.alg_bytes("fp64") == 609
    assert bench.alg_bytes("fp32") == 305
    assert bench.alg_bytes("fp16") == 153


def test_kernel_bytes_of_the_lattice_kernels():
    # density pass: populations + mask in, rho^A, rho^B and j^A + j^B out
    assert bench.kernel_bytes("k_density", "fp32") == 152 + 1 + 20
    # lean kernel: psi pairs, the three momentum rows and the link classes in,
    # populations out
    assert bench.kernel_bytes("k_lean", "fp32") == 152 + 20 + 4
    # the two passes together move more than the single-pass ideal
    assert bench.kernel_bytes("k_density", "fp32") + bench.kernel_bytes("k_lean", "fp32") > bench.alg_bytes("fp32")
    assert bench.kernel_bytes("k_fused", "fp16") == 2 * 76 + 1


def test_traffic_record_follows_the_kernel_sources(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "lattice_traffic_shear512_fp32.json")
    rec = json.load(open(path))["fp32"]
    monkeypatch.setattr(bench, "kernel_hash", lambda: rec["kernel_sha"])
    assert bench.recorded_traffic("fp32") == rec["bytes_per_launch_full_workload"]
    # ratio to the algorithmic bytes of the 512 x 512 x 256 step
    ratio = rec["bytes_per_launch_full_workload"] / (bench.alg_bytes("fp32") * 512 * 512 * 256)
    assert 1.0 < ratio < 1.3
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("fp32") is None
    assert bench.recorded_traffic("fp16") is None
