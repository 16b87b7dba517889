"""Host logic of bench.py: the kernel-source hash that ties the committed DRAM
traffic figures to the sources they were captured on."""
import os
import shutil

import pytest

import bench


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    """A copy of the hashed sources and the traffic summaries under a temporary root."""
    src = os.path.join(bench.ROOT, "paper_2606_02627_gb300", "csrc")
    dst = tmp_path / "paper_2606_02627_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("advect.cu", "rk4.cuh", "common.cuh", "tracer.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_hash_ignores_host_tracer_state(fake_root):
    h0 = bench.kernel_hash()
    p = fake_root / "paper_2606_02627_gb300" / "csrc" / "tracer.cuh"
    s = p.read_text()
    assert "\nstruct sg_tracer {" in s
    # a host-only field of the tracer state: no kernel reads it
    p.write_text(s.replace("\nstruct sg_tracer {\n", "\nstruct sg_tracer {\n    int host_only_field;\n", 1))
    assert bench.kernel_hash() == h0


def test_hash_sees_kernel_changes(fake_root):
    h0 = bench.kernel_hash()
    for f, edit in (("advect.cu", "\n// edit\n"), ("tracer.cuh", "\nstruct LineParamsEdit {};\n")):
        p = fake_root / "paper_2606_02627_gb300" / "csrc" / f
        s = p.read_text()
        p.write_text(s + edit)
        assert bench.kernel_hash() != h0
        p.write_text(s)
    assert bench.kernel_hash() == h0


def test_traffic_needs_matching_hash(fake_root):
    # a summary carrying the hash of the sources it was captured on is read;
    # once a kernel source changes, the figure no longer applies
    p = fake_root / "profiles" / "round_async_f32_traffic.txt"
    p.write_text("# capture notes\n"
                 f"kernel_source_hash: {bench.kernel_hash()}\n"
                 "dram_bytes_per_particle_step: 12.50\n")
    assert bench.traffic_per_step("f32", "async") == 12.5
    src = fake_root / "paper_2606_02627_gb300" / "csrc" / "advect.cu"
    src.write_text(src.read_text() + "\n// edit\n")
    assert bench.traffic_per_step("f32", "async") is None
    assert bench.traffic_per_step("f32", "missing_tag") is None
