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


def test_cpu_baseline_sizing():
    """The CPU baseline traces a prefix of the seeds: a calibration run, then
    rescaled runs until the sample takes at least half the target time (or
    every seed); with n_seeds it traces exactly that prefix."""
    import numpy as np
    from paper_2606_02627_gb300 import inputs
    import oracle
    g = inputs.cube_grid(17)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(3, n_modes=16, kmax=2)).numpy()
    seeds = inputs.uniform_seeds(g, 4000, 3)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    rate, cores, n, steps, secs = bench.cpu_oracle_rate(F, g, seeds, dt, 60, 0.2, nthreads=2)
    assert cores == 2 and 0 < n <= len(seeds) and steps > 0 and rate > 0
    assert secs >= 0.1 or n == len(seeds)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds[:n], dt, 60, eps=1e-6, nthreads=2)
    assert steps == int(ref.steps().sum())
    rate2, _, n2, steps2, _ = bench.cpu_oracle_rate(F, g, seeds, dt, 60, 0.2, nthreads=2, n_seeds=123)
    assert n2 == 123 and rate2 > 0
    assert steps2 == int(oracle.trace_streamlines(F, g.origin, g.spacing, seeds[:123], dt, 60, eps=1e-6,
                                                  nthreads=2).steps().sum())
    assert np.isfinite(rate) and np.isfinite(rate2)
