"""Host logic of bench.py (no GPU): the DRAM traffic record matches the
current kernel source, the anisotropic workload's recipe and its
sweeps-only guard, and the algorithmic byte count per launch."""
import subprocess
import sys

import bench
import synth


def test_recorded_traffic_matches_the_current_kernel_source():
    """profiles/dram_traffic.txt carries the ncu DRAM bytes of the step
    kernels under the hash of the code they were taken on; after a kernel
    change the record must be captured again."""
    fwd = bench.recorded_traffic("step_kernel<float,forward>", "large_257")
    adj = bench.recorded_traffic("step_kernel<float,adjoint>", "large_257")
    assert fwd is not None and adj is not None, bench.kernel_source_hash()
    assert 1.0e9 < fwd < 5.0e9 and 1.0e9 < adj < 5.0e9


def test_anisotropic_workload_recipe():
    w = bench.make_workload("anisotropic_box", 20)
    assert w.n == (257, 193, 321) and w.nsteps == 20 and len(w.sources) == 8
    assert w.hv == (2.0 / 256, 2.0 / 192, 2.0 / 320)
    assert w.fem_lo == (64, 48, 80) and w.fem_hi == (192, 144, 240)
    bound = 1.0 / (w.a_max * sum(1.0 / (d * d) for d in w.hv)) ** 0.5
    assert abs(w.dt - 0.9 * bound) < 1e-15
    assert w.refine is None and w.n_unknown == 126 * 94 * 158


def test_anisotropic_workload_needs_sweeps_only():
    r = subprocess.run([sys.executable, bench.__file__, "--workload", "anisotropic_box"], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode != 0 and "--sweeps-only" in r.stderr


def test_algorithmic_bytes_per_launch():
    """3 words per FDM-owned node, 4 (forward) / 5 (transposed) per FEM-owned
    node and per centre, times the sources."""
    class Info:
        n_fem_owned = 10
        n_centres = 2
    w = synth.small_problem(n=(7, 8, 9), fem=(2, 5))
    f, a = bench.algorithmic_bytes(w, Info, 3)
    n = 7 * 8 * 9
    assert f == 3 * ((n - 10) * 12 + 10 * 16 + 2 * 16)
    assert a == 3 * ((n - 10) * 12 + 10 * 20 + 2 * 20)
