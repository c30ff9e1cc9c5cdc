"""Planted mistakes in a copy of the oracle, on the CPU: each mutation below
of the per-axis-step arithmetic (a plausible slip: an axis, a step or a
factor taken from the wrong place) must make at least one pin of
tests/test_oracle_aniso.py fail, and the unmutated copy must pass them.  Each
run is a pytest subprocess with the copy first on the import path."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HYBRID = os.path.join(ROOT, "oracle", "hybrid.py")
PINS = os.path.join(ROOT, "tests", "test_oracle_aniso.py")

MUTANTS = {
    # the second difference of axis d over the step of the next axis
    "laplacian_axis": ("            inv_h2 = 1.0 / self.hv[d] ** 2",
                       "            inv_h2 = 1.0 / self.hv[(d + 1) % 3] ** 2"),
    # the absorbing coefficient of every face from the x step
    "abc_x_step": ("        return (self.hv - dt) / (self.hv + dt)",
                   "        return (self.hv[0] - dt) / (self.hv[0] + dt) + 0 * self.hv"),
    # a node on several absorbing faces: the sum of its faces' r, not the mean
    "abc_corner_sum": ("        return acc / np.maximum(level, 1)", "        return acc"),
    # the source ghost 2 h g with the x step on every face
    "source_ghost_x_step": ("dt * dt * 2.0 / self.hv[f // 2] * src.amp", "dt * dt * 2.0 / self.hv[0] * src.amp"),
    # the y delay of an oblique wave with the z step
    "delay_axis": ("d[1] * self.hv[1] * (self.I[:, 1] - i0[1])", "d[1] * self.hv[2] * (self.I[:, 1] - i0[1])"),
    # the face quadrature area dx_p dx_p
    "face_area": ("float(self.hv[p] * self.hv[q])", "float(self.hv[p] * self.hv[p])"),
    # the switch time of an entry face with the wrong in-face step
    "switch_time": ("abs(d[q]) * (self.n[q] - 1) * self.hv[q])", "abs(d[q]) * (self.n[q] - 1) * self.hv[p])"),
    # refined voxels' centres placed with the steps in reverse order
    "centre_position": ("(cvox + lo + 1 + 0.5) * self.hv", "(cvox + lo + 1 + 0.5) * self.hv[::-1]"),
    # the cell volume dx_1 dx_2 dx_2
    "cell_volume": ("float(self.hv[0] * self.hv[1] * self.hv[2])", "float(self.hv[0] * self.hv[1] * self.hv[1])"),
}


def _run_pins(tmp_path, src):
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg / "__init__.py")
    (pkg / "hybrid.py").write_text(src)
    env = dict(os.environ, PYTHONPATH=str(tmp_path) + os.pathsep + ROOT)
    which = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], env=env,
                           cwd=str(tmp_path), capture_output=True, text=True, timeout=300)
    assert which.stdout.strip().startswith(str(pkg)), which.stdout + which.stderr
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", PINS], env=env,
                          cwd=str(tmp_path), capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes_the_pins(tmp_path):
    r = _run_pins(tmp_path, open(HYBRID).read())
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(HYBRID).read()
    assert src.count(old) == 1, name
    r = _run_pins(tmp_path, src.replace(old, new))
    assert r.returncode == 1, r.stdout[-3000:]  # 1: some test failed (not a collection error)
