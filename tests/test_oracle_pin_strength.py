"""Planted mistakes in a copy of the oracle, on the CPU: each mutation below
(a plausible slip: a factor, a sign, an index, an axis or a step taken from
the wrong place) must make at least one of the oracle's pins fail, and the
unmutated copy must pass them all.  Each run is a pytest subprocess over the
pin files with the copy first on the import path."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HYBRID = os.path.join(ROOT, "oracle", "hybrid.py")
PINS = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins.py", "test_oracle_refinement.py",
                                                  "test_oracle_sources.py", "test_oracle_telegraph.py",
                                                  "test_oracle_aniso.py")]

MUTANTS = {
    # ---- the scheme
    # the mirror ghost's factor 2 dropped on the low faces
    "mirror_ghost": ("np.full(lowb.sum(), 2 * inv_h2), np.full(highb.sum(), 2 * inv_h2)]",
                     "np.full(lowb.sum(), inv_h2), np.full(highb.sum(), 2 * inv_h2)]"),
    # the absorbing coefficient (tau - h) / (h + tau)
    "abc_sign": ("        return (self.hv - dt) / (self.hv + dt)", "        return (dt - self.hv) / (self.hv + dt)"),
    # the absorbing row's coupling to the inward neighbour halved
    "abc_coupling": ("            vb.append(1.0 / Lb)", "            vb.append(0.5 / Lb)"),
    # corners before edges before faces
    "abc_order": ("            for L in (1, 2, 3):", "            for L in (3, 2, 1):"),
    # the flux ghost u_in + h g
    "source_factor": ("dt * dt * 2.0 / self.hv[f // 2] * src.amp", "dt * dt * 1.0 / self.hv[f // 2] * src.amp"),
    # an oblique wave's flux without its factor -(d . n)
    "oblique_factor": ("                entry[f] = -dn", "                entry[f] = 1.0"),
    # the lumped mass |K| / 3 per vertex
    "lumped_mass": ("weights=np.repeat(self.tet_vol / 4.0, 4),", "weights=np.repeat(self.tet_vol / 3.0, 4),"),
    # Algorithm 1's copy of omega_diamond into the FDM array left out
    "exchange": ("                # 3. FEM values at omega_diamond become FDM boundary values\n"
                 "                new_fd[self.omega_diamond] = new_fe[self.omega_diamond]",
                 "                # 3. FEM values at omega_diamond become FDM boundary values\n                pass"),
    # ---- adjoint, gradient, CG, telegraph
    "adjoint_data_index": ("            rhs[obs] += cot[j]\n            lam = self._solve_unit(NT, rhs)",
                           "            rhs[obs] += cot[j - 1]\n            lam = self._solve_unit(NT, rhs)"),
    "gradient_sign": ("        out = -dt * dt * Gacc", "        out = dt * dt * Gacc"),
    "pairing_time_index": ("                Gacc += self.pair(hist[j], lam1, ML)",
                           "                Gacc += self.pair(hist[j - 1], lam1, ML)"),
    "step_parabola": ("        alpha = -dJ0 * alpha_t * alpha_t / (2.0 * curv)",
                      "        alpha = -dJ0 * alpha_t * alpha_t / curv"),
    "fr_beta": ("    beta = gn2 / gn2_prev", "    beta = gn2_prev / gn2"),
    "face_weight_border": ("            w[edge] *= 0.5", "            w[edge] *= 1.0"),
    "damping_ratio": ("    s[own] = 0.5 * dt * D[own] / ML[own]", "    s[own] = dt * D[own] / ML[own]"),
    "telegraph_pair_sign": ("            G -= pair(j, lam1)", "            G += pair(j, lam1)"),
    # ---- elements, mesh, sources
    "tet_volume": ("    vol = np.abs(np.linalg.det(e)) / 6.0", "    vol = np.abs(np.linalg.det(e)) / 2.0"),
    "bisection_child": ("    ch1 = np.stack([pn[:, 0], pn[:, 1], pn[:, 2], c], axis=1)",
                        "    ch1 = np.stack([pn[:, 0], pn[:, 1], pn[:, 3], c], axis=1)"),
    "owned_nodes": ("            self.owned = np.all((self.I >= lo + 1) & (self.I <= hi - 1), axis=1)",
                    "            self.owned = np.all((self.I >= lo + 1) & (self.I <= hi - 2), axis=1)"),
    "unknown_voxels": ("            unk = np.all((vox >= lo + 1) & (vox <= hi - 2), axis=1)",
                       "            unk = np.all((vox >= lo + 1) & (vox <= hi - 3), axis=1)"),
    "exchange_omega_o": ("                # 4. FDM values at omega_o become FEM boundary values\n"
                         "                new_fe[self.omega_o] = new_fd[self.omega_o]",
                         "                # 4. FDM values at omega_o become FEM boundary values\n                pass"),
    "pulse_window": ("    return np.where((s >= 0.0) & (s <= t1), np.sin(omega * s), 0.0)",
                     "    return np.where((s >= 0.0) & (s <= 2 * t1), np.sin(omega * s), 0.0)"),
    "entry_corner": ("        i0 = [0 if d[ax] >= 0.0 else self.n[ax] - 1 for ax in range(3)]",
                     "        i0 = [0 for ax in range(3)]"),
    # ---- the paper's adjoint, the functional, the projection
    "paper_data_sign": ("            new_fd[obs] += -dt * cot[k] / M[obs]", "            new_fd[obs] += dt * cot[k] / M[obs]"),
    "paper_gradient_scale": ("        out = dt * G", "        out = dt * dt * G"),
    "time_weight_k0": ("    wk[0] = 0.0", "    wk[0] = 1.0"),
    "misfit_half": ("    return 0.5 * float(np.sum(wk[:, None] * mj[None, :] * d * d)), wk[:, None] * mj[None, :] * d",
                    "    return float(np.sum(wk[:, None] * mj[None, :] * d * d)), wk[:, None] * mj[None, :] * d"),
    "tikhonov_volume": ("    J = 0.5 * gamma * prob.voxel_volume * float(np.sum((a - a0) ** 2))",
                        "    J = 0.5 * gamma * float(np.sum((a - a0) ** 2))"),
    "projection_side": ("    blocked = ((a <= a_min) & (g > 0.0)) | ((a >= a_max) & (g < 0.0))",
                        "    blocked = ((a <= a_min) & (g < 0.0)) | ((a >= a_max) & (g > 0.0))"),
    # ---- per-axis steps
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
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] + PINS, env=env,
                          cwd=str(tmp_path), capture_output=True, text=True, timeout=900)


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
