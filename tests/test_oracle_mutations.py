"""Sensitivity of the oracle pins: plant one plausible mistake at a time in a
copy of the oracle (on the CPU, in a temporary directory) and check that the
pin suite fails for every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted mistake)
MUTATIONS = [
    ("rotation sign", "R[1] = 2 * (x * y - w * z)", "R[1] = 2 * (x * y + w * z)"),
    ("rotation jacobian entry", "{2 * z, 2 * y, 2 * x, 2 * w}", "{2 * z, 2 * y, 2 * x, -2 * w}"),
    ("adjugate vjp sign", "dM[r0 * 3 + c1] -= g * M[r1 * 3 + c0];", "dM[r0 * 3 + c1] += g * M[r1 * 3 + c0];"),
    ("background dropped in reverse pass",
     "double SC[3] = {tf * cfg.bg[0], tf * cfg.bg[1], tf * cfg.bg[2]}", "double SC[3] = {0, 0, 0}"),
    ("alpha-output term", "da += dA * tf / om;", "da += dA * tf;"),
    ("center gradient term", "dM[8] -= (gr[R_CX] * g.M[2] + gr[R_CY] * g.M[5]) / (m22 * m22);",
     "dM[8] -= (gr[R_CX] * g.M[2]) / (m22 * m22);"),
    ("pose cross order", "cross(g.nc, dnc, cr);", "cross(dnc, g.nc, cr);"),
    ("normal not turned to camera", "g->flip = (d > 0) ? -1.0 : 1.0;", "g->flip = 1.0;"),
    ("stop rule", "if (Tn < cfg->t_min) break;", "if (Tn < 0.5 * cfg->t_min) break;"),
    ("low-pass width", "(dx * dx + dy * dy) / (cfg->sigma_lp * cfg->sigma_lp)",
     "(dx * dx + dy * dy) / (2 * cfg->sigma_lp * cfg->sigma_lp)"),
    ("rect too small", "double lo = fmin(fmin(r1, r2), c0 - rlp)", "double lo = fmin(fmin(r1, r2), c0 - rlp) + 0.3"),
    ("rect too wide", "double lo = fmin(fmin(r1, r2), c0 - rlp)", "double lo = fmin(fmin(r1, r2), c0 - rlp) - 0.3"),
    ("low-pass square too wide", "double rlp = cfg.sigma_lp * kk;", "double rlp = 2.0 * cfg.sigma_lp * kk;"),
    ("dual conic root with a spare margin", "double r1 = (di2 + sqrt(disc)) / d22", "double r1 = (di2 + 1.02 * sqrt(disc)) / d22"),
    ("opacity-aware extent", "double k2 = 2.0 * log(op / cfg.alpha_min);", "double k2 = 1.5 * log(op / cfg.alpha_min);"),
    ("homogeneous divide gradient", "dcc = -(b->e.u * du + b->e.v * dv) / c;", "dcc = -(b->e.u * du - b->e.v * dv) / c;"),
    ("ray depth: divide term of its gradient", "g[R_A + 6 + j] -= dz * zi / c * x[j];",
     "g[R_A + 6 + j] -= 0.5 * dz * zi / c * x[j];"),
    ("ray depth: determinant jacobian transposed", "dM[i * 3 + j] += gr[R_DET] * g.A[j * 3 + i];",
     "dM[i * 3 + j] += gr[R_DET] * g.A[i * 3 + j];"),
    ("ray depth where the low-pass term decides", "e->zray = cfg->depth_ray && e->obj && e->c != 0;",
     "e->zray = cfg->depth_ray && e->c != 0;"),
    ("distortion: factor 2 dropped", "d += 2.0 * wi * wj * (list[i].e.z - list[j].e.z);",
     "d += wi * wj * (list[i].e.z - list[j].e.z);"),
    ("distortion adjoint: terms behind the entry dropped", "const double Wk = 2.0 * (zi * Ap - Bp + Bsuf - zi * Asuf);",
     "const double Wk = 2.0 * (zi * Ap - Bp);"),
    ("distortion adjoint: depth gradient sign", "dzd = gd * 2.0 * w * (Ap - Asuf);", "dzd = gd * 2.0 * w * (Asuf - Ap);"),
    ("distortion adjoint: transmittance term", "da += gd * (Wk * Ti - Wsuf / om);", "da += gd * (Wk * Ti);"),
    ("error attribution summed", "if (e > max_err[list[k].s]) max_err[list[k].s] = e;",
     "max_err[list[k].s] += e;"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,bad", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, bad):
    src = open(os.path.join(ROOT, "oracle", "splat2d_oracle.c")).read()
    assert orig in src, f"mutation anchor for {name!r} no longer in the oracle"
    for d in ("oracle", "tests", "paper_2604_03092_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_lib", "__pycache__", "golden"))
    (tmp_path / "oracle" / "splat2d_oracle.c").write_text(src.replace(orig, bad))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"


# planted mistakes in the map-maintenance statements (oracle/fusion.py)
FUSION_MUTATIONS = [
    ("quaternion alignment dropped", "acc += q if np.dot(q, q1) >= 0 else -q", "acc += q"),
    ("scales left unscaled", "s2[i] = s * np.asarray(scales[i], np.float64)", "s2[i] = np.asarray(scales[i], np.float64)"),
    ("rotation product order", "q2[i] = quat_mul(q / np.linalg.norm(q), np.asarray(quats[i], np.float64))",
     "q2[i] = quat_mul(np.asarray(quats[i], np.float64), q / np.linalg.norm(q))"),
    ("depth gate inverted", "if max(z) - min(z) > tau_d:", "if max(z) - min(z) < tau_d:"),
    ("edge block size", "n = len(idx)", "n = 4"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,bad", FUSION_MUTATIONS, ids=[m[0] for m in FUSION_MUTATIONS])
def test_fusion_pins_catch_planted_mistake(tmp_path, name, orig, bad):
    src = open(os.path.join(ROOT, "oracle", "fusion.py")).read()
    assert orig in src, f"mutation anchor for {name!r} no longer in the oracle"
    for d in ("oracle", "tests", "paper_2604_03092_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_lib", "__pycache__", "golden"))
    (tmp_path / "oracle" / "fusion.py").write_text(src.replace(orig, bad))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_fusion.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
