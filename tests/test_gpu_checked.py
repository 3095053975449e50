"""The checked build (SPLAT2D_CHECKS=1): every kernel index check compiled
in, a failed check recorded as SPLAT2D_ERR_BOUNDS in the status word and
the access skipped.  Each case runs in a child process that builds and loads
that library: on valid inputs it must give exactly the normal build's
results with a clean status, and a corrupted sorted list must be reported,
not read."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_2604_03092_gb300 import _abi, scenes
from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

sc = scenes.random_scene(n=3000, width=96, height=72, f=70.0, seed=3, n_views=2)
params = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb)]
rast = Rasterizer(sc.views, sc.n, RasterConfig())
im = rast.forward(*params)
g = torch.Generator(device="cuda").manual_seed(0)
d = (torch.randn(3 * rast.n_pixels, device="cuda", generator=g), torch.randn(rast.n_pixels, device="cuda", generator=g),
     None, None)
grads = rast.backward(*params, d)
torch.cuda.synchronize()
status = rast.status()
out = {{"status": np.array(status)}}
for k in ("rgb", "depth", "normal", "alpha"):
    out[k] = getattr(im, k).cpu().numpy()
for k in ("means", "scales", "quats", "opacity", "rgb", "pose"):
    out["g_" + k] = getattr(grads, k).cpu().numpy()
if {corrupt}:
    # a surfel index far outside every view's range in the sorted list
    n = int(rast.stats()["n_instances"])
    vals = rast.ws_tensor(rast.layout.vals, n, torch.int32)
    vals[:8] = -16
    rast.render_fwd(rast.new_images())
    torch.cuda.synchronize()
    out["status_after"] = np.array(rast.status())
np.savez({path!r}, **out)
"""


def _run(tmp_path, checked: bool, corrupt: bool = False):
    path = str(tmp_path / f"out_{int(checked)}_{int(corrupt)}.npz")
    env = dict(os.environ, SPLAT2D_CHECKS="1" if checked else "0")
    code = CHILD.format(root=ROOT, corrupt=corrupt, path=path)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(path))


def test_checked_build_matches_and_stays_clean(tmp_path):
    plain = _run(tmp_path, checked=False)
    checked = _run(tmp_path, checked=True)
    assert int(plain["status"]) == 0 and int(checked["status"]) == 0
    for k, v in plain.items():
        if k == "status":
            continue
        if k.startswith("g_"):
            # gradient sums meet in atomics, so the two runs round in different
            # orders: compare as vectors, far below the parity bar of 1e-3
            diff = np.linalg.norm((checked[k] - v).ravel().astype(np.float64))
            assert diff <= 1e-5 * np.linalg.norm(v.ravel().astype(np.float64)), k
        else:  # the forward has no atomics: bit-identical
            np.testing.assert_array_equal(checked[k], v, err_msg=k)


def test_checked_build_reports_a_corrupted_list(tmp_path):
    from paper_2604_03092_gb300 import _abi
    res = _run(tmp_path, checked=True, corrupt=True)
    assert int(res["status"]) == 0
    assert int(res["status_after"]) == _abi.ERR_BOUNDS
