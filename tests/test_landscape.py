"""2-D landscapes (App. A plots as data): the grid, the image and CSV writers
on the CPU; on the GPU, the grid values against the FP64 oracle at the same
points and, for a unimodal function, the minimum at the grid point next to
the optimum."""
import os

import numpy as np
import pytest

from paper_1407_7737_gb300 import landscape as ls


def test_grid_layout():
    p = ls.grid_points(3, -1.0, 1.0)
    assert p.shape == (9, 2)
    assert np.array_equal(p[:3, 0], [-1.0, 0.0, 1.0]) and np.all(p[:3, 1] == -1.0)
    assert np.all(p[6:, 1] == 1.0)


def test_pgm_and_csv_writers(tmp_path):
    f = 100.0 + np.add.outer(np.arange(4.0), np.arange(5.0)) ** 2  # min at (0, 0)
    g = ls.to_grey(f)
    assert g.dtype == np.uint16 and g[0, 0] == 0 and g.max() == 65535
    path = os.path.join(tmp_path, "f.pgm")
    ls.write_pgm(path, f)
    raw = open(path, "rb").read()
    head = b"P5\n5 4\n65535\n"
    assert raw.startswith(head) and len(raw) == len(head) + 2 * 20
    img = np.frombuffer(raw[len(head):], dtype=">u2").reshape(4, 5)
    assert img[-1, 0] == 0  # the bottom row is the lowest x_2
    cpath = os.path.join(tmp_path, "f.csv")
    ls.write_csv(cpath, np.full((2, 2), 101.5), -1.0, 1.0)
    rows = np.loadtxt(cpath, delimiter=",", skiprows=1)
    assert rows.shape == (4, 3) and np.all(rows[:, 2] == 101.5)


@pytest.mark.gpu
@pytest.mark.parametrize("fid", [0, 8, 12, 30])
def test_landscape_matches_oracle(orc, fid):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import gpu_util as gu
    gu.invalidate()  # the landscape initialises the library itself
    res, seed = 41, 3
    f = ls.landscape(fid, res, seed=seed)
    pts = ls.grid_points(res)
    ref = orc.evaluate(fid, 2, seed, pts).reshape(res, res)
    assert np.all(np.abs(f - ref) <= 1e-12 * np.abs(ref))
    if fid == 0:  # Sphere: the grid minimum sits next to the optimum
        o = orc.generate(fid, 2, seed)[0].o
        i, j = np.unravel_index(np.argmin(f), f.shape)
        step = 200.0 / (res - 1)
        assert abs(pts[i * res + j, 0] - o[0]) <= step / 2 + 1e-9
        assert abs(pts[i * res + j, 1] - o[1]) <= step / 2 + 1e-9
