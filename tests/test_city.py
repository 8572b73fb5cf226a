"""The aerial-city workload on the host: layout invariants, per-cell determinism, camera
poses, and the conservative tile-reach bound that lets the oracle check the 120M-Gaussian
step on sampled tiles from the Gaussians that can reach them."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

from city_util import reach_tiles, tile_sample


@pytest.fixture(scope="module")
def small_city():
    lay = I.city_layout(200_000, 9, 8)
    sc = [lay.cell_scene(k) for k in range(lay.K)]
    return lay, sc


def _concat(cells):
    return I.Scene(*(np.concatenate([getattr(c, a) for c in cells]) for a in
                     ("means", "log_scales", "quats", "opacity_logits", "sh")), cells[0].sh_degree)


def test_layout_cells_are_the_kd_boxes(small_city):
    lay, cells = small_city
    assert lay.offsets[-1] == 200_000 and np.all(np.diff(lay.offsets) == [c.n for c in cells])
    sizes = np.diff(lay.offsets)
    assert sizes.min() > 0.8 * sizes.mean()  # median splits of the surface mass
    for k, c in enumerate(cells):
        lo, hi = lay.boxes[k]
        m = c.means.astype(np.float64)
        for a in (0, 2):
            assert np.all(m[:, a] >= lo[a] - 1e-3) and np.all(m[:, a] <= hi[a] + 1e-3)
        assert np.all(m[:, 1] <= 1e-6) and np.all(m[:, 1] >= -200.0)  # ground up to roofs
    assert np.all(np.abs(np.linalg.norm(cells[0].quats, axis=1) - 1) < 1e-5)


def test_cells_regenerate_identically(small_city):
    lay, cells = small_city
    again = lay.cell_scene(3)
    for a, b in zip(again.arrays(), cells[3].arrays()):
        assert np.array_equal(a, b)


def test_aerial_cameras_look_down_from_altitude():
    cams = I.aerial_cameras(4, n=60)
    for c in cams:
        R = c.R.astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6) and np.linalg.det(R) > 0.999
        assert 150.0 <= -c.eye[1] <= 300.0
        fwd_down = R[2, 1]  # world +y is down
        assert np.sin(np.radians(45.0)) - 1e-6 <= fwd_down <= 1.0 + 1e-6
    v = I.step_views(4, 7, 500)
    assert len(set(v.tolist())) == 8 and v.max() < 500


def _camera_seeing(lay, cells):
    for c in I.aerial_cameras(9, n=40, size=(640, 360)):
        vis, _, _ = O.bin(_concat(cells), c)
        if vis.sum() > 5000:
            return c
    raise AssertionError("no camera sees the city")


def test_reach_bound_contains_the_binned_gaussians(small_city):
    lay, cells = small_city
    sc = _concat(cells)
    cam = _camera_seeing(lay, cells)
    mask, _ = tile_sample(cam, 60, 5)
    vis, rect, _ = O.bin(sc, cam)
    B = 16
    tw = (cam.width + B - 1) // B
    m2 = mask.reshape(-1, tw)
    binned = np.zeros(sc.n, bool)
    for g in np.nonzero(vis)[0]:
        x0, x1, y0, y1 = rect[g]
        binned[g] = m2[y0 // B:y1 // B + 1, x0 // B:x1 // B + 1].any()
    reach = reach_tiles(sc, cam, mask)
    assert binned.sum() > 100
    assert not np.any(binned & ~reach)
    assert reach.sum() < 0.5 * sc.n  # the bound still selects


def test_oracle_on_the_reaching_gaussians_equals_the_full_scene(small_city):
    lay, cells = small_city
    sc = _concat(cells)
    cam = _camera_seeing(lay, cells)
    mask, pix = tile_sample(cam, 24, 6)
    reach = reach_tiles(sc, cam, mask)
    sub = sc.take(np.nonzero(reach)[0])
    cell_of = np.searchsorted(lay.offsets, np.nonzero(reach)[0], side="right") - 1
    sub_off = np.zeros(lay.K + 1, np.int64)
    sub_off[1:] = np.cumsum(np.bincount(cell_of, minlength=lay.K))
    order = list(O.cell_order(lay.boxes, cam.eye))
    full = O.render_view(sc, lay.offsets, cam, O.opts(), tile_mask=mask, order=order)
    part = O.render_view(sub, sub_off, cam, O.opts(), tile_mask=mask, order=order)
    assert np.array_equal(full["image"][:, pix], part["image"][:, pix])
