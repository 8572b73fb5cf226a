"""Host-side helpers for the aerial-city tests: seeded samples of image tiles, and a
conservative bound on which Gaussians can reach them, so that the oracle needs to see only
those (in their global order) to reproduce the full scene on the sampled tiles."""
import numpy as np


def tile_sample(cam, n, seed, B=16):
    """n distinct seeded tiles of B x B pixels: (tile mask [tiles], pixel mask [H, W])."""
    tw, th = (cam.width + B - 1) // B, (cam.height + B - 1) // B
    rng = np.random.default_rng(seed)
    mask = np.zeros(tw * th, np.uint8)
    mask[rng.choice(tw * th, size=n, replace=False)] = 1
    pix = np.zeros((th * B, tw * B), bool)
    pix.reshape(th, B, tw, B)[:] = mask.reshape(th, 1, tw, 1).astype(bool)
    return mask, pix[:cam.height, :cam.width]


def reach_tiles(sc, cam, tile_mask, B=16):
    """Boolean [n]: the Gaussians whose pixel rectangle can meet a tile of tile_mask.

    A superset of what the FP32 binning keeps: FP64 camera-space depth above half the near
    plane, and a radius bound 3 sqrt(|J|_F^2 s_max^2 + 0.3 + 0.32) + 2 pixels, since the
    2-D covariance J W Sigma W^T J^T has largest eigenvalue at most |J|_2^2 s_max^2 (W is a
    rotation, |J|_2 <= |J|_F, and clamping the Jacobian's x/z, y/z only lowers |J|), the
    dilation adds 0.3 and the binning's floor of 0.1 under the root adds at most
    sqrt(0.1) < 0.32 to the eigenvalue; 2 pixels cover the ceil and FP32 rounding."""
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    pc = sc.means.astype(np.float64) @ R.T + t
    z = pc[:, 2]
    front = z > 0.5 * cam.near
    z = np.where(front, z, 1.0)
    u = cam.fx * pc[:, 0] / z + cam.cx
    v = cam.fy * pc[:, 1] / z + cam.cy
    smax2 = np.exp(2.0 * sc.log_scales.astype(np.float64).max(axis=1))
    j2 = ((cam.fx / z) ** 2 + (cam.fy / z) ** 2 + (cam.fx * pc[:, 0] / z ** 2) ** 2 +
          (cam.fy * pc[:, 1] / z ** 2) ** 2)
    r = 3.0 * np.sqrt(j2 * smax2 + 0.62) + 2.0
    tw, th = (cam.width + B - 1) // B, (cam.height + B - 1) // B
    with np.errstate(invalid="ignore"):
        x0 = np.clip(np.floor((u - r) / B), 0, tw - 1).astype(np.int64)
        x1 = np.clip(np.floor((u + r) / B), 0, tw - 1).astype(np.int64)
        y0 = np.clip(np.floor((v - r) / B), 0, th - 1).astype(np.int64)
        y1 = np.clip(np.floor((v + r) / B), 0, th - 1).astype(np.int64)
        on = front & np.isfinite(u) & np.isfinite(v) & (u + r >= 0) & (u - r <= cam.width) & \
            (v + r >= 0) & (v - r <= cam.height)
    sat = np.zeros((th + 1, tw + 1), np.int64)
    sat[1:, 1:] = np.asarray(tile_mask).reshape(th, tw).astype(np.int64).cumsum(0).cumsum(1)
    hits = sat[y1 + 1, x1 + 1] - sat[y0, x1 + 1] - sat[y1 + 1, x0] + sat[y0, x0]
    return on & (hits > 0)
