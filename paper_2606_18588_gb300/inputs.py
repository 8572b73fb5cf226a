"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only draws numbers and arranges them: Gaussian scenes, cameras, target
images and the k-d split that forms the K convex subsets.  It holds none of the
rendering arithmetic (projection, binning, blending, composition, gradients).

Layouts (all float32, C-contiguous):
  means [N,3], log_scales [N,3], quats [N,4] as (w,x,y,z), opacity_logits [N],
  sh [N,(deg+1)^2,3]  (coefficient-major, RGB innermost).
Camera: world->camera rotation R (3x3, rows = camera right, down, forward), t (3),
pinhole fx, fy, cx, cy, width, height, near.  Camera space is x right, y down, z forward.

The synthetic recipes stand in for the paper's MatrixCity scenes (Sec. 5), which are
not available; the scene shapes follow the workloads it describes (Sec. 5, Sec. 8.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Real spherical-harmonic DC normalisation Y_00 = 1/(2 sqrt(pi)).  Only used to turn
# a drawn RGB into the DC coefficient that reproduces it (colour = Y_00*dc + 0.5).
_INV_Y00 = 2.0 * math.sqrt(math.pi)


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, lo: int, hi: int) -> "Scene":
        return Scene(self.means[lo:hi], self.log_scales[lo:hi], self.quats[lo:hi],
                     self.opacity_logits[lo:hi], self.sh[lo:hi], self.sh_degree)

    def take(self, idx: np.ndarray) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in
                       (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)),
                     self.sh_degree)

    def arrays(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # (3,3) float32, world -> camera rotation
    t: np.ndarray          # (3,)  float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01

    @property
    def eye(self) -> np.ndarray:
        """Camera centre in world coordinates (float64)."""
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


def n_sh_coeffs(deg: int) -> int:
    return (deg + 1) * (deg + 1)


def look_at(eye, target, world_up=(0.0, -1.0, 0.0)):
    """Rotation/translation of a camera at `eye` looking at `target` (x right, y down, z forward)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(world_up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    return R, t


def pinhole(width: int, height: int, fov_x_deg: float, eye, target, near=0.01,
            world_up=(0.0, -1.0, 0.0)) -> Camera:
    R, t = look_at(eye, target, world_up)
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(R, t, float(np.float32(fx)), float(np.float32(fx)),
                  0.5 * width, 0.5 * height, int(width), int(height), float(near))


def _quats(rng, n):
    q = rng.standard_normal((n, 4), dtype=np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng, n, deg, rgb):
    c = n_sh_coeffs(deg)
    sh = np.zeros((n, c, 3), np.float32)
    sh[:, 0, :] = (rgb - 0.5) * _INV_Y00
    if c > 1:
        rest = rng.standard_normal((n, c - 1, 3), dtype=np.float32)
        rest *= np.float32(0.2)
        sh[:, 1:, :] = rest
    return sh


def uniform_scene(n: int, seed: int, sh_degree: int = 0, log_scale_mu=-3.5,
                  log_scale_sigma=0.5, extent=1.0) -> Scene:
    """Means ~ U[-extent,extent]^3, log-scales ~ N(mu, sigma), unit quaternions uniform
    on S^3, opacity = sigmoid(N(0,1)), RGB ~ U[0,1] (the 10k-Gaussian plain-forward case)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-extent, extent, (n, 3)).astype(np.float32)
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = _quats(rng, n)
    logits = rng.standard_normal(n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    return Scene(means, log_scales, quats, logits, _sh(rng, n, sh_degree, rgb), sh_degree)


def cluster_scene(n: int, seed: int, sh_degree: int = 3, n_clusters: int = 64,
                  box: float = 20.0, sigma_range=(0.5, 2.0), log_scale_sigma=0.5) -> Scene:
    """Means from an equal-weight mixture of isotropic clusters inside a cube of side
    `box` centred at the origin (points outside are redrawn); log-scale mean chosen so
    that a Gaussian's scale is about a third of the mean spacing (V_box/N)^(1/3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    half = 0.5 * box
    centres = rng.uniform(-half, half, (n_clusters, 3))
    sig = rng.uniform(sigma_range[0], sigma_range[1], n_clusters)
    lab = rng.integers(0, n_clusters, n)
    means = centres[lab] + sig[lab, None] * rng.standard_normal((n, 3))
    bad = np.nonzero(np.any(np.abs(means) > half, axis=1))[0]  # ascending indices
    while bad.size:
        means[bad] = centres[lab[bad]] + sig[lab[bad], None] * rng.standard_normal((bad.size, 3))
        bad = bad[np.any(np.abs(means[bad]) > half, axis=1)]
    means = means.astype(np.float32)
    mu = math.log(0.33 * (box ** 3 / n) ** (1.0 / 3.0))
    log_scales = rng.normal(mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = _quats(rng, n)
    logits = rng.standard_normal(n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    return Scene(means, log_scales, quats, logits, _sh(rng, n, sh_degree, rgb), sh_degree)


def morton_codes(points: np.ndarray) -> np.ndarray:
    """30-bit Morton (Z-order) codes of points quantised to 1024 cells per axis of their
    bounding box."""
    lo = points.min(axis=0)
    ext = np.maximum(points.max(axis=0) - lo, 1e-12)
    q = np.clip(((points - lo) / ext * 1023.0).astype(np.int64), 0, 1023)
    code = np.zeros(points.shape[0], np.int64)
    for a in range(3):  # bit b of axis a goes to bit 3 b + a
        v = q[:, a]
        v = (v | (v << 16)) & 0x030000FF
        v = (v | (v << 8)) & 0x0300F00F
        v = (v | (v << 4)) & 0x030C30C3
        v = (v | (v << 2)) & 0x09249249
        code |= v << a
    return code


def kd_partition(means: np.ndarray, K: int, axes=(0, 2), spatial_order: bool = True):
    """Recursive median split into K (a power of two) axis-aligned boxes.

    At every node the split axis is the one of `axes` with the largest extent of the
    node's means; the node's Gaussians are ordered by (coordinate, index) and the left
    child takes the first floor(n/2) (Sec. 8.1, partition strategy).  Within each box the
    Gaussians are then laid out in Morton order of their means (spatial_order), so that
    neighbours in memory are neighbours on screen.  Returns the permutation that makes
    subsets contiguous, the K+1 subset offsets, and each subset's (lo, hi) split-plane box
    (infinite on unsplit sides).
    """
    if K < 1 or (K & (K - 1)) != 0:
        raise ValueError("K must be a power of two")
    n = means.shape[0]
    m = means.astype(np.float64)
    groups = [(np.arange(n), np.full(3, -np.inf), np.full(3, np.inf))]
    while len(groups) < K:
        nxt = []
        for idx, lo, hi in groups:
            ext = [m[idx, a].max() - m[idx, a].min() if idx.size else 0.0 for a in axes]
            ax = axes[int(np.argmax(ext))]
            # idx is ascending, so a stable sort by coordinate orders by (coordinate, index)
            order = np.argsort(m[idx, ax], kind="stable")
            idx = idx[order]
            h = idx.size // 2
            left, right = idx[:h], idx[h:]
            if left.size and right.size:
                plane = 0.5 * (m[left[-1], ax] + m[right[0], ax])
            else:
                plane = 0.0
            lhi = hi.copy(); lhi[ax] = plane
            rlo = lo.copy(); rlo[ax] = plane
            nxt.append((np.sort(left), lo, lhi))
            nxt.append((np.sort(right), rlo, hi))
        groups = nxt
    if spatial_order:
        groups = [(idx[np.argsort(morton_codes(m[idx]), kind="stable")], lo, hi)
                  for idx, lo, hi in groups]
    perm = np.concatenate([g[0] for g in groups]).astype(np.int64)
    offsets = np.zeros(K + 1, np.int64)
    offsets[1:] = np.cumsum([g[0].size for g in groups])
    boxes = np.stack([np.stack([g[1], g[2]]) for g in groups])
    return perm, offsets, boxes


def orbit_cameras(n_views: int, seed: int, sizes, radius=25.0, height=(2.0, 10.0),
                  fov_x_deg=60.0, centre=(0.0, 0.0, 0.0), near=0.01):
    """Cameras on a seeded orbit around `centre` (world up is -y), looking at it.
    `sizes` is a list of (width, height) cycled over the views."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cams = []
    c = np.asarray(centre, np.float64)
    for i in range(n_views):
        phi = rng.uniform(0.0, 2.0 * math.pi)
        h = rng.uniform(height[0], height[1])
        eye = c + np.array([radius * math.cos(phi), -h, radius * math.sin(phi)])
        w, hh = sizes[i % len(sizes)]
        cams.append(pinhole(w, hh, fov_x_deg, eye, c, near))
    return cams


def random_image(height: int, width: int, seed: int) -> np.ndarray:
    """Target image ~ U[0,1], planar [3,H,W] float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)


def plain_forward_case(seed: int = 0, n: int = 10_000):
    """10k Gaussians, SH degree 0, means U[-1,1]^3, 256x256, fov 60 deg, eye at distance 3
    looking at the origin, near 0.01, one subset."""
    scene = uniform_scene(n, seed, 0)
    cam = pinhole(256, 256, 60.0, (0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 0.01)
    return scene, cam


def cluster_case(n: int, seed: int, K: int, n_views: int, sizes, sh_degree: int = 3):
    """A cluster scene reordered so its K k-d subsets (split on x/z) are contiguous,
    plus orbit cameras.  Returns (scene, offsets, boxes, cameras)."""
    scene = cluster_scene(n, seed, sh_degree)
    perm, offsets, boxes = kd_partition(scene.means, K)
    scene = scene.take(perm)
    cams = orbit_cameras(n_views, seed + 1, sizes)
    return scene, offsets, boxes, cams


# ---------------------------------------------------------------- city layout
# The 120M-Gaussian training step stands in for an aerial city capture (the paper's
# MatrixCity aerial scenes, Sec. 5): a street grid of square blocks over 1 km x 1 km, each
# block's lots holding a building box with a lognormal height; Gaussians lie on the ground,
# the facades and the roofs, with a lognormal density per block.  The scene is generated
# one k-d cell at a time, so that no host ever holds all of it.

@dataclasses.dataclass
class CityLayout:
    """Surface pieces of the city clipped to the K k-d cells, with their Gaussian counts.

    Piece p is the axis-aligned box [lo[p], hi[p]] with one degenerate axis (a flat
    rectangle); its count[p] Gaussians are uniform on it.  Cell k holds the pieces with
    cell[p] == k and becomes the contiguous subset [offsets[k], offsets[k+1]).
    """
    n: int
    seed: int
    K: int
    sh_degree: int
    lo: np.ndarray
    hi: np.ndarray
    cell: np.ndarray
    count: np.ndarray
    offsets: np.ndarray
    boxes: np.ndarray
    log_scale_mu: float

    def cell_scene(self, k: int) -> Scene:
        """The Gaussians of cell k, means in Morton order (deterministic in (seed, k)
        alone).  The other attributes are i.i.d., drawn after the means in their final
        order."""
        rng = np.random.Generator(np.random.PCG64([self.seed, 3, k]))
        sel = np.nonzero(self.cell == k)[0]
        n = int(self.count[sel].sum())
        means = np.empty((n, 3), np.float64)
        at = 0
        for p in sel:
            c = int(self.count[p])
            if c:
                u = rng.uniform(0.0, 1.0, (c, 3))
                means[at:at + c] = self.lo[p] + u * (self.hi[p] - self.lo[p])
                at += c
        means = means.astype(np.float32)
        if n:
            means = means[np.argsort(morton_codes(means), kind="stable")]
        log_scales = rng.normal(self.log_scale_mu, 0.5, (n, 3)).astype(np.float32)
        quats = _quats(rng, n)
        logits = rng.standard_normal(n).astype(np.float32)
        rgb = rng.uniform(0.0, 1.0, (n, 3))
        return Scene(means, log_scales, quats, logits, _sh(rng, n, self.sh_degree, rgb),
                     self.sh_degree)


def _city_surfaces(rng, extent, block, street):
    """Axis-aligned surface rectangles (lo, hi) of the city and their density weights."""
    nb = int(round(extent / block))
    half = 0.5 * extent
    lo, hi, dens = [], [], []

    def add(a, b, d):
        lo.append(a); hi.append(b); dens.append(d)

    for bi in range(nb):
        for bj in range(nb):
            x0, z0 = -half + bi * block, -half + bj * block
            d = float(rng.lognormal(0.0, 0.6))
            add((x0, 0.0, z0), (x0 + block, 0.0, z0 + block), d)  # ground, streets included
            g = int(rng.integers(2, 4))
            lot = (block - street) / g
            for li in range(g):
                for lj in range(g):
                    w, dp = lot * rng.uniform(0.6, 0.9), lot * rng.uniform(0.6, 0.9)
                    cx = x0 + 0.5 * street + (li + 0.5) * lot
                    cz = z0 + 0.5 * street + (lj + 0.5) * lot
                    h = float(np.clip(rng.lognormal(math.log(25.0), 0.6), 4.0, 200.0))
                    ax0, ax1, az0, az1 = cx - 0.5 * w, cx + 0.5 * w, cz - 0.5 * dp, cz + 0.5 * dp
                    add((ax0, -h, az0), (ax1, -h, az1), d)  # roof (world up is -y)
                    add((ax0, -h, az0), (ax0, 0.0, az1), d)  # facades
                    add((ax1, -h, az0), (ax1, 0.0, az1), d)
                    add((ax0, -h, az0), (ax1, 0.0, az0), d)
                    add((ax0, -h, az1), (ax1, 0.0, az1), d)
    return np.array(lo), np.array(hi), np.array(dens)


def _area(lo, hi):
    e = hi - lo
    return e[:, 0] * e[:, 1] + e[:, 1] * e[:, 2] + e[:, 0] * e[:, 2]  # one extent is zero


def city_layout(n: int, seed: int, K: int, sh_degree: int = 3, extent=1000.0, block=100.0,
                street=20.0, sample=1 << 20) -> CityLayout:
    """Lays out the city, splits it into K k-d cells on x/z (median splits of a 1M-point
    sample of the surface distribution) and draws each clipped piece's Gaussian count.
    Log-scales ~ N(ln(0.5 s), 0.5) with s = sqrt(surface area / n), the mean spacing of
    the Gaussians on the surfaces."""
    rng = np.random.Generator(np.random.PCG64([seed, 0]))
    lo, hi, dens = _city_surfaces(rng, extent, block, street)
    area = _area(lo, hi)
    w = area * dens
    srng = np.random.Generator(np.random.PCG64([seed, 1]))
    pick = srng.choice(len(w), size=sample, p=w / w.sum())
    pts = lo[pick] + srng.uniform(0.0, 1.0, (sample, 3)) * (hi[pick] - lo[pick])
    _, _, boxes = kd_partition(pts, K, spatial_order=False)
    # clip every surface to every cell; a flat side on a split plane belongs to the cell
    # whose box starts there (half-open cells)
    plo, phi, pcell, pw = [], [], [], []
    for k in range(K):
        blo, bhi = boxes[k, 0], boxes[k, 1]
        a, b = np.maximum(lo, blo), np.minimum(hi, bhi)
        flat = lo == hi
        ok = np.all(np.where(flat, (lo >= blo) & (lo < bhi), b > a), axis=1)
        a, b = np.where(flat, lo, a), np.where(flat, hi, b)
        idx = np.nonzero(ok)[0]
        plo.append(a[idx]); phi.append(b[idx]); pcell.append(np.full(idx.size, k))
        pw.append(_area(a[idx], b[idx]) * dens[idx])
    plo, phi = np.concatenate(plo), np.concatenate(phi)
    pcell, pw = np.concatenate(pcell), np.concatenate(pw)
    count = np.random.Generator(np.random.PCG64([seed, 2])).multinomial(n, pw / pw.sum())
    offsets = np.zeros(K + 1, np.int64)
    offsets[1:] = np.cumsum(np.bincount(pcell, weights=count, minlength=K).astype(np.int64))
    mu = math.log(0.5 * math.sqrt(area.sum() / n))
    return CityLayout(n, seed, K, sh_degree, plo, phi, pcell, count.astype(np.int64), offsets,
                      boxes, mu)


def aerial_cameras(seed: int, n: int = 500, grid=(25, 20), extent=1000.0, altitude=(150.0, 300.0),
                   pitch_deg=(45.0, 90.0), fov_x_deg=60.0, size=(1920, 1080), near=0.01):
    """Aerial cameras on a grid x grid[1] lattice over the city, altitude, heading and
    downward pitch uniform (world up is -y)."""
    rng = np.random.Generator(np.random.PCG64([seed, 4]))
    half = 0.5 * extent
    xs = np.linspace(-half, half, grid[0] + 2)[1:-1]
    zs = np.linspace(-half, half, grid[1] + 2)[1:-1]
    w, h = size
    fx = float(np.float32(0.5 * w / math.tan(math.radians(fov_x_deg) * 0.5)))
    cams = []
    for i in range(n):
        gx, gz = xs[i % grid[0]], zs[(i // grid[0]) % grid[1]]
        alt = rng.uniform(*altitude)
        head = rng.uniform(0.0, 2.0 * math.pi)
        p = math.radians(rng.uniform(*pitch_deg))
        f = np.array([math.cos(p) * math.cos(head), math.sin(p), math.cos(p) * math.sin(head)])
        r = np.array([math.sin(head), 0.0, -math.cos(head)])
        d = np.cross(f, r)
        R = np.stack([r, d, f]).astype(np.float32)
        eye = np.array([gx, -alt, gz])
        t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
        cams.append(Camera(R, t, fx, fx, 0.5 * w, 0.5 * h, int(w), int(h), float(near)))
    return cams


def step_views(seed: int, step: int, pool: int, n: int = 8) -> np.ndarray:
    """The n distinct camera indices a training step samples from the pool."""
    rng = np.random.Generator(np.random.PCG64([seed, 5, step]))
    return np.sort(rng.choice(pool, size=n, replace=False))


# Named workloads (sizes follow the five configurations the hot path is quoted on).
WORKLOADS = {
    "plain_fwd_10k": dict(n=10_000, sh_degree=0, K=1, sizes=[(256, 256)], views=1),
    "fwdbwd_1m_k4": dict(n=1_000_000, sh_degree=3, K=4, sizes=[(1920, 1080)], views=1),
    "batched_10m_k8": dict(n=10_000_000, sh_degree=3, K=8,
                           sizes=[(1600, 1064), (1280, 720)], views=16),
    "train_120m_k32": dict(n=120_000_000, sh_degree=3, K=32, sizes=[(1920, 1080)], views=8),
    "serve_20m_k8": dict(n=20_000_000, sh_degree=3, K=8,
                         sizes=[(512, 512), (1280, 720), (1920, 1080), (3840, 2160)], views=0),
}
