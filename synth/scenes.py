"""Seeded synthetic multi-camera scenes: the input generator shared by the
tests, the smoke check and the benchmark.

It holds none of the method's arithmetic.  It places pinhole cameras, builds
"players" as unions of ellipsoids, and renders exact silhouettes and flat
colour images by casting one ray per pixel centre (float64).  Both the CUDA
path and the CPU oracle consume what it returns; neither is imported here.

Workload shapes (the paper's volleyball and judo captures are not available,
so these stand in for them):

* ``tiny``        8 cameras 640x360 (f=500) on a 6 m ring at 3 m, one player,
                  volume 4x4x2.5 m, coarse 5 cm, fine 1 cm, 8 bisection steps.
* ``volleyball``  16 cameras 1920x1080 (f=1800) on an ellipse with semi-axes
                  30x20 m at 6-10 m height, 12 players (1.7-2.0 m) and a
                  0.21 m ball over an 18x9 m court, volume 20x11x4 m, coarse
                  5 cm (400x220x80), fine 1 cm, 10 bisection steps.
* ``judo``        12 cameras 3840x2160 (f=3600) on a 14 m ring at 6 m, two
                  interlocked players and a referee, volume 12x12x3 m,
                  coarse 4 cm, fine 5 mm, 12 bisection steps.
* ``hd720``       8 cameras 1280x720 (f=1000) on an 8 m ring at 4 m, three
                  players, volume 8x8x2.5 m, coarse 5 cm, fine 1 cm, 8 steps.

Silhouettes get i.i.d. Bernoulli(0.001) pixel flips.  Every random draw comes
from a ``torch.Generator`` seeded from (SEED_BASE, config, frame index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SEED_BASE = 1903_11785

STRICT = 0
ABSTAIN = 1

# Player model at height 1.8 m: (count, centre, semi-axes) in the player frame
# (x to the player's side, z up).  Each part is one ellipsoid with a flat colour.
PLAYER_PARTS = (
    ((-0.09, 0.0, 0.45), (0.08, 0.08, 0.45)),   # left leg
    ((0.09, 0.0, 0.45), (0.08, 0.08, 0.45)),    # right leg
    ((0.0, 0.0, 1.20), (0.20, 0.13, 0.35)),     # torso
    ((0.0, 0.0, 1.66), (0.10, 0.10, 0.12)),     # head
    ((-0.25, 0.0, 1.20), (0.06, 0.06, 0.33)),   # left arm
    ((0.25, 0.0, 1.20), (0.06, 0.06, 0.33)),    # right arm
)
BACKGROUND_RGB = (128, 128, 128)


@dataclass
class Ellipsoid:
    centre: np.ndarray      # (3,) float64
    rot: np.ndarray         # (3,3) float64, columns = the ellipsoid's axes in world
    axes: np.ndarray        # (3,) float64 semi-axes
    colour: tuple           # uint8 RGB
    obj: int = 0            # index of the object (player / ball) it belongs to


@dataclass
class Rig:
    """Cameras plus the reconstruction parameters of one capture setup."""
    name: str
    P: np.ndarray           # (N,3,4) float32 world -> pixel
    centre: np.ndarray      # (N,3) float32
    width: np.ndarray       # (N,) int32
    height: np.ndarray      # (N,) int32
    vol_min: tuple
    vol_max: tuple
    coarse_m: float
    fine_m: float
    bisect_steps: int
    t_np: int = 8
    t_nb: int = 2**31 - 1
    t_v: float = 0.5
    oob_policy: int = STRICT
    surface_rule: int = 0   # 0: bisection, 1: the paper's pixel walk and minimum ratio (Eqs. (2)-(3))
    P64: np.ndarray = field(default=None, repr=False)       # float64 originals
    K64: np.ndarray = field(default=None, repr=False)
    R64: np.ndarray = field(default=None, repr=False)
    C64: np.ndarray = field(default=None, repr=False)

    @property
    def n_cams(self) -> int:
        return int(self.P.shape[0])

    def grid_dims(self):
        def um(x):
            return int(round(float(np.float32(x)) * 1e6))
        s = um(self.coarse_m)
        return tuple(-(-(um(self.vol_max[a]) - um(self.vol_min[a])) // s) for a in range(3))


@dataclass
class Frame:
    masks: torch.Tensor     # (N,H,W) uint8, nonzero = foreground
    rgb: torch.Tensor       # (N,H,W,3) uint8
    ellipsoids: list
    viewpoint: np.ndarray   # (3,) float32 virtual viewpoint


# ----------------------------------------------------------------- cameras

def _rot_xyz(yaw, pitch, roll):
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1.0]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return Rz @ Ry @ Rx


def look_at_camera(C, target, f, W, H, jitter=(0.0, 0.0, 0.0)):
    """K, R (world->camera rows: right, down, forward) and P = K [R | -R C]."""
    C = np.asarray(C, np.float64)
    fwd = np.asarray(target, np.float64) - C
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    R = _rot_xyz(*jitter) @ R
    K = np.array([[f, 0.0, W / 2.0], [0.0, f, H / 2.0], [0.0, 0.0, 1.0]])
    P = K @ np.concatenate([R, -R @ C[:, None]], axis=1)
    return K, R, P


def _make_rig(name, centres, targets, f, W, H, gen, vol_min, vol_max, coarse, fine, steps,
              jitter_deg=2.0):
    Ks, Rs, Ps = [], [], []
    for C, T in zip(centres, targets):
        j = (torch.rand(3, generator=gen, dtype=torch.float64).numpy() * 2 - 1) * math.radians(jitter_deg)
        K, R, P = look_at_camera(C, T, f, W, H, tuple(j))
        Ks.append(K); Rs.append(R); Ps.append(P)
    n = len(centres)
    P64 = np.stack(Ps)
    return Rig(name=name, P=P64.astype(np.float32), centre=np.asarray(centres, np.float64).astype(np.float32),
               width=np.full(n, W, np.int32), height=np.full(n, H, np.int32),
               vol_min=tuple(float(x) for x in vol_min), vol_max=tuple(float(x) for x in vol_max),
               coarse_m=coarse, fine_m=fine, bisect_steps=steps,
               P64=P64, K64=np.stack(Ks), R64=np.stack(Rs), C64=np.asarray(centres, np.float64))


def _gen(config: str, index: int = 0, device="cpu") -> torch.Generator:
    """Generator seeded from (SEED_BASE, config, index) on `device` (the CPU and
    CUDA generators give different streams from the same seed)."""
    g = torch.Generator(device=device)
    code = sum((i + 1) * ord(c) for i, c in enumerate(config))
    g.manual_seed(SEED_BASE * 1000003 + code * 7919 + index)
    return g


def make_rig(config: str) -> Rig:
    g = _gen(config + "/rig")
    if config == "tiny":
        n, r, h = 8, 6.0, 3.0
        phase = float(torch.rand(1, generator=g, dtype=torch.float64)) * 2 * math.pi / n
        cs = [(r * math.cos(phase + 2 * math.pi * k / n), r * math.sin(phase + 2 * math.pi * k / n), h)
              for k in range(n)]
        return _make_rig("tiny", cs, [(0, 0, 0.9)] * n, 500.0, 640, 360, g,
                         (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 8)
    if config == "volleyball":
        n = 16
        cs = []
        for k in range(n):
            a = 2 * math.pi * (k + 0.5) / n
            hgt = 6.0 + 4.0 * float(torch.rand(1, generator=g, dtype=torch.float64))
            cs.append((30.0 * math.cos(a), 20.0 * math.sin(a), hgt))
        return _make_rig("volleyball", cs, [(0, 0, 1.0)] * n, 1800.0, 1920, 1080, g,
                         (-10.0, -5.5, 0.0), (10.0, 5.5, 4.0), 0.05, 0.01, 10)
    if config == "judo":
        n, r, h = 12, 14.0, 6.0
        cs = [(r * math.cos(2 * math.pi * (k + 0.25) / n), r * math.sin(2 * math.pi * (k + 0.25) / n), h)
              for k in range(n)]
        return _make_rig("judo", cs, [(0, 0, 0.8)] * n, 3600.0, 3840, 2160, g,
                         (-6.0, -6.0, 0.0), (6.0, 6.0, 3.0), 0.04, 0.005, 12)
    if config == "volleyball_t1":
        # the paper's volleyball capture shape (Table I): 10 cameras at 4K,
        # an 18 x 18 x 9 m volume, 50 mm coarse and 20 mm fine voxels
        n = 10
        cs = []
        for k in range(n):
            a = 2 * math.pi * (k + 0.5) / n
            hgt = 6.0 + 4.0 * float(torch.rand(1, generator=g, dtype=torch.float64))
            cs.append((30.0 * math.cos(a), 20.0 * math.sin(a), hgt))
        return _make_rig("volleyball_t1", cs, [(0, 0, 1.0)] * n, 3600.0, 3840, 2160, g,
                         (-9.0, -9.0, 0.0), (9.0, 9.0, 9.0), 0.05, 0.02, 10)
    if config == "judo_t1":
        # the paper's judo capture shape (Table I): 16 cameras at 1080p, a
        # 5 x 6 x 2.1 m volume, 80 mm coarse and 40 mm fine voxels
        n, r, h = 16, 14.0, 6.0
        cs = [(r * math.cos(2 * math.pi * (k + 0.25) / n), r * math.sin(2 * math.pi * (k + 0.25) / n), h)
              for k in range(n)]
        return _make_rig("judo_t1", cs, [(0, 0, 0.8)] * n, 1800.0, 1920, 1080, g,
                         (-2.5, -3.0, 0.0), (2.5, 3.0, 2.1), 0.08, 0.04, 10)
    if config == "hd720":
        n, r, h = 8, 8.0, 4.0
        cs = [(r * math.cos(2 * math.pi * (k + 0.5) / n), r * math.sin(2 * math.pi * (k + 0.5) / n), h)
              for k in range(n)]
        return _make_rig("hd720", cs, [(0, 0, 0.9)] * n, 1000.0, 1280, 720, g,
                         (-4.0, -4.0, 0.0), (4.0, 4.0, 2.5), 0.05, 0.01, 8)
    raise ValueError(f"unknown config {config!r}")


# ----------------------------------------------------------------- objects

def _random_colour(g):
    return tuple(int(x) for x in torch.randint(20, 236, (3,), generator=g))


def player(pos, yaw, height, g, obj=0):
    s = height / 1.8
    Rz = _rot_xyz(yaw, 0.0, 0.0)
    parts = []
    for c, ax in PLAYER_PARTS:
        c = np.asarray(c, np.float64) * s
        parts.append(Ellipsoid(centre=np.array([pos[0], pos[1], 0.0]) + Rz @ c, rot=Rz,
                               axes=np.asarray(ax, np.float64) * s, colour=_random_colour(g), obj=obj))
    return parts


def ball(pos, radius, g, obj=0):
    return [Ellipsoid(centre=np.asarray(pos, np.float64), rot=np.eye(3), axes=np.full(3, radius),
                      colour=_random_colour(g), obj=obj)]


def sphere_scene(centre, radius):
    return [Ellipsoid(centre=np.asarray(centre, np.float64), rot=np.eye(3), axes=np.full(3, float(radius)),
                      colour=(200, 40, 40), obj=0)]


def _u(g, lo, hi):
    return lo + (hi - lo) * float(torch.rand(1, generator=g, dtype=torch.float64))


def scene_objects(config: str, index: int = 0):
    """Ellipsoids of frame `index` of a config (players on smooth seeded paths)."""
    g = _gen(config + "/scene")
    t = index / 30.0
    if config == "tiny":
        pos = (_u(g, -1.5, 1.5), _u(g, -1.5, 1.5))
        return player(pos, _u(g, 0, 2 * math.pi), 1.8, g)
    if config == "volleyball_t1":
        return scene_objects("volleyball", index)
    if config == "judo_t1":
        # the judo pair near the middle of the 5 x 6 m volume and the referee
        # 2 m from it along y, on the side with more room
        cx, cy = _u(g, -0.5, 0.5), _u(g, -0.5, 0.5)
        yaw = _u(g, 0, 2 * math.pi)
        d = np.array([math.cos(yaw), math.sin(yaw)]) * 0.225
        objs = player((cx - d[0], cy - d[1]), yaw, _u(g, 1.7, 1.9), g, obj=0)
        objs += player((cx + d[0], cy + d[1]), yaw + math.pi, _u(g, 1.7, 1.9), g, obj=1)
        side = -1.0 if cy > 0 else 1.0
        objs += player((cx + _u(g, -0.3, 0.3), cy + 2.0 * side), _u(g, 0, 2 * math.pi), 1.75, g, obj=2)
        return objs
    if config == "volleyball":
        objs, placed = [], []
        for p in range(12):
            xlo, xhi = (-8.2, -0.8) if p < 6 else (0.8, 8.2)
            for _ in range(1000):
                base = (_u(g, xlo, xhi), _u(g, -3.8, 3.8))
                if all(math.hypot(base[0] - q[0], base[1] - q[1]) >= 0.9 for q in placed):
                    break
            placed.append(base)
            # sum of three sinusoids; amplitude*frequency sums to <= 6 m/s per axis pair
            amp = [(_u(g, 0.1, 0.5), _u(g, 0.1, 0.5)) for _ in range(3)]
            om = [_u(g, 0.5, 3.0) for _ in range(3)]
            ph = [(_u(g, 0, 2 * math.pi), _u(g, 0, 2 * math.pi)) for _ in range(3)]
            vmax = sum(math.hypot(*a) * w for a, w in zip(amp, om))
            k = min(1.0, 6.0 / vmax)
            x = base[0] + k * sum(a[0] * (math.sin(w * t + q[0]) - math.sin(q[0])) for a, w, q in zip(amp, om, ph))
            y = base[1] + k * sum(a[1] * (math.sin(w * t + q[1]) - math.sin(q[1])) for a, w, q in zip(amp, om, ph))
            x = min(max(x, -8.6), 8.6)
            y = min(max(y, -4.2), 4.2)
            yaw = _u(g, 0, 2 * math.pi) + 0.4 * math.sin(_u(g, 0.5, 2.0) * t)
            h = _u(g, 1.7, 2.0)
            objs += player((x, y), yaw, h, g, obj=p)
        bx, by = _u(g, -7.0, 7.0), _u(g, -3.5, 3.5)
        vx, vy = _u(g, -4.0, 4.0), _u(g, -2.0, 2.0)
        tau = (t + _u(g, 0.0, 1.0)) % 1.0
        bz = 1.0 + 4.905 * tau - 4.905 * tau * tau
        objs += ball((min(max(bx + vx * t, -9.0), 9.0), min(max(by + vy * t, -4.5), 4.5), bz), 0.105, g, obj=12)
        return objs
    if config == "judo":
        # two players 0.45 m apart whose arms (along each player's local x)
        # overlap between them, so that they form one connected component
        cx, cy = _u(g, -1.0, 1.0), _u(g, -1.0, 1.0)
        yaw = _u(g, 0, 2 * math.pi)
        d = np.array([math.cos(yaw), math.sin(yaw)]) * 0.225
        objs = player((cx - d[0], cy - d[1]), yaw, _u(g, 1.7, 1.9), g, obj=0)
        objs += player((cx + d[0], cy + d[1]), yaw + math.pi, _u(g, 1.7, 1.9), g, obj=1)
        ra = _u(g, 0, 2 * math.pi)
        objs += player((cx + 2.6 * math.cos(ra), cy + 2.6 * math.sin(ra)), _u(g, 0, 2 * math.pi), 1.75, g, obj=2)
        return objs
    if config == "hd720":
        objs = []
        for p in range(3):
            a = 2 * math.pi * p / 3 + _u(g, -0.3, 0.3)
            objs += player((1.6 * math.cos(a), 1.6 * math.sin(a)), _u(g, 0, 2 * math.pi), _u(g, 1.7, 1.9), g, obj=p)
        return objs
    raise ValueError(f"unknown config {config!r}")


def default_viewpoint(rig: Rig, index: int = 0) -> np.ndarray:
    """A virtual viewpoint between camera 0 and camera 1, lifted 0.5 m."""
    c = 0.6 * rig.C64[index % rig.n_cams] + 0.4 * rig.C64[(index + 1) % rig.n_cams]
    return (c + np.array([0.0, 0.0, 0.5])).astype(np.float32)


# --------------------------------------------------------------- rendering

def _ellipsoid_pixel_box(rig, n, e, W, H):
    """Pixel box containing the projection of ellipsoid e in camera n, or None."""
    half = np.sqrt(((e.rot * e.axes[None, :]) ** 2).sum(axis=1))
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * half + e.centre
    h = np.concatenate([corners, np.ones((8, 1))], axis=1) @ rig.P64[n].T
    if np.any(h[:, 2] <= 1e-9):
        return 0, W, 0, H
    u, v = h[:, 0] / h[:, 2], h[:, 1] / h[:, 2]
    x0, x1 = int(max(0, math.floor(u.min()) - 1)), int(min(W, math.ceil(u.max()) + 2))
    y0, y1 = int(max(0, math.floor(v.min()) - 1)), int(min(H, math.ceil(v.max()) + 2))
    if x0 >= x1 or y0 >= y1:
        return None
    return x0, x1, y0, y1


def _conic(rig, n, e):
    """3x3 image conic of ellipsoid e in camera n, scaled so inside is < 0."""
    T = np.eye(4)
    T[:3, :3] = e.rot * e.axes[None, :]
    T[:3, 3] = e.centre
    Qs = T @ np.diag([1.0, 1.0, 1.0, -1.0]) @ T.T          # dual quadric
    Cs = rig.P64[n] @ Qs @ rig.P64[n].T                     # dual conic
    C = np.linalg.inv(Cs)
    hc = rig.P64[n] @ np.append(e.centre, 1.0)
    x = hc / hc[2]
    if x @ C @ x > 0:
        C = -C
    return C


def render(rig: Rig, objects, index: int = 0, flip_prob: float = 1e-3, device="cpu",
           conservative: bool = False, with_rgb: bool = True, config_tag: str = "") -> Frame:
    """Silhouettes (and colour images) of `objects` seen by every camera of `rig`.

    Default: a pixel is foreground iff the ray through its centre meets an
    ellipsoid; its colour is that of the nearest ellipsoid hit, else grey.
    conservative=True: a pixel is foreground iff its unit square meets the
    exact image ellipse of an ellipsoid (no flips are added then).
    """
    N = rig.n_cams
    H, W = int(rig.height[0]), int(rig.width[0])
    assert all(int(w) == W for w in rig.width) and all(int(h) == H for h in rig.height)
    masks = torch.zeros((N, H, W), dtype=torch.uint8, device=device)
    rgb = None
    if with_rgb:
        rgb = torch.empty((N, H, W, 3), dtype=torch.uint8, device=device)
        rgb[..., 0] = BACKGROUND_RGB[0]; rgb[..., 1] = BACKGROUND_RGB[1]; rgb[..., 2] = BACKGROUND_RGB[2]
    g = _gen((config_tag or rig.name) + "/flips", index, device=device)
    groups = {}
    for e in objects:
        groups.setdefault(e.obj, []).append(e)
    for n in range(N):
        M = torch.tensor(rig.R64[n].T @ np.linalg.inv(rig.K64[n]), dtype=torch.float64, device=device)
        C = rig.C64[n]
        zbest = torch.full((H, W), float("inf"), dtype=torch.float64, device=device) if with_rgb else None
        for es in groups.values():
            boxes = [b for b in (_ellipsoid_pixel_box(rig, n, e, W, H) for e in es) if b is not None]
            if not boxes:
                continue
            x0, x1 = min(b[0] for b in boxes), max(b[1] for b in boxes)
            y0, y1 = min(b[2] for b in boxes), max(b[3] for b in boxes)
            ys = torch.arange(y0, y1, dtype=torch.float64, device=device)
            xs = torch.arange(x0, x1, dtype=torch.float64, device=device)
            if conservative:
                for e in es:
                    Cq = torch.tensor(_conic(rig, n, e), dtype=torch.float64, device=device)
                    masks[n, y0:y1, x0:x1] |= _square_meets_conic(Cq, xs, ys).to(torch.uint8)
                continue
            # rays d = R^T K^-1 (u, v, 1) through the pixel centres, in each
            # ellipsoid's unit-sphere frame: |p + t dq|^2 = 1
            uu = (xs + 0.5)[None, :].expand(len(ys), -1)
            vv = (ys + 0.5)[:, None].expand(-1, len(xs))
            d = M[:, 0, None, None] * uu[None] + M[:, 1, None, None] * vv[None] + M[:, 2, None, None]
            S = np.stack([(e.rot / e.axes[None, :]).T for e in es])             # (E,3,3) = A^-1 R^T
            P0 = np.stack([Si @ (C - e.centre) for Si, e in zip(S, es)])        # (E,3)
            S_t = torch.tensor(S, dtype=torch.float64, device=device)
            p_t = torch.tensor(P0, dtype=torch.float64, device=device)
            dq = torch.einsum("eij,jhw->eihw", S_t, d)
            a = (dq * dq).sum(1)
            b = (p_t[:, :, None, None] * dq).sum(1)
            c = (p_t * p_t).sum(1)[:, None, None] - 1.0
            disc = b * b - a * c
            sq = torch.sqrt(torch.clamp(disc, min=0.0))
            hit = (disc >= 0) & ((-b + sq) / a > 0)
            masks[n, y0:y1, x0:x1] |= hit.any(0).to(torch.uint8)
            if with_rgb:
                tz = torch.where(hit, torch.clamp((-b - sq) / a, min=0.0), torch.full_like(a, float("inf")))
                tmin, imin = tz.min(0)
                better = tmin < zbest[y0:y1, x0:x1]
                zbest[y0:y1, x0:x1] = torch.where(better, tmin, zbest[y0:y1, x0:x1])
                cols = torch.tensor([e.colour for e in es], dtype=torch.uint8, device=device)
                rgb[n, y0:y1, x0:x1] = torch.where(better[..., None], cols[imin], rgb[n, y0:y1, x0:x1])
        if flip_prob > 0 and not conservative:
            r = torch.rand((H, W), generator=g, dtype=torch.float32, device=device)
            masks[n] ^= (r < flip_prob).to(torch.uint8)
    return Frame(masks=masks, rgb=rgb, ellipsoids=list(objects), viewpoint=default_viewpoint(rig, index))


def _square_meets_conic(C, xs, ys, eps=1e-9):
    """Pixel squares [x,x+1]x[y,y+1] meeting the ellipse {p : p^T C p <= 0}."""
    X = xs[None, :].expand(len(ys), -1)
    Y = ys[:, None].expand(-1, len(xs))

    def q(u, v):
        return (C[0, 0] * u * u + 2 * C[0, 1] * u * v + C[1, 1] * v * v
                + 2 * C[0, 2] * u + 2 * C[1, 2] * v + C[2, 2])

    def seg_min(u0, v0, du, dv):
        # minimum of the convex quadratic q(p + t d), t in [0, 1]
        A = C[0, 0] * du * du + 2 * C[0, 1] * du * dv + C[1, 1] * dv * dv
        B = 2 * (C[0, 0] * u0 * du + C[0, 1] * (u0 * dv + v0 * du) + C[1, 1] * v0 * dv + C[0, 2] * du + C[1, 2] * dv)
        t = torch.clamp(-B / (2 * A), 0.0, 1.0)
        return q(u0 + t * du, v0 + t * dv)

    one = torch.ones_like(X)
    zero = torch.zeros_like(X)
    m = torch.minimum(seg_min(X, Y, one, zero), seg_min(X, Y + 1, one, zero))
    m = torch.minimum(m, seg_min(X, Y, zero, one))
    m = torch.minimum(m, seg_min(X + 1, Y, zero, one))
    scale = torch.abs(C).max()
    hit = m <= eps * scale
    # ellipse entirely inside the square: its centre is inside the square
    Ci = torch.linalg.inv(C)
    ctr = Ci[:2, 2] / Ci[2, 2]
    hit |= (X <= ctr[0]) & (ctr[0] <= X + 1) & (Y <= ctr[1]) & (ctr[1] <= Y + 1)
    return hit


def make_frame(config: str, index: int = 0, device="cpu", rig: Rig | None = None, **kw) -> tuple:
    rig = rig or make_rig(config)
    objs = scene_objects(config, index)
    return rig, render(rig, objs, index=index, device=device, config_tag=config, **kw)


def inside_any(objects, pts: np.ndarray, shrink: float = 0.0) -> np.ndarray:
    """Points (M,3) inside at least one ellipsoid shrunk by `shrink` metres
    (a point is inside the shrunk ellipsoid if it is inside the ellipsoid with
    every semi-axis reduced by `shrink`)."""
    out = np.zeros(len(pts), bool)
    for e in objects:
        q = (pts - e.centre) @ e.rot / (e.axes - shrink)[None, :]
        out |= (q * q).sum(1) <= 1.0
    return out
