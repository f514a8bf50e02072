"""Seeded synthetic scenes, cameras and targets shaped like the paper's workloads.

This module only draws random inputs (numpy PCG64 streams and scipy rotations).
It holds none of the renderer's arithmetic and imports nothing else from this
package, so the CPU oracle and the CUDA path can both be fed from it.

Layout of a scene (structure of arrays, float32):
  means  [N,3]   world-space centres
  scales [N,3]   activated scales (already exp'ed)
  quats  [N,4]   (w, x, y, z), unit length unless a test rescales them
  opac   [N]     activated opacities in (0, 1)
  sh     [N,16,3] SH coefficients, stride 16 whatever the degree
Cameras: views = list of dicts (fx, fy, cx, cy, width, height); poses float64
[V,12] = world->camera rotation (row-major 3x3) followed by the translation,
so that a world point x maps to R x + t.

The workloads stand in for the paper's datasets (LLFF, Replica, Tanks and
Temples are not available): forward-facing boxes of Gaussians seen by grids of
cameras at LLFF's 1/8 resolution (504x378) and at mixed resolutions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.transform import Rotation

# The DC coefficient range that makes the degree-0 colour uniform in [0, 1]:
# the constant SH basis function is 1/(2 sqrt(pi)), so f0 in [-sqrt(pi), sqrt(pi)]
# spans a colour offset of [-0.5, 0.5] around the renderer's +0.5.
DC_HALF_RANGE = math.sqrt(math.pi)

RESOLUTIONS_MIXED = ((256, 192), (504, 378), (1008, 756))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def sigmoid_normal(rng: np.random.Generator, n: int, mean=0.0, std=1.0) -> np.ndarray:
    z = rng.normal(mean, std, n)
    return (1.0 / (1.0 + np.exp(-z))).astype(np.float32)


def make_scene_tiny(seed: int = 0, n: int = 2000) -> dict:
    """2,000 Gaussians 3-5 units in front of an identity camera, SH degree 0."""
    rng = _rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3)) + np.array([0.0, 0.0, 4.0])
    scales = np.exp(rng.normal(-3.0, 0.5, (n, 3)))
    quats = random_unit_quats(rng, n)
    opac = sigmoid_normal(rng, n)
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-DC_HALF_RANGE, DC_HALF_RANGE, (n, 3))
    return dict(means=means.astype(np.float32), scales=scales.astype(np.float32),
                quats=quats, opac=opac, sh=sh, sh_degree=0)


def make_scene_box(seed: int, n: int, sh_degree: int = 3,
                   lo=(-2.0, -1.5, 3.0), hi=(2.0, 1.5, 7.0)) -> dict:
    """Forward-facing box of Gaussians; scales follow the mean spacing."""
    rng = _rng(seed)
    lo = np.asarray(lo); hi = np.asarray(hi)
    vol = float(np.prod(hi - lo))
    spacing = (vol / n) ** (1.0 / 3.0)
    means = rng.uniform(lo, hi, (n, 3))
    scales = np.exp(rng.normal(math.log(0.6 * spacing), 0.5, (n, 3)))
    quats = random_unit_quats(rng, n)
    opac = sigmoid_normal(rng, n)
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-DC_HALF_RANGE, DC_HALF_RANGE, (n, 3))
    if sh_degree > 0:
        ncoef = (sh_degree + 1) ** 2
        sh[:, 1:ncoef, :] = rng.normal(0.0, 0.1, (n, ncoef - 1, 3))
    return dict(means=means.astype(np.float32), scales=scales.astype(np.float32),
                quats=quats, opac=opac, sh=sh.astype(np.float32), sh_degree=sh_degree)


def intrinsics(width: int, height: int, focal_frac: float = 0.8, fx: float | None = None) -> dict:
    f = float(fx) if fx is not None else focal_frac * width
    return dict(fx=f, fy=f, cx=width / 2.0, cy=height / 2.0, width=int(width), height=int(height))


def pose_from_center(R_wc: np.ndarray, center: np.ndarray) -> np.ndarray:
    """World->camera pose [12] of a camera at `center` whose world->camera
    rotation is R_wc (t = -R c)."""
    R = np.asarray(R_wc, np.float64)
    t = -R @ np.asarray(center, np.float64)
    return np.concatenate([R.reshape(9), t])


def compose(delta_R: np.ndarray, delta_t: np.ndarray, pose: np.ndarray) -> np.ndarray:
    """Left-compose a rigid motion (delta_R, delta_t) with a world->camera pose."""
    R = pose[:9].reshape(3, 3); t = pose[9:]
    return np.concatenate([(delta_R @ R).reshape(9), delta_R @ t + delta_t])


def perturb_exact(rng: np.random.Generator, pose: np.ndarray, deg: float, trans: float) -> np.ndarray:
    """Rotation of exactly `deg` degrees about a random axis and a translation
    of norm `trans` in a random direction, applied on the left."""
    axis = rng.standard_normal(3); axis /= np.linalg.norm(axis)
    d = rng.standard_normal(3); d /= np.linalg.norm(d)
    dR = Rotation.from_rotvec(axis * math.radians(deg)).as_matrix()
    return compose(dR, trans * d, pose)


def perturb_normal(rng: np.random.Generator, pose: np.ndarray, deg_std: float, trans_std: float) -> np.ndarray:
    """Rotation about a uniform axis by an angle ~ N(0, deg_std) and a
    translation ~ N(0, trans_std)^3, applied on the left."""
    axis = rng.standard_normal(3); axis /= np.linalg.norm(axis)
    ang = math.radians(rng.normal(0.0, deg_std))
    dR = Rotation.from_rotvec(axis * ang).as_matrix()
    return compose(dR, rng.normal(0.0, trans_std, 3), pose)


def yaw_pitch(yaw_deg: float, pitch_deg: float) -> np.ndarray:
    return Rotation.from_euler("yx", [yaw_deg, pitch_deg], degrees=True).as_matrix()


def tiny_workload(seed: int = 0) -> dict:
    """One 64x48 camera (fx=fy=60) at the identity; the target pose is the
    identity perturbed by exactly 3 degrees and a 0.05 translation."""
    scene = make_scene_tiny(seed)
    rng = _rng(seed + 1000)
    view = dict(fx=60.0, fy=60.0, cx=32.0, cy=24.0, width=64, height=48)
    pose = pose_from_center(np.eye(3), np.zeros(3))
    target_pose = perturb_exact(rng, pose, 3.0, 0.05)
    return dict(scene=scene, views=[view], poses=pose[None, :].copy(),
                target_poses=target_pose[None, :].copy())


def grid_views(rng: np.random.Generator, nx: int, ny: int, resolutions, jitter: float = 0.0,
               max_angle_deg: float = 0.0, xr=(-0.5, 0.5), yr=(-0.4, 0.4), focal_frac: float = 0.8):
    """Cameras on a fronto-parallel grid at z = 0 looking along +z."""
    views, poses = [], []
    xs = np.linspace(xr[0], xr[1], nx); ys = np.linspace(yr[0], yr[1], ny)
    k = 0
    for y in ys:
        for x in xs:
            w, h = resolutions[k % len(resolutions)] if not callable(resolutions) else resolutions(rng)
            views.append(intrinsics(w, h, focal_frac))
            c = np.array([x, y, 0.0])
            if jitter > 0:
                c = c + rng.uniform(-jitter, jitter, 3) * np.array([1.0, 1.0, 0.0])
            R = np.eye(3)
            if max_angle_deg > 0:
                R = yaw_pitch(rng.uniform(-max_angle_deg, max_angle_deg),
                              rng.uniform(-max_angle_deg, max_angle_deg))
            poses.append(pose_from_center(R, c))
            k += 1
    return views, np.stack(poses)


def joint_workload(seed: int = 2, n: int = 300_000, n_views: int = 20) -> dict:
    """Forward-facing joint refinement: 300k SH3 Gaussians, 20 views at
    504x378 on a 5x4 grid; initial poses off by N(0,5 deg)/N(0,0.1)."""
    scene = make_scene_box(seed, n, 3)
    rng = _rng(seed + 1000)
    views, poses = grid_views(rng, 5, 4, [(504, 378)])
    init = np.stack([perturb_normal(rng, p, 5.0, 0.1) for p in poses])
    return dict(scene=scene, views=views[:n_views], poses=poses[:n_views],
                init_poses=init[:n_views])


def perturb_scene_raw(seed: int, scene: dict, means_std: float = 0.02, log_scale_std: float = 0.2,
                      logit_opac_std: float = 0.5, sh_std: float = 0.05) -> dict:
    """Raw (pre-activation) parameters of a perturbed copy of `scene`, the
    starting point of a joint refinement: means + N(0, 0.02), log-scales
    + N(0, 0.2), logit-opacities + N(0, 0.5), SH coefficients + N(0, 0.05);
    quaternions unchanged.  Keys: means, log_scales, quats, logit_opac, sh."""
    rng = _rng(seed)
    n = len(scene["opac"])
    o = np.clip(scene["opac"].astype(np.float64), 1e-6, 1 - 1e-6)
    nc = (int(scene["sh_degree"]) + 1) ** 2
    sh = scene["sh"].astype(np.float64).copy()
    sh[:, :nc] += rng.normal(0.0, sh_std, (n, nc, 3))
    return dict(means=(scene["means"] + rng.normal(0.0, means_std, (n, 3))).astype(np.float32),
                log_scales=(np.log(scene["scales"].astype(np.float64)) + rng.normal(0.0, log_scale_std, (n, 3))
                            ).astype(np.float32),
                quats=scene["quats"].copy(),
                logit_opac=(np.log(o / (1 - o)) + rng.normal(0.0, logit_opac_std, n)).astype(np.float32),
                sh=sh.astype(np.float32))


def batched_workload(seed: int = 3, n: int = 1_000_000, n_views: int = 64,
                     resolutions=RESOLUTIONS_MIXED, view_seed: int | None = None) -> dict:
    """1M SH3 Gaussians seen by 64 cameras of mixed resolution on a jittered
    8x8 grid with up to +-5 degrees of yaw and pitch.  view_seed (default:
    seed) draws the cameras, so that several GPUs can render different views
    of one scene."""
    scene = make_scene_box(seed, n, 3)
    rng = _rng((seed if view_seed is None else view_seed) + 1000)
    nx = int(math.ceil(math.sqrt(n_views)))
    ny = int(math.ceil(n_views / nx))
    pick = lambda r: resolutions[r.integers(len(resolutions))]
    views, poses = grid_views(rng, nx, ny, pick, jitter=0.05, max_angle_deg=5.0)
    target_poses = np.stack([perturb_normal(rng, p, 1.0, 0.02) for p in poses])
    return dict(scene=scene, views=views[:n_views], poses=poses[:n_views],
                target_poses=target_poses[:n_views])


def _box_surface_points(rng: np.random.Generator, n: int, lo, hi) -> np.ndarray:
    """n points uniform on the surface of the axis-aligned box [lo, hi]."""
    lo = np.asarray(lo, np.float64); hi = np.asarray(hi, np.float64)
    e = hi - lo
    areas = np.array([e[1] * e[2], e[1] * e[2], e[0] * e[2], e[0] * e[2], e[0] * e[1], e[0] * e[1]])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    pts = rng.uniform(lo, hi, (n, 3))
    axis = face // 2
    side = np.where(face % 2 == 0, lo[axis], hi[axis])
    pts[np.arange(n), axis] = side
    return pts


def room_geometry(seed: int = 5, room=(6.0, 3.0, 8.0), n_boxes: int = 6) -> dict:
    """The room of the trajectory workload: a room x*y*z box centred at the
    origin (floor at y = +room_y/2) and n_boxes furniture boxes standing on
    the floor near the side walls.  Returns dict(half [3], boxes [(lo, hi)])."""
    rng = _rng(seed + 17)
    half = np.asarray(room, np.float64) / 2.0
    sizes = rng.uniform(0.3, 0.9, (n_boxes, 3))
    boxes = []
    for k in range(n_boxes):
        sx = (1 if k % 2 == 0 else -1) * (half[0] - 0.2 - sizes[k, 0] / 2)
        cz = rng.uniform(-half[2] + 1.0, half[2] - 1.0)
        c = np.array([sx, half[1] - sizes[k, 1] / 2, cz])
        boxes.append((c - sizes[k] / 2, c + sizes[k] / 2))
    return dict(half=half, boxes=boxes)


def make_scene_room(seed: int = 5, n: int = 3_000_000, sh_degree: int = 3,
                    room=(6.0, 3.0, 8.0), n_boxes: int = 6, box_share: float = 0.25,
                    scale: float = 0.006) -> dict:
    """Room-scale scene: Gaussians on the walls, floor and ceiling of the
    room and on the surfaces of its furniture boxes (room_geometry);
    log-scales N(log scale, 0.4)."""
    geo = room_geometry(seed, room, n_boxes)
    rng = _rng(seed)
    half = geo["half"]
    n_box = int(n * box_share)
    n_room = n - n_box
    parts = [_box_surface_points(rng, n_room, -half, half)]
    ext = np.array([hi - lo for lo, hi in geo["boxes"]])
    areas = 2 * (ext[:, 0] * ext[:, 1] + ext[:, 1] * ext[:, 2] + ext[:, 0] * ext[:, 2])
    counts = np.floor(n_box * areas / areas.sum()).astype(int)
    counts[0] += n_box - counts.sum()
    for k, (lo, hi) in enumerate(geo["boxes"]):
        parts.append(_box_surface_points(rng, counts[k], lo, hi))
    means = np.concatenate(parts)
    scales = np.exp(rng.normal(math.log(scale), 0.4, (n, 3)))
    quats = random_unit_quats(rng, n)
    opac = sigmoid_normal(rng, n)
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-DC_HALF_RANGE, DC_HALF_RANGE, (n, 3))
    if sh_degree > 0:
        ncoef = (sh_degree + 1) ** 2
        sh[:, 1:ncoef, :] = 0.1 * rng.standard_normal((n, ncoef - 1, 3), dtype=np.float32)
    return dict(means=means.astype(np.float32), scales=scales.astype(np.float32),
                quats=quats, opac=opac, sh=sh, sh_degree=sh_degree)


def room_depth(geo: dict, view: dict, pose: np.ndarray) -> np.ndarray:
    """Ground-truth z-depth [H, W] (float32) of the room's surfaces seen by a
    pinhole camera (world->camera pose [12]): per pixel, the nearest hit of
    the ray through the pixel's sample point with the furniture boxes (slab
    test) or the room's inner walls.  This is the input stand-in for a
    monocular depth estimate."""
    W, H = view["width"], view["height"]
    R = np.asarray(pose[:9], np.float64).reshape(3, 3)
    t = np.asarray(pose[9:], np.float64)
    c = -R.T @ t
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dc = np.stack([(u - view["cx"]) / view["fx"], (v - view["cy"]) / view["fy"], np.ones_like(u)], -1)
    d = dc @ R                       # world directions (rows of R^T dc), camera z component 1
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        half = geo["half"]
        t_exit = np.min(np.where(d > 0, (half - c) * inv, np.where(d < 0, (-half - c) * inv, np.inf)), -1)
        best = t_exit
        for lo, hi in geo["boxes"]:
            t1 = (lo - c) * inv
            t2 = (hi - c) * inv
            tn = np.max(np.minimum(t1, t2), -1)
            tf = np.min(np.maximum(t1, t2), -1)
            hit = (tn <= tf) & (tn > 0)
            best = np.where(hit & (tn < best), tn, best)
    return best.astype(np.float32)     # the ray parameter is the z-depth (camera z of d is 1)


def spline_trajectory(rng: np.random.Generator, n_frames: int, n_ctrl: int = 8,
                      xr=(-1.8, 1.8), yr=(-0.4, 0.4), zr=(-3.0, 3.0)) -> np.ndarray:
    """World->camera poses [n_frames, 12] along a C2 (natural cubic) spline
    through n_ctrl interior control points, each camera looking along the
    path's tangent with its y axis close to world +y."""
    from scipy.interpolate import CubicSpline
    ctrl = np.stack([rng.uniform(xr[0], xr[1], n_ctrl), rng.uniform(yr[0], yr[1], n_ctrl),
                     np.linspace(zr[0], zr[1], n_ctrl)], 1)
    sp = CubicSpline(np.arange(n_ctrl), ctrl, bc_type="natural")
    u = np.linspace(0.0, n_ctrl - 1, n_frames)
    pos, tan = sp(u), sp(u, 1)
    out = []
    for c, d in zip(pos, tan):
        z = d / np.linalg.norm(d)
        x = np.cross(np.array([0.0, 1.0, 0.0]), z)
        x /= np.linalg.norm(x)
        y = np.cross(z, x)
        out.append(pose_from_center(np.stack([x, y, z]), c))
    return np.stack(out)


def trajectory_workload(seed: int = 5, n: int = 3_000_000, n_frames: int = 200,
                        width: int = 1280, height: int = 720, focal: float = 600.0, scale: float = 0.006) -> dict:
    """Large trajectory refinement: a 3M-Gaussian SH3 room seen by n_frames
    1280x720 cameras (fx = fy = 600) along a smooth spline; initial poses
    off by N(0, 1 deg)/N(0, 0.02)."""
    scene = make_scene_room(seed, n, scale=scale)
    rng = _rng(seed + 1000)
    poses = spline_trajectory(rng, n_frames)
    views = [intrinsics(width, height, fx=focal) for _ in range(n_frames)]
    init = np.stack([perturb_normal(rng, p, 1.0, 0.02) for p in poses])
    return dict(scene=scene, views=views, poses=poses, init_poses=init, geometry=room_geometry(seed))


def serving_requests(seed: int = 4, n_requests: int = 2000, rate_hz: float = 200.0,
                     steps: int = 100) -> list[dict]:
    """Poisson arrivals of pose-estimation requests at mixed image sizes.

    Each request: arrival time (s), intrinsics, the ground-truth pose the query
    image is rendered at, and an initial pose off by N(0,10 deg)/N(0,0.2)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        w = int(rng.integers(256, 1281))
        a = (3.0 / 4.0) if rng.integers(2) == 0 else (9.0 / 16.0)
        h = int(min(max(round(w * a), 192), 720))
        c = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), 0.0])
        R = yaw_pitch(rng.uniform(-5, 5), rng.uniform(-5, 5))
        gt = pose_from_center(R, c)
        init = perturb_normal(rng, gt, 10.0, 0.2)
        out.append(dict(id=k, arrival=t, view=intrinsics(w, h), gt_pose=gt, init_pose=init,
                        steps=steps))
    return out


def random_image_like(rng: np.random.Generator, views) -> np.ndarray:
    """Packed planar float32 images [sum 3*H*W], uniform in [0, 1]."""
    n = sum(3 * v["width"] * v["height"] for v in views)
    return rng.uniform(0.0, 1.0, n).astype(np.float32)


def random_dldc_like(rng: np.random.Generator, views, scale: float = 1.0) -> np.ndarray:
    n = sum(3 * v["width"] * v["height"] for v in views)
    return (scale * rng.standard_normal(n)).astype(np.float32)


def image_offsets(views):
    """Float offsets of each view's planar [3][H][W] image in a packed buffer
    and pixel offsets of its [H][W] per-pixel planes."""
    img, pix = [0], [0]
    for v in views:
        img.append(img[-1] + 3 * v["width"] * v["height"])
        pix.append(pix[-1] + v["width"] * v["height"])
    return img, pix
