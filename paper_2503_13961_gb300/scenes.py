"""Seeded synthetic scenes and cameras for the BG-Triangle rasterizer.

This module only builds inputs: triangle meshes lifted to degree-n Bezier
control points, per-primitive attributes and pinhole cameras. It contains none
of the rendering arithmetic (no Bernstein evaluation, projection of Gaussians,
blending or derivatives), so both the CUDA path and the CPU oracle can consume
its output without sharing any of the method's code.

Scenes stand in for the paper's Lego / NeRF-Synthetic / Tanks & Temples
workloads (Sec. 4, Table 4), which are not available offline. Control-point
layout follows the order i = n..0, then j = n-i..0, k = n-i-j, so that the
flat index of p_ijk is (n-i)(n-i+1)/2 + k and the corners p_n00, p_0n0, p_00n
sit under barycentric u, v, w = 1 (Sec. 3.1, Eq. 1).

Every array is float32 and C-contiguous; a scene is a plain dict:
  degree  int n
  ctrl      [M, Ncp, 3]  control points p_ijk (world units)
  color     [M, Ncp, 3]  colour control points p^c_ijk (RGB)
  opacity   [M]          per-primitive opacity o (Eq. 8)
  r_b       [M]          boundary scale r_b (Sec. 3.2, boundary Gaussians)
  log_scale [M, 3]       log of the sub-primitive Gaussian scales
  quat      [M, 4]       sub-primitive rotation, (w, x, y, z)
  bg        [3]          background colour
  attr_res  int R        (optional, default 1) leg resolution of the rotation
                         and scaling attribute maps (Sec. 3.2, Eq. 5); with
                         R > 1, log_scale is [M, T, 3] and quat [M, T, 4] over
                         the T = R (R + 1) / 2 texels (see with_attribute_maps)
  sh_degree int D        (optional, default 0) degree of the view-dependent
                         colour; with D > 0, sh [M, (D+1)^2 - 1, 3] holds the
                         coefficients of SH bands 1..D per primitive (see with_sh)
A camera is a dict with R [3,3], t [3] (world -> camera, x right, y down,
z forward), fx, fy, cx, cy (pixels, pixel centres at integer coordinates)
and width, height.
"""
import math

import numpy as np

__all__ = [
    "ncp", "cp_index", "look_at_camera", "crop_camera", "make_scene",
    "make_views", "config_scene", "tiny_scene", "random_gaussians", "triangles_scene",
]


def ncp(n):
    """Number of control points of a degree-n Bezier triangle."""
    return (n + 1) * (n + 2) // 2


def cp_index(n, i, j):
    """Flat index of p_ijk (k = n - i - j) in the i-descending, j-descending order."""
    k = n - i - j
    return (n - i) * (n - i + 1) // 2 + k


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at_camera(eye, target, width, height, fov_x_deg=60.0):
    """Pinhole camera at `eye` looking at `target` (horizontal FOV in degrees).

    up is +z unless the view direction is within ~8 deg of it, then +y.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(f @ up) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ eye
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return {
        "R": R.astype(np.float32), "t": t.astype(np.float32),
        "fx": np.float32(fx), "fy": np.float32(fx),
        "cx": np.float32((width - 1) / 2.0), "cy": np.float32((height - 1) / 2.0),
        "width": int(width), "height": int(height),
    }


def crop_camera(cam, x0, y0, width, height):
    """The window [x0, x0+width) x [y0, y0+height) of `cam` as its own camera."""
    c = dict(cam)
    c["cx"] = np.float32(float(cam["cx"]) - x0)
    c["cy"] = np.float32(float(cam["cy"]) - y0)
    c["width"], c["height"] = int(width), int(height)
    return c


# ----------------------------------------------------------------------------
# meshes (flat triangles + an object tag that says how to push points outward)
# ----------------------------------------------------------------------------

class _Mesh:
    """Flat triangles with, per object, a radial projector for lifted points."""

    def __init__(self):
        self.tris = []      # list of [3,3] arrays
        self.obj = []       # object index per triangle
        self.objects = []   # ("sphere", c, r) | ("ellipsoid", c, axes) | ("flat",)

    def add_object(self, desc, tris):
        oid = len(self.objects)
        self.objects.append(desc)
        for tr in tris:
            self.tris.append(np.asarray(tr, np.float64))
            self.obj.append(oid)


def _sphere_project(p, c, r):
    d = p - c
    return c + r * d / np.linalg.norm(d)


def _ellipsoid_project(p, c, axes):
    x = (p - c) / axes
    return c + axes * x / np.linalg.norm(x)


def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, phi, 0], [1, phi, 0], [-1, -phi, 0], [1, -phi, 0],
        [0, -1, phi], [0, 1, phi], [0, -1, -phi], [0, 1, -phi],
        [phi, 0, -1], [phi, 0, 1], [-phi, 0, -1], [-phi, 0, 1]], np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    return v, f


def _subdivide_face(a, b, c, freq):
    """freq^2 flat triangles of the lattice a + (b-a) i/f + (c-a) j/f."""
    def P(i, j):
        return a + (b - a) * (i / freq) + (c - a) * (j / freq)
    out = []
    for i in range(freq):
        for j in range(freq - i):
            out.append((P(i, j), P(i + 1, j), P(i, j + 1)))
            if i + j <= freq - 2:
                out.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    return out


def icosphere_tris(freq, center=(0, 0, 0), radius=1.0):
    """Geodesic sphere: 20 * freq^2 triangles with vertices on the sphere."""
    center = np.asarray(center, np.float64)
    v, faces = _icosahedron()
    tris = []
    for (i, j, k) in faces:
        for tr in _subdivide_face(v[i], v[j], v[k], freq):
            tris.append(tuple(center + radius * (p / np.linalg.norm(p)) for p in tr))
    return tris


def octahedron16_tris(radius=1.0):
    """Octahedron whose 8 faces are each split in two at the midpoint of the
    edge opposite their pole vertex (midpoint pushed onto the sphere)."""
    X, Y, Z = np.eye(3)
    ring = [X, Y, -X, -Y]
    tris = []
    for pole in (Z, -Z):
        for a in range(4):
            e1, e2 = ring[a], ring[(a + 1) % 4]
            m = (e1 + e2) / 2.0
            m = m / np.linalg.norm(m)
            tris.append((pole * radius, e1 * radius, m * radius))
            tris.append((pole * radius, m * radius, e2 * radius))
    return tris


def latlong_tris(center, axes, segments, bands):
    """Lat-long ellipsoid: `bands` rings of `segments` quads, two triangles each.

    Rings sit at polar angles pi (r+1) / (bands+2), r = 0..bands, leaving two
    small open caps so that no triangle is degenerate.
    """
    center = np.asarray(center, np.float64)
    axes = np.asarray(axes, np.float64)
    th = [math.pi * (r + 1) / (bands + 2) for r in range(bands + 1)]
    ph = [2 * math.pi * s / segments for s in range(segments)]

    def P(r, s):
        t, p = th[r], ph[s % segments]
        return center + axes * np.array([math.sin(t) * math.cos(p),
                                         math.sin(t) * math.sin(p), math.cos(t)])
    tris = []
    for r in range(bands):
        for s in range(segments):
            a, b, c, d = P(r, s), P(r, s + 1), P(r + 1, s), P(r + 1, s + 1)
            tris.append((a, c, b))
            tris.append((b, c, d))
    return tris


def grid_quad_tris(origin, eu, ev, n):
    """Square patch origin + eu*s + ev*t, s,t in [0,1], as an n x n grid (2 n^2 tris)."""
    origin, eu, ev = (np.asarray(x, np.float64) for x in (origin, eu, ev))
    tris = []
    for i in range(n):
        for j in range(n):
            p00 = origin + eu * (i / n) + ev * (j / n)
            p10 = origin + eu * ((i + 1) / n) + ev * (j / n)
            p01 = origin + eu * (i / n) + ev * ((j + 1) / n)
            p11 = origin + eu * ((i + 1) / n) + ev * ((j + 1) / n)
            tris.append((p00, p10, p01))
            tris.append((p10, p11, p01))
    return tris


def box_tris(center, half, n, inward=False):
    """Axis-aligned box surface, each face an n x n grid."""
    c = np.asarray(center, np.float64)
    h = np.asarray(half, np.float64) * np.ones(3)
    tris = []
    for ax in range(3):
        for sgn in (-1.0, 1.0):
            u_ax, v_ax = (ax + 1) % 3, (ax + 2) % 3
            eu = np.zeros(3)
            ev = np.zeros(3)
            eu[u_ax] = 2 * h[u_ax]
            ev[v_ax] = 2 * h[v_ax]
            o = c.copy()
            o[ax] += sgn * h[ax]
            o[u_ax] -= h[u_ax]
            o[v_ax] -= h[v_ax]
            face = grid_quad_tris(o, eu, ev, n)
            outward = (sgn > 0) != inward
            # orient so that the normal points outward (or inward for a room)
            if (np.cross(eu, ev)[ax] > 0) != outward:
                face = [(a, cc, b) for (a, b, cc) in face]
            tris.extend(face)
    return tris


# ----------------------------------------------------------------------------
# lifting flat triangles to degree-n Bezier control points
# ----------------------------------------------------------------------------

def _lift(mesh, n, noise_std, rng):
    """Degree-n control points of every triangle of `mesh`.

    Corners are the triangle's vertices. Non-corner lattice points start at
    the flat position (i P0 + j P1 + k P2) / n, are pushed onto the object's
    surface (spheres, ellipsoids) and then moved along the outward direction
    by N(0, noise_std). Points on an edge are shared by the two triangles of
    that edge (one draw per edge point), so neighbouring patches stay joined.
    """
    T = len(mesh.tris)
    m = ncp(n)
    ctrl = np.zeros((T, m, 3), np.float64)
    vkey = {}

    def vid(p):
        k = tuple(np.round(p, 9))
        if k not in vkey:
            vkey[k] = len(vkey)
        return vkey[k]

    edge_draw = {}
    interior = []
    for t_i, (tr, oid) in enumerate(zip(mesh.tris, mesh.obj)):
        desc = mesh.objects[oid]
        ids = [vid(p) for p in tr]
        if desc[0] == "flat":
            nrm = np.cross(tr[1] - tr[0], tr[2] - tr[0])
            nrm /= np.linalg.norm(nrm)
        for i in range(n, -1, -1):
            for j in range(n - i, -1, -1):
                k = n - i - j
                idx = cp_index(n, i, j)
                p = (i * tr[0] + j * tr[1] + k * tr[2]) / n
                if max(i, j, k) == n:
                    ctrl[t_i, idx] = p
                    continue
                if desc[0] == "sphere":
                    p = _sphere_project(p, desc[1], desc[2])
                    dirv = (p - desc[1]) / np.linalg.norm(p - desc[1])
                elif desc[0] == "ellipsoid":
                    p = _ellipsoid_project(p, desc[1], desc[2])
                    dirv = (p - desc[1]) / np.linalg.norm(p - desc[1])
                else:
                    dirv = nrm
                zero = [x for x, w in zip(ids, (i, j, k)) if w == 0]
                if len(zero) == 1:
                    # edge point: key by the edge's endpoints and position along it
                    ends = [(x, w) for x, w in zip(ids, (i, j, k)) if w > 0]
                    ends.sort()
                    key = (ends[0][0], ends[1][0], ends[0][1])
                    if key not in edge_draw:
                        edge_draw[key] = None
                    ctrl[t_i, idx] = p
                    interior.append((t_i, idx, dirv, key))
                else:
                    ctrl[t_i, idx] = p
                    interior.append((t_i, idx, dirv, None))
    # draw the noise in a deterministic order: edges (sorted keys), then interiors
    keys = sorted(edge_draw)
    vals = rng.normal(0.0, noise_std, size=len(keys)) if noise_std > 0 else np.zeros(len(keys))
    for kk, vv in zip(keys, vals):
        edge_draw[kk] = vv
    n_int = sum(1 for x in interior if x[3] is None)
    ivals = rng.normal(0.0, noise_std, size=n_int) if noise_std > 0 else np.zeros(n_int)
    ii = 0
    for (t_i, idx, dirv, key) in interior:
        if key is not None:
            ctrl[t_i, idx] += edge_draw[key] * dirv
        else:
            ctrl[t_i, idx] += ivals[ii] * dirv
            ii += 1
    return ctrl


def make_scene(mesh, n, noise_std, seed, opacity="uniform", r_b=1e-2,
               gauss_scale=0.005, bg=(0.0, 0.0, 0.0)):
    """Lift `mesh` to a degree-n BG-Triangle scene (see module docstring)."""
    rng = np.random.default_rng(seed)
    ctrl = _lift(mesh, n, noise_std, rng)
    M = ctrl.shape[0]
    m = ncp(n)
    rgb = rng.uniform(0.0, 1.0, size=(M, 3))
    color = np.repeat(rgb[:, None, :], m, axis=1)
    if opacity == "uniform":
        o = rng.uniform(0.5, 1.0, size=M)
    elif opacity == "beta":
        o = rng.beta(5.0, 1.0, size=M)
    else:
        o = np.full(M, float(opacity))
    rb = np.broadcast_to(np.asarray(r_b, np.float64), (M,)).copy()
    quat = np.zeros((M, 4))
    quat[:, 0] = 1.0
    log_scale = np.full((M, 3), math.log(gauss_scale))
    return {
        "degree": int(n),
        "ctrl": np.ascontiguousarray(ctrl, np.float32),
        "color": np.ascontiguousarray(color, np.float32),
        "opacity": np.ascontiguousarray(o, np.float32),
        "r_b": np.ascontiguousarray(rb, np.float32),
        "log_scale": np.ascontiguousarray(log_scale, np.float32),
        "quat": np.ascontiguousarray(quat, np.float32),
        "bg": np.asarray(bg, np.float32),
    }


def _gauss_scale(s_px, d_ref, width_ref, fov_x_deg=60.0):
    """World-space Gaussian scale that spans s_px pixels at distance d_ref."""
    f_ref = (width_ref / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return s_px * d_ref / f_ref


def _random_dir(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def make_views(rng, sizes, r_lo, r_hi, target=(0, 0, 0)):
    """Cameras uniform in direction on S^2 at radius U[r_lo, r_hi], looking at target."""
    cams = []
    for (w, h) in sizes:
        d = _random_dir(rng)
        r = rng.uniform(r_lo, r_hi)
        cams.append(look_at_camera(np.asarray(target) + r * d, target, w, h))
    return cams


def _blob_mesh(rng, ico_freq, n_blobs, segments, bands):
    mesh = _Mesh()
    mesh.add_object(("sphere", np.zeros(3), 1.0), icosphere_tris(ico_freq))
    for _ in range(n_blobs):
        axes = rng.uniform(0.3, 0.8, size=3)
        c = rng.uniform(-1.5, 1.5, size=3)
        mesh.add_object(("ellipsoid", c, axes), latlong_tris(c, axes, segments, bands))
    return mesh


def _room_mesh(rng):
    mesh = _Mesh()
    mesh.add_object(("flat",), box_tris((0, 0, 0), 5.0, 40, inward=True))
    centres = []
    for _ in range(100):
        e = rng.uniform(0.3, 1.0)
        c = rng.uniform(-4.0, 4.0, size=3)
        centres.append(c)
        mesh.add_object(("flat",), box_tris(c, e / 2.0, 4))
    for _ in range(100):
        r = rng.uniform(0.2, 0.6)
        c = rng.uniform(-4.0, 4.0, size=3)
        centres.append(c)
        mesh.add_object(("sphere", c, r), latlong_tris(c, (r, r, r), 22, 14))
    return mesh, centres


def with_attribute_maps(scene, R, seed=0, scale_noise=0.3, rot_noise=0.3):
    """The scene with rotation and scaling attribute maps of leg resolution R
    (Eq. 5): T = R (R + 1) / 2 texels per primitive at the nodes (i, j),
    i + j <= R - 1, of the level-(R - 1) barycentric lattice, in control-point
    order. Each texel is the primitive's attribute plus seeded noise (normal,
    std scale_noise on the log scales, rot_noise on the raw quaternion), so
    that the interpolation varies across a primitive."""
    rng = np.random.default_rng(1000 + seed)
    M = scene["ctrl"].shape[0]
    T = R * (R + 1) // 2
    ls = np.asarray(scene["log_scale"], np.float64).reshape(M, -1, 3)[:, :1, :]
    q = np.asarray(scene["quat"], np.float64).reshape(M, -1, 4)[:, :1, :]
    ls = np.repeat(ls, T, axis=1) + rng.normal(0.0, scale_noise, size=(M, T, 3))
    q = np.repeat(q, T, axis=1) + rng.normal(0.0, rot_noise, size=(M, T, 4))
    out = dict(scene)
    out["attr_res"] = int(R)
    out["log_scale"] = np.ascontiguousarray(ls, np.float32)
    out["quat"] = np.ascontiguousarray(q, np.float32)
    return out


def with_sh(scene, D, seed=0, scale=0.2):
    """The scene with view-dependent colour of SH degree D: per primitive the
    coefficients of the real SH bands 1..D for each RGB channel, normal with
    std `scale`, added to the diffuse colour of Eq. 4."""
    rng = np.random.default_rng(2000 + seed)
    M = scene["ctrl"].shape[0]
    K = (D + 1) ** 2 - 1
    out = dict(scene)
    out["sh_degree"] = int(D)
    out["sh"] = np.ascontiguousarray(rng.normal(0.0, scale, size=(M, K, 3)), np.float32)
    return out


def config_scene(cfg, seed=0, r_b=None):
    """The five synthetic workloads: (scene, cameras[, extras]).

    1  16 degree-2 triangles (split octahedron, r=1, noise 0.05), one 64x64
       view from distance 4; forward parity.
    2  2,000 degree-2 triangles (icosphere freq 10, noise 0.03), one 800x800
       view on a radius-4 sphere; also returns the noise-free target scene.
    3  20,000 degree-2 triangles (icosphere freq 20 + three 4,000-triangle
       ellipsoids, noise 0.02), one 1024x1024 view; gradient check.
    4  the config-3 scene under 64 views of mixed size {256,512,800,1024}^2
       at radius U[3.5, 5]; the batched fwd+bwd workload.
    5  100,000 degree-3 triangles (room of 19,200, 100 cubes of 192, 100
       spheres of 616, noise 0.01, opacity Beta(5,1)), 8 views 1600x1200.
    """
    rng = np.random.default_rng(seed)
    if cfg == 1:
        mesh = _Mesh()
        mesh.add_object(("sphere", np.zeros(3), 1.0), octahedron16_tris())
        s = _gauss_scale(0.7, 4.0, 64)
        scene = make_scene(mesh, 2, 0.05, seed, r_b=1e-2 if r_b is None else r_b, gauss_scale=s)
        cam = look_at_camera((4.0, 0.0, 0.0), (0, 0, 0), 64, 64)
        return scene, [cam]
    if cfg == 2:
        mesh = _Mesh()
        mesh.add_object(("sphere", np.zeros(3), 1.0), icosphere_tris(10))
        s = _gauss_scale(0.7, 4.0, 800)
        rb = 1e-2 if r_b is None else r_b
        scene = make_scene(mesh, 2, 0.03, seed, r_b=rb, gauss_scale=s)
        target = make_scene(mesh, 2, 0.0, seed, r_b=rb, gauss_scale=s)
        az = rng.uniform(0, 2 * math.pi)
        el = rng.uniform(-math.pi / 3, math.pi / 3)
        eye = 4.0 * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cam = look_at_camera(eye, (0, 0, 0), 800, 800)
        return scene, [cam], {"target_scene": target}
    if cfg in (3, 4):
        mesh = _blob_mesh(rng, 20, 3, 40, 50)
        s = _gauss_scale(0.7, 4.0, 800)
        rb = 1e-2 if r_b is None else r_b
        scene = make_scene(mesh, 2, 0.02, seed, r_b=rb, gauss_scale=s)
        if cfg == 3:
            cam = look_at_camera(4.0 * _random_dir(rng), (0, 0, 0), 1024, 1024)
            return scene, [cam]
        res = [256, 512, 800, 1024]
        sizes = [(r, r) for r in rng.choice(res, size=64)]
        return scene, make_views(rng, sizes, 3.5, 5.0)
    if cfg == 5:
        mesh, centres = _room_mesh(rng)
        s = _gauss_scale(0.7, 5.0, 1600)
        scene = make_scene(mesh, 3, 0.01, seed, opacity="beta",
                           r_b=1e-2 if r_b is None else r_b, gauss_scale=s)
        cams = []
        for _ in range(8):
            eye = rng.uniform(-3.0, 3.0, size=3)
            tgt = centres[rng.integers(len(centres))]
            while np.linalg.norm(tgt - eye) < 1e-3:
                tgt = centres[rng.integers(len(centres))]
            cams.append(look_at_camera(eye, tgt, 1600, 1200))
        return scene, cams
    raise ValueError(f"unknown config {cfg}")


def tiny_scene(kind, seed=0, n=2, noise=0.0, size=(32, 32), r_b=1e-2, opacity="uniform",
               gauss_scale=None, dist=4.0):
    """Small hand-built scenes for unit tests.

    kind "two"    two triangles sharing an edge (a flat square split in two)
                  plus a third triangle far to the side (Fig. 4's R_a, R_b, G_c)
    kind "one"    a single flat triangle facing the camera
    kind "octa"   the 16-triangle split octahedron
    kind "ico1"   icosphere freq 1 (20 triangles)
    """
    mesh = _Mesh()
    if kind == "two":
        a, b, c, d = (np.array(x, np.float64) for x in
                      ([0, -0.8, -0.8], [0, 0.8, -0.8], [0, -0.8, 0.8], [0, 0.8, 0.8]))
        mesh.add_object(("flat",), [(a, b, c), (b, d, c)])
        e, f, g = (np.array(x, np.float64) for x in ([0.2, -1.9, 1.2], [0.2, -1.2, 1.2], [0.2, -1.5, 1.9]))
        mesh.add_object(("flat",), [(e, f, g)])
    elif kind == "one":
        mesh.add_object(("flat",), [(np.array([0.0, -0.9, -0.7]), np.array([0.0, 0.8, -0.5]),
                                     np.array([0.0, 0.1, 0.9]))])
    elif kind == "octa":
        mesh.add_object(("sphere", np.zeros(3), 1.0), octahedron16_tris())
    elif kind == "ico1":
        mesh.add_object(("sphere", np.zeros(3), 1.0), icosphere_tris(1))
    else:
        raise ValueError(kind)
    w, h = size
    if gauss_scale is None:
        gauss_scale = _gauss_scale(0.7, dist, w)
    scene = make_scene(mesh, n, noise, seed, opacity=opacity, r_b=r_b, gauss_scale=gauss_scale)
    cam = look_at_camera((dist, 0.05, 0.03), (0, 0, 0), w, h)
    return scene, [cam]


def random_gaussians(seed, width, height, count, radius_px=(0.5, 3.0), depth_ties=True):
    """Synthetic projected Gaussians for binning/sort tests.

    Returns per Gaussian: pixel (qx, qy) it is attached to, sub-pixel offset
    of its mean, conic (a, b, c), opacity and depth, all float32 except the
    integer pixel. With depth_ties, a quarter of the depths repeat exactly,
    so the (depth, index) tie rule is exercised.
    """
    rng = np.random.default_rng(seed)
    qx = rng.integers(0, width, size=count).astype(np.int32)
    qy = rng.integers(0, height, size=count).astype(np.int32)
    off = rng.uniform(-0.5, 0.5, size=(count, 2)).astype(np.float32)
    sx = rng.uniform(*radius_px, size=count)
    sy = rng.uniform(*radius_px, size=count)
    th = rng.uniform(0, math.pi, size=count)
    c, s = np.cos(th), np.sin(th)
    # covariance = Rot diag(sx^2, sy^2) Rot^T, conic = its inverse
    A = c * c * sx * sx + s * s * sy * sy
    B = c * s * (sx * sx - sy * sy)
    C = s * s * sx * sx + c * c * sy * sy
    det = A * C - B * B
    conic = np.stack([C / det, -B / det, A / det], axis=1).astype(np.float32)
    opac = rng.uniform(0.3, 1.0, size=count).astype(np.float32)
    depth = rng.uniform(2.0, 6.0, size=count).astype(np.float32)
    if depth_ties and count >= 4:
        k = count // 4
        src = rng.integers(0, count, size=k)
        dst = rng.integers(0, count, size=k)
        depth[dst] = depth[src]
    return {"qx": qx, "qy": qy, "off": off, "conic": conic, "opacity": opac, "depth": depth}


def triangles_scene(tris, n=1, seed=0, **kw):
    """Scene from explicit flat triangles [(P0, P1, P2), ...] lifted to degree n
    without noise (the surfaces stay flat). Keyword arguments go to make_scene."""
    mesh = _Mesh()
    mesh.add_object(("flat",), [tuple(np.asarray(p, np.float64) for p in t) for t in tris])
    return make_scene(mesh, n, 0.0, seed, **kw)


def photo_pair(rng, width, height, noise=0.05):
    """A rendered-looking image and a target to train it against, [H, W, 3]
    float32 in [0, 1], for the photometric loss (Sec. 3.3, Eq. 9).

    The image is a flat background with a few flat rectangles (sharp edges,
    the flat areas where windowed variances are small) and sparse pixel
    noise; the target is the image with Gaussian noise of std `noise`,
    clipped, and one flat stripe every seventh row (structure that differs).
    """
    img = np.empty((height, width, 3), np.float64)
    img[:] = rng.uniform(0.0, 1.0, size=3)
    for _ in range(4):
        y0, x0 = rng.integers(0, max(1, height), 2) if height and width else (0, 0)
        y1 = y0 + rng.integers(1, max(2, height // 2 + 1))
        x1 = x0 + rng.integers(1, max(2, width // 2 + 1))
        img[y0:y1, x0:x1] = rng.uniform(0.0, 1.0, size=3)
    speck = rng.uniform(size=(height, width, 1)) < 0.3
    img += rng.normal(scale=0.02, size=img.shape) * speck
    img = np.clip(img, 0.0, 1.0)
    gt = np.clip(img + rng.normal(scale=noise, size=img.shape), 0.0, 1.0)
    gt[::7] = rng.uniform(0.0, 1.0, size=3)
    return img.astype(np.float32), gt.astype(np.float32)


def mixed_shapes_scene(count, n, seed=0, curve=0.15):
    """`count` degree-n primitives of mixed size and shape for the split and
    prune geometry (Sec. 3.3): corner triangles with longest edge log-uniform
    in [1e-3, 1] and height / edge log-uniform in [1e-3, 1] (from tiny to
    sliver-like), randomly oriented and placed in [-2, 2]^3, control points
    moved by N(0, curve * edge) (curved patches), colour control points
    U[0, 1] each, opacity U[0.5, 1], r_b U[5e-3, 2e-2], attribute maps of
    leg 1."""
    rng = np.random.default_rng(seed)
    tris = []
    for _ in range(count):
        e = 10.0 ** rng.uniform(-3.0, 0.0)
        h = e * 10.0 ** rng.uniform(-3.0, 0.0)
        t = rng.uniform(-0.5, 1.5)
        local = np.array([[0.0, 0.0, 0.0], [e, 0.0, 0.0], [t * e, h, 0.0]])
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        tris.append(local @ q.T + rng.uniform(-2.0, 2.0, size=3))
    sc = triangles_scene(tris, n=n, seed=seed)
    m = ncp(n)
    edge = np.array([np.linalg.norm(np.asarray(tr)[1] - np.asarray(tr)[0]) for tr in tris])
    noise = rng.normal(size=(count, m, 3)) * (curve * edge)[:, None, None]
    sc["ctrl"] = np.ascontiguousarray(sc["ctrl"] + noise, np.float32)
    sc["color"] = np.ascontiguousarray(rng.uniform(0.0, 1.0, size=(count, m, 3)), np.float32)
    sc["r_b"] = np.ascontiguousarray(rng.uniform(5e-3, 2e-2, size=count), np.float32)
    return sc
