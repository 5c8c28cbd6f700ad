"""Python front end of the FP64 CPU oracle (bgt_oracle.c).

TEST INFRASTRUCTURE: imported only by tests/, by __graft_entry__.smoke() and
by the CPU-baseline leg of bench.py. The CUDA library never imports it.

Functions take the scene / camera dicts produced by the seeded generator
(paper_2503_13961_gb300.scenes) and return numpy arrays in FP64. The C file is
compiled with gcc (-O2 -fopenmp -ffp-contract=off) into oracle/_build/.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libbgt_oracle.so")
_LOCK = threading.Lock()
_LIB = None

GREC = 14
BREC = 6
GGRAD = 9

F_AMIN, F_AMAX, F_TSTOP, F_DEPTH, F_SAT, F_ARGMIN, F_DZERO, F_DEPTHG = 1, 2, 4, 8, 16, 32, 64, 128
FWD_UNSTABLE = F_AMIN | F_AMAX | F_TSTOP | F_DEPTH

# Defaults shared by name (not by code) with the CUDA library's config.
DEFAULTS = {
    "tess_level": 8,
    "near_z": 0.2,
    "k_b": 3.0,
    "alpha_min": float(np.float32(1.0 / 255.0)),
    "alpha_max": float(np.float32(0.99)),
    "t_stop": float(np.float32(1e-4)),
    "dilation": float(np.float32(0.3)),
    "use_boundary": 1,
    "all_pairs": 0,
    "tol_alpha": 2e-5,
    "tol_T": 1e-4,
    "tol_z": 3e-9,
    "tol_rho": 1e-5,
    "tol_d": 1e-4,
}


def build(force=False):
    """Compile the oracle shared library (gcc, no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, f32, f64, i64 = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_int64
            L.bgto_bernstein.argtypes = [i32, f64, f64, f64, P]
            L.bgto_decasteljau.argtypes = [i32, P, f64, f64, f64, P]
            L.bgto_raster.argtypes = [i32, i32, P, i32, P, i32, i32, f32, i32, P, P, P, P]
            L.bgto_render.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, i32, i32, P, P, P, P,
                                      P, P, P, P, P, P, P, P]
            L.bgto_backward.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, i32, i32, P, P, P, P,
                                        P, P, P, P, P, P, P, P, P]
            L.bgto_sh_basis.argtypes = [i32, P, P]
            L.bgto_attr_weights.argtypes = [i32, f64, f64, P, P]
            L.bgto_pixel_lists.argtypes = [i32, i32, i32, P, P, P, P, P, P, f64, P, P, i64]
            L.bgto_pixel_lists.restype = i64
            L.bgto_num_threads.restype = i32
            L.bgto_gamma.argtypes = [f64, f64]
            L.bgto_gamma.restype = f64
            L.bgto_wvalues.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, i32, i32, P, P, P, i32,
                                       P, P, P, P]
            _LIB = L
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads():
    return int(lib().bgto_num_threads())


def cam_array(cam):
    """FP32 camera vector R[9], t[3], fx, fy, cx, cy."""
    v = np.concatenate([np.asarray(cam["R"], np.float32).ravel(), np.asarray(cam["t"], np.float32).ravel(),
                        np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"]], np.float32)])
    return np.ascontiguousarray(v, np.float32)


def _params(opts, scene=None):
    o = dict(DEFAULTS)
    o.update(opts or {})
    R = int(scene.get("attr_res", 1)) if scene is not None else 1
    D = int(scene.get("sh_degree", 0)) if scene is not None else 0
    return o, np.array([o["k_b"], o["alpha_min"], o["alpha_max"], o["t_stop"], o["dilation"],
                        o["use_boundary"], o["all_pairs"], o["tol_alpha"], o["tol_T"], o["tol_z"],
                        o["tol_rho"], o["tol_d"], R, D], np.float64)


def attr_weights(R, u, v):
    """Eq. 5 texture interpolation Theta on a leg-R triangular attribute map:
    (texel indices [3], weights [3]) of the lattice triangle holding (u, v)."""
    idx = np.zeros(3, np.int32)
    w = np.zeros(3, np.float64)
    rc = lib().bgto_attr_weights(int(R), float(u), float(v), _p(idx), _p(w))
    assert rc == 0, rc
    return idx, w


def sh_basis(D, direction):
    """Real spherical harmonics of bands 1..D at a direction (the SH colour's
    basis, from the associated Legendre definition), [(D + 1)^2 - 1]."""
    Y = np.zeros(max((D + 1) ** 2 - 1, 1), np.float64)
    d = np.ascontiguousarray(direction, np.float64)
    rc = lib().bgto_sh_basis(int(D), _p(d), _p(Y))
    assert rc == 0, rc
    return Y[:(D + 1) ** 2 - 1]


def bernstein(n, u, v, w):
    out = np.zeros((n + 1) * (n + 2) // 2, np.float64)
    assert lib().bgto_bernstein(n, u, v, w, _p(out)) == 0
    return out


def decasteljau(n, ctrl, u, v, w):
    c = np.ascontiguousarray(ctrl, np.float64)
    out = np.zeros(3, np.float64)
    assert lib().bgto_decasteljau(n, _p(c), u, v, w, _p(out)) == 0
    return out


def raster(scene, cam, tess_level=None, near_z=None, ztest=True, cover=False):
    """Tessellate + rasterize: returns (id [H,W] int32, uv [H,W,2] f64, key [H,W] u64[, cover])."""
    L = DEFAULTS["tess_level"] if tess_level is None else tess_level
    nz = DEFAULTS["near_z"] if near_z is None else near_z
    W, H = cam["width"], cam["height"]
    ctrl = np.ascontiguousarray(scene["ctrl"], np.float32)
    M = ctrl.shape[0]
    idm = np.empty((H, W), np.int32)
    uv = np.empty((H, W, 2), np.float64)
    key = np.empty((H, W), np.uint64)
    cov = np.empty((H, W), np.int32) if cover else None
    rc = lib().bgto_raster(scene["degree"], M, _p(ctrl), L, _p(cam_array(cam)), W, H, nz,
                           1 if ztest else 0, _p(idm), _p(uv), _p(key), _p(cov))
    assert rc == 0, rc
    return (idm, uv, key, cov) if cover else (idm, uv, key)


def _scene64(scene):
    f = lambda k: np.ascontiguousarray(scene[k], np.float64)
    out = {k: f(k) for k in ("ctrl", "color", "opacity", "r_b", "log_scale", "quat", "bg")}
    if scene.get("sh_degree", 0) > 0:
        out["sh"] = f("sh")
    return out


def render(scene, cam, idm=None, uv=None, opts=None, pixels=None, records=False, scene64=None):
    """Forward pass in FP64. Returns dict with image [H,W,3], T [H,W], n [H,W],
    flags [H,W], hash, F, Nb and (records=True) gauss [F,14] / bnd [Nb,6].

    idm / uv default to bgto_raster's output. `pixels` (bool [H,W]) limits
    compositing to those pixels. `scene64` overrides the parameters with FP64
    arrays (finite differences)."""
    o, par = _params(opts, scene)
    W, H = cam["width"], cam["height"]
    if idm is None:
        idm, uv, _ = raster(scene, cam, o["tess_level"], o["near_z"])
    s = scene64 if scene64 is not None else _scene64(scene)
    M = s["ctrl"].shape[0]
    img = np.zeros((H, W, 3), np.float64)
    T = np.zeros((H, W), np.float64)
    nn = np.zeros((H, W), np.int32)
    fl = np.zeros((H, W), np.int32)
    hsh = np.zeros(1, np.uint64)
    cnt = np.zeros(2, np.int32)
    mask = None if pixels is None else np.ascontiguousarray(pixels, np.int32)
    grec = np.zeros((max(W * H, 1), GREC), np.float64) if records else None
    brec = np.zeros((max(W * H, 1), BREC), np.float64) if records else None
    idm = np.ascontiguousarray(idm, np.int32)
    uv = np.ascontiguousarray(uv, np.float64)
    rc = lib().bgto_render(scene["degree"], M, _p(s["ctrl"]), _p(s["color"]), _p(s["opacity"]),
                           _p(s["r_b"]), _p(s["log_scale"]), _p(s["quat"]), _p(s["bg"]), _p(s.get("sh")),
                           _p(cam_array(cam)), W, H, _p(idm), _p(uv), _p(par), _p(mask), _p(img),
                           _p(T), _p(nn), _p(fl), _p(hsh), _p(grec), _p(brec), _p(cnt))
    assert rc == 0, rc
    out = {"image": img, "T": T, "n": nn, "flags": fl, "hash": int(hsh[0]), "F": int(cnt[0]),
           "Nb": int(cnt[1]), "id": idm, "uv": uv}
    if records:
        out["gauss"] = grec[: cnt[0]].copy()
        out["bnd"] = brec[: cnt[1]].copy()
    return out


def backward(scene, cam, dLdC, idm=None, uv=None, opts=None, scene64=None, intermediates=False):
    """Gradients of l = sum dLdC * C with the raster and all discrete choices frozen.
    Returns dict ctrl [M,Ncp,3], color [M,Ncp,3], opacity [M], r_b [M],
    log_scale and quat (shaped like the scene's attribute maps)
    (+ ggrad [F,9], bgrad [Nb,3] if intermediates)."""
    o, par = _params(opts, scene)
    W, H = cam["width"], cam["height"]
    if idm is None:
        idm, uv, _ = raster(scene, cam, o["tess_level"], o["near_z"])
    s = scene64 if scene64 is not None else _scene64(scene)
    M, m = s["ctrl"].shape[0], s["ctrl"].shape[1]
    gc = np.zeros((M, m, 3), np.float64)
    gcol = np.zeros((M, m, 3), np.float64)
    go = np.zeros(M, np.float64)
    grb = np.zeros(M, np.float64)
    P = max(W * H, 1)
    gg = np.zeros((P, GGRAD), np.float64) if intermediates else None
    gb = np.zeros((P, 3), np.float64) if intermediates else None
    dl = np.ascontiguousarray(dLdC, np.float64).reshape(H, W, 3)
    idm = np.ascontiguousarray(idm, np.int32)
    uv = np.ascontiguousarray(uv, np.float64)
    gls = np.zeros(s["log_scale"].shape, np.float64)
    gq = np.zeros(s["quat"].shape, np.float64)
    gsh = np.zeros(s["sh"].shape, np.float64) if "sh" in s else None
    rc = lib().bgto_backward(scene["degree"], M, _p(s["ctrl"]), _p(s["color"]), _p(s["opacity"]),
                             _p(s["r_b"]), _p(s["log_scale"]), _p(s["quat"]), _p(s["bg"]), _p(s.get("sh")),
                             _p(cam_array(cam)), W, H, _p(idm), _p(uv), _p(par), _p(dl), _p(gc),
                             _p(gcol), _p(go), _p(grb), _p(gg), _p(gb), _p(gls), _p(gq), _p(gsh))
    assert rc == 0, rc
    out = {"ctrl": gc, "color": gcol, "opacity": go, "r_b": grb, "log_scale": gls, "quat": gq}
    if gsh is not None:
        out["sh"] = gsh
    if intermediates:
        F = int((idm >= 0).sum())
        out["ggrad"] = gg[:F].copy()
        out["bgrad"] = gb
    return out


def pixel_lists(g, width, height, alpha_min=None):
    """Per-pixel (depth, index)-ordered support lists of synthetic Gaussians
    (see scenes.random_gaussians). Returns (ptr [P+1], idx)."""
    am = DEFAULTS["alpha_min"] if alpha_min is None else alpha_min
    P = width * height
    ptr = np.zeros(P + 1, np.int32)
    cnt = len(g["qx"])
    cap = max(16, 40 * cnt)
    while True:
        idx = np.zeros(cap, np.int32)
        tot = lib().bgto_pixel_lists(width, height, cnt, _p(g["qx"]), _p(g["qy"]),
                                     _p(np.ascontiguousarray(g["off"], np.float32)),
                                     _p(np.ascontiguousarray(g["conic"], np.float32)),
                                     _p(g["opacity"]), _p(g["depth"]), am, _p(ptr), _p(idx), cap)
        if tot >= 0:
            return ptr, idx[:tot]
        cap = -tot


def gamma(d, sigma):
    """Eq. 7 blur function."""
    return float(lib().bgto_gamma(float(d), float(sigma)))


def wvalues(scene, cam, pix, prim, idm=None, uv=None, opts=None):
    """Eq. 6 coefficient w(q, g) for pixel indices `pix` and primitives `prim`.
    Returns (w, most influential boundary index)."""
    o, par = _params(opts, scene)
    W, H = cam["width"], cam["height"]
    if idm is None:
        idm, uv, _ = raster(scene, cam, o["tess_level"], o["near_z"])
    s = _scene64(scene)
    pix = np.ascontiguousarray(pix, np.int32)
    prim = np.ascontiguousarray(prim, np.int32)
    w = np.zeros(len(pix), np.float64)
    b = np.zeros(len(pix), np.int32)
    rc = lib().bgto_wvalues(scene["degree"], s["ctrl"].shape[0], _p(s["ctrl"]), _p(s["color"]),
                            _p(s["opacity"]), _p(s["r_b"]), _p(s["log_scale"]), _p(s["quat"]),
                            _p(s["bg"]), _p(s.get("sh")), _p(cam_array(cam)), W, H,
                            _p(np.ascontiguousarray(idm, np.int32)),
                            _p(np.ascontiguousarray(uv, np.float64)), _p(par), len(pix), _p(pix),
                            _p(prim), _p(w), _p(b))
    assert rc == 0, rc
    return w, b


def scene_to64(scene):
    return _scene64(scene)
