"""ctypes binding of include/bgt.h (argument marshalling only).

Loads the in-tree libbgt.so (building it with nvcc first if it is missing or
older than its sources). There is no fallback: if the library cannot be
built or loaded, import of the renderer fails with the reason.
"""
import ctypes
import os
import re
import threading

from . import build as _build

_LOCK = threading.Lock()
_LIB = None

c_int, c_float, c_ll, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_longlong, ctypes.c_void_p

BGT_OK = 0
STATUS_NAMES = {0: "BGT_OK", 1: "BGT_ERR_INVALID_ARG", 2: "BGT_ERR_CAPACITY", 3: "BGT_ERR_CUDA",
                4: "BGT_ERR_TIMEOUT", 5: "BGT_ERR_NONFINITE", 6: "BGT_ERR_STATE"}
FLAG_NO_BOUNDARY = 1
FLAG_GRAPH = 2

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bgt.h")


class Config(ctypes.Structure):
    _fields_ = [("degree", c_int), ("max_prims", c_int), ("max_views", c_int), ("max_pixels", c_ll),
                ("max_pairs", c_ll), ("max_boundary_pairs", c_ll), ("max_blend_pairs", c_ll),
                ("tess_level", c_int), ("tile_size", c_int),
                ("k_b", c_float), ("alpha_min", c_float), ("alpha_max", c_float), ("t_stop", c_float),
                ("dilation", c_float), ("near_z", c_float), ("flags", c_int)]


class Camera(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int), ("height", c_int)]


class Scene(ctypes.Structure):
    _fields_ = [("ctrl", c_void_p), ("color", c_void_p), ("opacity", c_void_p), ("r_b", c_void_p),
                ("log_scale", c_void_p), ("quat", c_void_p), ("num_prims", c_int), ("bg", c_float * 3),
                ("attr_res", c_int), ("sh", c_void_p), ("sh_degree", c_int)]


class Grads(ctypes.Structure):
    _fields_ = [("ctrl", c_void_p), ("color", c_void_p), ("opacity", c_void_p), ("r_b", c_void_p),
                ("log_scale", c_void_p), ("quat", c_void_p), ("sh", c_void_p)]


class Tuning(ctypes.Structure):
    """bgt_tuning: scheduling knobs of the batched launches."""
    _fields_ = [("tile_size", c_int), ("raster_prims", c_int), ("bwd_dequeue", c_int),
                ("chain_blocks_per_sm", c_int)]


PRIMS_KEYS = ("ctrl", "color", "opacity", "r_b", "log_scale", "quat", "sh")


class Prims(ctypes.Structure):
    """bgt_prims: output arrays of bgt_subdivide."""
    _fields_ = [(k, c_void_p) for k in PRIMS_KEYS]


class BGTError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _declare(L):
    P = c_void_p
    L.bgt_default_config.argtypes = [ctypes.POINTER(Config)]
    L.bgt_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(c_void_p)]
    L.bgt_destroy.argtypes = [P]
    L.bgt_destroy.restype = None
    L.bgt_render_fwd.argtypes = [P, ctypes.POINTER(Scene), ctypes.POINTER(Camera), c_int, P, P]
    L.bgt_render_bwd.argtypes = [P, ctypes.POINTER(Scene), ctypes.POINTER(Camera), c_int, P, ctypes.POINTER(Grads), P]
    L.bgt_sync_status.argtypes = [P, P]
    L.bgt_last_error.argtypes = [P]
    L.bgt_last_error.restype = ctypes.c_char_p
    L.bgt_get_counts.argtypes = [P, ctypes.POINTER(c_ll), P]
    L.bgt_set_tile_size.argtypes = [P, c_int]
    L.bgt_get_tile_size.argtypes = [P]
    L.bgt_autotune.argtypes = [P, ctypes.POINTER(Scene), ctypes.POINTER(Camera), c_int, P, P, ctypes.POINTER(Grads),
                               c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_float), P]
    L.bgt_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    L.bgt_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    L.bgt_l1_loss_grad.argtypes = [P, P, c_ll, c_float, P, P, P]
    L.bgt_l2_dssim_loss_grad.argtypes = [P, P, c_int, P, c_float, c_float, P, P, P]
    L.bgt_prim_metrics.argtypes = [c_int, ctypes.POINTER(Scene), P, c_float, c_float, c_float, P, P, c_float, P,
                                   c_int, P, c_int, c_float, c_float, P, P, P, P, P]
    L.bgt_edge_magnitude.argtypes = [P, c_int, P, P, P]
    L.bgt_edge_prior.argtypes = [P, P, P, P, P]
    L.bgt_visibility.argtypes = [P, P, P, P]
    L.bgt_subdivide.argtypes = [c_int, ctypes.POINTER(Scene), P, c_int, ctypes.POINTER(Prims), P]
    L.bgt_get_stage.argtypes = [P, c_int, P, c_ll, ctypes.POINTER(c_ll), P]
    L.bgt_bin_sort.argtypes = [P, c_int, c_int, c_int, P, P, P, P, P, P]
    L.bgt_bin_sort_static.argtypes = [c_int, c_int, c_int, c_int, P, P, P, P, P, c_float, P, P, c_ll, P]
    L.bgt_set_profiling.argtypes = [P, c_int]
    L.bgt_get_profile.argtypes = [P, ctypes.POINTER(c_float), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                  ctypes.POINTER(ctypes.c_ulonglong)]
    return L


def header_functions(path=HEADER):
    """Names of the functions declared in include/bgt.h."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"\b(bgt_[a-z0-9_]+)\s*\(", text)


def library_path():
    return _build.LIB


def load(build=True):
    """Load libbgt.so (building it first if needed). Raises if unavailable."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"libbgt.so not found at {path}; run paper_2503_13961_gb300/build.py")
            _LIB = _declare(ctypes.CDLL(path))
    return _LIB


def check(status, handle=None):
    if status != BGT_OK:
        msg = ""
        if handle:
            msg = (load().bgt_last_error(handle) or b"").decode(errors="replace")
        raise BGTError(status, msg)


def make_camera(cam):
    c = Camera()
    R = [float(x) for x in list(_flat(cam["R"]))]
    t = [float(x) for x in list(_flat(cam["t"]))]
    c.R[:] = R
    c.t[:] = t
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def _flat(x):
    try:
        import numpy as np
        return np.asarray(x, dtype=np.float32).ravel()
    except Exception:  # pragma: no cover
        return x


def camera_array(cams):
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = make_camera(c)
    return arr
