"""PyTorch front end of the BG-Triangle CUDA rasterizer.

`Renderer` owns one library handle (workspace sized at construction) and
marshals torch CUDA tensors into the C ABI of include/bgt.h; `render()`
wraps forward + backward in a torch.autograd.Function. PyTorch only provides
device memory and the stream: every stage runs in the library's kernels.
"""
import ctypes

import numpy as np
import torch

from . import _abi

SCENE_KEYS = ("ctrl", "color", "opacity", "r_b", "log_scale", "quat")
GRAD_KEYS = ("ctrl", "color", "opacity", "r_b", "log_scale", "quat", "sh")

STAGE_ID = {"id": 0, "uv": 1, "gauss": 2, "bnd": 3, "g_ranges": 4, "g_keys": 5, "b_ranges": 6,
            "b_keys": 7, "T": 8, "n": 9, "ggrad": 10, "bgrad": 11}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def scene_to_device(scene, device="cuda"):
    """Numpy scene dict (see scenes.py) -> dict of contiguous float32 CUDA tensors."""
    out = {k: torch.as_tensor(np.ascontiguousarray(scene[k]), dtype=torch.float32, device=device)
           for k in SCENE_KEYS}
    out["degree"] = int(scene["degree"])
    out["bg"] = [float(x) for x in np.asarray(scene["bg"]).ravel()]
    out["attr_res"] = int(scene.get("attr_res", 1))
    out["sh_degree"] = int(scene.get("sh_degree", 0))
    if out["sh_degree"] > 0:
        out["sh"] = torch.as_tensor(np.ascontiguousarray(scene["sh"]), dtype=torch.float32, device=device)
    return out


def _grads_struct(grads):
    """bgt_grads of a dict of tensors; absent keys (or None) are not computed."""
    return _abi.Grads(*((grads[k].data_ptr() if grads.get(k) is not None else None) for k in GRAD_KEYS))


def _device_f32(t, name, numel=None):
    """A contiguous float32 CUDA tensor (the library writes or reads it on the
    device), of `numel` elements if given; else ValueError."""
    if t is None:
        return None
    if not (torch.is_tensor(t) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} floats, not {t.numel()}")
    return t


def _scene_struct(sc):
    """bgt_scene of a device scene dict (see scene_to_device)."""
    s = _abi.Scene()
    for k in SCENE_KEYS:
        t = sc[k]
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous(), k
        setattr(s, k, t.data_ptr())
    s.num_prims = int(sc["ctrl"].shape[0])
    s.bg[:] = [float(x) for x in sc["bg"]]
    s.attr_res = int(sc.get("attr_res", 1))
    s.sh_degree = int(sc.get("sh_degree", 0))
    if s.sh_degree > 0:
        t = sc["sh"]
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous(), "sh"
        s.sh = t.data_ptr()
    return s


# thresholds of the splitting and pruning criteria (Sec. 3.3 and its implementation details)
TAU_A, TAU_S, TAU_G = 3e-4, 10.0, 0.0018


TAU_V, TAU_R, TAU_B = 0.08, 0.4, 13.0


def prim_metrics(scene, g_ctrl=None, tau_a=TAU_A, tau_s=TAU_S, tau_g=TAU_G, view_count=None, n_views=0,
                 cell_mask=None, tess_level=8, tau_v=TAU_V, tau_r=TAU_R, edge_sum=None, edge_count=None,
                 tau_b=TAU_B, stream=None):
    """Area, aspect ratio, mean control-point gradient and the flags of the
    splitting and pruning criteria (bit 0 prune by area / aspect, bit 1
    split by gradient or edge prior, bit 2 occluded in the views, bit 3
    occluded in the visibility texture) of every primitive of a device scene
    (bgt_prim_metrics); view_count / cell_mask come from Renderer.visibility
    over n_views views, edge_sum / edge_count from Renderer.edge_prior."""
    lib = _abi.load()
    M = int(scene["ctrl"].shape[0])
    dev = scene["ctrl"].device
    out = {"area": torch.empty(M, device=dev), "aspect": torch.empty(M, device=dev),
           "flags": torch.empty(M, dtype=torch.uint8, device=dev)}
    if g_ctrl is not None:
        if not (g_ctrl.is_cuda and g_ctrl.dtype == torch.float32 and g_ctrl.is_contiguous()
                and g_ctrl.shape == scene["ctrl"].shape):
            raise ValueError("g_ctrl must be a contiguous float32 CUDA tensor shaped like scene['ctrl']")
        out["grad"] = torch.empty(M, device=dev)
    if (edge_sum is None) != (edge_count is None):
        raise ValueError("edge_sum and edge_count go together")
    for name, t, dt in (("view_count", view_count, torch.int32), ("cell_mask", cell_mask, torch.int64),
                        ("edge_sum", edge_sum, torch.float32), ("edge_count", edge_count, torch.int32)):
        if t is not None and not (t.is_cuda and t.dtype == dt and t.is_contiguous() and t.shape[0] == M):
            raise ValueError(f"{name} must be a contiguous {dt} CUDA tensor with one row per primitive")
    sc = _scene_struct(scene)
    _abi.check(lib.bgt_prim_metrics(int(scene["degree"]), ctypes.byref(sc), _ptr(g_ctrl), float(tau_a), float(tau_s),
                                    float(tau_g), _ptr(edge_sum), _ptr(edge_count), float(tau_b),
                                    _ptr(view_count), int(n_views), _ptr(cell_mask), int(tess_level),
                                    float(tau_v), float(tau_r), _ptr(out["area"]), _ptr(out["aspect"]),
                                    _ptr(out.get("grad")), _ptr(out["flags"]), _stream(stream)))
    return out


def edge_magnitude(images, cams, edges=None, stream=None):
    """Sobel magnitude of the 8-bit luma of training images in the renderer's
    layout (bgt_edge_magnitude): [sum W H] float32."""
    lib = _abi.load()
    n = sum(int(c["width"]) * int(c["height"]) for c in cams)
    _device_f32(images, "images", 3 * n)
    if edges is None:
        edges = torch.empty(n, dtype=torch.float32, device=images.device)
    _device_f32(edges, "edges", n)
    sizes = (ctypes.c_int * (2 * len(cams)))(*[int(x) for c in cams for x in (c["width"], c["height"])])
    _abi.check(lib.bgt_edge_magnitude(_ptr(images), len(cams), sizes, _ptr(edges), _stream(stream)))
    return edges


def subdivide(scene, sel, stream=None):
    """Device scene of the 1 -> 4 midpoint split of the primitives `sel`
    (int32 CUDA tensor): piece 4 s + p of sel[s], p = U, V, W corner, middle
    (bgt_subdivide)."""
    lib = _abi.load()
    sel = torch.as_tensor(sel).to(device=scene["ctrl"].device, dtype=torch.int32).contiguous()
    n = int(sel.numel())
    out = {"degree": scene["degree"], "bg": list(scene["bg"]), "attr_res": int(scene.get("attr_res", 1)),
           "sh_degree": int(scene.get("sh_degree", 0))}
    for k in SCENE_KEYS + (("sh",) if out["sh_degree"] > 0 else ()):
        t = scene[k]
        out[k] = torch.empty((4 * n,) + tuple(t.shape[1:]), dtype=torch.float32, device=t.device)
    if n == 0:
        return out
    sc = _scene_struct(scene)
    pr = _abi.Prims(*(out[k].data_ptr() if k in out else None for k in _abi.PRIMS_KEYS))
    _abi.check(lib.bgt_subdivide(int(scene["degree"]), ctypes.byref(sc), _ptr(sel), n, ctypes.byref(pr),
                                 _stream(stream)))
    return out


def view_pixels(cams):
    if isinstance(cams, Cameras):
        return cams.pixels
    return int(sum(int(c["width"]) * int(c["height"]) for c in cams))


class Cameras(list):
    """A list of camera dicts whose C array is built once, for loops that
    render the same views every step (a snapshot: later edits of the dicts
    are not seen)."""

    def __init__(self, cams):
        super().__init__(cams)
        self.array = _abi.camera_array(self)
        self.pixels = int(sum(int(c["width"]) * int(c["height"]) for c in self))


def _camera_array(cams):
    return cams.array if isinstance(cams, Cameras) else _abi.camera_array(cams)


class Renderer:
    """One handle of the BG-Triangle library on the current CUDA device.

    Capacities: max_prims, max_views, max_pixels (sum of W*H of one call),
    max_pairs / max_boundary_pairs ((Gaussian, tile) and (boundary point,
    tile) pairs; default 8 per pixel), max_blend_pairs (composited
    (pixel, Gaussian) pairs the forward records for the backward; default
    8 per pixel; blocks whose records do not fit are re-walked by the
    backward). Options: tess_level L, tile_size
    (8/16/32), use_boundary (False = the paper's "w/o B" ablation), graph
    (capture forward / backward in CUDA graphs) and the blending cutoffs.
    """

    def __init__(self, degree=2, max_prims=100_000, max_views=64, max_pixels=1 << 20, max_pairs=None,
                 max_boundary_pairs=None, max_blend_pairs=0, tess_level=8, tile_size=16, use_boundary=True, graph=False,
                 k_b=3.0, alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4, dilation=0.3, near_z=0.2):
        self.lib = _abi.load()
        cfg = _abi.Config()
        _abi.check(self.lib.bgt_default_config(ctypes.byref(cfg)))
        cfg.degree = degree
        cfg.max_prims = max_prims
        cfg.max_views = max_views
        cfg.max_pixels = max_pixels
        cfg.max_pairs = max_pairs if max_pairs is not None else 8 * max_pixels
        cfg.max_boundary_pairs = max_boundary_pairs if max_boundary_pairs is not None else 8 * max_pixels
        cfg.max_blend_pairs = max_blend_pairs
        cfg.tess_level = tess_level
        self.tess_level = int(tess_level)
        cfg.tile_size = tile_size
        cfg.k_b, cfg.alpha_min, cfg.alpha_max = k_b, alpha_min, alpha_max
        cfg.t_stop, cfg.dilation, cfg.near_z = t_stop, dilation, near_z
        cfg.flags = (0 if use_boundary else _abi.FLAG_NO_BOUNDARY) | (_abi.FLAG_GRAPH if graph else 0)
        self.cfg = cfg
        h = ctypes.c_void_p()
        _abi.check(self.lib.bgt_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self._last_pixels = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.bgt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling -----------------------------------------------------
    def _scene(self, sc):
        return _scene_struct(sc)

    def _check(self, st):
        _abi.check(st, self.h)

    # -- calls -----------------------------------------------------------
    def forward(self, scene, cams, images=None, stream=None):
        """Images [sum W*H, 3] (views packed in order) of `scene` seen by `cams`."""
        P = view_pixels(cams)
        self._last_pixels = P
        if images is None:
            images = torch.empty((P, 3), dtype=torch.float32, device=scene["ctrl"].device)
        _device_f32(images, "images", 3 * P)
        cam_arr = _camera_array(cams)
        sc = self._scene(scene)
        self._check(self.lib.bgt_render_fwd(self.h, ctypes.byref(sc), cam_arr, len(cams), _ptr(images),
                                            _stream(stream)))
        return images

    def backward(self, scene, cams, d_images, grads=None, stream=None):
        """dl/d(ctrl, color, opacity, r_b, log_scale, quat[, sh]) for the last
        forward, given dl/dimages; keys missing from `grads` are not computed."""
        if grads is None:
            grads = {k: torch.empty_like(scene[k]) for k in GRAD_KEYS if scene.get(k) is not None}
        d_images = _device_f32(d_images.contiguous(), "d_images", 3 * view_pixels(cams))
        for k, t in grads.items():
            if t is not None:
                _device_f32(t, f"grads[{k!r}]", scene[k].numel())
        g = _grads_struct(grads)
        sc = self._scene(scene)
        cam_arr = _camera_array(cams)
        self._check(self.lib.bgt_render_bwd(self.h, ctypes.byref(sc), cam_arr, len(cams), _ptr(d_images),
                                            ctypes.byref(g), _stream(stream)))
        return grads

    def sync_status(self, stream=None):
        self._check(self.lib.bgt_sync_status(self.h, _stream(stream)))

    def status_code(self, stream=None):
        return int(self.lib.bgt_sync_status(self.h, _stream(stream)))

    def counts(self, stream=None):
        out = (ctypes.c_longlong * 8)()
        self._check(self.lib.bgt_get_counts(self.h, out, _stream(stream)))
        return {"F": out[0], "Nb": out[1], "K": out[2], "Kb": out[3], "tiles": out[4], "rec_headers": out[5],
                "rec_fill_units": out[6], "walked_blocks": out[7]}

    def set_tile_size(self, t):
        self._check(self.lib.bgt_set_tile_size(self.h, int(t)))

    @property
    def tile_size(self):
        return int(self.lib.bgt_get_tile_size(self.h))

    TUNING_KEYS = ("tile_size", "raster_prims", "bwd_dequeue", "chain_blocks_per_sm")

    def tuning(self):
        """The scheduling of the handle (bgt_tuning) as a dict."""
        t = _abi.Tuning()
        self._check(self.lib.bgt_get_tuning(self.h, ctypes.byref(t)))
        return {k: int(getattr(t, k)) for k in self.TUNING_KEYS}

    def set_tuning(self, **knobs):
        """Change scheduling knobs (tile_size, raster_prims, bwd_dequeue,
        chain_blocks_per_sm); images do not depend on them."""
        cur = self.tuning()
        unknown = set(knobs) - set(cur)
        if unknown:
            raise ValueError(f"unknown tuning knobs {sorted(unknown)}")
        cur.update(knobs)
        t = _abi.Tuning(*(int(cur[k]) for k in self.TUNING_KEYS))
        self._check(self.lib.bgt_set_tuning(self.h, ctypes.byref(t)))

    def autotune(self, scene, cams, images, d_images, grads, iters=3, stream=None):
        best = ctypes.c_int(0)
        ms = (ctypes.c_float * 3)()
        g = _grads_struct(grads)
        self._check(self.lib.bgt_autotune(self.h, ctypes.byref(self._scene(scene)), _camera_array(cams),
                                          len(cams), _ptr(images), _ptr(d_images), ctypes.byref(g), iters,
                                          ctypes.byref(best), ms, _stream(stream)))
        return best.value, {8: ms[0], 16: ms[1], 32: ms[2]}

    STAGES = ("prep", "raster", "resolve", "generate", "binning", "composite_fwd", "composite_bwd", "chain")

    def set_profiling(self, on=True, count_units=True):
        """Stage events on (`on`); with count_units the blending kernels also
        count their work units (their counting build), else the step's own
        kernels are timed."""
        self._check(self.lib.bgt_set_profiling(self.h, (1 if count_units else 2) if on else 0))

    UNITS = ("fwd_support", "fwd_composited", "fwd_candidates", "fwd_warp_visits", "bwd_support",
             "bwd_composited", "bwd_candidates", "bwd_warp_visits")

    def profile(self):
        """Device ms per stage of the last profiled forward + backward, kernel counts
        per pass, and the blending kernels' work units."""
        ms = (ctypes.c_float * 8)()
        kf, kb = ctypes.c_int(0), ctypes.c_int(0)
        units = (ctypes.c_ulonglong * 8)()
        self._check(self.lib.bgt_get_profile(self.h, ms, ctypes.byref(kf), ctypes.byref(kb), units))
        u = {k: int(v) for k, v in zip(self.UNITS, units) if k}
        return dict(zip(self.STAGES, list(ms))), kf.value, kb.value, u

    def l1_loss_grad(self, images, target, scale, d_images=None, loss=None, stream=None):
        if d_images is None:
            d_images = torch.empty_like(images)
        for name, t in (("images", images), ("target", target), ("d_images", d_images)):
            _device_f32(t, name, images.numel())
        _device_f32(loss, "loss", 1)
        _abi.check(self.lib.bgt_l1_loss_grad(_ptr(images), _ptr(target), images.numel(), float(scale),
                                             _ptr(d_images), _ptr(loss), _stream(stream)))
        return d_images

    def l2_dssim_loss_grad(self, images, target, cams, lam=0.2, scale=1.0, d_images=None, loss=None, stream=None):
        """Eq. 9 per view of `images` (the forward's layout, views sized by `cams`): writes
        scale * dL/dC to d_images and adds scale * the sum of the views' losses to `loss`."""
        if d_images is None:
            d_images = torch.empty_like(images)
        sizes = (ctypes.c_int * (2 * len(cams)))(*[int(x) for c in cams for x in (c["width"], c["height"])])
        n = 3 * sum(c["width"] * c["height"] for c in cams)
        for name, t in (("images", images), ("target", target), ("d_images", d_images)):
            _device_f32(t, name, n)
        _device_f32(loss, "loss", 1)
        _abi.check(self.lib.bgt_l2_dssim_loss_grad(_ptr(images), _ptr(target), len(cams), sizes, float(lam),
                                                   float(scale), _ptr(d_images), _ptr(loss), _stream(stream)))
        return d_images

    def visibility(self, num_prims, view_count=None, cell_mask=None, stream=None):
        """Visibility measures of the last forward's views (bgt_visibility),
        accumulated into view_count [M] int32 and cell_mask [M, words] int64
        (zeros when not given; words = ceil(2 L^2 / 64) of the tessellation
        level L): views a primitive owns pixels in, and the lattice flat
        triangles it is seen through."""
        L = self.tess_level
        words = (2 * L * L + 63) // 64
        dev = torch.device("cuda", torch.cuda.current_device())
        if view_count is None:
            view_count = torch.zeros(num_prims, dtype=torch.int32, device=dev)
        if cell_mask is None:
            cell_mask = torch.zeros((num_prims, words), dtype=torch.int64, device=dev)
        if not (view_count.is_cuda and view_count.dtype == torch.int32 and view_count.is_contiguous()
                and view_count.numel() == num_prims):
            raise ValueError("view_count must be a contiguous int32 CUDA tensor of num_prims entries")
        if not (cell_mask.is_cuda and cell_mask.dtype == torch.int64 and cell_mask.is_contiguous()
                and cell_mask.numel() == num_prims * words):
            raise ValueError(f"cell_mask must be a contiguous int64 CUDA tensor of num_prims x {words}")
        self._check(self.lib.bgt_visibility(self.h, _ptr(view_count), _ptr(cell_mask), _stream(stream)))
        return view_count, cell_mask

    def edge_prior(self, edges, num_prims, edge_sum=None, edge_count=None, stream=None):
        """Edge values of the last forward's views back-projected onto the
        primitives through I_id (bgt_edge_prior), accumulated into edge_sum
        [M] float32 and edge_count [M] int32 (zeros when not given)."""
        dev = edges.device
        if edge_sum is None:
            edge_sum = torch.zeros(num_prims, dtype=torch.float32, device=dev)
        if edge_count is None:
            edge_count = torch.zeros(num_prims, dtype=torch.int32, device=dev)
        _device_f32(edges, "edges", self._last_pixels)
        _device_f32(edge_sum, "edge_sum", num_prims)
        if not (edge_count.is_cuda and edge_count.dtype == torch.int32 and edge_count.is_contiguous()
                and edge_count.numel() == num_prims):
            raise ValueError("edge_count must be a contiguous int32 CUDA tensor of num_prims entries")
        self._check(self.lib.bgt_edge_prior(self.h, _ptr(edges), _ptr(edge_sum), _ptr(edge_count), _stream(stream)))
        return edge_sum, edge_count

    def stage(self, name, stream=None):
        """Copy an intermediate buffer of the last forward to a numpy array."""
        which = STAGE_ID[name]
        c = self.counts(stream)
        P = int(self.lib_last_pixels())
        size = {0: 4 * P, 1: 8 * P, 2: 48 * c["F"], 3: 32 * c["Nb"], 4: 8 * (c["tiles"] + 1),
                5: 8 * c["K"], 6: 8 * (c["tiles"] + 1), 7: 8 * c["Kb"], 8: 4 * P, 9: 4 * P,
                10: 48 * c["F"], 11: 16 * c["Nb"]}[which]
        buf = np.empty(max(size, 8), np.uint8)
        written = ctypes.c_longlong(0)
        self._check(self.lib.bgt_get_stage(self.h, which, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes,
                                           ctypes.byref(written), _stream(stream)))
        raw = buf[: written.value]
        if which == 0:
            return raw.view(np.int32)
        if which in (1, 8):
            return raw.view(np.float32).reshape(-1, 2) if which == 1 else raw.view(np.float32)
        if which == 2:
            return raw.view(np.float32).reshape(-1, 12)
        if which == 3:
            return raw.view(np.float32).reshape(-1, 8)
        if which in (4, 6):
            return raw.view(np.int64)
        if which == 9:
            return raw.view(np.int32)
        if which in (5, 7):
            return raw.view(np.uint64)
        if which == 10:
            return raw.view(np.float32).reshape(-1, 12)
        return raw.view(np.float32).reshape(-1, 4)

    def lib_last_pixels(self):
        return self._last_pixels

    def bin_sort(self, g, width, height, stream=None):
        """Binning + per-tile sort of synthetic projected Gaussians (scenes.random_gaussians)."""
        dev = torch.device("cuda")
        qxy = torch.as_tensor((g["qx"].astype(np.int64) | (g["qy"].astype(np.int64) << 16)).astype(np.int32),
                              device=dev)
        off = torch.as_tensor(np.ascontiguousarray(g["off"], np.float32), device=dev)
        conic = torch.as_tensor(np.ascontiguousarray(g["conic"], np.float32), device=dev)
        op = torch.as_tensor(g["opacity"], device=dev)
        dp = torch.as_tensor(g["depth"], device=dev)
        self._check(self.lib.bgt_bin_sort(self.h, int(width), int(height), len(g["qx"]), _ptr(qxy), _ptr(off),
                                          _ptr(conic), _ptr(op), _ptr(dp), _stream(stream)))
        torch.cuda.synchronize()
        self._last_pixels = width * height
        return {"ranges": self.stage("g_ranges", stream), "keys": self.stage("g_keys", stream)}


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, cams, scene_meta, ctrl, color, opacity, r_b, log_scale, quat, sh):
        scene = dict(scene_meta, ctrl=ctrl, color=color, opacity=opacity, r_b=r_b, log_scale=log_scale, quat=quat)
        if scene_meta.get("sh_degree", 0) > 0:
            scene["sh"] = sh
        img = renderer.forward(scene, cams)
        ctx.renderer, ctx.cams, ctx.scene = renderer, cams, scene
        return img

    @staticmethod
    def backward(ctx, d_img):
        g = ctx.renderer.backward(ctx.scene, ctx.cams, d_img.contiguous())
        return (None, None, None, g["ctrl"], g["color"], g["opacity"], g["r_b"], g["log_scale"], g["quat"],
                g.get("sh"))


def render(renderer, scene, cams):
    """Differentiable render: images [sum W*H, 3]; gradients flow to
    scene['ctrl'], ['color'], ['opacity'], ['r_b'], ['log_scale'], ['quat'] and ['sh']."""
    meta = {"degree": scene["degree"], "bg": scene["bg"], "attr_res": scene.get("attr_res", 1),
            "sh_degree": scene.get("sh_degree", 0)}
    sh = scene.get("sh")
    if sh is None:
        sh = scene["opacity"].new_zeros(0)
    return _RenderFn.apply(renderer, cams, meta, scene["ctrl"], scene["color"], scene["opacity"], scene["r_b"],
                           scene["log_scale"], scene["quat"], sh)


class _LossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, cams, lam, images, target):
        loss = images.new_zeros(1)
        d = renderer.l2_dssim_loss_grad(images.contiguous(), target.contiguous(), cams, lam, 1.0, loss=loss)
        ctx.save_for_backward(d)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (d,) = ctx.saved_tensors
        return None, None, None, d * g, None


def photometric_loss(renderer, images, target, cams, lam=0.2):
    """Differentiable Eq. 9 loss, (1 - lam) L2 + lam (1 - SSIM) summed over the
    views of `images` (the forward's layout); its gradient with respect to
    `images` comes from the same fused kernel call as the value."""
    return _LossFn.apply(renderer, cams, float(lam), images, target)


def split_views(images, cams):
    """Packed images [sum W*H, 3] -> list of [H, W, 3] views."""
    out, off = [], 0
    for c in cams:
        n = int(c["width"]) * int(c["height"])
        out.append(images[off: off + n].view(int(c["height"]), int(c["width"]), 3))
        off += n
    return out
