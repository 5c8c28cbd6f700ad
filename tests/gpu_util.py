"""Helpers shared by the GPU parity tests: run the CUDA path through the
C ABI binding and fetch the oracle's reference for the same seeded inputs."""
import numpy as np

FWD_TOL = 1e-4       # absolute per channel, images (stable pixels)
UNSTABLE_MAX = 5e-3  # fraction of pixels the oracle may flag as near a discontinuity
GRAD_TOL = 1e-3      # relative


def make_renderer(scene, cams, tile=16, use_boundary=True, graph=False, pairs_per_px=8, **kw):
    from paper_2503_13961_gb300 import render as R
    P = sum(c["width"] * c["height"] for c in cams)
    return R.Renderer(degree=scene["degree"], max_prims=max(1, scene["ctrl"].shape[0]), max_views=len(cams),
                      max_pixels=max(P, 1), max_pairs=max(1024, pairs_per_px * P),
                      max_boundary_pairs=max(1024, pairs_per_px * P), tile_size=tile,
                      use_boundary=use_boundary, graph=graph, **kw)


def gpu_forward(scene, cams, tile=16, use_boundary=True, renderer=None, stages=("id", "uv")):
    import torch
    from paper_2503_13961_gb300 import render as R
    rd = renderer or make_renderer(scene, cams, tile=tile, use_boundary=use_boundary)
    dev = R.scene_to_device(scene)
    img = rd.forward(dev, cams)
    rd.sync_status()
    torch.cuda.synchronize()
    out = {"renderer": rd, "dev": dev, "images_flat": img,
           "images": [v.cpu().numpy().astype(np.float64) for v in R.split_views(img, cams)],
           "counts": rd.counts()}
    for s in stages:
        out[s] = rd.stage(s)
    return out


def oracle_opts(use_boundary=True, **kw):
    o = {"use_boundary": 1 if use_boundary else 0}
    o.update(kw)
    return o


def split_flat(arr, cams, width=1):
    out, off = [], 0
    for c in cams:
        n = c["width"] * c["height"]
        a = arr[off * width:(off + n) * width]
        out.append(a.reshape(c["height"], c["width"], *((width,) if width > 1 else ())))
        off += n
    return out


def compare_images(got, ref, flags, oracle):
    stable = (flags & oracle.FWD_UNSTABLE) == 0
    err = np.abs(got - ref["image"])
    return float(err[stable].max()) if stable.any() else 0.0, float((~stable).mean())


def grad_rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
