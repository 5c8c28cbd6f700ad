"""bgt_bin_sort_static: the binning + sort stage for callers that cannot
allocate device memory (no handle; scratch in a static device array).

Its tile ranges and sorted keys must equal those of bgt_bin_sort (integer
outputs: exact) on the same Gaussians, for two calls in a row (the second on
different inputs, so nothing left in the shared scratch may leak into it),
and must pass the same check against the oracle's per-pixel lists as the
handle's binning (every Gaussian whose FP64 support holds a pixel listed in
the pixel's tile in the oracle's (depth, index) order, every other entry
valid); inputs beyond its limits must be rejected. This file is collected
last.
"""
import ctypes

import numpy as np
import pytest

from tests.test_gpu_sort import _check_lists

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    qxy = (g["qx"].astype(np.int64) | (g["qy"].astype(np.int64) << 16)).astype(np.int32)
    return {"qxy": torch.as_tensor(qxy, device="cuda"),
            "off": torch.as_tensor(np.ascontiguousarray(g["off"], np.float32), device="cuda"),
            "conic": torch.as_tensor(np.ascontiguousarray(g["conic"], np.float32), device="cuda"),
            "opacity": torch.as_tensor(g["opacity"], device="cuda"),
            "depth": torch.as_tensor(g["depth"], device="cuda")}


def _static_call(lib, d, count, W, H, tile, alpha_min, cap):
    import torch
    tiles = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    ranges = torch.full((tiles + 1,), -1, dtype=torch.int64, device="cuda")
    keys = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.bgt_bin_sort_static(W, H, tile, count, P(d["qxy"]), P(d["off"]), P(d["conic"]), P(d["opacity"]),
                                 P(d["depth"]), ctypes.c_float(alpha_min), P(ranges), P(keys), cap,
                                 ctypes.c_void_p(st))
    torch.cuda.synchronize()
    r = ranges.cpu().numpy()
    return rc, r, keys.cpu().numpy().view(np.uint64)[: max(int(r[-1]), 0)]


@pytest.mark.parametrize("W,H,n,tile,radius", [(70, 45, 700, 16, (0.5, 3.0)), (40, 36, 9000, 32, (2.0, 5.0))])
def test_static_entry_matches_bin_sort_twice(oracle, scenes, W, H, n, tile, radius):
    from paper_2503_13961_gb300 import _abi
    from paper_2503_13961_gb300 import render as R
    lib = _abi.load()
    rd = R.Renderer(degree=2, max_prims=1, max_views=1, max_pixels=max(W * H, n), max_pairs=64 * max(W * H, n),
                    max_boundary_pairs=1024, tile_size=tile)
    am = float(np.float32(rd.cfg.alpha_min))
    for seed in (tile, tile + 100):  # two calls in a row on different inputs
        g = scenes.random_gaussians(seed, W, H, n, radius_px=radius)
        ref = rd.bin_sort(g, W, H)
        rd.sync_status()
        rc, ranges, keys = _static_call(lib, _dev(g), n, W, H, tile, am, 262144)
        assert rc == 0, _abi.STATUS_NAMES.get(rc, rc)
        assert np.array_equal(ranges, ref["ranges"])
        assert np.array_equal(keys, ref["keys"])
        ptr, idx = oracle.pixel_lists(g, W, H, alpha_min=am)
        _check_lists(g, W, H, tile, ranges, keys, ptr, idx, am)
    rd.close()


def test_static_entry_rejects_sizes_beyond_its_limits(scenes):
    from paper_2503_13961_gb300 import _abi
    lib = _abi.load()
    g = scenes.random_gaussians(1, 64, 64, 8)
    d = _dev(g)
    am = float(np.float32(1.0 / 255.0))
    # more Gaussians than the scratch holds: rejected before any work
    rc, _, _ = _static_call(lib, d, 65537, 64, 64, 16, am, 1024)
    assert rc == 2
    # more tiles than the scratch holds (4096 x 4096 px at tile 8)
    rc, _, _ = _static_call(lib, d, 8, 4096, 4096, 8, am, 1024)
    assert rc == 2
    # key capacity too small for this input: rejected after the counting pass
    rc, _, _ = _static_call(lib, d, 8, 64, 64, 8, am, 1)
    assert rc == 2
    # and a valid call afterwards still works
    rc, r, _ = _static_call(lib, d, 8, 64, 64, 8, am, 1024)
    assert rc == 0 and r[-1] > 0
