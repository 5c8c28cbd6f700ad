"""Tile binning + (tile, depth) sort and the per-tile boundary lists vs the
oracle's per-pixel lists (Sec. 3.2 "Rendering Acceleration").

For every pixel, the Gaussians whose support o exp(-1/2 d^T K d) >= alpha_min
contains it (oracle, FP64, exact ellipse test) must all appear in the pixel's
tile list, in exactly the oracle's (depth, index) order. Every other entry of
a tile list must be valid: its conservative support box overlaps the tile.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _renderer(width, height, count, tile):
    from paper_2503_13961_gb300 import render as R
    P = max(width * height, count)
    return R.Renderer(degree=2, max_prims=1, max_views=1, max_pixels=P, max_pairs=64 * P,
                      max_boundary_pairs=1024, tile_size=tile)


def _check_lists(g, W, H, tile, ranges, keys, ptr, idx, alpha_min):
    tx = (W + tile - 1) // tile
    ty = (H + tile - 1) // tile
    assert len(ranges) == tx * ty + 1
    gi = (keys & np.uint64((1 << 27) - 1)).astype(np.int64)
    dbits = (keys >> np.uint64(32)).astype(np.uint32)
    # keys carry the Gaussians' FP32 depth bits; FP32 inputs sit mid-interval (sub = 16)
    assert np.array_equal(dbits, g["depth"].view(np.uint32)[gi])
    assert np.all(((keys >> np.uint64(27)) & np.uint64(31)) == 16)
    lists = []
    for t in range(tx * ty):
        seg = keys[ranges[t]:ranges[t + 1]]
        assert np.all(seg[1:] > seg[:-1]), "tile not sorted"
        lists.append(gi[ranges[t]:ranges[t + 1]])
    # validity: every entry's box overlaps its tile
    cx = g["qx"] + g["off"][:, 0].astype(np.float64)
    cy = g["qy"] + g["off"][:, 1].astype(np.float64)
    a, b, c = (g["conic"][:, k].astype(np.float64) for k in range(3))
    det = a * c - b * b
    lvl = 2 * np.log(np.maximum(g["opacity"].astype(np.float64) / alpha_min, 1.0))
    rx = np.sqrt(lvl * c / det) + 0.01
    ry = np.sqrt(lvl * a / det) + 0.01
    for t, lst in enumerate(lists):
        x0, y0 = (t % tx) * tile, (t // tx) * tile
        ok = (cx[lst] + rx[lst] >= x0) & (cx[lst] - rx[lst] <= x0 + tile - 1) & \
             (cy[lst] + ry[lst] >= y0) & (cy[lst] - ry[lst] <= y0 + tile - 1)
        assert ok.all(), f"tile {t}: entry outside its support box"
    # completeness and order per pixel
    for y in range(H):
        for x in range(W):
            p = y * W + x
            want = idx[ptr[p]:ptr[p + 1]]
            lst = lists[(y // tile) * tx + x // tile]
            keep = np.isin(lst, want)
            assert np.array_equal(lst[keep], want), f"pixel ({x},{y})"
    return sorted(len(x) for x in lists)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_sort_matches_oracle_pixel_lists(oracle, scenes, tile):
    W, H, n = 70, 45, 700
    g = scenes.random_gaussians(tile, W, H, n)
    rd = _renderer(W, H, n, tile)
    res = rd.bin_sort(g, W, H)
    rd.sync_status()
    ptr, idx = oracle.pixel_lists(g, W, H)
    _check_lists(g, W, H, tile, res["ranges"], res["keys"], ptr, idx, oracle.DEFAULTS["alpha_min"])


@pytest.mark.parametrize("n, low, high", [(3000, 1024, 4096), (9000, 4096, 1 << 30)])
def test_bin_sort_large_tiles(oracle, scenes, n, low, high):
    # more than 1,024 keys in one tile go to the block sort: bitonic in shared
    # memory up to 4,096 keys, the stable block-wide radix sort beyond
    W, H = 40, 36
    g = scenes.random_gaussians(5, W, H, n, radius_px=(2.0, 5.0))
    rd = _renderer(W, H, n, 32)
    res = rd.bin_sort(g, W, H)
    rd.sync_status()
    ptr, idx = oracle.pixel_lists(g, W, H)
    lengths = _check_lists(g, W, H, 32, res["ranges"], res["keys"], ptr, idx, oracle.DEFAULTS["alpha_min"])
    assert any(low < x <= high for x in lengths), lengths


def test_bin_sort_warp_sized_tiles(oracle, scenes):
    # tiles of 33..64, 65..128 keys (one warp, bitonic network in shared
    # memory) and 129..256, 257..512 keys (one warp, radix sort)
    W, H = 64, 64
    seen = []
    for seed, n in ((21, 150), (22, 400), (23, 900), (24, 1800)):
        g = scenes.random_gaussians(seed, W, H, n, radius_px=(1.0, 4.0))
        rd = _renderer(W, H, n, 16)
        res = rd.bin_sort(g, W, H)
        rd.sync_status()
        ptr, idx = oracle.pixel_lists(g, W, H)
        seen += _check_lists(g, W, H, 16, res["ranges"], res["keys"], ptr, idx, oracle.DEFAULTS["alpha_min"])
        rd.close()
    for lo, hi in ((32, 64), (64, 128), (128, 256), (256, 512)):
        assert any(lo < m <= hi for m in seen), (lo, hi, seen)


def test_bin_sort_mid_size_tiles(oracle, scenes):
    # tiles of 513..1024 and 1025..4096 keys (one block, bitonic network in
    # shared memory) in the same call
    W, H, n = 40, 36, 2000
    g = scenes.random_gaussians(7, W, H, n, radius_px=(2.0, 5.0))
    rd = _renderer(W, H, n, 32)
    res = rd.bin_sort(g, W, H)
    rd.sync_status()
    ptr, idx = oracle.pixel_lists(g, W, H)
    lengths = _check_lists(g, W, H, 32, res["ranges"], res["keys"], ptr, idx, oracle.DEFAULTS["alpha_min"])
    assert any(512 < m <= 1024 for m in lengths)
    assert any(1024 < m <= 4096 for m in lengths)


def test_bin_sort_empty_and_single(oracle, scenes):
    for n in (0, 1):
        W, H = 20, 10
        g = scenes.random_gaussians(3, W, H, max(n, 1))
        if n == 0:
            g = {k: v[:0] for k, v in g.items()}
        rd = _renderer(W, H, max(n, 1), 8)
        res = rd.bin_sort(g, W, H)
        rd.sync_status()
        ptr, idx = oracle.pixel_lists(g, W, H)
        _check_lists(g, W, H, 8, res["ranges"], res["keys"], ptr, idx, oracle.DEFAULTS["alpha_min"])


@pytest.mark.parametrize("tile", [8, 32])
def test_boundary_tile_lists(oracle, scenes, tile):
    from tests.gpu_util import gpu_forward
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.06)
    cam = cams[0]
    g = gpu_forward(sc, cams, tile=tile, stages=("b_ranges", "b_keys"))
    ref = oracle.render(sc, cam, records=True)
    bnd = ref["bnd"]
    W, H = cam["width"], cam["height"]
    tx = (W + tile - 1) // tile
    ranges, keys = g["b_ranges"], g["b_keys"]
    prim = (keys >> np.uint64(32)).astype(np.int64)
    bidx = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(prim, bnd[bidx, 1].astype(np.int64))
    for t in range(len(ranges) - 1):
        seg = keys[ranges[t]:ranges[t + 1]]
        assert np.all(seg[1:] > seg[:-1])
    ys, xs = np.mgrid[0:H, 0:W]
    for t in range(len(ranges) - 1):
        x0, y0 = (t % tx) * tile, (t // tx) * tile
        lst = set(bidx[ranges[t]:ranges[t + 1]].tolist())
        px = xs[y0:y0 + tile, x0:x0 + tile].ravel()
        py = ys[y0:y0 + tile, x0:x0 + tile].ravel()
        d = np.hypot(px[:, None] - bnd[None, :, 2], py[:, None] - bnd[None, :, 3])
        need = np.flatnonzero((d < bnd[None, :, 4]).any(0))
        assert set(need.tolist()) <= lst, f"tile {t} misses boundary points"
        for b in lst:  # validity: disc of radius sigma reaches the tile's box
            bx, by, s = bnd[b, 2], bnd[b, 3], bnd[b, 4]
            assert bx + s >= x0 - 0.01 and bx - s <= x0 + tile - 1 + 0.01
            assert by + s >= y0 - 0.01 and by - s <= y0 + tile - 1 + 0.01
    assert math.isfinite(float(len(keys)))
