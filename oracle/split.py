"""FP64 oracle of the geometric half of splitting and pruning (Sec. 3.3
"Splitting and Pruning"; implementation details of the same name):

  * the 1 -> 4 split of a degree-n BG-triangle at the midpoints of its edges,
    with the exact control points of each piece (the restriction of the
    Bezier triangle to a sub-triangle of its parameter domain);
  * the area estimate from four planar triangles and the bounding-box aspect
    ratio that the pruning criteria threshold (tau_a = 3e-4, tau_s = 10);
  * the average control-point gradient that the split criterion thresholds
    (tau_g = 0.0018);
  * the visibility measures of the other two pruning criteria: in how many
    training views a primitive owns pixels of I_id (tau_v = 0.08 of them)
    and how much of its visibility texture is seen (tau_r = 0.4);
  * the edge prior of the split criterion: edge magnitudes of the training
    images back-projected onto the primitives through I_id (tau_b = 13).

TEST INFRASTRUCTURE: imported only by tests/. The CUDA library never imports
it, and it shares no code with it.

Control points follow the order of Eq. 1: i = n..0, then j = n - i..0,
k = n - i - j, flat index (n - i)(n - i + 1) / 2 + k; corners p_n00, p_0n0,
p_00n sit at barycentric u, v, w = 1.

The pieces come from the polar form (blossom) of the patch: the piece with
corners A, B, C (barycentric points of the parent domain, in that order) has
control points q_ijk = f(A, .., A, B, .., B, C, .., C) with i, j, k copies,
f evaluated by de Casteljau's algorithm with a different parameter at each
level (Ramshaw's blossoming; Farin, "Curves and Surfaces for CAGD", ch. 17).

Readings (the paper is brief here):
  * pieces in the order (U corner, V corner, W corner, middle) with corners
    (U, M_uv, M_uw), (M_uv, V, M_vw), (M_uw, M_vw, W), (M_vw, M_uw, M_uv),
    M the edge midpoints; every piece keeps the parent's orientation;
  * per-primitive attributes (opacity, r_b, SH coefficients) are copied;
    rotation / scaling attribute maps of leg R > 1 are resampled: a piece's
    texel takes the parent map's Theta (Eq. 5 interpolation) at the texel's
    node mapped into the parent's domain;
  * area = sum of the areas of the four planar triangles through the
    corners and the surface points at the edge midpoints, in the split's
    pattern;
  * aspect ratio = longer / shorter side of the bounding rectangle of the
    control points in the plane of the three corners, its first axis along
    the longest corner edge (a flat sliver has a large ratio; a primitive
    whose corners are collinear has an infinite one);
  * average gradient = mean over the control points of |dL/dp_ijk|.
"""
import math

import numpy as np

TAU_G = 0.0018
TAU_A = 3e-4
TAU_S = 10.0

U, V, W = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)
M_UV, M_VW, M_UW = (0.5, 0.5, 0.0), (0.0, 0.5, 0.5), (0.5, 0.0, 0.5)
PIECES = ((U, M_UV, M_UW), (M_UV, V, M_VW), (M_UW, M_VW, W), (M_VW, M_UW, M_UV))


def ncp(n):
    return (n + 1) * (n + 2) // 2


def index(n, i, j):
    """Flat index of p_ijk (k = n - i - j) in the order of Eq. 1."""
    k = n - i - j
    return (n - i) * (n - i + 1) // 2 + k


def triples(n):
    """(i, j, k) in storage order."""
    out = []
    for i in range(n, -1, -1):
        for j in range(n - i, -1, -1):
            out.append((i, j, n - i - j))
    return out


def blossom(ctrl, n, params):
    """Polar form f(params[0], .., params[n-1]) of the patch with control
    points ctrl [Ncp, D]: level r replaces the degree-(n - r) net by the
    combination u b_(i+1)jk + v b_i(j+1)k + w b_ij(k+1) with (u, v, w) = params[r]."""
    ctrl = np.asarray(ctrl, np.float64)
    net = {(i, j, k): ctrl[index(n, i, j)] for (i, j, k) in triples(n)}
    for r in range(n):
        u, v, w = params[r]
        m = n - r - 1
        net = {(i, j, k): u * net[(i + 1, j, k)] + v * net[(i, j + 1, k)] + w * net[(i, j, k + 1)]
               for (i, j, k) in triples(m)}
    return net[(0, 0, 0)]


def evaluate(ctrl, n, uvw):
    """Surface point: the blossom with every argument equal to (u, v, w)."""
    return blossom(ctrl, n, [uvw] * n)


def subdivide(ctrl, n):
    """Control points of the four pieces, [4, Ncp, D]."""
    ctrl = np.asarray(ctrl, np.float64)
    out = np.zeros((4,) + ctrl.shape)
    for p, (A, B, C) in enumerate(PIECES):
        for (i, j, k) in triples(n):
            out[p, index(n, i, j)] = blossom(ctrl, n, [A] * i + [B] * j + [C] * k)
    return out


def piece_point(p, uvw):
    """Parent-domain barycentric point of a piece's (u, v, w)."""
    A, B, C = (np.array(x) for x in PIECES[p])
    u, v, w = uvw
    return u * A + v * B + w * C


def texel_nodes(R):
    """(u, v) of the texels of a leg-R map in storage order (control-point order)."""
    if R == 1:
        return [(1.0 / 3.0, 1.0 / 3.0)]
    n = R - 1
    return [(i / n, j / n) for (i, j, _) in triples(n)]


def subdivide_map(tex, R, attr_weights):
    """Texels of the four pieces' attribute maps [4, T, C] from the parent's
    [T, C]: Theta of the parent at each piece texel's node in the parent's
    domain. `attr_weights(R, u, v)` is the Eq. 5 interpolation."""
    tex = np.asarray(tex, np.float64)
    out = np.zeros((4,) + tex.shape)
    if R == 1:
        out[:] = tex
        return out
    for p in range(4):
        for t, (u, v) in enumerate(texel_nodes(R)):
            pu, pv, _ = piece_point(p, (u, v, 1.0 - u - v))
            idx, w = attr_weights(R, pu, pv)
            out[p, t] = (w[:, None] * tex[idx]).sum(axis=0)
    return out


def _tri_area(a, b, c):
    return 0.5 * float(np.linalg.norm(np.cross(b - a, c - a)))


def area(ctrl, n):
    """Area estimate: four planar triangles through the corners and the
    surface points at the edge midpoints."""
    pts = {name: evaluate(ctrl, n, x) for name, x in
           (("U", U), ("V", V), ("W", W), ("uv", M_UV), ("vw", M_VW), ("uw", M_UW))}
    return (_tri_area(pts["U"], pts["uv"], pts["uw"]) + _tri_area(pts["uv"], pts["V"], pts["vw"])
            + _tri_area(pts["uw"], pts["vw"], pts["W"]) + _tri_area(pts["vw"], pts["uw"], pts["uv"]))


def aspect(ctrl, n):
    """Bounding-rectangle aspect ratio in the corners' plane (>= 1, inf if
    the corners are collinear)."""
    ctrl = np.asarray(ctrl, np.float64)
    P = [ctrl[index(n, n, 0)], ctrl[index(n, 0, n)], ctrl[index(n, 0, 0)]]
    edges = [(P[0], P[1]), (P[1], P[2]), (P[2], P[0])]
    lens = [float(np.linalg.norm(b - a)) for a, b in edges]
    e = int(np.argmax(lens))
    a, b = edges[e]
    if lens[e] == 0.0:
        return math.inf
    x = (b - a) / lens[e]
    nrm = np.cross(P[1] - P[0], P[2] - P[0])
    nn = float(np.linalg.norm(nrm))
    if nn == 0.0:
        return math.inf
    y = np.cross(nrm / nn, x)
    px, py = (ctrl - a) @ x, (ctrl - a) @ y
    ex, ey = px.max() - px.min(), py.max() - py.min()
    lo, hi = min(ex, ey), max(ex, ey)
    return math.inf if lo == 0.0 else hi / lo


def avg_grad(g_ctrl):
    """Mean over the control points of |dL/dp|, g_ctrl [Ncp, 3]."""
    return float(np.linalg.norm(np.asarray(g_ctrl, np.float64), axis=1).mean())


def decisions(ctrl, n, g_ctrl=None, tau_a=TAU_A, tau_s=TAU_S, tau_g=TAU_G):
    """(prune, split) of one primitive from the geometric criteria and the
    control-point gradient."""
    prune = area(ctrl, n) < tau_a or aspect(ctrl, n) > tau_s
    split = g_ctrl is not None and avg_grad(g_ctrl) > tau_g
    return prune, split


TAU_V = 0.08
TAU_R = 0.4


def visibility(rasters, M, tess_level=8):
    """Visibility measures of the pruning criteria from the raster of each
    training view: rasters = [(I_id [H, W], key [H, W]), ...], key the depth
    key whose low 32 bits are prim * 2 L^2 + sub-triangle id.

    Readings: a primitive is visible in a view when it owns at least one
    pixel of I_id there (view_count = number of such views); its visibility
    texture has one cell per flat triangle of the level-L lattice (the L^2
    sub-triangles of the raster, id 2 (a L + b) + down), and a cell is
    visible when the primitive owns a pixel through that flat triangle in
    any view. Returns (view_count [M] int, cells: list of M sets of ids)."""
    L = tess_level
    nsub = 2 * L * L
    count = np.zeros(M, np.int64)
    cells = [set() for _ in range(M)]
    for idm, key in rasters:
        fg = idm >= 0
        ids = idm[fg].astype(np.int64)
        sub = (key[fg].astype(np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.int64) - ids * nsub
        for m in np.unique(ids):
            count[m] += 1
        for m, s in zip(ids.tolist(), sub.tolist()):
            cells[m].add(s)
    return count, cells


def occluded(view_count, n_views, cells, tess_level=8, tau_v=TAU_V, tau_r=TAU_R):
    """(seen in too few views, too little of the texture visible) per
    primitive: view_count / n_views < tau_v, |cells| / L^2 < tau_r."""
    L2 = tess_level * tess_level
    by_views = [n_views > 0 and c / n_views < tau_v for c in view_count]
    by_area = [len(s) / L2 < tau_r for s in cells]
    return by_views, by_area


TAU_B = 13.0
LUMA = (0.299, 0.587, 0.114)


def edge_magnitude(img):
    """Edge prior of the split criterion: the Sobel gradient magnitude of a
    training image's luma in 8-bit units. Readings (the paper names an edge
    detector, not which): luma 255 (0.299 R + 0.587 G + 0.114 B) of an
    [H, W, 3] image in [0, 1]; the unnormalised 3 x 3 Sobel pair
    Gx = [1 2 1]^T [-1 0 1], Gy its transpose, with the border replicated;
    magnitude sqrt(Gx^2 + Gy^2). Returns [H, W]."""
    img = np.asarray(img, np.float64)
    y = 255.0 * (LUMA[0] * img[..., 0] + LUMA[1] * img[..., 1] + LUMA[2] * img[..., 2])
    H, W = y.shape
    p = np.pad(y, 1, mode="edge")

    def at(dy, dx):
        return p[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]

    gx = (at(-1, 1) - at(-1, -1)) + 2 * (at(0, 1) - at(0, -1)) + (at(1, 1) - at(1, -1))
    gy = (at(1, -1) - at(-1, -1)) + 2 * (at(1, 0) - at(-1, 0)) + (at(1, 1) - at(-1, 1))
    return np.sqrt(gx * gx + gy * gy)


def edge_prior(ids, edges, M):
    """Edge values back-projected onto the primitives through I_id: per
    primitive the sum of the edge magnitudes of the pixels it owns and their
    count, over the views (ids, edges: lists of [H, W] arrays)."""
    s = np.zeros(M)
    n = np.zeros(M, np.int64)
    for idm, e in zip(ids, edges):
        fg = idm >= 0
        np.add.at(s, idm[fg], e[fg])
        np.add.at(n, idm[fg], 1)
    return s, n


def split_by_edges(edge_sum, edge_count, tau_b=TAU_B):
    """Split criterion of the edge prior: the accumulated average edge value
    of a primitive exceeds tau_b."""
    return [c > 0 and s / c > tau_b for s, c in zip(edge_sum, edge_count)]
