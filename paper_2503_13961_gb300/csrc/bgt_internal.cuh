// Internal declarations of the BG-Triangle CUDA library (sm_103a).
//
// Data layout in HBM (one call renders V views of mixed size):
//   pixels   the views' pixels concatenated in view order, row-major inside a
//            view; global pixel index p = view.pix_off + y * W + x.
//   tiles    t x t screen tiles, concatenated the same way (view.tile_off).
//   gaussians one per foreground pixel (Sec. 3.2, sub-primitive generation),
//            compacted in global pixel order; gaussian index = rank.
//   boundary  one point per pixel of B, compacted in global pixel order.
//   pairs    (tile, gaussian) and (tile, boundary point) pairs bucketed by
//            tile, then sorted inside each tile (see binning.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bgt {

constexpr int kMaxDegree = 4;
constexpr int kMaxCp = 15;
constexpr int kMaxTess = 16;
constexpr int kMaxViews = 4096;
constexpr int kGuardPx = 1 << 20;  // vertices beyond +-2^20 px cull their flat triangles

// status word bits (device-side errors, reported by bgt_sync_status)
constexpr int kStatusPairOverflow = 1;
constexpr int kStatusBoundaryOverflow = 2;
constexpr int kStatusTileOverflow = 4;
constexpr int kStatusNonFinite = 8;
constexpr int kStatusBadPrim = 16;
constexpr int kStatusBlendOverflow = 32;  // reserved (blend-record overflow falls back to a tile-list walk)

// blend records (forward -> backward): headers in chunks of kRecChunk per warp
// block, fill records in chunks of kFillChunk per warp
constexpr int kRecChunk = 32;
constexpr int kFillChunk = 8;

struct View {                 // one camera and its place in the batch (128 B)
  float R[9];                 // world -> camera rotation, row-major
  float t[3];
  float fx, fy, cx, cy;
  int W, H;
  int pix_off;                // first global pixel of the view
  int tile_off;               // first global tile of the view
  int tiles_x, tiles_y;
  int pad[10];
};
static_assert(sizeof(View) == 128, "View is 128 bytes");

struct Params {
  int n, ncp, M, L;
  float near_z, k_b, alpha_min, alpha_max, t_stop, dilation;
  float log_alpha_min;
  int use_boundary;
  int tile;                   // tile edge in pixels (8, 16 or 32)
  int V, P, tiles;            // views, total pixels, total tiles of this call
  float bg[3];
  long long max_pairs, max_bpairs;
  int stats;                  // 1: blending kernels count their work units into Work::stats
  int attr_res, ntex;         // attribute maps: leg resolution R, texels R (R + 1) / 2
  int sh_deg, sh_k;           // SH colour: degree D, coefficients per channel (D + 1)^2 - 1
  // scheduling (bgt_tuning): primitives per rasterizer warp and block, warp
  // blocks per backward dequeue, persistent blocks per SM of the chain kernels
  int raster_prims, bwd_dequeue, chain_bps;
};

struct Scene {                // device pointers, caller-owned
  const float *ctrl, *color, *opacity, *r_b, *log_scale, *quat;
  const float *sh;            // [M][K][3] SH coefficients of bands 1..D, or null
};

struct Grads {                // device pointers, caller-owned outputs
  float *ctrl, *color, *opacity, *r_b;
  float *log_scale, *quat;    // attribute-map texel gradients, nullable
  float *sh;                  // SH coefficient gradients, nullable
};

// Per-Gaussian gradient of the blending backward from the sums in Work::gg
// and the Gaussian's conic K = (a, b, c) and opacity o: out = (dl/dmu x, y,
// dl/dK a, b, c, dl/do, dl/dcolour r, g, b).
__device__ inline void gauss_grad_from_sums(const float *gs, float4 Ko, float *out) {
  const float o = Ko.w;
  out[0] = o * (Ko.x * gs[0] + Ko.y * gs[1]);
  out[1] = o * (Ko.y * gs[0] + Ko.z * gs[1]);
  out[2] = -0.5f * o * gs[2];
  out[3] = -o * gs[3];
  out[4] = -0.5f * o * gs[4];
  out[5] = gs[5];
  out[6] = gs[6];
  out[7] = gs[7];
  out[8] = gs[8];
}

// Gaussian record (one per foreground pixel), three float4 per Gaussian:
//   A = (off_x, off_y, bits(qx | qy << 16), support radius)
//        mean = pixel centre (qx, qy) + off; the support {o G >= alpha_min}
//        lies inside the square of this half-width around the mean
//   B = (K_a, K_b, K_c, opacity)   conic of the projected Gaussian
//   C = (r, g, b, bits(prim))
// Boundary record (one per pixel of B):
//   R = (bits(qx | qy << 16), off_x, off_y, 1 / sigma)
struct Work {
  const View *views;
  const int *view_pix_off;    // V + 1 entries
  const int *view_tile_off;   // V + 1 entries
  unsigned long long *zbuf;   // [P] depth key of the nearest flat triangle
  int *pid;                   // [P] I_id, -1 background
  unsigned long long *vis_seen;  // [M] views (bit v - v0) a primitive owns pixels in, for the visibility measures
  float2 *puv;                // [P] I_uv (u, v)
  int *pix_gidx;              // [P] gaussian index of a foreground pixel, else -1
  int *blk_cnt;               // [2][nblk] foreground / boundary pixels per warp chunk of 128 pixels
  long long *blk_off;         // [2][nblk + 1] their exclusive prefix sums (totals last)
  int *counters;              // [16] F, Nb, K, Kb, queue heads...
  int *status;                // [1]
  // per primitive
  // gaussians
  float4 *gA, *gB, *gC;       // [Fcap]
  int *g_pix;                 // [Fcap] global pixel index
  int *g_view;                // [Fcap]
  int *g_bidx;                // [Fcap] boundary point of the Gaussian's pixel, -1 if not in B
  int *g_prim;                // [Fcap] primitive of the Gaussian's pixel (I_id)
  float2 *g_uv;               // [Fcap]
  uint2 *g_rect;              // [Fcap] tile rect x0 | y0 << 16, x1 | y1 << 16 (view-local tiles)
  float *g_depth;             // [Fcap] camera depth (FP32)
  unsigned char *g_dsub;      // [Fcap] 5 extra depth-key bits (position of the exact depth
                              //        inside the rounding interval of its FP32 value)
  // boundary points
  float4 *bR;                 // [Fcap]
  int *b_pix, *b_prim, *b_view;
  float2 *b_uv;
  float *b_sigma, *b_z;
  uint2 *b_rect;
  // tiles
  int *g_tcount, *g_tfill;    // [tiles + 1] per-tile pair counts / fill cursors
  int *b_tcount, *b_tfill;
  long long *g_tstart, *b_tstart;  // [tiles + 1] exclusive prefix sums (64-bit: no wrap)
  long long *scan_aux, *scan_aux2; // scratch of the two tile-count (and chunk-count) scans
  int *big_list;              // [2 tiles] segments too long for one warp to sort
  int4 *tile_desc;            // [2 tiles] (view, x0 | y0 << 16, W | H << 16, view pixel offset),
                              // (Gaussian list start, length, boundary list start, length)
  // Blend records written by the forward pass for the backward pass. A fill
  // record is written when a warp's primitive cache takes in primitive g: per
  // pixel plane k and lane, the index of the pixel's most influential boundary
  // point of g in the tile's boundary list, or -1 (w follows from it). A
  // header is written per (warp visit of a listed Gaussian, plane k) with at
  // least one composited pixel: (Gaussian index, lane mask of the composited
  // pixels, first unit of the fill record of its primitive, k).
  uint4 *rec_hdr;             // [rec_chunk_cap * kRecChunk]
  int *rec_prev;              // [rec_chunk_cap] previous header chunk of the same warp block, -1
  int *rec_fill;              // [fill_unit_cap * 32] one unit = one plane of one fill record
  int2 *blk_rec;              // [warp blocks] last header chunk (-1 none, -2 overflow), records in it
  int *walk_list;             // [warp blocks] blocks whose records overflowed (counters[kWalkCount] of them):
                              // the backward re-walks their tile lists instead of replaying records
  int rec_chunk_cap, fill_unit_cap;
  // pairs
  unsigned long long *gkeys;  // [Kcap] depth key (FP32 bits << 5 | sub) << 27 | gaussian index
  unsigned long long *bkeys;  // [Kbcap] (prim << 32) | boundary index
  int *bl_prim;               // [Kbcap] prim of each sorted boundary entry
  float4 *bl_rec;             // [Kbcap] boundary record of each sorted entry
  // forward state for the backward pass
  float *T_final;             // [P]
  int *n_contrib;             // [P] tile-list position after the last composited pair
  // intermediate gradients
  float *prim_cov;            // [Mcap][6] Sigma3D per primitive (maps of leg resolution 1): xx xy xz yy yz zz
  float *prim_gcov;           // [Mcap][6] dl/dSigma3D per primitive, summed over its Gaussians (same order)
  float *gg;                  // [Fcap][12] per-Gaussian sums of the blending backward over its composited
                              // pairs, s = dl/dalpha w G of a pair, d = q - mu: s dx, s dy, s dx^2,
                              // s dx dy, s dy^2, s (= dl/do), dl/dcolour r, g, b; pad (dl/dmu = o K (s d),
                              // dl/dK = -o/2 (s dx^2, 2 s dx dy, s dy^2) are formed per Gaussian)
  float4 *bg_grad;            // [Fcap] (db x, db y, dsigma, 0)
  // per-primitive gradient records of the chain rule: each Gaussian's and
  // each boundary point's dl/dS (and the rest) in its primitive's segment
  int *prim_gcnt, *prim_bcnt;     // [Mcap] records per primitive, then fill counters
  long long *prim_gseg, *prim_bseg;  // [Mcap + 1] segment starts
  float4 *pg_rec;             // [Fcap][4] Gaussian: (dl/dS, dl/do), (dl/dc, u), (v, dl/dSigma3D xx xy xz), (yy yz zz, 0)
  float4 *pb_rec;             // [Fcap][2] boundary point: (dl/dS, dl/dr_b), (u, v, 0, 0)
  unsigned long long *stats;  // [8] work units of the last profiled call (see Stat)
  long long Fcap;
  int nblk;
};

// Work units counted by the blending kernels when Params::stats is set:
// pairs inside a Gaussian's support (o G >= alpha_min), pairs composited,
// boundary candidates scanned by the coefficient search; forward then backward.
enum Stat { kFwdSupport = 0, kFwdComposited = 1, kFwdCandidates = 2, kFwdVisits = 3, kBwdSupport = 4,
            kBwdComposited = 5, kBwdCandidates = 6, kBwdVisits = 7 };

constexpr int kIndexBits = 27;  // Gaussian index field of a pair key (<= 134M Gaussians per call)
constexpr unsigned long long kIndexMask = (1ull << kIndexBits) - 1ull;

enum Counter { kF = 0, kNb = 1, kK = 2, kKb = 3, kQueueFwd = 4, kQueueBwd = 5, kQueueSort = 6, kBigCount = 7,
               kRecChunks = 8, kFillChunks = 9, kWalkCount = 10, kQueueWalk = 11, kMidCount = 12 };

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__host__ __device__ inline int ncp_of(int n) { return (n + 1) * (n + 2) / 2; }

__device__ inline int find_view(const int *off, int V, int idx) {
  int lo = 0, hi = V;  // off[lo] <= idx < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= idx) lo = mid; else hi = mid;
  }
  return lo;
}

// n! / (i! j! k!) for n <= 4 (exact in FP32)
__host__ __device__ constexpr int factorial(int k) { return k <= 1 ? 1 : k * factorial(k - 1); }
__host__ __device__ constexpr float multinom(int n, int i, int j, int k) {
  return (float)(factorial(n) / (factorial(i) * factorial(j) * factorial(k)));
}

// Warp-segmented sums: lanes holding equal keys in a run of consecutive
// lanes form a segment; seg_sum leaves the segment's sum (inclusive scan) in
// its last lane (tail), so that one atomic per run replaces one per lane.
struct Seg {
  int start;
  bool tail;
};

__device__ inline Seg seg_info(int key) {
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const int next = __shfl_down_sync(0xffffffffu, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned upto = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
  Seg s;
  s.start = 31 - __clz(heads & upto);
  s.tail = lane == 31 || next != key;
  return s;
}

__device__ inline float seg_sum(float v, const Seg &s) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= s.start) v += y;
  }
  return v;
}

// Calls f(Degree<N>()) for the degree n (1..kMaxDegree), so that every loop
// over Bernstein terms is unrolled at compile time.
template <int N> struct Degree { static constexpr int value = N; };
template <class F>
inline void dispatch_degree(int n, F &&f) {
  switch (n) {
    case 1: f(Degree<1>()); break;
    case 2: f(Degree<2>()); break;
    case 3: f(Degree<3>()); break;
    default: f(Degree<4>()); break;
  }
}

// ---------------------------------------------------------------------------
// FP32 lattice vertex with one fixed sequence of IEEE-rounded operations.
// Coverage and the depth test are integer decisions taken from these values,
// so every operation is an explicit correctly rounded intrinsic (no
// contraction): Bernstein weights ((coef u^i) v^j) w^k, fused multiply-add
// accumulation in control-point order, world->camera rows as
// fma(r2, z, fma(r1, y, r0 * x)) + t, projection fma(f, X / Z, c), and a
// snap to the 1/256-pixel grid with round-to-nearest-even.
// ---------------------------------------------------------------------------
struct RVert {
  int X, Y;     // 1/256-pixel fixed point
  float Z, iz;  // camera depth and its reciprocal
  bool valid;
};

// lattice coordinate k / L, correctly rounded
__device__ inline float lattice_frac(int k, int L) { return __fdiv_rn((float)k, (float)L); }

template <int N>
__device__ inline RVert raster_vertex(const float *cp, float u, float vv, float w, const View &v, float near_z);

template <int N>
__device__ inline RVert raster_vertex(const float *cp, int a, int b, int L, const View &v, float near_z) {
  return raster_vertex<N>(cp, lattice_frac(a, L), lattice_frac(b, L), lattice_frac(L - a - b, L), v, near_z);
}

// Bernstein weights ((coef u^i) v^j) w^k of a lattice vertex, in control-point
// order, each product one IEEE rounding
template <int N>
__device__ inline void lattice_bernstein(float u, float vv, float w, float *B) {
  float pu[N + 1], pv[N + 1], pw[N + 1];
  pu[0] = pv[0] = pw[0] = 1.0f;
#pragma unroll
  for (int m = 1; m <= N; m++) {
    pu[m] = __fmul_rn(pu[m - 1], u);
    pv[m] = __fmul_rn(pv[m - 1], vv);
    pw[m] = __fmul_rn(pw[m - 1], w);
  }
  int idx = 0;
#pragma unroll
  for (int i = N; i >= 0; i--)
#pragma unroll
    for (int j = N - i; j >= 0; j--) {
      const int k = N - i - j;
      B[idx++] = __fmul_rn(__fmul_rn(__fmul_rn(multinom(N, i, j, k), pu[i]), pv[j]), pw[k]);
    }
}

// The vertex of Bernstein weights B (lattice_bernstein) of control points
// cp[Ncp][3]: fused multiply-add accumulation in control-point order, camera
// transform, projection and snap. cp may point to registers or memory.
template <int N>
__device__ inline RVert vertex_from_weights(const float *B, const float *cp, const View &v, float near_z) {
  RVert o;
  float Sx = 0.f, Sy = 0.f, Sz = 0.f;
#pragma unroll
  for (int idx = 0; idx < (N + 1) * (N + 2) / 2; idx++) {
    Sx = __fmaf_rn(B[idx], cp[3 * idx + 0], Sx);
    Sy = __fmaf_rn(B[idx], cp[3 * idx + 1], Sy);
    Sz = __fmaf_rn(B[idx], cp[3 * idx + 2], Sz);
  }
  float Xc = __fmul_rn(v.R[0], Sx); Xc = __fmaf_rn(v.R[1], Sy, Xc); Xc = __fmaf_rn(v.R[2], Sz, Xc); Xc = __fadd_rn(Xc, v.t[0]);
  float Yc = __fmul_rn(v.R[3], Sx); Yc = __fmaf_rn(v.R[4], Sy, Yc); Yc = __fmaf_rn(v.R[5], Sz, Yc); Yc = __fadd_rn(Yc, v.t[1]);
  float Zc = __fmul_rn(v.R[6], Sx); Zc = __fmaf_rn(v.R[7], Sy, Zc); Zc = __fmaf_rn(v.R[8], Sz, Zc); Zc = __fadd_rn(Zc, v.t[2]);
  o.valid = (Zc >= near_z);
  o.Z = Zc;
  o.iz = __fdiv_rn(1.0f, Zc);
  const float x = __fmaf_rn(v.fx, __fmul_rn(Xc, o.iz), v.cx);
  const float y = __fmaf_rn(v.fy, __fmul_rn(Yc, o.iz), v.cy);
  if (!(fabsf(x) <= (float)kGuardPx && fabsf(y) <= (float)kGuardPx)) o.valid = false;
  if (o.valid) {
    o.X = __float2int_rn(__fmul_rn(x, 256.0f));
    o.Y = __float2int_rn(__fmul_rn(y, 256.0f));
  } else {
    o.X = o.Y = 0;
  }
  return o;
}

// vertex at barycentric (u, vv, w) = (a, b, L - a - b) / L
template <int N>
__device__ inline RVert raster_vertex(const float *cp, float u, float vv, float w, const View &v, float near_z) {
  float B[(N + 1) * (N + 2) / 2];
  lattice_bernstein<N>(u, vv, w, B);
  float c[3 * (N + 1) * (N + 2) / 2];
#pragma unroll
  for (int k = 0; k < 3 * (N + 1) * (N + 2) / 2; k++) c[k] = __ldg(cp + k);
  return vertex_from_weights<N>(B, c, v, near_z);
}

// exact edge function (b - a) x (P - a) on the fixed-point grid
__device__ inline long long edge_fn(int ax, int ay, int bx, int by, int px, int py) {
  return (long long)(bx - ax) * (long long)(py - ay) - (long long)(by - ay) * (long long)(px - ax);
}

// fill rule: a zero edge function counts as inside on edges with dy < 0 or (dy == 0, dx > 0)
__device__ inline bool owns_zero_edge(int ax, int ay, int bx, int by) {
  const int dx = bx - ax, dy = by - ay;
  return (dy < 0) || (dy == 0 && dx > 0);
}

// sub-triangle s = 2 (a L + b) + down of the level-L lattice
__device__ inline void subtri_verts(int L, int s, int *va, int *vb) {
  const int down = s & 1, cell = s >> 1;
  const int a = cell / L, b = cell - a * L;
  if (!down) {
    va[0] = a; vb[0] = b; va[1] = a + 1; vb[1] = b; va[2] = a; vb[2] = b + 1;
  } else {
    va[0] = a + 1; vb[0] = b; va[1] = a + 1; vb[1] = b + 1; va[2] = a; vb[2] = b + 1;
  }
}

// ---------------------------------------------------------------------------
// Attribute maps (Sec. 3.2, Eq. 5): per primitive T = R (R + 1) / 2 texels at
// the nodes (i, j), i + j <= R - 1, of the level-(R - 1) barycentric lattice,
// in control-point order; Theta interpolates linearly on the lattice triangle
// holding (u, v). Rotation maps hold raw quaternions (w, x, y, z), normalised
// after interpolation; scaling maps hold log scales.
// ---------------------------------------------------------------------------
__device__ inline int tex_index(int R, int i, int j) {
  const int n = R - 1;
  return (n - i) * (n - i + 1) / 2 + (n - i - j);
}

__device__ inline void attr_weights(int R, float u, float v, int *idx, float *w) {
  const int n = R - 1;
  if (n <= 0) {
    idx[0] = idx[1] = idx[2] = 0;
    w[0] = 1.f;
    w[1] = w[2] = 0.f;
    return;
  }
  const float x = u * (float)n, y = v * (float)n;
  int a = (int)floorf(x), b = (int)floorf(y);
  a = max(0, min(a, n - 1));
  b = max(0, min(b, n - 1));
  if (a + b > n - 1) a = n - 1 - b;
  const float fx = x - (float)a, fy = y - (float)b;
  if (fx + fy <= 1.f) {
    idx[0] = tex_index(R, a, b);     w[0] = 1.f - fx - fy;
    idx[1] = tex_index(R, a + 1, b); w[1] = fx;
    idx[2] = tex_index(R, a, b + 1); w[2] = fy;
  } else {
    idx[0] = tex_index(R, a + 1, b + 1); w[0] = fx + fy - 1.f;
    idx[1] = tex_index(R, a + 1, b);     w[1] = 1.f - fy;
    idx[2] = tex_index(R, a, b + 1);     w[2] = 1.f - fx;
  }
}

// interpolated raw quaternion and log scales of the Gaussian of primitive g at (u, v)
__device__ inline void gauss_attrs(const float *quat, const float *log_scale, int R, int T, int g, float u, float v,
                                   float *q, float *ls, int *tex, float *tw) {
  attr_weights(R, u, v, tex, tw);
  q[0] = q[1] = q[2] = q[3] = 0.f;
  ls[0] = ls[1] = ls[2] = 0.f;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    if (tw[e] == 0.f) continue;
    const size_t t = (size_t)g * T + tex[e];
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = fmaf(tw[e], __ldg(quat + 4 * t + k), q[k]);
#pragma unroll
    for (int k = 0; k < 3; k++) ls[k] = fmaf(tw[e], __ldg(log_scale + 3 * t + k), ls[k]);
  }
}

// Sigma3D = (R(q) S)(R(q) S)^T, S = diag(exp(ls)): upper triangle (xx, xy, xz,
// yy, yz, zz); Rm and sc receive R(q / |q|) and exp(ls)
__device__ inline void cov3d_f32(const float *q, const float *ls, float *S6, float *Rm, float *sc) {
  const float nq = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const float r = q[0] * nq, x = q[1] * nq, y = q[2] * nq, z = q[3] * nq;
  Rm[0] = 1.f - 2.f * (y * y + z * z); Rm[1] = 2.f * (x * y - r * z);       Rm[2] = 2.f * (x * z + r * y);
  Rm[3] = 2.f * (x * y + r * z);       Rm[4] = 1.f - 2.f * (x * x + z * z); Rm[5] = 2.f * (y * z - r * x);
  Rm[6] = 2.f * (x * z - r * y);       Rm[7] = 2.f * (y * z + r * x);       Rm[8] = 1.f - 2.f * (x * x + y * y);
  sc[0] = expf(ls[0]);
  sc[1] = expf(ls[1]);
  sc[2] = expf(ls[2]);
  float Mx[9];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) Mx[3 * i + j] = Rm[3 * i + j] * sc[j];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = i; j < 3; j++) S6[k++] = Mx[3 * i] * Mx[3 * j] + Mx[3 * i + 1] * Mx[3 * j + 1] + Mx[3 * i + 2] * Mx[3 * j + 2];
}

// dl/d(log scales) and dl/d(raw quaternion) of Sigma3D = M M^T, M = R(q / |q|)
// diag(exp(ls)), from G3 = dl/dSigma3D (symmetric, row-major 3 x 3), with
// Rm = R(q / |q|) and sc = exp(ls) of cov3d_f32: dl/dM = 2 G3 M,
// dl/dls_c = exp(ls_c) sum_r dM_rc R_rc, dl/dR_rc = dM_rc exp(ls_c), then
// through the normalisation of q
__device__ inline void cov_grad_to_attrs(const float *qa, const float *G3, const float *Rm, const float *sc3,
                                         float *gls, float *gq) {
  float GR[9];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float ds = 0.f;
#pragma unroll
    for (int r = 0; r < 3; r++) {
      float dm = 0.f;
#pragma unroll
      for (int k = 0; k < 3; k++) dm += 2.f * G3[3 * r + k] * Rm[3 * k + c] * sc3[c];
      GR[3 * r + c] = dm * sc3[c];
      ds += dm * Rm[3 * r + c];
    }
    gls[c] = ds * sc3[c];
  }
  const float nq = rsqrtf(qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3]);
  const float r = qa[0] * nq, x = qa[1] * nq, y = qa[2] * nq, z = qa[3] * nq;
  float h[4];
  h[0] = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
  h[1] = 2.f * (-2.f * x * GR[4] + y * GR[1] + z * GR[2] + y * GR[3] - r * GR[5] + z * GR[6] + r * GR[7] -
                2.f * x * GR[8]);
  h[2] = 2.f * (-2.f * y * GR[0] + x * GR[1] + r * GR[2] + x * GR[3] + z * GR[5] - r * GR[6] + z * GR[7] -
                2.f * y * GR[8]);
  h[3] = 2.f * (-2.f * z * GR[0] - r * GR[1] + x * GR[2] + r * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] +
                y * GR[7]);
  const float dot = r * h[0] + x * h[1] + y * h[2] + z * h[3];
  gq[0] = (h[0] - r * dot) * nq;
  gq[1] = (h[1] - x * dot) * nq;
  gq[2] = (h[2] - y * dot) * nq;
  gq[3] = (h[3] - z * dot) * nq;
}

// ---------------------------------------------------------------------------
// View-dependent colour: real spherical harmonics of bands 1..D (D <= 3) at a
// unit direction (x, y, z), in the Cartesian forms that the associated
// Legendre definition (Condon-Shortley phase) gives on the unit sphere, order
// m = -l..l within a band; constants sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) times
// the Legendre factors, as noted.
// ---------------------------------------------------------------------------
__device__ inline void sh_eval(int D, float x, float y, float z, float *Y) {
  const float c1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
  const float c2a = 1.09254843059207907f;  // sqrt(15 / (4 pi))
  const float c2b = 0.31539156525252005f;  // sqrt(5 / (16 pi))
  const float c2c = 0.54627421529603959f;  // sqrt(15 / (16 pi))
  const float c3a = 0.59004358992664352f;  // sqrt(35 / (32 pi))
  const float c3b = 2.89061144264055405f;  // sqrt(105 / (4 pi))
  const float c3c = 0.45704579946446574f;  // sqrt(21 / (32 pi))
  const float c3d = 0.37317633259011540f;  // sqrt(7 / (16 pi))
  const float c3e = 1.44530572132027703f;  // sqrt(105 / (16 pi))
  Y[0] = -c1 * y; Y[1] = c1 * z; Y[2] = -c1 * x;
  if (D < 2) return;
  Y[3] = c2a * x * y; Y[4] = -c2a * y * z; Y[5] = c2b * (3.f * z * z - 1.f); Y[6] = -c2a * x * z;
  Y[7] = c2c * (x * x - y * y);
  if (D < 3) return;
  Y[8] = -c3a * y * (3.f * x * x - y * y); Y[9] = c3b * x * y * z; Y[10] = -c3c * y * (5.f * z * z - 1.f);
  Y[11] = c3d * z * (5.f * z * z - 3.f); Y[12] = -c3c * x * (5.f * z * z - 1.f); Y[13] = c3e * z * (x * x - y * y);
  Y[14] = -c3a * x * (x * x - 3.f * y * y);
}

// g = sum_k w_k grad P_k(x, y, z) of the Cartesian forms above
__device__ inline void sh_grad(int D, float x, float y, float z, const float *w, float *g) {
  const float c1 = 0.48860251190291992f, c2a = 1.09254843059207907f, c2b = 0.31539156525252005f;
  const float c2c = 0.54627421529603959f, c3a = 0.59004358992664352f, c3b = 2.89061144264055405f;
  const float c3c = 0.45704579946446574f, c3d = 0.37317633259011540f, c3e = 1.44530572132027703f;
  g[0] = -c1 * w[2];
  g[1] = -c1 * w[0];
  g[2] = c1 * w[1];
  if (D < 2) return;
  g[0] += c2a * y * w[3] - c2a * z * w[6] + 2.f * c2c * x * w[7];
  g[1] += c2a * x * w[3] - c2a * z * w[4] - 2.f * c2c * y * w[7];
  g[2] += -c2a * y * w[4] + 6.f * c2b * z * w[5] - c2a * x * w[6];
  if (D < 3) return;
  g[0] += -6.f * c3a * x * y * w[8] + c3b * y * z * w[9] - c3c * (5.f * z * z - 1.f) * w[12] +
          2.f * c3e * x * z * w[13] - 3.f * c3a * (x * x - y * y) * w[14];
  g[1] += -3.f * c3a * (x * x - y * y) * w[8] + c3b * x * z * w[9] - c3c * (5.f * z * z - 1.f) * w[10] -
          2.f * c3e * y * z * w[13] + 6.f * c3a * x * y * w[14];
  g[2] += c3b * x * y * w[9] - 10.f * c3c * y * z * w[10] + c3d * (15.f * z * z - 3.f) * w[11] -
          10.f * c3c * x * z * w[12] + c3e * (x * x - y * y) * w[13];
}

// ---------------------------------------------------------------------------
// double-float arithmetic (Dekker 1971 / Knuth TAOCP vol. 2, 4.2.2): a value
// is hi + lo with |lo| <= ulp(hi) / 2. Used to place Gaussian means and
// boundary points to ~1e-12 px before storing them relative to their pixel.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ inline df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ inline df df_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ inline df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ inline df df_add(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  const df t = df_two_sum(a.lo, b.lo);
  df r = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_fast_two_sum(r.hi, __fadd_rn(r.lo, t.lo));
}
__device__ inline df df_add_f(df a, float b) {
  const df s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ inline df df_mul_f(df a, float b) {
  const df p = df_two_prod(a.hi, b);
  return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ inline df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = df_add(a, df_mul_f(b, -q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df_fast_two_sum(q1, q2);
}

// Surface point S(u, v) of Eq. 1 and its camera-space position, accurate to
// a few 1e-9 world units: S = p_ref + sum_ijk B_ijk (p_ijk - p_ref) (the
// weights sum to one), p_ref = first control point; the camera transform of
// p_ref is taken in double-float.
template <int N>
struct SurfPoint {
  static constexpr int M = (N + 1) * (N + 2) / 2;
  df t[3];        // camera-space position
  float S[3];     // world position (FP32, for derivatives)
  float B[M];
};

template <int N>
__device__ inline void bernstein_f32(float u, float v, float *B) {
  const float w = 1.0f - u - v;
  float pu[N + 1], pv[N + 1], pw[N + 1];
  pu[0] = pv[0] = pw[0] = 1.0f;
#pragma unroll
  for (int m = 1; m <= N; m++) {
    pu[m] = pu[m - 1] * u;
    pv[m] = pv[m - 1] * v;
    pw[m] = pw[m - 1] * w;
  }
  int idx = 0;
#pragma unroll
  for (int i = N; i >= 0; i--)
#pragma unroll
    for (int j = N - i; j >= 0; j--) {
      const int k = N - i - j;
      B[idx++] = multinom(N, i, j, k) * pu[i] * pv[j] * pw[k];
    }
}

template <int N>
__device__ inline void surface_point(const float *__restrict__ cp, float u, float v, const View &vw,
                                     SurfPoint<N> &sp) {
  constexpr int m = SurfPoint<N>::M;
  bernstein_f32<N>(u, v, sp.B);
  const float r0 = __ldg(cp + 0), r1 = __ldg(cp + 1), r2 = __ldg(cp + 2);
  float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
  for (int a = 1; a < m; a++) {
    d0 = fmaf(sp.B[a], __ldg(cp + 3 * a + 0) - r0, d0);
    d1 = fmaf(sp.B[a], __ldg(cp + 3 * a + 1) - r1, d1);
    d2 = fmaf(sp.B[a], __ldg(cp + 3 * a + 2) - r2, d2);
  }
  sp.S[0] = r0 + d0;
  sp.S[1] = r1 + d1;
  sp.S[2] = r2 + d2;
#pragma unroll
  for (int r = 0; r < 3; r++) {
    df acc = df_two_prod(vw.R[3 * r + 0], r0);
    acc = df_add(acc, df_two_prod(vw.R[3 * r + 1], r1));
    acc = df_add(acc, df_two_prod(vw.R[3 * r + 2], r2));
    acc = df_add_f(acc, vw.t[r]);
    const float delta = vw.R[3 * r + 0] * d0 + vw.R[3 * r + 1] * d1 + vw.R[3 * r + 2] * d2;
    sp.t[r] = df_add_f(acc, delta);
  }
}

// projected position of a camera-space point relative to pixel centre (qx, qy)
__device__ inline float2 project_offset(const df *t, const View &vw, int qx, int qy) {
  const df xz = df_div(t[0], t[2]);
  const df yz = df_div(t[1], t[2]);
  df mx = df_add_f(df_mul_f(xz, vw.fx), vw.cx);
  df my = df_add_f(df_mul_f(yz, vw.fy), vw.cy);
  mx = df_add_f(mx, -(float)qx);
  my = df_add_f(my, -(float)qy);
  return make_float2(mx.hi + mx.lo, my.hi + my.lo);
}

// ---------------------------------------------------------------------------
// Support box of a projected Gaussian given by its conic K = Sigma2D^-1 and
// opacity o, for the binning stage run on its own (bgt_bin_sort and its
// allocation-free variant, which must agree bit for bit): the support
// {o G >= alpha_min} lies inside |dx| <= sqrt(lvl Sigma_xx), |dy| <= sqrt(lvl
// Sigma_yy), lvl = 2 ln(o / alpha_min), widened slightly, clipped to the W x H
// view; rect = tile rect (x0 | y0 << 16, x1 | y1 << 16) at tile size t, empty
// as x0 = 1 > x1 = 0; r = the box's larger half-width, or -1 when empty.
// ---------------------------------------------------------------------------
struct ConicBox {
  uint2 rect;
  float r;
};

__device__ inline ConicBox conic_support_box(float Ka, float Kb, float Kc, float o, float cx, float cy, int W,
                                             int H, int t, float alpha_min, float log_alpha_min) {
  ConicBox b;
  b.rect = make_uint2(1u, 0u);
  b.r = -1.0f;
  const float det = Ka * Kc - Kb * Kb;
  if (!(o > alpha_min && det > 0.f)) return b;
  const float lvl = 2.0f * (logf(o) - log_alpha_min);
  const float rx = sqrtf(lvl * Kc / det) * 1.0001f + 1e-3f;
  const float ry = sqrtf(lvl * Ka / det) * 1.0001f + 1e-3f;
  int x0 = (int)ceilf(cx - rx), x1 = (int)floorf(cx + rx), y0 = (int)ceilf(cy - ry), y1 = (int)floorf(cy + ry);
  x0 = max(x0, 0); y0 = max(y0, 0); x1 = min(x1, W - 1); y1 = min(y1, H - 1);
  if (x0 > x1 || y0 > y1) return b;
  x0 /= t; x1 /= t; y0 /= t; y1 /= t;
  b.rect = make_uint2((unsigned)x0 | ((unsigned)y0 << 16), (unsigned)x1 | ((unsigned)y1 << 16));
  b.r = fmaxf(rx, ry);
  return b;
}

// depth key of a Gaussian given only its FP32 depth: the exact depth is the
// FP32 value itself, the middle (16) of the 32 finer sub-steps
__device__ inline unsigned long long plain_depth_key(float depth) {
  return ((unsigned long long)__float_as_uint(depth) << 5) | 16ull;
}

// ---------------------------------------------------------------------------
// host-side launchers (one per kernel family)
// ---------------------------------------------------------------------------
// host-side launchers; each returns the number of kernels it enqueued
int launch_raster(const Params &p, const Scene &s, const Work &w, cudaStream_t st);
int launch_resolve(const Params &p, const Scene &s, const Work &w, cudaStream_t st);
int launch_generate(const Params &p, const Scene &s, const Work &w, cudaStream_t st);
int launch_binning(const Params &p, const Work &w, cudaStream_t st);
cudaError_t configure_composite();  // opt the blending kernels into > 48 KB shared memory
cudaError_t configure_binning();    // the same for the per-tile sort
int launch_composite_fwd(const Params &p, const Work &w, float *image, cudaStream_t st);
int launch_composite_bwd(const Params &p, const Work &w, const float *dimage, cudaStream_t st);
int launch_chain(const Params &p, const Scene &s, const Work &w, const Grads &g, cudaStream_t st);
int launch_prim_cov(const Params &p, const Scene &s, const Work &w, cudaStream_t st);
int launch_l1_grad(const float *img, const float *target, long long n, float scale, float *dimg,
                   float *loss, cudaStream_t st);
int launch_l2_dssim_grad(const float *img, const float *gt, int n_views, const int *sizes, float lambda,
                         float scale, float *dimg, float *loss, cudaStream_t st);
int launch_prim_metrics(int degree, const float *ctrl, int M, const float *g_ctrl, float tau_a, float tau_s,
                        float tau_g, const float *edge_sum, const int *edge_count, float tau_b,
                        const int *view_count, int n_views, const unsigned long long *cell_mask, int tess_level,
                        float tau_v, float tau_r, float *area, float *aspect, float *grad, unsigned char *flags,
                        cudaStream_t st);
int launch_edge_magnitude(const float *img, int n_views, const int *sizes, float *edges, cudaStream_t st);
int launch_edge_prior(const Params &p, const Work &w, const float *edges, float *edge_sum, int *edge_count,
                      cudaStream_t st);
int launch_visibility(const Params &p, const Work &w, const int *view_off, int *view_count,
                      unsigned long long *cell_mask, cudaStream_t st);
int launch_exclusive_scan(const int *in, long long *out, int n, long long *aux, cudaStream_t st);
int launch_bin_sort_only(const Params &p, const Work &w, cudaStream_t st);

}  // namespace bgt
