// Splitting and pruning (Sec. 3.3 "Splitting and Pruning"): the
// per-primitive area / aspect / gradient measures that the criteria
// threshold, the visibility measures (views in which a primitive owns pixels
// of I_id, and its visibility texture: the flat triangles of its lattice it
// is seen through) gathered from a forward's raster, and the exact 1 -> 4
// midpoint subdivision of the selected primitives.
//
// A piece of the split is the parent patch restricted to a sub-triangle
// (A, B, C) of its parameter domain; its control point q_ijk is the polar
// form of the parent at (A x i, B x j, C x k), evaluated by de Casteljau's
// algorithm with parameter A at the first i levels, B at the next j and C at
// the last k. The corners of the four pieces (U, V, W corner, middle) are
// (U, M_uv, M_uw), (M_uv, V, M_vw), (M_uw, M_vw, W), (M_vw, M_uw, M_uv), M
// the edge midpoints, so every weight is 0, 1/2 or 1.
#include <cmath>

#include <cuda/atomic>

#include "../../include/bgt.h"
#include "bgt_internal.cuh"

namespace bgt {
namespace {

// piece p, corner c (u-, v-, w-corner of the piece) -> parent barycentrics x 2
__constant__ signed char c_piece[4][3][3] = {
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}},
    {{1, 1, 0}, {0, 2, 0}, {0, 1, 1}},
    {{1, 0, 1}, {0, 1, 1}, {0, 0, 2}},
    {{0, 1, 1}, {1, 0, 1}, {1, 1, 0}},
};

// control point with a = n - i, b = k sits at a (a + 1) / 2 + b
__host__ __device__ constexpr int slot(int a, int b) { return a * (a + 1) / 2 + b; }
template <int N> constexpr int kNcp = (N + 1) * (N + 2) / 2;

struct SplitArgs {
  const float *ctrl, *color, *opacity, *r_b, *log_scale, *quat, *sh;
  int M, R, T, K;  // primitives, map leg, texels, SH coefficients per channel
  const int *sel;
  int n_sel;
  bgt_prims out;
};

// de Casteljau with one parameter per level, in place: at level r the
// degree-(d + 1) net becomes the degree-d net, slot(a, b) <- u net[slot(a, b)]
// + v net[slot(a + 1, b)] + w net[slot(a + 1, b + 1)]; ascending slots only
// overwrite values no later slot reads.
template <int N, int C>
__device__ __forceinline__ void blossom(float (&net)[kNcp<N>][C], const float (&par)[N][3]) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int d = N - 1 - r;
    const float u = par[r][0], v = par[r][1], w = par[r][2];
#pragma unroll
    for (int a = 0; a <= d; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b)
#pragma unroll
        for (int ch = 0; ch < C; ++ch)
          net[slot(a, b)][ch] = u * net[slot(a, b)][ch] + v * net[slot(a + 1, b)][ch] +
                                w * net[slot(a + 1, b + 1)][ch];
  }
}

// one thread per (selected primitive, piece, control point or texel)
template <int N>
__global__ void __launch_bounds__(256) k_subdivide(const SplitArgs s) {
  constexpr int NC = kNcp<N>;
  const int per = max(NC, s.T);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 4LL * s.n_sel * per) return;
  const int e = (int)(gid % per);
  const long long sp = gid / per;
  const int piece = (int)(sp & 3);
  const long long child = sp;  // output primitive 4 sel_index + piece
  const int m = __ldg(s.sel + (sp >> 2));
  const bool valid = m >= 0 && m < s.M;

  if (e < NC) {
    // target control point q_ijk, a = n - i, b = k
    int a = 0;
    while (slot(a + 1, 0) <= e) ++a;
    const int b = e - slot(a, 0);
    const int i = N - a, k = b, j = N - i - k;
    float par[N][3];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const int corner = r < i ? 0 : (r < i + j ? 1 : 2);
#pragma unroll
      for (int c = 0; c < 3; ++c) par[r][c] = 0.5f * (float)c_piece[piece][corner][c];
    }
    float net[NC][6];
#pragma unroll
    for (int t = 0; t < NC; ++t)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        net[t][c] = valid ? __ldg(s.ctrl + ((size_t)m * NC + t) * 3 + c) : __int_as_float(0x7fc00000);
        net[t][3 + c] = valid ? __ldg(s.color + ((size_t)m * NC + t) * 3 + c) : __int_as_float(0x7fc00000);
      }
    blossom<N, 6>(net, par);
    const size_t o = ((size_t)child * NC + e) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s.out.ctrl[o + c] = net[0][c];
      s.out.color[o + c] = net[0][3 + c];
    }
  }

  if (e < s.T) {
    // texel (ti, tj) of the piece's maps: the parent's Theta at its node
    float lsv[3], qv[4];
    if (!valid) {
      for (int c = 0; c < 3; ++c) lsv[c] = __int_as_float(0x7fc00000);
      for (int c = 0; c < 4; ++c) qv[c] = __int_as_float(0x7fc00000);
    } else if (s.R <= 1) {
      for (int c = 0; c < 3; ++c) lsv[c] = __ldg(s.log_scale + (size_t)m * 3 + c);
      for (int c = 0; c < 4; ++c) qv[c] = __ldg(s.quat + (size_t)m * 4 + c);
    } else {
      const int n = s.R - 1;
      int a = 0;
      while (slot(a + 1, 0) <= e) ++a;
      const int b = e - slot(a, 0);
      const float nu = (float)(n - a) / (float)n, nv = (float)(a - b) / (float)n;
      const float nw = 1.f - nu - nv;
      float pu = 0.f, pv = 0.f;
#pragma unroll
      for (int corner = 0; corner < 3; ++corner) {
        const float wc = corner == 0 ? nu : (corner == 1 ? nv : nw);
        pu += wc * 0.5f * (float)c_piece[piece][corner][0];
        pv += wc * 0.5f * (float)c_piece[piece][corner][1];
      }
      int idx[3];
      float w[3];
      attr_weights(s.R, pu, pv, idx, w);
      for (int c = 0; c < 3; ++c) lsv[c] = 0.f;
      for (int c = 0; c < 4; ++c) qv[c] = 0.f;
      for (int t = 0; t < 3; ++t) {
        const size_t base = (size_t)m * s.T + idx[t];
        for (int c = 0; c < 3; ++c) lsv[c] = fmaf(w[t], __ldg(s.log_scale + base * 3 + c), lsv[c]);
        for (int c = 0; c < 4; ++c) qv[c] = fmaf(w[t], __ldg(s.quat + base * 4 + c), qv[c]);
      }
    }
    const size_t o = (size_t)child * s.T + e;
    for (int c = 0; c < 3; ++c) s.out.log_scale[o * 3 + c] = lsv[c];
    for (int c = 0; c < 4; ++c) s.out.quat[o * 4 + c] = qv[c];
  }

  if (e == 0) {
    const float nanv = __int_as_float(0x7fc00000);
    s.out.opacity[child] = valid ? __ldg(s.opacity + m) : nanv;
    s.out.r_b[child] = valid ? __ldg(s.r_b + m) : nanv;
    for (int c = 0; c < 3 * s.K; ++c)
      s.out.sh[(size_t)child * 3 * s.K + c] = valid ? __ldg(s.sh + (size_t)m * 3 * s.K + c) : nanv;
  }
}

struct MetricArgs {
  const float *ctrl, *g_ctrl;
  int M;
  float tau_a, tau_s, tau_g;
  const float *edge_sum;
  const int *edge_count;
  float tau_b;
  const int *view_count;
  int n_views;
  const unsigned long long *cell_mask;
  int words, cells;  // mask words per primitive, lattice cells L^2
  float tau_v, tau_r;
  float *area, *aspect, *grad;
  unsigned char *flags;
};

__device__ __forceinline__ float tri_area(const float3 &a, const float3 &b, const float3 &c) {
  const float3 e1 = make_float3(b.x - a.x, b.y - a.y, b.z - a.z);
  const float3 e2 = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
  const float cx = e1.y * e2.z - e1.z * e2.y, cy = e1.z * e2.x - e1.x * e2.z, cz = e1.x * e2.y - e1.y * e2.x;
  return 0.5f * sqrtf(cx * cx + cy * cy + cz * cz);
}

// one thread per primitive
template <int N>
__global__ void __launch_bounds__(256) k_prim_metrics(const MetricArgs s) {
  constexpr int NC = kNcp<N>;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= s.M) return;
  float3 p[NC];
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    const float *q = s.ctrl + ((size_t)m * NC + t) * 3;
    p[t] = make_float3(__ldg(q), __ldg(q + 1), __ldg(q + 2));
  }
  // corners p_n00, p_0n0, p_00n and the surface points at the edge
  // midpoints: binomial weights 2^-n C(n, .) along each edge
  const float3 U = p[slot(0, 0)], V = p[slot(N, 0)], W = p[slot(N, N)];
  float3 muv = make_float3(0.f, 0.f, 0.f), muw = muv, mvw = muv;
#pragma unroll
  for (int a = 0; a <= N; ++a) {
    const float wgt = (float)(factorial(N) / (factorial(a) * factorial(N - a))) / (float)(1 << N);
    const float3 e_uv = p[slot(a, 0)], e_uw = p[slot(a, a)], e_vw = p[slot(N, a)];
    muv = make_float3(fmaf(wgt, e_uv.x, muv.x), fmaf(wgt, e_uv.y, muv.y), fmaf(wgt, e_uv.z, muv.z));
    muw = make_float3(fmaf(wgt, e_uw.x, muw.x), fmaf(wgt, e_uw.y, muw.y), fmaf(wgt, e_uw.z, muw.z));
    mvw = make_float3(fmaf(wgt, e_vw.x, mvw.x), fmaf(wgt, e_vw.y, mvw.y), fmaf(wgt, e_vw.z, mvw.z));
  }
  const float area = tri_area(U, muv, muw) + tri_area(muv, V, mvw) + tri_area(muw, mvw, W) + tri_area(mvw, muw, muv);

  // bounding rectangle in the corners' plane, first axis along the longest corner edge
  const float3 c3[3] = {U, V, W};
  float best = -1.f;
  int e0 = 0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const float3 a = c3[e], b = c3[(e + 1) % 3];
    const float l2 = (b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y) + (b.z - a.z) * (b.z - a.z);
    if (l2 > best) {
      best = l2;
      e0 = e;
    }
  }
  const float3 o = c3[e0], b = c3[(e0 + 1) % 3];
  float aspect = INFINITY;
  const float len = sqrtf(best);
  const float nx0 = (V.y - U.y) * (W.z - U.z) - (V.z - U.z) * (W.y - U.y);
  const float ny0 = (V.z - U.z) * (W.x - U.x) - (V.x - U.x) * (W.z - U.z);
  const float nz0 = (V.x - U.x) * (W.y - U.y) - (V.y - U.y) * (W.x - U.x);
  const float nl = sqrtf(nx0 * nx0 + ny0 * ny0 + nz0 * nz0);
  if (len > 0.f && nl > 0.f) {
    const float xx = (b.x - o.x) / len, xy = (b.y - o.y) / len, xz = (b.z - o.z) / len;
    const float nx = nx0 / nl, ny = ny0 / nl, nz = nz0 / nl;
    const float yx = ny * xz - nz * xy, yy = nz * xx - nx * xz, yz = nx * xy - ny * xx;
    float lox = INFINITY, hix = -INFINITY, loy = INFINITY, hiy = -INFINITY;
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      const float dx = p[t].x - o.x, dy = p[t].y - o.y, dz = p[t].z - o.z;
      const float px = dx * xx + dy * xy + dz * xz, py = dx * yx + dy * yy + dz * yz;
      lox = fminf(lox, px);
      hix = fmaxf(hix, px);
      loy = fminf(loy, py);
      hiy = fmaxf(hiy, py);
    }
    const float ex = hix - lox, ey = hiy - loy;
    const float lo = fminf(ex, ey), hi = fmaxf(ex, ey);
    aspect = lo > 0.f ? hi / lo : INFINITY;
  }

  float grad = 0.f;
  if (s.g_ctrl) {
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      const float *g = s.g_ctrl + ((size_t)m * NC + t) * 3;
      const float gx = __ldg(g), gy = __ldg(g + 1), gz = __ldg(g + 2);
      grad += sqrtf(gx * gx + gy * gy + gz * gz);
    }
    grad /= (float)NC;
  }
  if (s.area) s.area[m] = area;
  if (s.aspect) s.aspect[m] = aspect;
  if (s.grad && s.g_ctrl) s.grad[m] = grad;
  if (s.flags) {
    // split: the mean control-point gradient, or the accumulated average edge value
    const bool by_edges = s.edge_sum && s.edge_count && s.edge_count[m] > 0 &&
                          (double)s.edge_sum[m] > (double)s.tau_b * (double)s.edge_count[m];
    unsigned char f = (unsigned char)((area < s.tau_a || aspect > s.tau_s ? 1 : 0) |
                                      ((s.g_ctrl && grad > s.tau_g) || by_edges ? 2 : 0));
    // visibility ratios compared in FP64: integer counts over integer totals
    if (s.view_count && s.n_views > 0 && (double)s.view_count[m] < (double)s.tau_v * (double)s.n_views) f |= 4;
    if (s.cell_mask) {
      int seen = 0;
      for (int k = 0; k < s.words; ++k) seen += __popcll(s.cell_mask[(size_t)m * s.words + k]);
      if ((double)seen < (double)s.tau_r * (double)s.cells) f |= 8;
    }
    s.flags[m] = f;
  }
}

// a word other threads set bits of: a relaxed atomic read (a stale value
// only costs one redundant atomicOr)
__device__ __forceinline__ unsigned long long relaxed_load(unsigned long long *p) {
  return cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>(*p).load(cuda::memory_order_relaxed);
}

// Visibility measures from the raster of views [v0, v0 + 64): per foreground
// pixel, the bit of the flat triangle it is seen through (the low 32 bits of
// its depth key are prim * nsub + sub-triangle) in cell_mask[prim], and bit
// v - v0 in seen[prim]. A bit already set is read, not written again.
__global__ void __launch_bounds__(256) k_vis_pixels(const int *pid, const unsigned long long *zbuf,
                                                    const int *view_off, int V, int pix0, int pix1, int v0,
                                                    int nsub, int words, unsigned long long *cell_mask,
                                                    unsigned long long *seen) {
  const int pix = pix0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= pix1) return;
  const int id = pid[pix];
  if (id < 0) return;
  if (cell_mask) {
    const int sub = (int)((unsigned)(zbuf[pix] & 0xffffffffull) - (unsigned)id * (unsigned)nsub);
    unsigned long long *c = cell_mask + (size_t)id * words + (sub >> 6);
    const unsigned long long bit = 1ull << (sub & 63);
    if (!(relaxed_load(c) & bit)) atomicOr(c, bit);
  }
  if (seen) {
    const int view = find_view(view_off, V, pix);
    const unsigned long long bit = 1ull << (view - v0);
    if (!(relaxed_load(seen + id) & bit)) atomicOr(seen + id, bit);
  }
}

// view_count[m] += the views of the group primitive m was seen in; clears seen
__global__ void __launch_bounds__(256) k_vis_count(int M, unsigned long long *seen, int *view_count) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const unsigned long long v = seen[m];
  if (v) {
    view_count[m] += __popcll(v);
    seen[m] = 0ull;
  }
}

constexpr int kMaxEdgeViews = 200;  // views per launch: the table stays in 4 KB of parameters

struct EdgeArgs {
  const float *img;
  float *edges;
  int n_views;
  int off[kMaxEdgeViews + 1];  // first pixel of each view of the launch, last: end
  int W[kMaxEdgeViews];
};
static_assert(sizeof(EdgeArgs) <= 4000, "kernel parameters");

// 8-bit luma of pixel (x, y) of a W-wide view at pixel offset base (clamped to the view)
__device__ __forceinline__ float luma255(const float *img, int base, int W, int H, int x, int y) {
  x = min(max(x, 0), W - 1);
  y = min(max(y, 0), H - 1);
  const float *c = img + 3 * ((size_t)base + (size_t)y * W + x);
  return 255.0f * (0.299f * __ldg(c) + 0.587f * __ldg(c + 1) + 0.114f * __ldg(c + 2));
}

// Edge prior of the split criterion: Sobel gradient magnitude of the 8-bit
// luma, border replicated, one thread per pixel of the launch's views
__global__ void __launch_bounds__(256) k_edge_magnitude(const __grid_constant__ EdgeArgs a) {
  const int i = a.off[0] + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.off[a.n_views]) return;
  int lo = 0, hi = a.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  const int base = a.off[lo], W = a.W[lo], H = (a.off[lo + 1] - base) / W;
  const int y = (i - base) / W, x = (i - base) - y * W;
  float p[3][3];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) p[dy + 1][dx + 1] = luma255(a.img, base, W, H, x + dx, y + dy);
  const float gx = (p[0][2] - p[0][0]) + 2.0f * (p[1][2] - p[1][0]) + (p[2][2] - p[2][0]);
  const float gy = (p[2][0] - p[0][0]) + 2.0f * (p[2][1] - p[0][1]) + (p[2][2] - p[0][2]);
  a.edges[i] = sqrtf(gx * gx + gy * gy);
}

// edge values back-projected through I_id of the last forward: per run of
// consecutive pixels of one primitive, one atomic for the sum and one for the count
__global__ void __launch_bounds__(256) k_edge_prior(const int *pid, const float *edges, int P, float *edge_sum,
                                                    int *edge_count) {
  const int lane = threadIdx.x & 31;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  const int id = pix < P ? pid[pix] : -1;
  const bool on = id >= 0;
  if (!__any_sync(0xffffffffu, on)) return;
  const Seg sg = seg_info(on ? id : -1 - lane);
  const float e = seg_sum(on ? edges[pix] : 0.f, sg);
  const float c = seg_sum(on ? 1.f : 0.f, sg);
  if (sg.tail && on) {
    if (edge_sum) atomicAdd(edge_sum + id, e);
    if (edge_count) atomicAdd(edge_count + id, (int)c);
  }
}

}  // namespace

int launch_subdivide(int degree, const bgt_scene &sc, const int *sel, int n_sel, const bgt_prims &out,
                     cudaStream_t st) {
  if (n_sel <= 0) return 0;
  SplitArgs s;
  s.ctrl = sc.ctrl;
  s.color = sc.color;
  s.opacity = sc.opacity;
  s.r_b = sc.r_b;
  s.log_scale = sc.log_scale;
  s.quat = sc.quat;
  s.sh = sc.sh;
  s.M = sc.num_prims;
  s.R = sc.attr_res <= 0 ? 1 : sc.attr_res;
  s.T = s.R * (s.R + 1) / 2;
  s.K = sc.sh_degree > 0 ? (sc.sh_degree + 1) * (sc.sh_degree + 1) - 1 : 0;
  s.sel = sel;
  s.n_sel = n_sel;
  s.out = out;
  const long long per = std::max(ncp_of(degree), s.T);
  const long long threads = 4LL * n_sel * per;
  const int blocks = (int)((threads + 255) / 256);
  dispatch_degree(degree, [&](auto d) { k_subdivide<decltype(d)::value><<<blocks, 256, 0, st>>>(s); });
  return 1;
}

int launch_prim_metrics(int degree, const float *ctrl, int M, const float *g_ctrl, float tau_a, float tau_s,
                        float tau_g, const float *edge_sum, const int *edge_count, float tau_b,
                        const int *view_count, int n_views, const unsigned long long *cell_mask, int tess_level,
                        float tau_v, float tau_r, float *area, float *aspect, float *grad, unsigned char *flags,
                        cudaStream_t st) {
  if (M <= 0) return 0;
  const int nsub = 2 * tess_level * tess_level;
  MetricArgs s{ctrl, g_ctrl, M, tau_a, tau_s, tau_g, edge_sum, edge_count, tau_b, view_count, n_views, cell_mask,
               (nsub + 63) / 64, tess_level * tess_level, tau_v, tau_r, area, aspect, grad, flags};
  dispatch_degree(degree, [&](auto d) { k_prim_metrics<decltype(d)::value><<<(M + 255) / 256, 256, 0, st>>>(s); });
  return 1;
}

int launch_edge_magnitude(const float *img, int n_views, const int *sizes, float *edges, cudaStream_t st) {
  EdgeArgs a;
  a.img = img;
  a.edges = edges;
  int launches = 0, off = 0;
  for (int v0 = 0; v0 < n_views; v0 += kMaxEdgeViews) {
    a.n_views = 0;
    const int first = off;
    for (int v = v0; v < n_views && v < v0 + kMaxEdgeViews; ++v) {
      const int W = sizes[2 * v], H = sizes[2 * v + 1];
      if (W > 0 && H > 0) {
        a.off[a.n_views] = off;
        a.W[a.n_views] = W;
        a.n_views++;
      }
      off += W * H;
    }
    a.off[a.n_views] = off;
    if (a.n_views == 0 || off == first) continue;
    k_edge_magnitude<<<(off - first + 255) / 256, 256, 0, st>>>(a);
    ++launches;
  }
  return launches;
}

int launch_edge_prior(const Params &p, const Work &w, const float *edges, float *edge_sum, int *edge_count,
                      cudaStream_t st) {
  if (p.P <= 0) return 0;
  k_edge_prior<<<(p.P + 255) / 256, 256, 0, st>>>(w.pid, edges, p.P, edge_sum, edge_count);
  return 1;
}

int launch_visibility(const Params &p, const Work &w, const int *view_off, int *view_count,
                      unsigned long long *cell_mask, cudaStream_t st) {
  // view_off: host copy of the forward's pixel offsets per view (V + 1)
  const int nsub = 2 * p.L * p.L, words = (nsub + 63) / 64;
  int launches = 0;
  if (view_count && p.M > 0) {
    cudaMemsetAsync(w.vis_seen, 0, sizeof(unsigned long long) * (size_t)p.M, st);
    launches++;
  }
  for (int v0 = 0; v0 < p.V; v0 += 64) {
    const int v1 = v0 + 64 < p.V ? v0 + 64 : p.V;
    const int pix0 = view_off[v0], pix1 = view_off[v1];
    if (pix1 > pix0) {
      k_vis_pixels<<<(pix1 - pix0 + 255) / 256, 256, 0, st>>>(w.pid, w.zbuf, w.view_pix_off, p.V, pix0, pix1, v0,
                                                             nsub, words, cell_mask,
                                                             view_count ? w.vis_seen : nullptr);
      launches++;
    }
    if (view_count && p.M > 0) {
      k_vis_count<<<(p.M + 255) / 256, 256, 0, st>>>(p.M, w.vis_seen, view_count);
      launches++;
    }
  }
  return launches;
}

}  // namespace bgt
