// Tessellation + rasterization with a depth test (Sec. 3.2, "Tessellation and
// Rasterization"): every Bezier triangle is cut into the L^2 flat triangles
// of a uniform barycentric lattice whose vertices are exact evaluations of
// Eq. 1; each flat triangle is rasterized against pixel centres with exact
// 64-bit edge functions on a 1/256-pixel grid, and the nearest one per pixel
// is kept by a 64-bit atomicMin on (~bits(1/z) << 32 | sub-triangle id), 1/z
// the perspective-correct interpolation sum(e_i / z_i) / area2 (the nearest
// surface has the largest 1/z). The resolve pass turns the winning key into
// I_id and perspective-correct I_uv.
//
// Grid: one block row per view (blockIdx.y), warps take primitives of that
// view two at a time. Per block, the Bernstein weights of the (L+1)(L+2)/2
// lattice vertices and the vertex slots of the L^2 flat triangles are
// tabulated once in shared memory. Per pair of primitives, the lanes evaluate
// the lattice vertices of both from the table and their control points (in
// shared memory) into shared memory (2 x 45 vertices at L = 8 fill three
// rounds of 32 lanes where one primitive alone leaves the second of two
// rounds mostly idle); then each lane rasterizes its flat triangles: an empty
// pixel box is rejected before any edge function, and the pixel centres of the
// box are walked in one loop with incrementally updated edge functions, in
// 32-bit integers when the box is under 125 px (exact: every product stays
// below 2^30) and in 64-bit ones otherwise. Every operation that decides
// coverage or the depth order is an explicit IEEE-rounded intrinsic, so the
// result is reproducible bit for bit.
#include <climits>

#include "bgt_internal.cuh"

namespace bgt {

namespace {

constexpr int kRasterWarps = 4;
constexpr int kMaxVerts = (kMaxTess + 1) * (kMaxTess + 2) / 2;
constexpr int kSpan32 = 32000;    // box spans (1/256 px) below which edge functions fit 32 bits

__device__ inline int vslot(int a, int b, int L) { return a * (L + 1) - a * (a - 1) / 2 + b; }

__device__ inline void slot_to_ab(int vi, int L, int &a, int &b) {
  int rem = vi;
  a = 0;
  while (rem >= L + 1 - a) {
    rem -= L + 1 - a;
    a++;
  }
  b = rem;
}

__device__ __forceinline__ float to_f32(int x) { return __int2float_rn(x); }
__device__ __forceinline__ float to_f32(long long x) { return __ll2float_rn(x); }

// depth test of one covered pixel: the interpolated 1/z = sum(e_i / z_i) /
// area2, every operation IEEE-rounded; the key complements its bits so that
// the nearest surface has the smallest key
__device__ __forceinline__ void depth_test(float f0, float f1, float f2, float af, const float *IZ, int pix,
                                           unsigned gid, unsigned long long *zb) {
  float sd = __fmul_rn(f0, IZ[0]);
  sd = __fmaf_rn(f1, IZ[1], sd);
  sd = __fmaf_rn(f2, IZ[2], sd);
  const float inv_z = __fdiv_rn(sd, af);
  atomicMin(zb + pix, ((unsigned long long)(~__float_as_uint(inv_z)) << 32) | (unsigned long long)gid);
}

// Pixel centres of the box [px0, px1] x [py0, py1] inside the flat triangle
// (X, Y, IZ) (counter-clockwise after the swap, area2 > 0, fill-rule flags
// t0..t2 of the edges 1-2, 2-0, 0-1): edge functions (b - a) x (P - a) start
// at the box corner and step by their constant differences, row by row in one
// loop (lanes with boxes of different shapes stay in step); I is int when
// every value stays below 2^31 (box span < kSpan32), else long long. Covered
// pixels take the depth test.
template <typename I>
__device__ __forceinline__ void raster_box(const int *X, const int *Y, const float *IZ, bool t0, bool t1, bool t2,
                                           float af, int px0, int px1, int py0, int py1, unsigned gid,
                                           unsigned long long *zb, int W) {
  const I a0 = (I)(X[2] - X[1]), b0 = (I)(Y[2] - Y[1]);
  const I a1 = (I)(X[0] - X[2]), b1 = (I)(Y[0] - Y[2]);
  const I a2 = (I)(X[1] - X[0]), b2 = (I)(Y[1] - Y[0]);
  const int Px0 = px0 * 256, Py0 = py0 * 256;
  I r0 = a0 * (I)(Py0 - Y[1]) - b0 * (I)(Px0 - X[1]);
  I r1 = a1 * (I)(Py0 - Y[2]) - b1 * (I)(Px0 - X[2]);
  I r2 = a2 * (I)(Py0 - Y[0]) - b2 * (I)(Px0 - X[0]);
  const I sx0 = b0 * (I)256, sx1 = b1 * (I)256, sx2 = b2 * (I)256;  // per pixel step in x (subtracted)
  const I sy0 = a0 * (I)256, sy1 = a1 * (I)256, sy2 = a2 * (I)256;  // per pixel step in y (added)
  // one loop over the box's pixel centres, row by row
  const int n = (px1 - px0 + 1) * (py1 - py0 + 1);
  I e0 = r0, e1 = r1, e2 = r2;
  int px = px0, pix = py0 * W + px0;
  for (int k = 0; k < n; k++) {
    if ((e0 > 0 || (e0 == 0 && t0)) && (e1 > 0 || (e1 == 0 && t1)) && (e2 > 0 || (e2 == 0 && t2)))
      depth_test(to_f32(e0), to_f32(e1), to_f32(e2), af, IZ, pix, gid, zb);
    if (px < px1) {
      px++;
      pix++;
      e0 -= sx0;
      e1 -= sx1;
      e2 -= sx2;
    } else {
      r0 += sy0;
      r1 += sy1;
      r2 += sy2;
      e0 = r0;
      e1 = r1;
      e2 = r2;
      pix += W - (px1 - px0);
      px = px0;
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kRasterWarps * 32, N <= 2 ? 8 : 6) k_raster(Params p, Scene s, Work w) {
  constexpr int NCP = (N + 1) * (N + 2) / 2;
  __shared__ float sB[kMaxVerts * NCP];  // Bernstein weights of the lattice vertices
  __shared__ int2 s_tri[kMaxTess * kMaxTess];  // vertex slots (8 bits each) and sub-triangle id
  __shared__ int sX[kRasterWarps][2 * kMaxVerts];
  __shared__ int sY[kRasterWarps][2 * kMaxVerts];
  __shared__ float sIZ[kRasterWarps][2 * kMaxVerts];
  __shared__ __align__(16) float sC[kRasterWarps][2][3 * NCP + 2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = p.L;
  const int NV = (L + 1) * (L + 2) / 2;
  const int up_count = L * (L + 1) / 2;
  const int nsub = 2 * L * L;
  for (int vi = threadIdx.x; vi < NV; vi += blockDim.x) {
    int a, b;
    slot_to_ab(vi, L, a, b);
    float Bw[NCP];
    lattice_bernstein<N>(lattice_frac(a, L), lattice_frac(b, L), lattice_frac(L - a - b, L), Bw);
#pragma unroll
    for (int t = 0; t < NCP; t++) sB[vi * NCP + t] = Bw[t];
  }
  for (int ti = threadIdx.x; ti < L * L; ti += blockDim.x) {
    int a, down, rem;
    if (ti < up_count) {
      down = 0;
      rem = ti;
      a = 0;
      while (rem >= L - a) { rem -= L - a; a++; }
    } else {
      down = 1;
      rem = ti - up_count;
      a = 0;
      while (rem >= L - 1 - a) { rem -= L - 1 - a; a++; }
    }
    const int sid = 2 * (a * L + rem) + down;
    int va[3], vb[3];
    subtri_verts(L, sid, va, vb);
    s_tri[ti] = make_int2(vslot(va[0], vb[0], L) | (vslot(va[1], vb[1], L) << 8) | (vslot(va[2], vb[2], L) << 16), sid);
  }
  __syncthreads();
  // the block row's camera in shared memory, its fields read where used
  // (held in registers it costs spills at the 64-register budget)
  __shared__ View s_view;
  if (threadIdx.x < (int)(sizeof(View) / 4))
    reinterpret_cast<int *>(&s_view)[threadIdx.x] = reinterpret_cast<const int *>(w.views + blockIdx.y)[threadIdx.x];
  __syncthreads();
  const View &vw = s_view;
  const int W = vw.W, H = vw.H;
  unsigned long long *zb = w.zbuf + vw.pix_off;
  const int stride = gridDim.x * kRasterWarps;
  for (int prim0 = blockIdx.x * kRasterWarps + warp; prim0 < p.M; prim0 += 2 * stride) {
    const int nitem = prim0 + stride < p.M ? 2 : 1;
    for (int k = lane; k < nitem * 3 * NCP; k += 32) {
      const int it = k >= 3 * NCP;
      sC[warp][it][k - it * 3 * NCP] = __ldg(s.ctrl + (size_t)(prim0 + it * stride) * NCP * 3 + (k - it * 3 * NCP));
    }
    __syncwarp();
    for (int vi = lane; vi < nitem * NV; vi += 32) {
      const int it = vi >= NV;
      const RVert r = vertex_from_weights<N>(sB + (vi - it * NV) * NCP, sC[warp][it], vw, p.near_z);
      sX[warp][vi] = r.valid ? r.X : INT_MIN;
      sY[warp][vi] = r.Y;
      sIZ[warp][vi] = r.iz;
    }
    __syncwarp();
    for (int it = 0; it < nitem; it++) {
    const int prim = prim0 + it * stride;
    const int vb = it * NV;
    for (int ti = lane; ti < L * L; ti += 32) {
      const int2 tri = s_tri[ti];
      int X[3], Y[3];
      float IZ[3];
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const int sl = vb + ((tri.x >> (8 * k)) & 0xff);
        X[k] = sX[warp][sl];
        Y[k] = sY[warp][sl];
        IZ[k] = sIZ[warp][sl];
        ok = ok && (X[k] != INT_MIN);
      }
      if (!ok) continue;
      const int xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
      const int ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
      // pixel range: ceil(xmin / 256) .. floor(xmax / 256) (arithmetic shift = floor)
      const int px0 = max(-((-xmin) >> 8), 0), px1 = min(xmax >> 8, W - 1);
      const int py0 = max(-((-ymin) >> 8), 0), py1 = min(ymax >> 8, H - 1);
      if (px0 > px1 || py0 > py1) continue;  // no pixel centre in the box
      long long area2 = edge_fn(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
      if (area2 == 0) continue;
      if (area2 < 0) {
        int tx = X[1]; X[1] = X[2]; X[2] = tx;
        tx = Y[1]; Y[1] = Y[2]; Y[2] = tx;
        const float tz = IZ[1]; IZ[1] = IZ[2]; IZ[2] = tz;
        area2 = -area2;
      }
      const bool t0 = owns_zero_edge(X[1], Y[1], X[2], Y[2]);
      const bool t1 = owns_zero_edge(X[2], Y[2], X[0], Y[0]);
      const bool t2 = owns_zero_edge(X[0], Y[0], X[1], Y[1]);
      const float af = __ll2float_rn(area2);
      const unsigned gid = (unsigned)prim * (unsigned)nsub + (unsigned)tri.y;
      if (xmax - xmin < kSpan32 && ymax - ymin < kSpan32)
        raster_box<int>(X, Y, IZ, t0, t1, t2, af, px0, px1, py0, py1, gid, zb, W);
      else
        raster_box<long long>(X, Y, IZ, t0, t1, t2, af, px0, px1, py0, py1, gid, zb, W);
    }
    }
    __syncwarp();
  }
}

// Resolve: the winning key of each pixel -> I_id and perspective-correct
// I_uv. Persistent blocks tabulate the lattice Bernstein weights once (the
// raster's table, same operations) and recompute the winning flat triangle's
// three vertices from it with the primitive's control points in registers.
template <int N>
__global__ void __launch_bounds__(256) k_resolve(Params p, Scene s, Work w) {
  constexpr int NCP = (N + 1) * (N + 2) / 2;
  __shared__ float sB[kMaxVerts * NCP];
  const int L = p.L, nsub = 2 * L * L;
  const int NV = (L + 1) * (L + 2) / 2;
  for (int vi = threadIdx.x; vi < NV; vi += blockDim.x) {
    int a, b;
    slot_to_ab(vi, L, a, b);
    float Bw[NCP];
    lattice_bernstein<N>(lattice_frac(a, L), lattice_frac(b, L), lattice_frac(L - a - b, L), Bw);
#pragma unroll
    for (int t = 0; t < NCP; t++) sB[vi * NCP + t] = Bw[t];
  }
  __syncthreads();
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < p.P; pix += gridDim.x * blockDim.x) {
    const unsigned long long key = w.zbuf[pix];
    if (key == ~0ull) {
      w.pid[pix] = -1;
      w.puv[pix] = make_float2(0.f, 0.f);
      continue;
    }
    const unsigned int gid = (unsigned int)(key & 0xffffffffu);
    const int prim = (int)(gid / (unsigned int)nsub);
    const int sid = (int)(gid - (unsigned int)prim * (unsigned int)nsub);
    if (prim >= p.M) {
      atomicOr(w.status, kStatusBadPrim);
      w.pid[pix] = -1;
      continue;
    }
    const int view = find_view(w.view_pix_off, p.V, pix);
    const View &vw = w.views[view];
    const float *cp = s.ctrl + (size_t)prim * NCP * 3;
    float c[3 * NCP];
#pragma unroll
    for (int k = 0; k < 3 * NCP; k++) c[k] = __ldg(cp + k);
    int va[3], vb[3];
    subtri_verts(L, sid, va, vb);
    RVert r[3];
#pragma unroll
    for (int k = 0; k < 3; k++) r[k] = vertex_from_weights<N>(sB + vslot(va[k], vb[k], L) * NCP, c, vw, p.near_z);
    long long area2 = edge_fn(r[0].X, r[0].Y, r[1].X, r[1].Y, r[2].X, r[2].Y);
    if (area2 < 0) {
      RVert t = r[1]; r[1] = r[2]; r[2] = t;
      int x = va[1]; va[1] = va[2]; va[2] = x;
      x = vb[1]; vb[1] = vb[2]; vb[2] = x;
      area2 = -area2;
    }
    const int local = pix - vw.pix_off;
    const int qy = local / vw.W, qx = local - qy * vw.W;
    const int Px = qx * 256, Py = qy * 256;
    const long long e0 = edge_fn(r[1].X, r[1].Y, r[2].X, r[2].Y, Px, Py);
    const long long e1 = edge_fn(r[2].X, r[2].Y, r[0].X, r[0].Y, Px, Py);
    const long long e2 = edge_fn(r[0].X, r[0].Y, r[1].X, r[1].Y, Px, Py);
    const float af = (float)area2;
    const float w0 = ((float)e0 / af) / r[0].Z;
    const float w1 = ((float)e1 / af) / r[1].Z;
    const float w2 = ((float)e2 / af) / r[2].Z;
    const float ws = (w0 + w1) + w2;
    const float u = (w0 * (float)va[0] + w1 * (float)va[1] + w2 * (float)va[2]) / (ws * (float)L);
    const float v = (w0 * (float)vb[0] + w1 * (float)vb[1] + w2 * (float)vb[2]) / (ws * (float)L);
    w.pid[pix] = prim;
    w.puv[pix] = make_float2(u, v);
  }
}

}  // namespace

int launch_raster(const Params &p, const Scene &s, const Work &w, cudaStream_t st) {
  if (p.V == 0 || p.M == 0) return 0;
  // each warp rasterizes p.raster_prims primitives per block (amortises the tables)
  const int per_block = kRasterWarps * p.raster_prims;
  const dim3 grid((unsigned)((p.M + per_block - 1) / per_block), (unsigned)p.V);
  dispatch_degree(p.n, [&](auto d) { k_raster<decltype(d)::value><<<grid, kRasterWarps * 32, 0, st>>>(p, s, w); });
  return 1;
}

int launch_resolve(const Params &p, const Scene &s, const Work &w, cudaStream_t st) {
  if (p.P == 0) return 0;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = min((p.P + 255) / 256, (sms > 0 ? sms : 152) * 8);
  dispatch_degree(p.n, [&](auto d) { k_resolve<decltype(d)::value><<<blocks, 256, 0, st>>>(p, s, w); });
  return 1;
}

}  // namespace bgt
