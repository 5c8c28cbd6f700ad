// Tessellation + rasterization with a depth test (Sec. 3.2, "Tessellation and
// Rasterization"): every Bezier triangle is cut into the L^2 flat triangles
// of a uniform barycentric lattice whose vertices are exact evaluations of
// Eq. 1; each flat triangle is rasterized against pixel centres with exact
// 64-bit edge functions on a 1/256-pixel grid, and the nearest one per pixel
// is kept by a 64-bit atomicMin on (depth bits << 32 | sub-triangle id). The
// resolve pass turns the winning key into I_id and perspective-correct I_uv.
//
// One warp per (view, primitive): the lanes evaluate the (L+1)(L+2)/2 lattice
// vertices into shared memory once, then each lane rasterizes its flat
// triangles. Every operation that decides coverage or the depth order is an
// explicit IEEE-rounded intrinsic, so the result is reproducible bit for bit.
#include <climits>

#include "bgt_internal.cuh"

namespace bgt {

namespace {

constexpr int kRasterWarps = 4;
constexpr int kMaxVerts = (kMaxTess + 1) * (kMaxTess + 2) / 2;

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

template <int N>
__global__ void __launch_bounds__(kRasterWarps * 32) k_raster(Params p, Scene s, Work w) {
  __shared__ int sX[kRasterWarps][kMaxVerts];
  __shared__ int sY[kRasterWarps][kMaxVerts];
  __shared__ float sIZ[kRasterWarps][kMaxVerts];
  // lattice tables of this launch's level L: k / L, vertex (a, b), and per flat
  // triangle its three vertex slots and its id
  __shared__ float s_frac[kMaxTess + 1];
  __shared__ int s_vab[kMaxVerts];
  __shared__ int2 s_tri[kMaxTess * kMaxTess];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long items = (long long)p.V * p.M;
  const int L = p.L;
  const int NV = (L + 1) * (L + 2) / 2;
  const int up_count = L * (L + 1) / 2;
  const int nsub = 2 * L * L;
  for (int i = threadIdx.x; i <= L; i += blockDim.x) s_frac[i] = lattice_frac(i, L);
  for (int vi = threadIdx.x; vi < NV; vi += blockDim.x) {
    int a, b;
    slot_to_ab(vi, L, a, b);
    s_vab[vi] = a | (b << 8);
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
  for (long long item = (long long)blockIdx.x * kRasterWarps + warp; item < items;
       item += (long long)gridDim.x * kRasterWarps) {
    const int view = (int)(item / p.M);
    const int prim = (int)(item - (long long)view * p.M);
    const View vw = w.views[view];
    const float *cp = s.ctrl + (size_t)prim * p.ncp * 3;
    for (int vi = lane; vi < NV; vi += 32) {
      const int ab = s_vab[vi], a = ab & 0xff, b = ab >> 8;
      const RVert r = raster_vertex<N>(cp, s_frac[a], s_frac[b], s_frac[L - a - b], vw, p.near_z);
      sX[warp][vi] = r.valid ? r.X : INT_MIN;
      sY[warp][vi] = r.Y;
      sIZ[warp][vi] = r.iz;
    }
    __syncwarp();
    const int W = vw.W, H = vw.H;
    unsigned long long *zb = w.zbuf + vw.pix_off;
    for (int ti = lane; ti < L * L; ti += 32) {
      const int2 tri = s_tri[ti];
      const int sid = tri.y;
      int X[3], Y[3];
      float IZ[3];
      bool ok = true;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const int sl = (tri.x >> (8 * c)) & 0xff;
        X[c] = sX[warp][sl];
        Y[c] = sY[warp][sl];
        IZ[c] = sIZ[warp][sl];
        ok = ok && (X[c] != INT_MIN);
      }
      if (!ok) continue;
      long long area2 = edge_fn(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
      if (area2 == 0) continue;
      if (area2 < 0) {
        int tx = X[1]; X[1] = X[2]; X[2] = tx;
        tx = Y[1]; Y[1] = Y[2]; Y[2] = tx;
        const float tz = IZ[1]; IZ[1] = IZ[2]; IZ[2] = tz;
        area2 = -area2;
      }
      const int xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
      const int ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
      // pixel range: ceil(xmin / 256) .. floor(xmax / 256) (arithmetic shift = floor)
      int px0 = -((-xmin) >> 8), px1 = xmax >> 8;
      int py0 = -((-ymin) >> 8), py1 = ymax >> 8;
      px0 = max(px0, 0); py0 = max(py0, 0);
      px1 = min(px1, W - 1); py1 = min(py1, H - 1);
      if (px0 > px1 || py0 > py1) continue;
      const bool t0 = owns_zero_edge(X[1], Y[1], X[2], Y[2]);
      const bool t1 = owns_zero_edge(X[2], Y[2], X[0], Y[0]);
      const bool t2 = owns_zero_edge(X[0], Y[0], X[1], Y[1]);
      const float af = __ll2float_rn(area2);
      const unsigned int gid = (unsigned int)prim * (unsigned int)nsub + (unsigned int)sid;
      for (int py = py0; py <= py1; py++) {
        const int Py = py * 256;
        for (int px = px0; px <= px1; px++) {
          const int Px = px * 256;
          const long long e0 = edge_fn(X[1], Y[1], X[2], Y[2], Px, Py);
          const long long e1 = edge_fn(X[2], Y[2], X[0], Y[0], Px, Py);
          const long long e2 = edge_fn(X[0], Y[0], X[1], Y[1], Px, Py);
          const bool in = (e0 > 0 || (e0 == 0 && t0)) && (e1 > 0 || (e1 == 0 && t1)) &&
                          (e2 > 0 || (e2 == 0 && t2));
          if (!in) continue;
          const float l0 = __fdiv_rn(__ll2float_rn(e0), af);
          const float l1 = __fdiv_rn(__ll2float_rn(e1), af);
          const float l2 = __fdiv_rn(__ll2float_rn(e2), af);
          float sd = __fmul_rn(l0, IZ[0]);
          sd = __fmaf_rn(l1, IZ[1], sd);
          sd = __fmaf_rn(l2, IZ[2], sd);
          const float z = __fdiv_rn(1.0f, sd);
          const unsigned long long key =
              ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)gid;
          atomicMin(zb + (size_t)py * W + px, key);
        }
      }
    }
    __syncwarp();
  }
}

template <int N>
__global__ void k_resolve(Params p, Scene s, Work w) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= p.P) return;
  const unsigned long long key = w.zbuf[pix];
  if (key == ~0ull) {
    w.pid[pix] = -1;
    w.puv[pix] = make_float2(0.f, 0.f);
    return;
  }
  const int view = find_view(w.view_pix_off, p.V, pix);
  const View vw = w.views[view];
  const int L = p.L, nsub = 2 * L * L;
  const unsigned int gid = (unsigned int)(key & 0xffffffffu);
  const int prim = (int)(gid / (unsigned int)nsub);
  const int sid = (int)(gid - (unsigned int)prim * (unsigned int)nsub);
  if (prim >= p.M) {
    atomicOr(w.status, kStatusBadPrim);
    w.pid[pix] = -1;
    return;
  }
  const float *cp = s.ctrl + (size_t)prim * p.ncp * 3;
  int va[3], vb[3];
  subtri_verts(L, sid, va, vb);
  RVert r[3];
#pragma unroll
  for (int c = 0; c < 3; c++) r[c] = raster_vertex<N>(cp, va[c], vb[c], L, vw, p.near_z);
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

}  // namespace

int launch_raster(const Params &p, const Scene &s, const Work &w, cudaStream_t st) {
  const long long items = (long long)p.V * p.M;
  if (items == 0) return 0;
  long long blocks = (items + kRasterWarps - 1) / kRasterWarps;
  if (blocks > (1ll << 30)) blocks = 1ll << 30;
  dispatch_degree(p.n, [&](auto d) { k_raster<decltype(d)::value><<<(unsigned)blocks, kRasterWarps * 32, 0, st>>>(p, s, w); });
  return 1;
}

int launch_resolve(const Params &p, const Scene &s, const Work &w, cudaStream_t st) {
  if (p.P == 0) return 0;
  dispatch_degree(p.n, [&](auto d) { k_resolve<decltype(d)::value><<<(p.P + 255) / 256, 256, 0, st>>>(p, s, w); });
  return 1;
}

}  // namespace bgt
