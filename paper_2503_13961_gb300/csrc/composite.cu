// Discontinuity-aware alpha blending, forward and backward (Sec. 3.2, Eq. 6-8;
// supplementary "Backward Derivative").
//
// One CTA per screen tile, persistent over a work queue of tiles. The tile's
// Gaussian list (sorted by depth, index) is staged in shared memory in
// batches; its boundary list (sorted by primitive, index) is staged once. For
// pixel q and a Gaussian of primitive g, the coefficient w (Eq. 6) is
// gamma* = min over g's boundary points b of gamma(|q - b|; sigma_b) (Eq. 7),
// found by a binary search for g in the tile's list; w = gamma* if I_id(q) = g
// else 1 - gamma*. alpha = min(alpha_max, o w G) (Eq. 8); pairs with
// alpha < alpha_min are skipped; blending stops before the pair that would
// take T below t_stop. Pair evaluation uses explicit IEEE-rounded intrinsics
// so that the backward pass reproduces the forward decisions exactly.
//
// The backward pass re-traverses each pixel's list back to front from its
// last composited entry, recovering T_i = T_{i+1} / (1 - alpha_i), and
// accumulates per-Gaussian gradients (mean, conic, opacity, colour; warp-
// reduced before the atomics) and per-boundary-point gradients (position,
// radius).
#include "bgt_internal.cuh"

namespace bgt {

namespace {

constexpr int kBCap = 1536;  // boundary entries staged in shared memory

// Block layout: NT threads; every warp owns a WX x WY block of the tile's
// pixels (PPT pixels per lane), so that a chunk of 32 staged Gaussians can be
// culled against the warp's block with one ballot.
template <int T>
struct TileCfg {
  static constexpr int NT = (T == 8) ? 64 : 256;
  static constexpr int NW = NT / 32;
  static constexpr int PPT = T * T / NT;     // 1, 1, 4
  static constexpr int WX = (T == 32) ? 16 : 8;
  static constexpr int WY = (T == 32) ? 8 : 4;
  static constexpr int WPR = T / WX;         // warp blocks per tile row
  static constexpr int NC = (PPT == 1) ? 8 : 4;  // coefficient cache entries per pixel
};

template <int T>
__device__ __forceinline__ void lane_pixel(int warp, int lane, int k, int &lx, int &ly) {
  using C = TileCfg<T>;
  lx = (warp % C::WPR) * C::WX + (lane & 7) + 8 * (k & 1);
  ly = (warp / C::WPR) * C::WY + (lane >> 3) + 4 * (k >> 1);
}

struct WRes {
  float w, gamma, rho;
  int best;   // position in the tile's boundary list, -1 if none within range
  int cands;  // boundary candidates scanned
};

// Eq. 6-7 for pixel (px, py) and primitive g over the tile's boundary list.
__device__ __forceinline__ WRes w_search(int g, int px, int py, int idq, const int *bprim,
                                         const float4 *brec, int bn, int use_boundary) {
  WRes r;
  r.best = -1;
  r.rho = 3.0e38f;
  r.gamma = 1.0f;
  r.cands = 0;
  if (!use_boundary) {  // the paper's "w/o B" ablation: no blending coefficient
    r.w = 1.0f;
    return r;
  }
  int lo = 0, hi = bn;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (bprim[mid] < g) lo = mid + 1; else hi = mid;
  }
  float best = 3.0e38f;
  for (int i = lo; i < bn && bprim[i] == g; i++) {
    const float4 b = brec[i];
    const unsigned qxy = __float_as_uint(b.x);
    const float dx = __fsub_rn((float)(px - (int)(qxy & 0xffffu)), b.y);
    const float dy = __fsub_rn((float)(py - (int)(qxy >> 16)), b.z);
    const float r2 = __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), __fmul_rn(b.w, b.w));
    if (r2 < best) {
      best = r2;
      r.best = i;
    }
    r.cands++;
  }
  if (r.best >= 0) {
    r.rho = __fsqrt_rn(best);
    if (best < 1.0f) r.gamma = exp2f(__fsub_rn(r.rho, 1.0f));
  }
  r.w = (idq == g) ? r.gamma : __fsub_rn(1.0f, r.gamma);
  return r;
}

struct PairGeo {
  float dx, dy, power;
};


// Warp-uniform cache of (primitive -> coefficient). All lanes of a warp hold
// the same primitive ids; each lane holds its own pixel's w and most
// influential boundary entry for them. On a miss every lane of the warp runs
// the same search (same primitive, same candidate list), so the search never
// diverges, and each primitive is searched about once per warp block.
template <int NC, bool BEST>
struct WarpCache {
  int key[NC];
  float w[NC];
  int best[BEST ? NC : 1];
  int next;
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int e = 0; e < NC; e++) key[e] = -2;
    next = 0;
  }
  // coefficient of primitive g for this lane's pixel; must be called by all lanes
  // with the same g
  __device__ __forceinline__ void get(int g, int px, int py, int idq, const int *bprim, const float4 *brec, int bn,
                                      int use_boundary, float &wv, int &bi, unsigned &cands) {
    int hit = -1;
#pragma unroll
    for (int e = 0; e < NC; e++) hit = (key[e] == g) ? e : hit;
    if (hit >= 0) {
      wv = w[0];
      bi = BEST ? best[0] : -1;
#pragma unroll
      for (int e = 1; e < NC; e++) {
        wv = (hit == e) ? w[e] : wv;
        if (BEST) bi = (hit == e) ? best[e] : bi;
      }
      return;
    }
    const WRes r = w_search(g, px, py, idq, bprim, brec, bn, use_boundary);
    cands += (unsigned)r.cands;
    wv = r.w;
    bi = (r.best >= 0 && r.rho < 1.0f) ? r.best : -1;
#pragma unroll
    for (int e = 0; e < NC; e++)
      if (e == next) {
        key[e] = g;
        w[e] = wv;
        if (BEST) best[e] = bi;
      }
    next = (next + 1 == NC) ? 0 : next + 1;
  }
};

struct TileInfo {
  int view, W, H, pix_off, x0, y0;
  long long gs, gn, bs, bn;
};

__device__ inline TileInfo tile_info(const Params &p, const Work &w, int tile, int T) {
  TileInfo t;
  t.view = find_view(w.view_tile_off, p.V, tile);
  const View *vw = w.views + t.view;
  t.W = __ldg(&vw->W);
  t.H = __ldg(&vw->H);
  t.pix_off = __ldg(&vw->pix_off);
  const int lt = tile - __ldg(&vw->tile_off);
  const int tx = __ldg(&vw->tiles_x);
  t.y0 = (lt / tx) * T;
  t.x0 = (lt - (lt / tx) * tx) * T;
  // an overflowed call (reported through the status word) leaves key slots
  // unwritten: its lists are treated as empty so that no slot is read
  const bool g_over = w.g_tstart[p.tiles] > p.max_pairs, b_over = w.b_tstart[p.tiles] > p.max_bpairs;
  t.gs = g_over ? 0 : w.g_tstart[tile];
  t.gn = g_over ? 0 : w.g_tstart[tile + 1] - t.gs;
  t.bs = b_over ? 0 : w.b_tstart[tile];
  t.bn = b_over ? 0 : w.b_tstart[tile + 1] - t.bs;
  return t;
}

// does the support square of the Gaussian cover any pixel of [x0,x1] x [y0,y1]?
__device__ __forceinline__ bool covers(const float4 &A, int x0, int x1, int y0, int y1) {
  const unsigned qxy = __float_as_uint(A.z);
  const float cx = (float)(int)(qxy & 0xffffu) + A.x, cy = (float)(int)(qxy >> 16) + A.y;
  const float r = A.w;
  return r >= 0.f && cx + r >= (float)x0 && cx - r <= (float)x1 && cy + r >= (float)y0 && cy - r <= (float)y1;
}

__device__ __forceinline__ PairGeo pair_geo2(int px, int py, const float4 &A, const float4 &B) {
  PairGeo p;
  const unsigned qxy = __float_as_uint(A.z);
  p.dx = __fsub_rn((float)(px - (int)(qxy & 0xffffu)), A.x);
  p.dy = __fsub_rn((float)(py - (int)(qxy >> 16)), A.y);
  const float q = __fmaf_rn(B.x, __fmul_rn(p.dx, p.dx), __fmul_rn(B.z, __fmul_rn(p.dy, p.dy)));
  p.power = __fsub_rn(__fmul_rn(-0.5f, q), __fmul_rn(B.y, __fmul_rn(p.dx, p.dy)));
  return p;
}

__device__ __forceinline__ void flush_stats(unsigned long long *stats, int base, unsigned a, unsigned b, unsigned c) {
  unsigned long long v[3] = {a, b, c};
#pragma unroll
  for (int q = 0; q < 3; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; q++)
      if (v[q]) atomicAdd(stats + base + q, v[q]);
}

template <int NT>
__device__ __forceinline__ void load_boundary_cache(const TileInfo &ti, const Work &w, int *s_bprim, float4 *s_brec,
                                                    const int *&bprim, const float4 *&brec) {
  const bool bsm = ti.bn <= kBCap;
  if (bsm) {
    for (int i = threadIdx.x; i < ti.bn; i += NT) {
      s_bprim[i] = w.bl_prim[ti.bs + i];
      s_brec[i] = w.bl_rec[ti.bs + i];
    }
  }
  bprim = bsm ? s_bprim : w.bl_prim + ti.bs;
  brec = bsm ? s_brec : w.bl_rec + ti.bs;
}

template <int T>
__global__ void __launch_bounds__(TileCfg<T>::NT) k_composite_fwd(Params p, Work w, float *image) {
  using Cfg = TileCfg<T>;
  constexpr int NT = Cfg::NT, NW = Cfg::NW, PPT = Cfg::PPT;
  __shared__ float4 sA[NW][32], sB[NW][32], sC[NW][32];
  __shared__ int s_bprim[kBCap];
  __shared__ float4 s_brec[kBCap];
  __shared__ int s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(w.counters + kQueueFwd, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= p.tiles) break;
    const TileInfo ti = tile_info(p, w, tile, T);
    const int *bprim;
    const float4 *brec;
    load_boundary_cache<NT>(ti, w, s_bprim, s_brec, bprim, brec);
    __syncthreads();
    const int bn = (int)ti.bn;
    const int wx0 = ti.x0 + (warp % Cfg::WPR) * Cfg::WX, wy0 = ti.y0 + (warp / Cfg::WPR) * Cfg::WY;
    const int wx1 = wx0 + Cfg::WX - 1, wy1 = wy0 + Cfg::WY - 1;

    float C[PPT][3], Tr[PPT];
    int last[PPT], idq[PPT], px[PPT], py[PPT];
    bool done[PPT];
    WarpCache<Cfg::NC, false> cache[PPT];
    unsigned n_sup = 0, n_comp = 0, n_cand = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      int lx, ly;
      lane_pixel<T>(warp, lane, k, lx, ly);
      px[k] = ti.x0 + lx;
      py[k] = ti.y0 + ly;
      const bool inside = px[k] < ti.W && py[k] < ti.H;
      done[k] = !inside;
      idq[k] = inside ? w.pid[ti.pix_off + py[k] * ti.W + px[k]] : -1;
      C[k][0] = C[k][1] = C[k][2] = 0.f;
      Tr[k] = 1.0f;
      last[k] = 0;
      cache[k].reset();
    }
    const int gn = (int)ti.gn;
    for (int c0 = 0; c0 < gn; c0 += 32) {
      bool alldone = true;
#pragma unroll
      for (int k = 0; k < PPT; k++) alldone = alldone && done[k];
      if (__all_sync(0xffffffffu, alldone)) break;
      // stage the chunk's Gaussians that touch this warp's block
      const int jl = c0 + lane;
      bool hit = false;
      if (jl < gn) {
        const unsigned gi = (unsigned)(w.gkeys[ti.gs + jl] & kIndexMask);
        const float4 A = w.gA[gi];
        hit = covers(A, wx0, wx1, wy0, wy1);
        if (hit) {
          sA[warp][lane] = A;
          sB[warp][lane] = w.gB[gi];
          sC[warp][lane] = w.gC[gi];
        }
      }
      unsigned mask = __ballot_sync(0xffffffffu, hit);
      __syncwarp();
      while (mask) {
        const int l = __ffs(mask) - 1;
        mask &= mask - 1;
        const float4 A = sA[warp][l], B = sB[warp][l];
        const int g = __float_as_int(sC[warp][l].w);
#pragma unroll
        for (int k = 0; k < PPT; k++) {
          const PairGeo pg = pair_geo2(px[k], py[k], A, B);
          const float G = __expf(pg.power);
          const float og = __fmul_rn(B.w, G);
          const bool cand = !done[k] && og >= p.alpha_min;  // w <= 1: else alpha < alpha_min
          if (!__any_sync(0xffffffffu, cand)) continue;
          float wv;
          int bi;
          cache[k].get(g, px[k], py[k], idq[k], bprim, brec, bn, p.use_boundary, wv, bi, n_cand);
          if (!cand) continue;
          n_sup++;
          const float alpha = fminf(p.alpha_max, __fmul_rn(og, wv));
          if (alpha < p.alpha_min) continue;
          const float testT = __fmul_rn(Tr[k], __fsub_rn(1.0f, alpha));
          if (testT < p.t_stop) {
            done[k] = true;
            continue;
          }
          const float4 Cc = sC[warp][l];
          const float ta = __fmul_rn(Tr[k], alpha);
          C[k][0] = __fmaf_rn(ta, Cc.x, C[k][0]);
          C[k][1] = __fmaf_rn(ta, Cc.y, C[k][1]);
          C[k][2] = __fmaf_rn(ta, Cc.z, C[k][2]);
          Tr[k] = testT;
          last[k] = c0 + l + 1;
          n_comp++;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      if (px[k] < ti.W && py[k] < ti.H) {
        const int pix = ti.pix_off + py[k] * ti.W + px[k];
        image[3 * (size_t)pix + 0] = __fmaf_rn(Tr[k], p.bg[0], C[k][0]);
        image[3 * (size_t)pix + 1] = __fmaf_rn(Tr[k], p.bg[1], C[k][1]);
        image[3 * (size_t)pix + 2] = __fmaf_rn(Tr[k], p.bg[2], C[k][2]);
        w.T_final[pix] = Tr[k];
        w.n_contrib[pix] = last[k];
      }
    }
    if (p.stats) flush_stats(w.stats, kFwdSupport, n_sup, n_comp, n_cand);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce-scatter of 8 values over a warp in 9 shuffles: on return lane l holds
// the warp total of value ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1).
__device__ __forceinline__ float warp_reduce_scatter8(const float *v) {
  const int lane = threadIdx.x & 31;
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
  float a[4], b[2];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const float send = h4 ? v[i] : v[i + 4];
    a[i] = (h4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const float send = h3 ? a[i] : a[i + 2];
    b[i] = (h3 ? a[i + 2] : a[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float c = (h2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h2 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

template <int T>
__global__ void __launch_bounds__(TileCfg<T>::NT) k_composite_bwd(Params p, Work w, const float *dimage) {
  using Cfg = TileCfg<T>;
  constexpr int NT = Cfg::NT, NW = Cfg::NW, PPT = Cfg::PPT;
  __shared__ float4 sA[NW][32], sB[NW][32], sC[NW][32];
  __shared__ int sG[NW][32];
  __shared__ int s_bprim[kBCap];
  __shared__ float4 s_brec[kBCap];
  __shared__ int s_tile;
  const float LN2 = 0.69314718055994531f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(w.counters + kQueueBwd, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= p.tiles) break;
    const TileInfo ti = tile_info(p, w, tile, T);
    const int *bprim;
    const float4 *brec;
    load_boundary_cache<NT>(ti, w, s_bprim, s_brec, bprim, brec);
    __syncthreads();
    const unsigned long long *bkeys = w.bkeys + ti.bs;
    const int bn = (int)ti.bn;
    const int wx0 = ti.x0 + (warp % Cfg::WPR) * Cfg::WX, wy0 = ti.y0 + (warp / Cfg::WPR) * Cfg::WY;
    const int wx1 = wx0 + Cfg::WX - 1, wy1 = wy0 + Cfg::WY - 1;

    // R: colour behind the current pair, seen through the pairs behind it
    float Tr[PPT], R[PPT][3], dC[PPT][3];
    int last[PPT], idq[PPT], px[PPT], py[PPT];
    WarpCache<Cfg::NC, true> cache[PPT];
    unsigned n_sup = 0, n_comp = 0, n_cand = 0;
    int mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      int lx, ly;
      lane_pixel<T>(warp, lane, k, lx, ly);
      px[k] = ti.x0 + lx;
      py[k] = ti.y0 + ly;
      last[k] = 0;
      idq[k] = -1;
      Tr[k] = 1.f;
      cache[k].reset();
      R[k][0] = R[k][1] = R[k][2] = 0.f;
      dC[k][0] = dC[k][1] = dC[k][2] = 0.f;
      if (px[k] < ti.W && py[k] < ti.H) {
        const int pix = ti.pix_off + py[k] * ti.W + px[k];
        idq[k] = w.pid[pix];
        last[k] = w.n_contrib[pix];
        Tr[k] = w.T_final[pix];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          dC[k][c] = dimage[3 * (size_t)pix + c];
          R[k][c] = p.bg[c];
        }
      }
      mylast = max(mylast, last[k]);
    }
    int wlast = mylast;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    for (int c1 = wlast; c1 > 0; c1 -= 32) {
      const int c0 = max(0, c1 - 32);
      const int jl = c0 + lane;
      bool hit = false;
      if (jl < c1) {
        const unsigned gi = (unsigned)(w.gkeys[ti.gs + jl] & kIndexMask);
        const float4 A = w.gA[gi];
        hit = covers(A, wx0, wx1, wy0, wy1);
        if (hit) {
          sA[warp][lane] = A;
          sB[warp][lane] = w.gB[gi];
          sC[warp][lane] = w.gC[gi];
          sG[warp][lane] = (int)gi;
        }
      }
      unsigned mask = __ballot_sync(0xffffffffu, hit);
      __syncwarp();
      while (mask) {
        const int l = 31 - __clz(mask);
        mask &= ~(1u << l);
        const int j = c0 + l;
        const float4 A = sA[warp][l], B = sB[warp][l], Cc = sC[warp][l];
        const int g = __float_as_int(Cc.w);
        float acc[9];
#pragma unroll
        for (int q = 0; q < 9; q++) acc[q] = 0.f;
        bool any = false;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
          const PairGeo pg = pair_geo2(px[k], py[k], A, B);
          const float G = __expf(pg.power);
          const float og = __fmul_rn(B.w, G);
          const bool cand = j < last[k] && og >= p.alpha_min;
          if (!__any_sync(0xffffffffu, cand)) continue;
          float wv;
          int bi;
          cache[k].get(g, px[k], py[k], idq[k], bprim, brec, bn, p.use_boundary, wv, bi, n_cand);
          if (!cand) continue;
          n_sup++;
          const float raw = __fmul_rn(og, wv);
          const float alpha = fminf(p.alpha_max, raw);
          if (alpha < p.alpha_min) continue;
          any = true;
          n_comp++;
          const float oma = 1.0f - alpha;
          Tr[k] = __fdividef(Tr[k], oma);  // T_i
          const float ta = Tr[k] * alpha;
          // dl/dalpha_i = dl/dC . (T_i c_i - S_i / (1 - alpha_i)) with
          // S_i / (1 - alpha_i) = T_i R_i, R <- alpha_i c_i + (1 - alpha_i) R:
          // the form T_i (c_i - R_i) avoids amplifying rounding by 1 / (1 - alpha_i)
          float dl_da = 0.f;
          const float col[3] = {Cc.x, Cc.y, Cc.z};
#pragma unroll
          for (int c = 0; c < 3; c++) {
            acc[6 + c] += ta * dC[k][c];
            dl_da += dC[k][c] * (col[c] - R[k][c]);
            R[k][c] = alpha * col[c] + oma * R[k][c];
          }
          dl_da *= Tr[k];
          if (raw >= p.alpha_max) continue;  // clamped: alpha is constant
          acc[5] += dl_da * wv * G;
          const float dl_dw = dl_da * B.w * G;
          const float dl_dpow = dl_da * og * wv;
          const float dx = pg.dx, dy = pg.dy;  // q - mu
          acc[2] += dl_dpow * (-0.5f * dx * dx);
          acc[3] += dl_dpow * (-dx * dy);
          acc[4] += dl_dpow * (-0.5f * dy * dy);
          acc[0] += dl_dpow * (B.x * dx + B.y * dy);
          acc[1] += dl_dpow * (B.y * dx + B.z * dy);
          if (bi >= 0) {
            // rho and gamma of the most influential boundary point, by the
            // same operations as the search
            const float4 b = brec[bi];
            const unsigned qxy = __float_as_uint(b.x);
            const float bx = __fsub_rn((float)(px[k] - (int)(qxy & 0xffffu)), b.y);
            const float by = __fsub_rn((float)(py[k] - (int)(qxy >> 16)), b.z);
            const float r2 = __fmul_rn(__fmaf_rn(bx, bx, __fmul_rn(by, by)), __fmul_rn(b.w, b.w));
            const float rho = __fsqrt_rn(r2);
            const float gam = exp2f(__fsub_rn(rho, 1.0f));
            const float d = sqrtf(bx * bx + by * by);
            if (d > 0.f) {
              const float sgn = (idq[k] == g) ? 1.0f : -1.0f;
              const float dl_drho = sgn * dl_dw * LN2 * gam;
              const float isig = b.w;
              const unsigned bidx = (unsigned)(bkeys[bi] & 0xffffffffull);
              float *gb = reinterpret_cast<float *>(w.bg_grad + bidx);
              atomicAdd(gb + 0, dl_drho * (-bx / d) * isig);
              atomicAdd(gb + 1, dl_drho * (-by / d) * isig);
              atomicAdd(gb + 2, dl_drho * (-rho) * isig);
            }
          }
        }
        if (__any_sync(0xffffffffu, any)) {
          // gradient slots: 0 dmu x, 1 dmu y, 2-4 dK, 5 do, 6-8 dcol; slots 0-7
          // by reduce-scatter (lanes 4m hold slot m), slot 8 by a butterfly
          const float part = warp_reduce_scatter8(acc);
          const float s8 = warp_sum(acc[8]);
          float *gg = w.gg + 12 * (size_t)sG[warp][l];
          const int slot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
          if ((lane & 3) == 0 && part != 0.f) atomicAdd(gg + slot, part);
          if (lane == 1 && s8 != 0.f) atomicAdd(gg + 8, s8);
        }
      }
      __syncwarp();
    }
    if (p.stats) flush_stats(w.stats, kBwdSupport, n_sup, n_comp, n_cand);
  }
}

template <int T>
int launch_fwd_t(const Params &p, const Work &w, float *image, cudaStream_t st, int sms) {
  int grid = p.tiles < sms * 8 ? p.tiles : sms * 8;
  if (grid > 0) k_composite_fwd<T><<<grid, TileCfg<T>::NT, 0, st>>>(p, w, image);
  return grid > 0 ? 1 : 0;
}

template <int T>
int launch_bwd_t(const Params &p, const Work &w, const float *dimage, cudaStream_t st, int sms) {
  int grid = p.tiles < sms * 8 ? p.tiles : sms * 8;
  if (grid > 0) k_composite_bwd<T><<<grid, TileCfg<T>::NT, 0, st>>>(p, w, dimage);
  return grid > 0 ? 1 : 0;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

}  // namespace

int launch_composite_fwd(const Params &p, const Work &w, float *image, cudaStream_t st) {
  cudaMemsetAsync(w.counters + kQueueFwd, 0, sizeof(int), st);
  const int sms = num_sms();
  if (p.tile == 8) return launch_fwd_t<8>(p, w, image, st, sms);
  if (p.tile == 32) return launch_fwd_t<32>(p, w, image, st, sms);
  return launch_fwd_t<16>(p, w, image, st, sms);
}

int launch_composite_bwd(const Params &p, const Work &w, const float *dimage, cudaStream_t st) {
  cudaMemsetAsync(w.counters + kQueueBwd, 0, sizeof(int), st);
  const int sms = num_sms();
  if (p.tile == 8) return launch_bwd_t<8>(p, w, dimage, st, sms);
  if (p.tile == 32) return launch_bwd_t<32>(p, w, dimage, st, sms);
  return launch_bwd_t<16>(p, w, dimage, st, sms);
}

}  // namespace bgt
