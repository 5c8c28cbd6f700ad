// Discontinuity-aware alpha blending, forward and backward (Sec. 3.2, Eq. 6-8;
// supplementary "Backward Derivative").
//
// Forward: persistent CTAs take screen tiles from an atomic queue. The tile's
// boundary list (sorted by primitive, index) is staged once in shared memory;
// each warp owns an 8 x 4 (16 x 8 at tile 32) block of the tile's pixels and
// walks the tile's Gaussian list (sorted by depth, index) in chunks of 32,
// culling each chunk against its block with one ballot. For pixel q and a
// Gaussian of primitive g, w (Eq. 6) is gamma* = min over g's boundary points b
// of gamma(|q - b|; sigma_b) (Eq. 7), w = gamma* if I_id(q) = g else 1 - gamma*;
// a warp-parallel search finds g's range in the boundary list, and a per-warp
// cache keyed by primitive keeps w per pixel for the primitives seen last.
// alpha = min(alpha_max, o w G) (Eq. 8); pairs with alpha < alpha_min are
// skipped; blending stops before the pair that would take T below t_stop.
// Every composited (warp visit, Gaussian) is recorded for the backward pass:
// a header (Gaussian, lane mask of the composited pixels, fill record) and,
// per cache fill, each pixel's most influential boundary point.
//
// Backward: warps take warp blocks from a queue and replay the block's
// records back to front: w is rebuilt from the recorded boundary point with
// the forward's operations, alpha recomputed bit for bit, T_i recovered as
// T_{i+1} / (1 - alpha_i); per-Gaussian gradients (mean, conic, opacity,
// colour) are reduced over the warp before the atomics, per-boundary-point
// gradients (position, radius) summed per (pixel, primitive) in the cache.
#include "bgt_internal.cuh"

namespace bgt {

namespace {

constexpr int kBCap = 1024;        // boundary candidates staged in shared memory per tile
constexpr float kLog2e = 1.4426950408889634f;

// Block layout: NT threads; every warp owns a WX x WY block of the tile's
// pixels (PPT pixels per lane), so that a chunk of 32 listed Gaussians can be
// culled against the warp's block with one ballot.
template <int T>
struct TileCfg {
  static constexpr int NT = (T == 8) ? 64 : 256;
  static constexpr int NW = NT / 32;
  static constexpr int PPT = T * T / NT;     // 1, 1, 4
  static constexpr int WX = (T == 32) ? 16 : 8;
  static constexpr int WY = (T == 32) ? 8 : 4;
  static constexpr int WPR = T / WX;         // warp blocks per tile row
  // primitive cache per warp (fully associative, FIFO): slot keys one per lane
  static constexpr int SLOTS_FWD = (PPT == 1) ? 16 : 8;
  static constexpr int SLOTS_BWD = (PPT == 1) ? 6 : 4;
  // resident blocks per SM the kernels are compiled for (their shared memory
  // allows this many; the register budget follows)
  static constexpr int MINB_FWD = (T == 8) ? 6 : (T == 16) ? 4 : 2;
  static constexpr int MINB_BWD = (T == 8) ? 6 : (T == 16) ? 3 : 2;
};

template <int T>
__device__ __forceinline__ void lane_pixel(int warp, int lane, int k, int &lx, int &ly) {
  using C = TileCfg<T>;
  lx = (warp % C::WPR) * C::WX + (lane & 7) + 8 * (k & 1);
  ly = (warp / C::WPR) * C::WY + (lane >> 3) + 4 * (k >> 1);
}

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Conic (a, b, c) and opacity o of a Gaussian record, with the conic scaled
// for the exponent: (-a/2, -b, -c/2) log2(e), so that G = 2^(a' dx^2 + b' dx dy
// + c' dy^2). Forward and backward stage the same scaled values.
__device__ __forceinline__ float4 scaled_conic(const float4 K) {
  return make_float4(__fmul_rn(K.x, -0.5f * kLog2e), __fmul_rn(K.y, -kLog2e), __fmul_rn(K.z, -0.5f * kLog2e), K.w);
}

// G = exp(-1/2 (a dx^2 + 2 b dx dy + c dy^2)) = 2^(dx (a' dx + b' dy) + c' dy^2)
// for a conic scaled by scaled_conic
__device__ __forceinline__ float gauss(float dx, float dy, const float4 &Qs) {
  const float t = __fmaf_rn(Qs.x, dx, __fmul_rn(Qs.y, dy));
  return ex2(__fmaf_rn(dx, t, __fmul_rn(__fmul_rn(Qs.z, dy), dy)));
}

// A boundary record in the form the search uses, relative to the 32 x 32 pixel
// cell (cx, cy) holding the tile (cells do not depend on the tile size, so
// neither do images): (x, y, 1/sigma^2, 1/sigma) with x = (qx_b - cx) +
// off_x, the first difference exact. For a pixel at (pxr, pyr) = (px - cx,
// py - cy) (exact), q - b = (pxr - x, pyr - y).
__device__ __forceinline__ float4 cell_record(const float4 rec, int cx, int cy) {
  const unsigned qxy = __float_as_uint(rec.x);
  return make_float4(__fadd_rn((float)((int)(qxy & 0xffffu) - cx), rec.y),
                     __fadd_rn((float)((int)(qxy >> 16) - cy), rec.z), __fmul_rn(rec.w, rec.w), rec.w);
}

// the tile's boundary candidates, sorted by (primitive, index)
struct BList {
  const int *prim;
  const float4 *loc;   // cell-relative records in shared memory (if cached)
  const float4 *glob;  // pixel-relative records in global memory
  int n, cx, cy;       // candidates; the cell of the tile
  bool cached;
  __device__ __forceinline__ float4 get(int i) const { return cached ? loc[i] : cell_record(glob[i], cx, cy); }
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One round of a warp-wide search in the sorted prim[a, a + len): 32 evenly
// spaced probes narrow the range holding the first index whose entry fails
// pred (entry < g, or entry <= g) 32-fold.
template <bool LE>
__device__ __forceinline__ void search_round(const int *prim, int g, int &a, int &len) {
  const int lane = threadIdx.x & 31;
  const int step = (len + 31) >> 5, end = a + len;
  const int idx = a + (lane + 1) * step - 1;
  const int v = idx < end ? prim[idx] : 0x7fffffff;
  a += __popc(__ballot_sync(0xffffffffu, LE ? v <= g : v < g)) * step;
  len = min(step, end - a);
}

// [lo, hi): the entries equal to g in the sorted prim[0, n), found by the
// whole warp (g warp-uniform); both bounds are narrowed in the same rounds,
// so n <= 1024 takes two rounds.
__device__ __forceinline__ void warp_equal_range(const int *prim, int n, int g, int &lo, int &hi) {
  const int lane = threadIdx.x & 31;
  int a = 0, la = n, b = 0, lb = n;
  while (la > 32 || lb > 32) {
    if (la > 32) search_round<false>(prim, g, a, la);
    if (lb > 32) search_round<true>(prim, g, b, lb);
  }
  const int va = lane < la ? prim[a + lane] : 0x7fffffff;
  const int vb = lane < lb ? prim[b + lane] : 0x7fffffff;
  lo = a + __popc(__ballot_sync(0xffffffffu, va < g));
  hi = b + __popc(__ballot_sync(0xffffffffu, vb <= g));
}

// |q - b|^2 / sigma^2 of a cell-relative record b at the cell-relative pixel (pxr, pyr)
__device__ __forceinline__ float rec_r2(const float4 &b, float pxr, float pyr) {
  const float dx = __fsub_rn(pxr, b.x), dy = __fsub_rn(pyr, b.y);
  return __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), b.z);
}

// |q - b|^2 / sigma^2 for boundary candidate i at the cell-relative pixel (pxr, pyr)
__device__ __forceinline__ float cand_r2(const BList &bl, int i, float pxr, float pyr) {
  return rec_r2(bl.get(i), pxr, pyr);
}

// gamma = min(2^(rho - 1), 1) (Eq. 7) for rho^2 = r2 < 1
__device__ __forceinline__ float gamma_of(float r2) { return ex2(__fsub_rn(sqrt_approx(r2), 1.0f)); }

// Eq. 6-7 at the cell-relative pixel (pxr, pyr) for primitive g, whose boundary candidates are
// [lo, hi): gamma* = min over g's boundary points of min(2^(rho - 1), 1),
// rho = |q - b| / sigma_b; w = gamma* inside g, 1 - gamma* outside.
// best: the first candidate of least rho if rho < 1, else -1. U candidates
// are evaluated per iteration (instruction-level parallelism vs registers).
template <int U>
__device__ __forceinline__ float w_search(const BList &bl, int lo, int hi, float pxr, float pyr, bool inside,
                                          int &best, unsigned &cands) {
  float r2min = 3.0e38f;
  best = -1;
  for (int i = lo; i < hi; i += U) {
    float r[U];
#pragma unroll
    for (int u = 0; u < U; u++) r[u] = cand_r2(bl, min(i + u, hi - 1), pxr, pyr);
#pragma unroll
    for (int u = 0; u < U; u++)
      if (r[u] < r2min) {  // a repeated last candidate never replaces itself
        r2min = r[u];
        best = min(i + u, hi - 1);
      }
  }
  cands += hi - lo;
  float gamma = 1.0f;
  if (best >= 0 && r2min < 1.0f) gamma = gamma_of(r2min);
  else best = -1;
  return inside ? gamma : __fsub_rn(1.0f, gamma);
}

struct TileInfo {
  int view, W, H, pix_off, x0, y0;
  long long gs, gn, bs, bn;
};

__device__ inline TileInfo tile_info(const Params &p, const Work &w, int tile) {
  TileInfo t;
  const int4 d = w.tile_desc[2 * tile], r = w.tile_desc[2 * tile + 1];
  t.view = d.x;
  t.x0 = d.y & 0xffff;
  t.y0 = (int)((unsigned)d.y >> 16);
  t.W = d.z & 0xffff;
  t.H = (int)((unsigned)d.z >> 16);
  t.pix_off = d.w;
  // an overflowed call (reported through the status word) has empty lists,
  // so that no unwritten key slot is read
  t.gs = r.x;
  t.gn = r.y;
  t.bs = r.z;
  t.bn = r.w;
  return t;
}

template <int NT>
__device__ __forceinline__ BList load_boundary(const TileInfo &ti, const Work &w, int *s_bprim, float4 *s_bloc) {
  BList bl;
  bl.n = (int)ti.bn;
  bl.glob = w.bl_rec + ti.bs;
  bl.cx = ti.x0 & ~31;
  bl.cy = ti.y0 & ~31;
  bl.cached = ti.bn <= kBCap;
  if (bl.cached) {
    for (int i = threadIdx.x; i < ti.bn; i += NT) {
      s_bprim[i] = w.bl_prim[ti.bs + i];
      s_bloc[i] = cell_record(w.bl_rec[ti.bs + i], bl.cx, bl.cy);
    }
  }
  bl.prim = bl.cached ? s_bprim : w.bl_prim + ti.bs;
  bl.loc = s_bloc;
  return bl;
}

// Stage this warp's hits of a chunk of 32 entries of the tile's list (this
// lane's sort key, prefetched, if valid):
// P = (pixel x, y of the Gaussian as exact floats, offset x, y of its mean),
// Q = (conic a, b, c, opacity), C = (colour, bits(prim)). The warp block is
// [bx0, bx1] x [by0, by1] in pixel coordinates. Returns the ballot of hits.
__device__ __forceinline__ unsigned stage_chunk(const Work &w, unsigned long long key, bool valid, float bx0,
                                                float bx1, float by0, float by1, float4 *sP, float4 *sQ, float4 *sC,
                                                int *sG) {
  const int lane = threadIdx.x & 31;
  bool hit = false;
  if (valid) {
    const unsigned gi = (unsigned)(key & kIndexMask);
    const float4 A = w.gA[gi];
    const unsigned qxy = __float_as_uint(A.z);
    const float gx = (float)(int)(qxy & 0xffffu), gy = (float)(int)(qxy >> 16);
    const float cx = gx + A.x, cy = gy + A.y, r = A.w;
    hit = r >= 0.f && cx + r >= bx0 && cx - r <= bx1 && cy + r >= by0 && cy - r <= by1;
    if (hit) {
      sP[lane] = make_float4(gx, gy, A.x, A.y);
      sQ[lane] = scaled_conic(w.gB[gi]);
      sC[lane] = w.gC[gi];
      if (sG) sG[lane] = (int)gi;
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, hit);
  __syncwarp();
  return mask;
}

// per-lane counts a, b, c summed over the warp; d is warp-uniform
__device__ __forceinline__ void flush_stats(unsigned long long *stats, int base, unsigned a, unsigned b, unsigned c,
                                            unsigned d) {
  unsigned long long v[3] = {a, b, c};
#pragma unroll
  for (int q = 0; q < 3; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if ((threadIdx.x & 31) == 0) {
    for (int q = 0; q < 3; q++)
      if (v[q]) atomicAdd(stats + base + q, v[q]);
    if (d) atomicAdd(stats + base + 3, (unsigned long long)d);
  }
}

// shared memory of the blending kernels (dynamic: above the 48 KB static limit)
template <int T>
struct FwdShared {
  using Cfg = TileCfg<T>;
  static constexpr int S = Cfg::SLOTS_FWD;
  float4 sP[Cfg::NW][32], sQ[Cfg::NW][32], sC[Cfg::NW][32];
  float4 s_bloc[kBCap];
  float s_cw[Cfg::NW][S][Cfg::PPT][32];  // cached w per slot and pixel
  int sG[Cfg::NW][32];
  int s_bprim[kBCap];
  int s_tile;
};

template <int T>
struct BwdShared {
  using Cfg = TileCfg<T>;
  static constexpr int S = Cfg::SLOTS_BWD;
  float4 sP[Cfg::NW][32], sQ[Cfg::NW][32], sC[Cfg::NW][32];
  uint4 sH[Cfg::NW][32];                 // staged record headers
  float s_cw[Cfg::NW][S][Cfg::PPT][32];  // w of the slot's primitive per pixel
  int s_cb[Cfg::NW][S][Cfg::PPT][32];    // the slot's boundary candidate per pixel (-1: none)
  float s_cacc[Cfg::NW][S][Cfg::PPT][32];  // sum of dl/dw over the slot's Gaussians per pixel
  // one pixel per lane: per-pair values of the last 16 records (row = record,
  // column = pixel, stride 33) and dl/dC of the warp block's pixels
  static constexpr int TR = (Cfg::PPT == 1) ? 16 : 1;
  float s_sg[Cfg::NW][TR][33];  // s = dl/dalpha w G of the pair (0 if not composited or clamped)
  float s_ta[Cfg::NW][TR][33];  // T alpha of the pair
  float4 s_dc[Cfg::NW][(Cfg::PPT == 1) ? 32 : 1];
};

// Warp-wide lookup of primitive g in the warp's cache: lane s < SLOTS holds
// the key of slot s. Returns the slot, or -1 (warp-uniform) on a miss.
__device__ __forceinline__ int cache_find(int ckey, int g) {
  const unsigned m = __ballot_sync(0xffffffffu, ckey == g);
  return m ? __ffs(m) - 1 : -1;
}

// Writer of the blend records of one warp. Headers are stashed one per lane
// (lane i holds the block's i-th pending header) and stored as one coalesced
// chunk of kRecChunk; fill records come from chunks of kFillChunk units owned
// by the warp across the blocks it blends. Running out of either capacity
// marks the block's records invalid and lists the block for the tile-list
// walk of the backward pass.
struct RecWriter {
  int chunk, last_n;  // the block's last stored header chunk (-1: none) and its headers
  int count;          // pending headers
  uint4 hdr;          // this lane's pending header
  int fill, fill_end; // the warp's current fill units [fill, fill_end)
  bool ok;

  __device__ __forceinline__ void begin_block() {
    chunk = -1;
    last_n = 0;
    count = 0;
    ok = true;
  }

  __device__ __forceinline__ void fail(const Work &) { ok = false; }

  // first unit of a new fill record of `units` planes, or -1
  __device__ __forceinline__ int new_fill(const Work &w, int units) {
    if (!ok) return -1;
    if (fill + units > fill_end) {
      int c = 0;
      if ((threadIdx.x & 31) == 0) c = atomicAdd(w.counters + kFillChunks, 1);
      c = __shfl_sync(0xffffffffu, c, 0);
      if ((long long)(c + 1) * kFillChunk * units > w.fill_unit_cap) {
        fail(w);
        return -1;
      }
      fill = c * kFillChunk * units;
      fill_end = fill + kFillChunk * units;
    }
    const int f = fill;
    fill += units;
    return f;
  }

  __device__ __forceinline__ void flush(const Work &w) {
    const int lane = threadIdx.x & 31;
    if (count == 0 || !ok) return;
    int id = 0;
    if (lane == 0) {
      id = atomicAdd(w.counters + kRecChunks, 1);
      if (id < w.rec_chunk_cap) w.rec_prev[id] = chunk;
    }
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= w.rec_chunk_cap) {
      fail(w);
      return;
    }
    if (lane < count) w.rec_hdr[(size_t)id * kRecChunk + lane] = hdr;
    chunk = id;
    last_n = count;
    count = 0;
  }

  // header: Gaussian gi composited at the pixels k of the lanes in cm; its
  // primitive's fill record starts at unit f
  __device__ __forceinline__ void put(const Work &w, unsigned gi, unsigned cm, int f, int k) {
    if ((threadIdx.x & 31) == count) hdr = make_uint4(gi, cm, (unsigned)f, (unsigned)k);
    if (++count == kRecChunk) flush(w);
  }

  __device__ __forceinline__ void end_block(const Work &w, int blk) {
    flush(w);
    if ((threadIdx.x & 31) == 0) {
      w.blk_rec[blk] = ok ? make_int2(chunk, last_n) : make_int2(-2, 0);
      if (!ok) w.walk_list[atomicAdd(w.counters + kWalkCount, 1)] = blk;
    }
  }
};

// STATS: count the work units of bench.py's roofline (a separate instantiation,
// launched only when profiling, so the production kernel carries no counters)
template <int T, bool STATS>
__global__ void __launch_bounds__(TileCfg<T>::NT, TileCfg<T>::MINB_FWD) k_composite_fwd(Params p, Work w, float *image) {
  using Cfg = TileCfg<T>;
  constexpr int NT = Cfg::NT, PPT = Cfg::PPT, S = Cfg::SLOTS_FWD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &sh = *reinterpret_cast<FwdShared<T> *>(smem_raw);
  auto &s_tile = sh.s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this warp's staging slots and primitive cache (w per slot, plane and lane)
  float4 *sP = sh.sP[warp], *sQ = sh.sQ[warp], *sC = sh.sC[warp];
  int *sG = sh.sG[warp];
  float *cw = &sh.s_cw[warp][0][0][0];
  RecWriter rw;
  rw.fill = rw.fill_end = 0;
  if (threadIdx.x == 0) s_tile = atomicAdd(w.counters + kQueueFwd, 1);
  __syncthreads();
  for (;;) {
    const int tile = s_tile;
    if (tile >= p.tiles) break;
    const TileInfo ti = tile_info(p, w, tile);
    const BList bl = load_boundary<NT>(ti, w, sh.s_bprim, sh.s_bloc);
    __syncthreads();  // boundary list staged, s_tile read by every thread
    // the next tile, fetched while this one is blended
    if (threadIdx.x == 0) s_tile = atomicAdd(w.counters + kQueueFwd, 1);
    // the warp's pixel block
    const int wx = ti.x0 + (warp % Cfg::WPR) * Cfg::WX, wy = ti.y0 + (warp / Cfg::WPR) * Cfg::WY;
    const float bx0 = (float)wx, bx1 = (float)(wx + Cfg::WX - 1);
    const float by0 = (float)wy, by1 = (float)(wy + Cfg::WY - 1);

    float C[PPT][3], Tr[PPT], pxf[PPT], pyf[PPT], pxr[PPT], pyr[PPT];
    int last[PPT], idq[PPT], pix[PPT];
    bool done[PPT];
    unsigned n_sup = 0, n_comp = 0, n_cand = 0, n_visit = 0;
    int ckey = -2, cnext = 0, cfill = -1;  // lane s: primitive and fill record of cache slot s
    rw.begin_block();
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      int lx, ly;
      lane_pixel<T>(warp, lane, k, lx, ly);
      const int px = ti.x0 + lx, py = ti.y0 + ly;
      pxf[k] = (float)px;
      pyf[k] = (float)py;
      pxr[k] = (float)(px - bl.cx);
      pyr[k] = (float)(py - bl.cy);
      const bool inside = px < ti.W && py < ti.H;
      pix[k] = inside ? ti.pix_off + py * ti.W + px : -1;
      done[k] = !inside;
      idq[k] = inside ? w.pid[pix[k]] : -1;
      C[k][0] = C[k][1] = C[k][2] = 0.f;
      Tr[k] = 1.0f;
      last[k] = 0;
    }
    const int gn = (int)ti.gn;
    const unsigned long long *gkeys = w.gkeys + ti.gs;
    unsigned long long knext = lane < gn ? gkeys[lane] : 0ull;
    for (int c0 = 0; c0 < gn; c0 += 32) {
      bool alldone = true;
#pragma unroll
      for (int k = 0; k < PPT; k++) alldone = alldone && done[k];
      if (__all_sync(0xffffffffu, alldone)) break;
      const unsigned long long key = knext;
      if (c0 + 32 + lane < gn) knext = gkeys[c0 + 32 + lane];  // prefetch the next chunk's keys
      unsigned mask = stage_chunk(w, key, c0 + lane < gn, bx0, bx1, by0, by1, sP, sQ, sC, sG);
      while (mask) {
        const int l = __ffs(mask) - 1;
        mask &= mask - 1;
        const float4 P = sP[l], Q = sQ[l];
        float og[PPT];
        bool cand[PPT];
        bool anyc = false;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
          // q - mu: the first difference is exact
          const float dx = __fsub_rn(__fsub_rn(pxf[k], P.x), P.z), dy = __fsub_rn(__fsub_rn(pyf[k], P.y), P.w);
          og[k] = __fmul_rn(Q.w, gauss(dx, dy, Q));
          cand[k] = !done[k] && og[k] >= p.alpha_min;  // w <= 1: else alpha < alpha_min
          anyc = anyc || cand[k];
        }
        if (!__any_sync(0xffffffffu, anyc)) continue;
        if constexpr (STATS) n_visit++;
        const float4 Cc = sC[l];
        const int g = __float_as_int(Cc.w);
        int slot = cache_find(ckey, g);
        if (slot < 0) {  // warp-uniform miss: every lane searches, coherently
          slot = cnext;
          cnext = (cnext + 1 == S) ? 0 : cnext + 1;
          int lo = 0, hi = 0, f = -1;
          if (p.use_boundary) {
            warp_equal_range(bl.prim, bl.n, g, lo, hi);
            // a primitive without boundary points in the tile has w = 1 inside and
            // 0 outside: no fill record (the backward reads -1 the same way)
            if (hi > lo) f = rw.new_fill(w, PPT);
          }
#pragma unroll
          for (int k = 0; k < PPT; k++) {
            int best = -1;
            cw[(slot * PPT + k) * 32 + lane] = p.use_boundary
                ? w_search<2>(bl, lo, hi, pxr[k], pyr[k], idq[k] == g, best, n_cand) : 1.0f;
            if (f >= 0) w.rec_fill[(size_t)(f + k) * 32 + lane] = best;
          }
          if (lane == slot) {
            ckey = g;
            cfill = f;
          }
        }
        // compositing without branches: a pixel composites when it is a
        // candidate, alpha >= alpha_min and T would stay >= t_stop; the pair
        // that would take T below t_stop ends the pixel's list
        bool comp[PPT];
#pragma unroll
        for (int k = 0; k < PPT; k++) {
          const float alpha = fminf(p.alpha_max, __fmul_rn(og[k], cw[(slot * PPT + k) * 32 + lane]));
          const float testT = __fmul_rn(Tr[k], __fsub_rn(1.0f, alpha));
          const bool ok = cand[k] && alpha >= p.alpha_min;
          const bool stop = ok && testT < p.t_stop;
          comp[k] = ok && !stop;
          done[k] = done[k] || stop;
          const float ta = comp[k] ? __fmul_rn(Tr[k], alpha) : 0.0f;
          C[k][0] = __fmaf_rn(ta, Cc.x, C[k][0]);
          C[k][1] = __fmaf_rn(ta, Cc.y, C[k][1]);
          C[k][2] = __fmaf_rn(ta, Cc.z, C[k][2]);
          Tr[k] = comp[k] ? testT : Tr[k];
          last[k] = comp[k] ? c0 + l + 1 : last[k];
          if constexpr (STATS) {
            n_sup += cand[k];
            n_comp += comp[k];
          }
        }
        // record the pixels composited for the backward pass
#pragma unroll
        for (int k = 0; k < PPT; k++) {
          const unsigned cm = __ballot_sync(0xffffffffu, comp[k]);
          if (cm) rw.put(w, (unsigned)sG[l], cm, __shfl_sync(0xffffffffu, cfill, slot), k);
        }
      }
      __syncwarp();
    }
    rw.end_block(w, tile * Cfg::NW + warp);
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      if (pix[k] >= 0) {
        image[3 * (size_t)pix[k] + 0] = __fmaf_rn(Tr[k], p.bg[0], C[k][0]);
        image[3 * (size_t)pix[k] + 1] = __fmaf_rn(Tr[k], p.bg[1], C[k][1]);
        image[3 * (size_t)pix[k] + 2] = __fmaf_rn(Tr[k], p.bg[2], C[k][2]);
        w.T_final[pix[k]] = Tr[k];
        w.n_contrib[pix[k]] = last[k];
      }
    }
    if constexpr (STATS) flush_stats(w.stats, kFwdSupport, n_sup, n_comp, n_cand, n_visit);
    __syncthreads();  // the staged boundary list is free again
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

// Backward of one composited pair (Gaussian with colour Cc at offset (dx, dy)
// of the pixel from its mean, G, og = o G, w, raw = og w, alpha): T_{i+1} ->
// T_i = T_{i+1} / (1 - alpha_i) in Tr, the colour behind the pair R updated
// (R <- R + alpha_i (c_i - R)), and the per-Gaussian sums accumulated in acc:
// with s = dl/dalpha w G (the pair's dl/do), acc[0..4] += s (dx, dy, dx^2,
// dx dy, dy^2), acc[5] += s, acc[6..8] += T_i alpha_i dl/dC (the chain kernel
// turns the moments into dl/dmu = o K (acc0, acc1) and dl/dK = -o/2 (acc2,
// 2 acc3, acc4)). dl/dalpha_i = dl/dC . T_i (c_i - R_i) (the supplementary's
// T_i c_i - S_i / (1 - alpha_i), without the 1 / (1 - alpha_i) amplification
// of rounding). Returns dl/dw (0 when alpha is clamped at alpha_max).
__device__ __forceinline__ float pair_values(float G, float og, float wv, float raw, float alpha, float alpha_max,
                                             const float4 &Cc, const float *dC, float &Tr, float *R, float &sg,
                                             float &ta) {
  Tr = __fdividef(Tr, 1.0f - alpha);  // T_i
  ta = Tr * alpha;
  const float col[3] = {Cc.x, Cc.y, Cc.z};
  float dl_da = 0.f;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const float d = col[c] - R[c];
    dl_da = fmaf(dC[c], d, dl_da);
    R[c] = fmaf(alpha, d, R[c]);
  }
  dl_da *= Tr;
  sg = 0.f;
  if (raw >= alpha_max) return 0.f;  // clamped: alpha is constant
  sg = dl_da * wv * G;
  return dl_da * og;
}

__device__ __forceinline__ void add_pair_sums(float sg, float ta, float dx, float dy, const float *dC, float *acc) {
  const float a = sg * dx, b = sg * dy;
  acc[0] += a;
  acc[1] += b;
  acc[2] = fmaf(a, dx, acc[2]);
  acc[3] = fmaf(a, dy, acc[3]);
  acc[4] = fmaf(b, dy, acc[4]);
  acc[5] += sg;
#pragma unroll
  for (int c = 0; c < 3; c++) acc[6 + c] = fmaf(ta, dC[c], acc[6 + c]);
}

__device__ __forceinline__ float pair_backward(float dx, float dy, float G, float og, float wv, float raw, float alpha,
                                               float alpha_max, const float4 &Cc, const float *dC, float &Tr, float *R,
                                               float *acc) {
  float sg, ta;
  const float dl_dw = pair_values(G, og, wv, raw, alpha, alpha_max, Cc, dC, Tr, R, sg, ta);
  add_pair_sums(sg, ta, dx, dy, dC, acc);
  return dl_dw;
}

// Boundary-point gradient of the cell-relative pixel (pxr, pyr) (cell (cx,
// cy)) and boundary candidate bi of the tile's list, given sum = the pixel's
// dl/dw over Gaussians of the candidate's primitive (inside: the pixel
// belongs to it). w = gamma (inside) or 1 - gamma with gamma = 2^(rho - 1),
// so dl/drho = +-ln2 gamma sum, taken through rho = |q - b| / sigma:
// drho/db = -(q - b) / (|q - b| sigma), drho/dsigma = -rho / sigma. brec and
// bkeys are the tile's boundary list (records in pixel-relative form, keys
// holding the boundary point's index).
__device__ __forceinline__ void boundary_grad(const float4 *brec, const unsigned long long *bkeys, float4 *bg_grad,
                                              int bi, float sum, bool inside, float pxr, float pyr, int cx, int cy) {
  const float LN2 = 0.69314718055994531f;
  if (bi < 0 || sum == 0.f) return;
  // rho and gamma with the operations of the forward search
  const float4 b = cell_record(brec[bi], cx, cy);
  const float isig = b.w;
  const float ex = __fsub_rn(pxr, b.x), ey = __fsub_rn(pyr, b.y);
  const float r2 = __fmul_rn(__fmaf_rn(ex, ex, __fmul_rn(ey, ey)), b.z);
  const float rho = sqrt_approx(r2);
  if (!(rho > 0.f)) return;
  const float gam = gamma_of(r2);
  const float dl_drho = (inside ? LN2 : -LN2) * gam * sum;
  const float s = dl_drho * isig * __frcp_rn(rho);  // (q - b) isig / rho is the unit direction
  const unsigned bidx = (unsigned)(bkeys[bi] & 0xffffffffull);
  float *gb = reinterpret_cast<float *>(bg_grad + bidx);
  atomicAdd(gb + 0, -(ex * isig) * s);
  atomicAdd(gb + 1, -(ey * isig) * s);
  atomicAdd(gb + 2, -dl_drho * rho * isig);
}

// Boundary-point gradients of one cache slot (primitive g): for every pixel
// all of g's Gaussians use the same boundary point, so their dl/dw were
// summed (cacc) before the gradient is taken once per (pixel, slot).
template <int PPT>
__device__ __forceinline__ void flush_boundary(const float4 *brec, const unsigned long long *bkeys, float4 *bg_grad,
                                               const int *cb, const float *cacc, int g, const int *idq,
                                               const float *pxr, const float *pyr, int cx, int cy) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < PPT; k++)
    boundary_grad(brec, bkeys, bg_grad, cb[k * 32 + lane], cacc[k * 32 + lane], idq[k] == g, pxr[k], pyr[k], cx,
                  cy);
}

// w (Eq. 6-7) at the cell-relative pixel (pxr, pyr) for the primitive whose
// most influential boundary point is candidate bi of the tile's list (-1: none
// within rho < 1), with the operations of the forward search, so the value is
// bit-identical
__device__ __forceinline__ float w_from_candidate(const float4 *brec, int bi, float pxr, float pyr, int cx, int cy,
                                                  bool inside) {
  if (bi < 0) return inside ? 1.0f : 0.0f;
  const float gamma = gamma_of(rec_r2(cell_record(brec[bi], cx, cy), pxr, pyr));
  return inside ? gamma : __fsub_rn(1.0f, gamma);
}

// Backward pass over the forward pass's blend records. Every warp takes warp
// blocks (tile, block) from a queue and replays the block's records back to
// front: T_i = T_{i+1} / (1 - alpha_i) with alpha_i recomputed from the
// recorded w by the forward pass's operations, R (colour behind) updated as
// R <- alpha_i c_i + (1 - alpha_i) R. Per record, the per-Gaussian gradient is
// reduced over the warp; boundary-point gradients are summed per (pixel,
// primitive) in a cache slot and flushed on eviction and at the block's end.
template <int T, bool STATS>
__global__ void __launch_bounds__(TileCfg<T>::NT, TileCfg<T>::MINB_BWD) k_composite_bwd(Params p, Work w, const float *dimage) {
  using Cfg = TileCfg<T>;
  constexpr int PPT = Cfg::PPT, S = Cfg::SLOTS_BWD, NW = Cfg::NW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &sh = *reinterpret_cast<BwdShared<T> *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4 *sP = sh.sP[warp], *sQ = sh.sQ[warp], *sC = sh.sC[warp];
  uint4 *sH = sh.sH[warp];
  auto &s_cw = sh.s_cw[warp];
  auto &s_cb = sh.s_cb[warp];
  auto &s_cacc = sh.s_cacc[warp];
  const int items = p.tiles * NW;
  const int deq = p.bwd_dequeue;  // warp blocks per dequeue
  int base = 0;
  if (lane == 0) base = atomicAdd(w.counters + kQueueBwd, deq);
  base = __shfl_sync(0xffffffffu, base, 0);
  while (base < items) {
    int next = 0;  // the next warp blocks, fetched while these are processed
    if (lane == 0) next = atomicAdd(w.counters + kQueueBwd, deq);
    const int end = min(base + deq, items);
    for (int item = base; item < end; item++) {
      const int tile = item / NW, wb = item - tile * NW;
      const int4 d = w.tile_desc[2 * tile];
      const int x0 = d.y & 0xffff, y0 = (int)((unsigned)d.y >> 16);
      const int W = d.z & 0xffff, H = (int)((unsigned)d.z >> 16);
      const long long bs = w.tile_desc[2 * tile + 1].z;
      const float4 *brec = w.bl_rec + bs;
      const unsigned long long *bkeys = w.bkeys + bs;
      const int2 br = w.blk_rec[item];

      const int cx = x0 & ~31, cy = y0 & ~31;  // the tile's cell (boundary records are cell-relative)
      float Tr[PPT], R[PPT][3], dC[PPT][3], pxf[PPT], pyf[PPT], pxr[PPT], pyr[PPT];
      int idq[PPT];
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        int lx, ly;
        lane_pixel<T>(wb, lane, k, lx, ly);
        const int px = x0 + lx, py = y0 + ly;
        pxf[k] = (float)px;
        pyf[k] = (float)py;
        pxr[k] = (float)(px - cx);
        pyr[k] = (float)(py - cy);
        idq[k] = -1;
        Tr[k] = 1.f;
        R[k][0] = R[k][1] = R[k][2] = 0.f;
        dC[k][0] = dC[k][1] = dC[k][2] = 0.f;
        if (br.x >= 0 && px < W && py < H) {
          const int pix = d.w + py * W + px;
          idq[k] = w.pid[pix];
          Tr[k] = w.T_final[pix];
#pragma unroll
          for (int c = 0; c < 3; c++) {
            dC[k][c] = dimage[3 * (size_t)pix + c];
            R[k][c] = p.bg[c];
          }
        }
      }
      unsigned n_comp = 0, n_rec = 0;
      int ckey = -2, cnext = 0;
      int chunk = br.x, n = br.y;
      // one pixel per lane: the block origin and dl/dC of every pixel, for the
      // per-Gaussian sums taken record by record over the block's pixels
      const float wx0 = (float)(x0 + (wb % Cfg::WPR) * Cfg::WX), wy0 = (float)(y0 + (wb / Cfg::WPR) * Cfg::WY);
      if constexpr (PPT == 1) sh.s_dc[warp][lane] = make_float4(dC[0][0], dC[0][1], dC[0][2], 0.f);
      while (chunk >= 0) {
        const int prev = w.rec_prev[chunk];
        // stage the chunk's records: headers and their Gaussians
        if (lane < n) {
          const uint4 h = w.rec_hdr[(size_t)chunk * kRecChunk + lane];
          const float4 A = w.gA[h.x];
          const unsigned qxy = __float_as_uint(A.z);
          sH[lane] = h;
          sP[lane] = make_float4((float)(int)(qxy & 0xffffu), (float)(int)(qxy >> 16), A.x, A.y);
          sQ[lane] = scaled_conic(w.gB[h.x]);
          sC[lane] = w.gC[h.x];
        }
        __syncwarp();
        for (int r = n - 1; r >= 0; r--) {
          const uint4 h = sH[r];
          const bool mine = (h.y >> lane) & 1u;
          const int rk = (int)h.w;
          const float4 P = sP[r], Q = sQ[r], Cc = sC[r];
          const int g = __float_as_int(Cc.w);
          if constexpr (STATS) n_rec++;
          // w of (pixel, g): from the cache slot, filled from g's fill record
          int slot = 0;
          if (p.use_boundary) {
            slot = cache_find(ckey, g);
            if (slot < 0) {  // warp-uniform miss: flush the evicted slot, take in g
              slot = cnext;
              cnext = (cnext + 1 == S) ? 0 : cnext + 1;
              const int old = __shfl_sync(0xffffffffu, ckey, slot);
              if (old >= 0)
                flush_boundary<PPT>(brec, bkeys, w.bg_grad, &s_cb[slot][0][0], &s_cacc[slot][0][0], old, idq, pxr,
                                    pyr, cx, cy);
#pragma unroll
              for (int k = 0; k < PPT; k++) {
                const int bi = (int)h.z >= 0 ? w.rec_fill[(size_t)((int)h.z + k) * 32 + lane] : -1;
                s_cw[slot][k][lane] = w_from_candidate(brec, bi, pxr[k], pyr[k], cx, cy, idq[k] == g);
                s_cb[slot][k][lane] = bi;
                s_cacc[slot][k][lane] = 0.f;
              }
              if (lane == slot) ckey = g;
            }
          }
          if constexpr (PPT == 1) {
            // the pair's values go to row r % 16 of the warp's transposition rows;
            // every 16 records, lane i (and i + 16, for the other half of the
            // pixels) sums record i's values over the block's pixels: the
            // per-Gaussian sums without a warp reduction per record
            float sg = 0.f, ta = 0.f, dl_dw = 0.f;
            if (mine) {
              if constexpr (STATS) n_comp++;
              const float dx = __fsub_rn(__fsub_rn(pxf[0], P.x), P.z), dy = __fsub_rn(__fsub_rn(pyf[0], P.y), P.w);
              const float G = gauss(dx, dy, Q);
              const float og = __fmul_rn(Q.w, G);
              const float wv = p.use_boundary ? s_cw[slot][0][lane] : 1.0f;
              const float raw = __fmul_rn(og, wv);
              const float alpha = fminf(p.alpha_max, raw);
              dl_dw = pair_values(G, og, wv, raw, alpha, p.alpha_max, Cc, dC[0], Tr[0], R[0], sg, ta);
              if (p.use_boundary) s_cacc[slot][0][lane] += dl_dw;
            }
            sh.s_sg[warp][r & 15][lane] = sg;
            sh.s_ta[warp][r & 15][lane] = ta;
            if ((r & 15) == 0) {
              __syncwarp();
              const int i = lane & 15, half = lane >> 4, rec = r + i;
              float acc[9];
#pragma unroll
              for (int q = 0; q < 9; q++) acc[q] = 0.f;
              if (rec < n) {
                const float4 Pm = sP[rec];
                const float bxm = __fsub_rn(__fsub_rn(wx0, Pm.x), Pm.z), bym = __fsub_rn(__fsub_rn(wy0, Pm.y), Pm.w);
#pragma unroll
                for (int j = 0; j < 16; j++) {
                  const int l = half * 16 + j;
                  const float4 dc = sh.s_dc[warp][l];
                  const float dcv[3] = {dc.x, dc.y, dc.z};
                  add_pair_sums(sh.s_sg[warp][i][l], sh.s_ta[warp][i][l], bxm + (float)(l & 7), bym + (float)(l >> 3),
                                dcv, acc);
                }
              }
#pragma unroll
              for (int q = 0; q < 9; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 16);
              if (rec < n && half == 0) {
                float *gg = w.gg + 12 * (size_t)sH[rec].x;
#pragma unroll
                for (int q = 0; q < 9; q++)
                  if (acc[q] != 0.f) atomicAdd(gg + q, acc[q]);
              }
              __syncwarp();
            }
          } else {
            float acc[9];
#pragma unroll
            for (int q = 0; q < 9; q++) acc[q] = 0.f;
            float dl_dw = 0.f;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
              if (k != rk || !mine) continue;
              if constexpr (STATS) n_comp++;
              const float dx = __fsub_rn(__fsub_rn(pxf[k], P.x), P.z), dy = __fsub_rn(__fsub_rn(pyf[k], P.y), P.w);
              const float G = gauss(dx, dy, Q);
              const float og = __fmul_rn(Q.w, G);
              const float wv = p.use_boundary ? s_cw[slot][k][lane] : 1.0f;
              const float raw = __fmul_rn(og, wv);
              const float alpha = fminf(p.alpha_max, raw);
              dl_dw = pair_backward(dx, dy, G, og, wv, raw, alpha, p.alpha_max, Cc, dC[k], Tr[k], R[k], acc);
            }
            if (p.use_boundary && mine) s_cacc[slot][rk][lane] += dl_dw;
            // per-Gaussian sums (see pair_backward); slots 0-7 by reduce-scatter
            // (lanes 4m hold slot m), slot 8 by a butterfly
            const float part = warp_reduce_scatter8(acc);
            const float s8 = warp_sum(acc[8]);
            float *gg = w.gg + 12 * (size_t)h.x;
            const int gslot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
            if ((lane & 3) == 0 && part != 0.f) atomicAdd(gg + gslot, part);
            if (lane == 1 && s8 != 0.f) atomicAdd(gg + 8, s8);
          }
        }
        __syncwarp();
        chunk = prev;
        n = kRecChunk;
      }
      if (p.use_boundary) {
        for (int sl = 0; sl < S; sl++) {
          const int old = __shfl_sync(0xffffffffu, ckey, sl);
          if (old >= 0)
            flush_boundary<PPT>(brec, bkeys, w.bg_grad, &s_cb[sl][0][0], &s_cacc[sl][0][0], old, idq, pxr, pyr, cx,
                                cy);
        }
      }
      if constexpr (STATS) flush_stats(w.stats, kBwdSupport, n_comp, n_comp, 0u, n_rec);
    }
    base = __shfl_sync(0xffffffffu, next, 0);
  }
}

// Backward pass of the warp blocks whose blend records did not fit (listed
// by the forward pass): each warp re-walks its block's tile list back to
// front from the last composited entry of its pixels. Every decision of the
// forward (support, w by the same Eq. 6 search over the tile's boundary
// list, alpha, the alpha_min cut) is retaken with the forward's operations,
// so exactly the forward's composited pairs are visited; T_i = T_{i+1} /
// (1 - alpha_i) and the gradients follow as in the record replay. As in the
// forward, the list is staged 32 entries at a time and culled against the
// warp's block with one ballot, and w of (pixel, primitive) is kept per
// primitive in a small per-warp cache (the same search, so the same values).
// Boundary gradients are added per pair (the most influential boundary point
// of the pair's search).
template <int T>
__global__ void __launch_bounds__(TileCfg<T>::NT) k_composite_bwd_walk(Params p, Work w, const float *dimage) {
  using Cfg = TileCfg<T>;
  constexpr int PPT = Cfg::PPT, NW = Cfg::NW;
  constexpr int kWalkSlots = PPT == 1 ? 8 : 2;  // primitive cache slots per warp (static shared memory)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ float4 s_P[NW][32], s_Q[NW][32], s_C[NW][32];
  __shared__ int s_G[NW][32];
  __shared__ float s_ww[NW][kWalkSlots][PPT][32];  // w of the slot's primitive per pixel
  __shared__ int s_wb[NW][kWalkSlots][PPT][32];    // its most influential boundary candidate
  float4 *sP = s_P[warp], *sQ = s_Q[warp], *sC = s_C[warp];
  int *sG = s_G[warp];
  const int nwalk = w.counters[kWalkCount];
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(w.counters + kQueueWalk, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= nwalk) break;
    const int item = w.walk_list[q];
    const int tile = item / NW, wb = item - tile * NW;
    const TileInfo ti = tile_info(p, w, tile);
    BList bl;
    bl.n = (int)ti.bn;
    bl.glob = w.bl_rec + ti.bs;
    bl.cx = ti.x0 & ~31;
    bl.cy = ti.y0 & ~31;
    bl.cached = false;
    bl.prim = w.bl_prim + ti.bs;
    bl.loc = nullptr;
    const float4 *brec = w.bl_rec + ti.bs;
    const unsigned long long *bkeys = w.bkeys + ti.bs;
    float Tr[PPT], R[PPT][3], dC[PPT][3], pxf[PPT], pyf[PPT], pxr[PPT], pyr[PPT];
    int idq[PPT], nlast[PPT];
    int emax = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      int lx, ly;
      lane_pixel<T>(wb, lane, k, lx, ly);
      const int px = ti.x0 + lx, py = ti.y0 + ly;
      pxf[k] = (float)px;
      pyf[k] = (float)py;
      pxr[k] = (float)(px - bl.cx);
      pyr[k] = (float)(py - bl.cy);
      idq[k] = -1;
      nlast[k] = 0;
      Tr[k] = 1.f;
      R[k][0] = R[k][1] = R[k][2] = 0.f;
      dC[k][0] = dC[k][1] = dC[k][2] = 0.f;
      if (px < ti.W && py < ti.H) {
        const int pix = ti.pix_off + py * ti.W + px;
        idq[k] = w.pid[pix];
        Tr[k] = w.T_final[pix];
        nlast[k] = w.n_contrib[pix];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          dC[k][c] = dimage[3 * (size_t)pix + c];
          R[k][c] = p.bg[c];
        }
      }
      emax = max(emax, nlast[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    const unsigned long long *gkeys = w.gkeys + ti.gs;
    // the warp's pixel block: entries whose support box misses it have no
    // candidate pixel there (the box holds every pixel with o G >= alpha_min)
    const int wx = ti.x0 + (wb % Cfg::WPR) * Cfg::WX, wy = ti.y0 + (wb / Cfg::WPR) * Cfg::WY;
    const float bx0 = (float)wx, bx1 = (float)(wx + Cfg::WX - 1);
    const float by0 = (float)wy, by1 = (float)(wy + Cfg::WY - 1);
    int ckey = -2, cnext = 0;  // lane s: primitive of cache slot s (w and best per pixel in shared memory)
    for (int c0 = ((emax - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
      const bool valid = c0 + lane < emax;
      unsigned mask = stage_chunk(w, valid ? gkeys[c0 + lane] : 0ull, valid, bx0, bx1, by0, by1, sP, sQ, sC, sG);
      while (mask) {  // back to front
      const int l = 31 - __clz(mask);
      mask &= ~(1u << l);
      const int e = c0 + l;
      const unsigned gi = (unsigned)sG[l];
      const float4 P = sP[l], Q = sQ[l], Cc = sC[l];
      const int g = __float_as_int(Cc.w);
      float og[PPT], Gk[PPT];
      bool cand[PPT];
      bool anyc = false;
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        const float dx = __fsub_rn(__fsub_rn(pxf[k], P.x), P.z), dy = __fsub_rn(__fsub_rn(pyf[k], P.y), P.w);
        Gk[k] = gauss(dx, dy, Q);
        og[k] = __fmul_rn(Q.w, Gk[k]);
        cand[k] = e < nlast[k] && og[k] >= p.alpha_min;
        anyc = anyc || cand[k];
      }
      if (!__any_sync(0xffffffffu, anyc)) continue;
      // w of (pixel, g) by the forward's search, kept per primitive in a cache slot
      int slot = 0;
      if (p.use_boundary) {
        slot = cache_find(ckey, g);
        if (slot < 0) {
          slot = cnext;
          cnext = (cnext + 1 == kWalkSlots) ? 0 : cnext + 1;
          int lo = 0, hi = 0;
          warp_equal_range(bl.prim, bl.n, g, lo, hi);
#pragma unroll
          for (int k = 0; k < PPT; k++) {
            int best = -1;
            unsigned ncand = 0;
            s_ww[warp][slot][k][lane] = w_search<2>(bl, lo, hi, pxr[k], pyr[k], idq[k] == g, best, ncand);
            s_wb[warp][slot][k][lane] = best;
          }
          if (lane == slot) ckey = g;
          __syncwarp();
        }
      }
      float acc[9];
#pragma unroll
      for (int c = 0; c < 9; c++) acc[c] = 0.f;
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        const int best = p.use_boundary ? s_wb[warp][slot][k][lane] : -1;
        const float wv = p.use_boundary ? s_ww[warp][slot][k][lane] : 1.0f;
        if (!cand[k]) continue;
        const float raw = __fmul_rn(og[k], wv);
        const float alpha = fminf(p.alpha_max, raw);
        if (alpha < p.alpha_min) continue;
        const float dx = __fsub_rn(__fsub_rn(pxf[k], P.x), P.z), dy = __fsub_rn(__fsub_rn(pyf[k], P.y), P.w);
        const float dl_dw = pair_backward(dx, dy, Gk[k], og[k], wv, raw, alpha, p.alpha_max, Cc, dC[k], Tr[k], R[k], acc);
        if (p.use_boundary)
          boundary_grad(brec, bkeys, w.bg_grad, best, dl_dw, idq[k] == g, pxr[k], pyr[k], bl.cx, bl.cy);
      }
      const float part = warp_reduce_scatter8(acc);
      const float s8 = warp_sum(acc[8]);
      float *gg = w.gg + 12 * (size_t)gi;
      const int gslot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
      if ((lane & 3) == 0 && part != 0.f) atomicAdd(gg + gslot, part);
      if (lane == 1 && s8 != 0.f) atomicAdd(gg + 8, s8);
      }
      __syncwarp();
    }
  }
}

template <int T>
int launch_fwd_t(const Params &p, const Work &w, float *image, cudaStream_t st, int sms) {
  int grid = p.tiles < sms * 8 ? p.tiles : sms * 8;
  if (grid > 0) {
    if (p.stats) k_composite_fwd<T, true><<<grid, TileCfg<T>::NT, sizeof(FwdShared<T>), st>>>(p, w, image);
    else k_composite_fwd<T, false><<<grid, TileCfg<T>::NT, sizeof(FwdShared<T>), st>>>(p, w, image);
  }
  return grid > 0 ? 1 : 0;
}

template <int T>
int launch_bwd_t(const Params &p, const Work &w, const float *dimage, cudaStream_t st, int sms) {
  int grid = p.tiles < sms * 8 ? p.tiles : sms * 8;
  if (grid > 0) {
    if (p.stats) k_composite_bwd<T, true><<<grid, TileCfg<T>::NT, sizeof(BwdShared<T>), st>>>(p, w, dimage);
    else k_composite_bwd<T, false><<<grid, TileCfg<T>::NT, sizeof(BwdShared<T>), st>>>(p, w, dimage);
    // warp blocks whose records overflowed (none in the common case: the
    // kernel reads the count and returns)
    k_composite_bwd_walk<T><<<sms * 3, TileCfg<T>::NT, 0, st>>>(p, w, dimage);  // 3 blocks per SM by registers
  }
  return grid > 0 ? 2 : 0;
}

template <int T, bool STATS>
cudaError_t configure_ts() {
  cudaError_t e = cudaFuncSetAttribute(k_composite_fwd<T, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(FwdShared<T>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_composite_bwd<T, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BwdShared<T>));
  return e;
}

template <int T>
cudaError_t configure_t() {
  cudaError_t e = configure_ts<T, false>();
  return e == cudaSuccess ? configure_ts<T, true>() : e;
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

cudaError_t configure_composite() {
  cudaError_t e = configure_t<8>();
  if (e == cudaSuccess) e = configure_t<16>();
  if (e == cudaSuccess) e = configure_t<32>();
  return e;
}

int launch_composite_fwd(const Params &p, const Work &w, float *image, cudaStream_t st) {
  cudaMemsetAsync(w.counters + kQueueFwd, 0, sizeof(int), st);
  const int sms = num_sms();
  if (p.tile == 8) return launch_fwd_t<8>(p, w, image, st, sms);
  if (p.tile == 32) return launch_fwd_t<32>(p, w, image, st, sms);
  return launch_fwd_t<16>(p, w, image, st, sms);
}

int launch_composite_bwd(const Params &p, const Work &w, const float *dimage, cudaStream_t st) {
  cudaMemsetAsync(w.counters + kQueueBwd, 0, sizeof(int), st);
  cudaMemsetAsync(w.counters + kQueueWalk, 0, sizeof(int), st);
  const int sms = num_sms();
  if (p.tile == 8) return launch_bwd_t<8>(p, w, dimage, st, sms);
  if (p.tile == 32) return launch_bwd_t<32>(p, w, dimage, st, sms);
  return launch_bwd_t<16>(p, w, dimage, st, sms);
}

}  // namespace bgt
