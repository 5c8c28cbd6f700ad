// Sub-primitive generation (Sec. 3.2, "Sub-Primitive Generation") and the
// boundary points of discontinuity-aware blending (same section, first
// paragraph of "Discontinuity-Aware Alpha Blending").
//
// For every foreground pixel q (I_id(q) = g >= 0) one Gaussian is placed at
// S_q = S(I_uv(q)) of primitive g (Eq. 3) with colour c_q (Eq. 4), the
// primitive's rotation / scale (Eq. 5 at attribute-map resolution 1) and the
// primitive's opacity; it is projected with the EWA approximation (J W
// Sigma3D W^T J^T + dilation) as in 3DGS. Pixels of B (a 4-neighbour with a
// different id) also yield a boundary point b = projection of the same S_q
// with radius sigma = k_b fx r_b / z.
//
// Gaussians and boundary points are compacted in global pixel order: a count
// pass per warp chunk of 128 pixels, exclusive scans of the chunk counts, a
// compaction pass in which every warp writes its chunk's foreground pixels
// (pixel, view, boundary index) at their ranks with ballots, and the
// generation pass with one thread per Gaussian; indices do not depend on
// scheduling. Each record counts its screen tiles into per-tile counters for
// the binning pass.
#include <algorithm>

#include "bgt_internal.cuh"

namespace bgt {

namespace {

constexpr int kGenThreads = 256;
constexpr int kGenRounds = 4;                  // pixels per lane: a warp chunk covers 128 pixels
constexpr int kChunk = 32 * kGenRounds;
constexpr int kGenWarps = kGenThreads / 32;

// A warp chunk of kChunk pixels from `first`: its view when the whole chunk
// lies in one view (the usual case: one search and one division per chunk),
// with the view's size and the column and row of `first`; view = -1 otherwise.
struct ChunkPos {
  int view, W, H, x0, y0;
};

__device__ inline ChunkPos chunk_pos(const Params &p, const Work &w, int first) {
  ChunkPos c{-1, 1, 1, 0, 0};
  if (first >= p.P) return c;
  const int v = find_view(w.view_pix_off, p.V, first);
  if (min(first + kChunk, p.P) > __ldg(w.view_pix_off + v + 1)) return c;
  c.view = v;
  c.W = __ldg(&w.views[v].W);
  c.H = __ldg(&w.views[v].H);
  const int local = first - __ldg(w.view_pix_off + v);
  c.y0 = local / c.W;
  c.x0 = local - c.y0 * c.W;
  return c;
}

// foreground / boundary flags of global pixel `pix`, the k-th of its chunk
__device__ inline void pixel_flags(const Params &p, const Work &w, int pix, int k, const ChunkPos &cp, bool &fg,
                                   bool &bnd, int &view) {
  fg = false;
  bnd = false;
  view = 0;
  if (pix >= p.P) return;
  int W, H, x, y;
  if (cp.view >= 0) {
    view = cp.view;
    W = cp.W;
    H = cp.H;
    x = cp.x0 + k;
    y = cp.y0;
    if (x >= W) {  // the chunk wraps to the following row(s)
      y += x / W;
      x -= (x / W) * W;
    }
  } else {
    view = find_view(w.view_pix_off, p.V, pix);
    W = __ldg(&w.views[view].W);
    H = __ldg(&w.views[view].H);
    const int local = pix - __ldg(w.view_pix_off + view);
    y = local / W;
    x = local - y * W;
  }
  // the pixel and its 4-neighbours, loaded together (clamped to the pixel
  // itself where a neighbour lies outside the view)
  const int id = w.pid[pix];
  const int il = w.pid[x > 0 ? pix - 1 : pix], ir = w.pid[x < W - 1 ? pix + 1 : pix];
  const int iu = w.pid[y > 0 ? pix - W : pix], idn = w.pid[y < H - 1 ? pix + W : pix];
  fg = id >= 0;
  bnd = fg && (il != id || ir != id || iu != id || idn != id);
}

// foreground and boundary pixels of each warp chunk of 128 pixels
__global__ void __launch_bounds__(kGenThreads) k_count(Params p, Work w) {
  const int lane = threadIdx.x & 31;
  const int chunk = blockIdx.x * kGenWarps + (threadIdx.x >> 5);
  if (chunk >= w.nblk) return;
  int cf = 0, cb = 0;
  const ChunkPos cp = chunk_pos(p, w, chunk * kChunk);
#pragma unroll
  for (int r = 0; r < kGenRounds; r++) {
    bool fg, bnd;
    int view;
    pixel_flags(p, w, chunk * kChunk + r * 32 + lane, r * 32 + lane, cp, fg, bnd, view);
    cf += __popc(__ballot_sync(0xffffffffu, fg));
    cb += __popc(__ballot_sync(0xffffffffu, bnd));
  }
  if (lane == 0) {
    w.blk_cnt[chunk] = cf;
    w.blk_cnt[w.nblk + chunk] = cb;
  }
}

// F and Nb: the totals of the two chunk scans
__global__ void k_totals(Work w) {
  w.counters[kF] = (int)w.blk_off[w.nblk];
  w.counters[kNb] = (int)w.blk_off[2 * w.nblk + 1];
}

// one count per tile of the rect; the active lanes of the warp that count the
// same tile add their counts with one atomic (consecutive Gaussians mostly
// share tiles)
__device__ inline void count_tiles(int *cnt, int tile_off, int tiles_x, uint2 rect) {
  const int lane = threadIdx.x & 31;
  const int x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff, y1 = rect.y >> 16;
  for (int ty = y0; ty <= y1; ty++)
    for (int tx = x0; tx <= x1; tx++) {
      const int t = tile_off + ty * tiles_x + tx;
      const unsigned peers = __match_any_sync(__activemask(), t);
      if (lane == __ffs(peers) - 1) atomicAdd(cnt + t, __popc(peers));
    }
}

// tile rect of the pixel box [cx - rx, cx + rx] x [cy - ry, cy + ry]; empty -> x0 > x1
__device__ inline uint2 tile_rect(float cx, float cy, float rx, float ry, const View &vw, int t) {
  int x0 = (int)ceilf(cx - rx), x1 = (int)floorf(cx + rx);
  int y0 = (int)ceilf(cy - ry), y1 = (int)floorf(cy + ry);
  x0 = max(x0, 0); y0 = max(y0, 0);
  x1 = min(x1, vw.W - 1); y1 = min(y1, vw.H - 1);
  if (x0 > x1 || y0 > y1) return make_uint2(1u, 0u);  // x0 = 1 > x1 = 0: empty
  x0 /= t; x1 /= t; y0 /= t; y1 /= t;
  return make_uint2((unsigned)x0 | ((unsigned)y0 << 16), (unsigned)x1 | ((unsigned)y1 << 16));
}

// compaction: each warp writes its chunk's foreground pixels at their ranks in
// pixel order (the Gaussian and boundary indices)
__global__ void __launch_bounds__(kGenThreads) k_compact(Params p, Work w) {
  const int lane = threadIdx.x & 31;
  const int chunk = blockIdx.x * kGenWarps + (threadIdx.x >> 5);
  if (chunk >= w.nblk) return;
  int nf = (int)w.blk_off[chunk];
  int nb = (int)w.blk_off[w.nblk + 1 + chunk];
  const unsigned lt = (1u << lane) - 1u;
  const ChunkPos cp = chunk_pos(p, w, chunk * kChunk);
#pragma unroll
  for (int r = 0; r < kGenRounds; r++) {
    const int pix = chunk * kChunk + r * 32 + lane;
    bool fg, bnd;
    int view;
    pixel_flags(p, w, pix, r * 32 + lane, cp, fg, bnd, view);
    const unsigned mf = __ballot_sync(0xffffffffu, fg), mb = __ballot_sync(0xffffffffu, bnd);
    const int gi = nf + __popc(mf & lt);
    if (pix < p.P) w.pix_gidx[pix] = fg ? gi : -1;
    if (fg) {
      w.g_pix[gi] = pix;
      w.g_view[gi] = view;
      w.g_bidx[gi] = bnd ? nb + __popc(mb & lt) : -1;
      w.g_prim[gi] = w.pid[pix];
      w.g_uv[gi] = w.puv[pix];
    }
    nf += __popc(mf);
    nb += __popc(mb);
  }
}

// one thread per Gaussian (sub-primitive) and boundary point
template <int N>
__global__ void __launch_bounds__(kGenThreads) k_generate(Params p, Scene s, Work w) {
  const int F = w.counters[kF];
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < F; gi += gridDim.x * blockDim.x) {
    const int pix = w.g_pix[gi], view = w.g_view[gi], bi = w.g_bidx[gi], prim = w.g_prim[gi];
    const float2 uv = w.g_uv[gi];
    const bool bnd = bi >= 0;
    const View vw = w.views[view];
    const int local = pix - vw.pix_off;
    const int qy = local / vw.W, qx = local - qy * vw.W;
    const float *cp = s.ctrl + (size_t)prim * p.ncp * 3;
    SurfPoint<N> sp;
    surface_point<N>(cp, uv.x, uv.y, vw, sp);
    const float2 off = project_offset(sp.t, vw, qx, qy);
    const float tx = sp.t[0].hi + sp.t[0].lo, ty = sp.t[1].hi + sp.t[1].lo, tz = sp.t[2].hi + sp.t[2].lo;
    // depth sort key refinement: the exact depth hi + lo lies in the rounding
    // interval of tz; its position there, in 1/32 ulp, extends the FP32 bits
    // by 5 monotone bits (|lo| <= ulp / 2 maps to 0..31)
    unsigned char dsub = 16;
    {
      const df z = df_fast_two_sum(sp.t[2].hi, sp.t[2].lo);
      const float r = __fsub_rn(z.hi, tz) + z.lo;  // exact depth minus tz
      const float ulp = __int_as_float(__float_as_int(tz) & 0x7f800000) * 1.1920928955078125e-7f;
      if (ulp > 0.f) {
        const float c = floorf(r / ulp * 32.0f) + 16.0f;
        dsub = (unsigned char)fminf(fmaxf(c, 0.0f), 31.0f);
      }
    }
    // EWA: T = J W, Sigma2D = T Sigma3D T^T + dilation I
    const float iz = 1.0f / tz;
    const float j00 = vw.fx * iz, j02 = -vw.fx * tx * iz * iz;
    const float j11 = vw.fy * iz, j12 = -vw.fy * ty * iz * iz;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      T0[k] = j00 * vw.R[k] + j02 * vw.R[6 + k];
      T1[k] = j11 * vw.R[3 + k] + j12 * vw.R[6 + k];
    }
    // Sigma3D from the attribute maps interpolated at I_uv (Eq. 5); maps of leg
    // resolution 1 hold one texel, so Sigma3D is the primitive's
    float S3[6];
    if (p.attr_res == 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) S3[k] = w.prim_cov[6 * (size_t)prim + k];
    } else {
      float qa[4], ls[3], Rm[9], sc3[3], tw[3];
      int tex[3];
      gauss_attrs(s.quat, s.log_scale, p.attr_res, p.ntex, prim, uv.x, uv.y, qa, ls, tex, tw);
      cov3d_f32(qa, ls, S3, Rm, sc3);
    }
    const float Sxx = S3[0], Sxy = S3[1], Sxz = S3[2], Syy = S3[3], Syz = S3[4], Szz = S3[5];
    const float a0 = T0[0] * Sxx + T0[1] * Sxy + T0[2] * Sxz;
    const float a1 = T0[0] * Sxy + T0[1] * Syy + T0[2] * Syz;
    const float a2 = T0[0] * Sxz + T0[1] * Syz + T0[2] * Szz;
    const float b0 = T1[0] * Sxx + T1[1] * Sxy + T1[2] * Sxz;
    const float b1 = T1[0] * Sxy + T1[1] * Syy + T1[2] * Syz;
    const float b2 = T1[0] * Sxz + T1[1] * Syz + T1[2] * Szz;
    const float cA = a0 * T0[0] + a1 * T0[1] + a2 * T0[2] + p.dilation;
    const float cB = a0 * T1[0] + a1 * T1[1] + a2 * T1[2];
    const float cC = b0 * T1[0] + b1 * T1[1] + b2 * T1[2] + p.dilation;
    const float det = cA * cC - cB * cB;
    const float idet = 1.0f / det;
    const float Ka = cC * idet, Kb = -cB * idet, Kc = cA * idet;
    float col[3] = {0.f, 0.f, 0.f};
    const float *cc = s.color + (size_t)prim * p.ncp * 3;
#pragma unroll
    for (int a = 0; a < SurfPoint<N>::M; a++) {
      col[0] = fmaf(sp.B[a], __ldg(cc + 3 * a + 0), col[0]);
      col[1] = fmaf(sp.B[a], __ldg(cc + 3 * a + 1), col[1]);
      col[2] = fmaf(sp.B[a], __ldg(cc + 3 * a + 2), col[2]);
    }
    const float o = __ldg(s.opacity + prim);
    const bool finite = isfinite(off.x) && isfinite(off.y) && isfinite(Ka) && isfinite(Kb) &&
                        isfinite(Kc) && det > 0.f && tz > 0.f;
    if (!finite) atomicOr(w.status, kStatusNonFinite);
    uint2 rect = make_uint2(1u, 0u);
    float rsup = -1.0f;
    if (finite && o > p.alpha_min) {
      // support {o G >= alpha_min} lies in the box |dx| <= sqrt(lvl Sigma_xx),
      // |dy| <= sqrt(lvl Sigma_yy), lvl = 2 ln(o / alpha_min); widened slightly
      const float lvl = 2.0f * (logf(o) - p.log_alpha_min);
      const float rx = sqrtf(lvl * cA) * 1.0001f + 1e-3f;
      const float ry = sqrtf(lvl * cC) * 1.0001f + 1e-3f;
      rsup = fmaxf(rx, ry);
      rect = tile_rect((float)qx + off.x, (float)qy + off.y, rx, ry, vw, p.tile);
      if ((rect.x & 0xffff) <= (rect.y & 0xffff)) count_tiles(w.g_tcount, vw.tile_off, vw.tiles_x, rect);
    }
    const unsigned qxy = (unsigned)qx | ((unsigned)qy << 16);
    w.gA[gi] = make_float4(off.x, off.y, __uint_as_float(qxy), rsup);
    w.gB[gi] = make_float4(Ka, Kb, Kc, o);
    w.gC[gi] = make_float4(col[0], col[1], col[2], __int_as_float(prim));
    w.g_depth[gi] = tz;
    w.g_rect[gi] = rect;
    w.g_dsub[gi] = dsub;
    float4 *ggz = reinterpret_cast<float4 *>(w.gg + 12 * (size_t)gi);
    ggz[0] = ggz[1] = ggz[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!bnd) continue;
    // boundary point: the same surface point, radius sigma = k_b fx r_b / z
    const float sigma = p.k_b * vw.fx * __ldg(s.r_b + prim) / tz;
    uint2 brect = make_uint2(1u, 0u);
    if (finite && sigma > 0.f && isfinite(sigma)) {
      const float rr = sigma * 1.0001f + 1e-3f;
      brect = tile_rect((float)qx + off.x, (float)qy + off.y, rr, rr, vw, p.tile);
      if ((brect.x & 0xffff) <= (brect.y & 0xffff)) count_tiles(w.b_tcount, vw.tile_off, vw.tiles_x, brect);
    }
    w.bR[bi] = make_float4(__uint_as_float(qxy), off.x, off.y, 1.0f / sigma);
    w.b_pix[bi] = pix;
    w.b_prim[bi] = prim;
    w.b_view[bi] = view;
    w.b_uv[bi] = uv;
    w.b_sigma[bi] = sigma;
    w.b_z[bi] = tz;
    w.b_rect[bi] = brect;
    w.bg_grad[bi] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

}  // namespace

// View-dependent colour (SH bands 1..D of the primitive) added to the diffuse
// colour of every Gaussian, at the direction from the camera centre to S_q
// (R^T t in world coordinates, t the camera-space point of Eq. 3)
template <int N>
__global__ void __launch_bounds__(256) k_sh_color(Params p, Scene s, Work w) {
  const int F = w.counters[kF];
  constexpr int m = SurfPoint<N>::M;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F; i += gridDim.x * blockDim.x) {
    float4 C = w.gC[i];
    const int g = __float_as_int(C.w);
    const View &vw = w.views[w.g_view[i]];
    const float2 uv = w.g_uv[i];
    float B[m], S[3] = {0.f, 0.f, 0.f};
    bernstein_f32<N>(uv.x, uv.y, B);
    const float *cp = s.ctrl + (size_t)g * m * 3;
#pragma unroll
    for (int a = 0; a < m; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) S[c] = fmaf(B[a], __ldg(cp + 3 * a + c), S[c]);
    float t[3], dv[3];
#pragma unroll
    for (int r = 0; r < 3; r++) t[r] = vw.R[3 * r] * S[0] + vw.R[3 * r + 1] * S[1] + vw.R[3 * r + 2] * S[2] + vw.t[r];
#pragma unroll
    for (int k = 0; k < 3; k++) dv[k] = vw.R[k] * t[0] + vw.R[3 + k] * t[1] + vw.R[6 + k] * t[2];
    const float inv = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    float Y[15];
    sh_eval(p.sh_deg, dv[0] * inv, dv[1] * inv, dv[2] * inv, Y);
    const float *shp = s.sh + (size_t)g * p.sh_k * 3;
#pragma unroll
    for (int k = 0; k < 15; k++) {
      if (k >= p.sh_k) break;
      C.x = fmaf(Y[k], __ldg(shp + 3 * k + 0), C.x);
      C.y = fmaf(Y[k], __ldg(shp + 3 * k + 1), C.y);
      C.z = fmaf(Y[k], __ldg(shp + 3 * k + 2), C.z);
    }
    w.gC[i] = C;
  }
}

// Sigma3D of every primitive whose rotation / scaling maps hold one texel
// (leg resolution 1), shared by its Gaussians
__global__ void k_prim_cov(Params p, Scene s, Work w) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= p.M) return;
  float qa[4], ls[3], Rm[9], sc3[3], S3[6];
#pragma unroll
  for (int k = 0; k < 4; k++) qa[k] = s.quat[4 * (size_t)m + k];
#pragma unroll
  for (int k = 0; k < 3; k++) ls[k] = s.log_scale[3 * (size_t)m + k];
  cov3d_f32(qa, ls, S3, Rm, sc3);
#pragma unroll
  for (int k = 0; k < 6; k++) w.prim_cov[6 * (size_t)m + k] = S3[k];
}

int launch_prim_cov(const Params &p, const Scene &s, const Work &w, cudaStream_t st) {
  if (p.attr_res != 1 || p.M == 0) return 0;
  k_prim_cov<<<(p.M + 255) / 256, 256, 0, st>>>(p, s, w);
  return 1;
}

int launch_generate(const Params &p, const Scene &s, const Work &w, cudaStream_t st) {
  const int nchunk = (p.P + kChunk - 1) / kChunk;
  if (nchunk == 0) {
    cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), st);
    return 0;
  }
  Work wc = w;
  wc.nblk = nchunk;  // chunks of this call (the arrays hold the capacity's)
  const int blocks = (nchunk + kGenWarps - 1) / kGenWarps;
  k_count<<<blocks, kGenThreads, 0, st>>>(p, wc);
  int k = 1;
  k += launch_exclusive_scan(wc.blk_cnt, wc.blk_off, nchunk, wc.scan_aux, st);
  k += launch_exclusive_scan(wc.blk_cnt + nchunk, wc.blk_off + nchunk + 1, nchunk, wc.scan_aux2, st);
  k_totals<<<1, 1, 0, st>>>(wc);
  k_compact<<<blocks, kGenThreads, 0, st>>>(p, wc);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one thread per Gaussian over a persistent grid (F is known on the device only)
  const int gblocks = std::min((p.P + kGenThreads - 1) / kGenThreads, (sms > 0 ? sms : 152) * 8);
  dispatch_degree(p.n, [&](auto d) { k_generate<decltype(d)::value><<<gblocks, kGenThreads, 0, st>>>(p, s, wc); });
  k += 3;
  if (p.sh_deg > 0) {
    dispatch_degree(p.n, [&](auto d) { k_sh_color<decltype(d)::value><<<152 * 8, 256, 0, st>>>(p, s, w); });
    k++;
  }
  return k;
}

}  // namespace bgt
