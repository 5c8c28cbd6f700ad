// Chain rule from the per-Gaussian and per-boundary-point gradients of the
// blending pass to the primitive parameters (supplementary "Backward
// Derivative": dl/dp_ijk = dl/dS_q B_ijk(I_uv(q)); the projection and EWA
// factors that the paper leaves to 3DGS are derived here).
//
// Gaussian of primitive g at S_q, camera point t = W S_q + t_cam:
//   mean  mu = (fx tx/tz + cx, fy ty/tz + cy)
//   conic K = Sigma2D^-1, Sigma2D = (J W) Sigma3D (J W)^T + dilation I
//   dl/dSigma2D = -K (dl/dK) K, dl/d(JW) = 2 dl/dSigma2D (JW) Sigma3D,
//   dl/dJ = dl/d(JW) W^T, J depends on t; dl/dS_q = W^T dl/dt.
// Boundary point b = projection of S_b, sigma = k_b fx r_b / z_b.
// Two passes take these to the primitives: pass one (one thread per Gaussian,
// one per boundary point) computes dl/dS_q and the other per-record
// gradients and writes them, with the record's (u, v), into its primitive's
// segment of a record array (segments from a count and a scan over the
// primitives); pass two sums each primitive's records with their Bernstein
// weights. A primitive covers a few pixels of a view, so records in pixel
// order change primitive every two or so; grouped, a primitive's records of
// all views are contiguous and its sums take a few atomics instead of one
// per short run and value.
#include <cstdint>

#include "bgt_internal.cuh"

namespace bgt {

namespace {

template <int N>
__device__ inline void camera_point_f32(const float *cp, float u, float v, const View &vw, float *B, float *t) {
  bernstein_f32<N>(u, v, B);
  float S[3] = {0.f, 0.f, 0.f};
  constexpr int m = SurfPoint<N>::M;
#pragma unroll
  for (int a = 0; a < m; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) S[c] = fmaf(B[a], __ldg(cp + 3 * a + c), S[c]);
#pragma unroll
  for (int r = 0; r < 3; r++) t[r] = vw.R[3 * r] * S[0] + vw.R[3 * r + 1] * S[1] + vw.R[3 * r + 2] * S[2] + vw.t[r];
}

// Per-primitive sums of NV values per lane over the warp's runs of lanes with
// equal key (the primitive; -1 for lanes with nothing to add), one atomic per
// (run, value): each lane writes its values to its row of the warp's shared
// memory `sw` (32 rows of NV | 1 floats: the odd stride keeps the row writes
// and the column reads free of bank conflicts), then lane j adds column j
// over the rows of each run and adds the sum to dst(key, j).
template <int NV, class Dst>
__device__ __forceinline__ void scatter_runs(float *sw, const float *v, int key, Dst dst) {
  constexpr int NS = NV | 1;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; j++) sw[lane * NS + j] = v[j];
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
  __syncwarp();
  while (heads) {
    const int start = __ffs(heads) - 1;
    heads &= heads - 1;
    const int end = heads ? __ffs(heads) - 1 : 32;
    const int g = __shfl_sync(0xffffffffu, key, start);
    if (g < 0) continue;
    for (int j = lane; j < NV; j += 32) {
      float sum = 0.f;
      for (int r = start; r < end; r++) sum += sw[r * NS + j];
      if (sum != 0.f) atomicAdd(dst(g, j), sum);
    }
  }
  __syncwarp();
}

constexpr int kChainWarps = 8;
constexpr int kStagedViews = 64;  // cameras a chain block keeps in shared memory

// the call's first kStagedViews cameras copied to shared memory, so that a
// thread reads the fields it uses instead of holding a 128-byte View in
// registers; returns how many were staged
__device__ inline int stage_views(const Params &p, const Work &w, View *s_views) {
  const int nsv = p.V < kStagedViews ? p.V : kStagedViews;
  for (int v = threadIdx.x; v < nsv * (int)(sizeof(View) / 4); v += blockDim.x)
    reinterpret_cast<int *>(s_views)[v] = reinterpret_cast<const int *>(w.views)[v];
  __syncthreads();
  return nsv;
}

template <int N>
__global__ void __launch_bounds__(256) k_chain_gauss(Params p, Scene s, Work w, Grads out) {
  constexpr int m = SurfPoint<N>::M;
  __shared__ View s_views[kStagedViews];
  const int nsv = stage_views(p, w, s_views);
  const int F = w.counters[kF];
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < F; base += warps_total * 32) {
    const int i = base + lane;
    bool active = i < F;
    int g = -1;
    float gS[3] = {0.f, 0.f, 0.f}, gcol[3] = {0.f, 0.f, 0.f}, gop = 0.f;
    float gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};  // map gradients (interpolated attrs)
    float gc6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dl/dSigma3D (xx xy xz yy yz zz), leg resolution 1
    int tex[3] = {0, 0, 0};
    float tw[3] = {0.f, 0.f, 0.f};
    float B[m];
    float2 uv = make_float2(0.f, 0.f);
    if (active) {
      const float *gg = w.gg + 12 * (size_t)i;
      const float4 q0 = reinterpret_cast<const float4 *>(gg)[0];
      const float4 q1 = reinterpret_cast<const float4 *>(gg)[1];
      const float4 q2 = reinterpret_cast<const float4 *>(gg)[2];
      const float4 Bq = w.gB[i];
      const float sums[9] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x};
      float gd[9];
      gauss_grad_from_sums(sums, Bq, gd);
      const float gmx = gd[0], gmy = gd[1], gKa = gd[2], gKb = gd[3], gKc = gd[4];
      gop = gd[5];
      gcol[0] = gd[6]; gcol[1] = gd[7]; gcol[2] = gd[8];
      g = w.g_prim[i];
      const int vi = w.g_view[i];
      const View &vw = vi < nsv ? s_views[vi] : w.views[vi];
      uv = w.g_uv[i];
      float t[3];
      camera_point_f32<N>(s.ctrl + (size_t)g * m * 3, uv.x, uv.y, vw, B, t);
      const bool any = gmx != 0.f || gmy != 0.f || gKa != 0.f || gKb != 0.f || gKc != 0.f;
      if (any) {
        const float Ka = Bq.x, Kb = Bq.y, Kc = Bq.z;
        const float tx = t[0], ty = t[1], tz = t[2];
        const float iz = 1.0f / tz, iz2 = iz * iz;
        // dl/dSigma2D = -K GK K, GK = [[gKa, gKb/2], [gKb/2, gKc]]
        const float hb = 0.5f * gKb;
        const float a00 = Ka * gKa + Kb * hb, a01 = Ka * hb + Kb * gKc;
        const float a10 = Kb * gKa + Kc * hb, a11 = Kb * hb + Kc * gKc;
        const float GS00 = -(a00 * Ka + a01 * Kb);
        const float GS01 = -0.5f * ((a00 * Kb + a01 * Kc) + (a10 * Ka + a11 * Kb));
        const float GS11 = -(a10 * Kb + a11 * Kc);
        const float j00 = vw.fx * iz, j02 = -vw.fx * tx * iz2;
        const float j11 = vw.fy * iz, j12 = -vw.fy * ty * iz2;
        float T0[3], T1[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
          T0[k] = j00 * vw.R[k] + j02 * vw.R[6 + k];
          T1[k] = j11 * vw.R[3 + k] + j12 * vw.R[6 + k];
        }
        // Sigma3D from the attribute maps at I_uv (Eq. 5), as in the forward
        // (the primitive's own with maps of leg resolution 1)
        float qa[4], lsa[3], Rm[9], sc3[3], S3[6];
        if (p.attr_res == 1) {
#pragma unroll
          for (int k = 0; k < 6; k++) S3[k] = w.prim_cov[6 * (size_t)g + k];
        } else {
          gauss_attrs(s.quat, s.log_scale, p.attr_res, p.ntex, g, uv.x, uv.y, qa, lsa, tex, tw);
          cov3d_f32(qa, lsa, S3, Rm, sc3);
        }
        const float Sg[9] = {S3[0], S3[1], S3[2], S3[1], S3[3], S3[4], S3[2], S3[4], S3[5]};
        if (out.log_scale || out.quat) {
          // dl/dSigma3D = T^T dl/dSigma2D T (symmetric): summed per primitive
          // for maps of leg resolution 1 (taken to the texel once per
          // primitive), else through the Gaussian's interpolated attributes
          float G3[9];
#pragma unroll
          for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++)
              G3[3 * a + b] = GS00 * T0[a] * T0[b] + GS01 * (T0[a] * T1[b] + T1[a] * T0[b]) + GS11 * T1[a] * T1[b];
          if (p.attr_res == 1) {
            gc6[0] = G3[0]; gc6[1] = G3[1]; gc6[2] = G3[2]; gc6[3] = G3[4]; gc6[4] = G3[5]; gc6[5] = G3[8];
          } else {
            cov_grad_to_attrs(qa, G3, Rm, sc3, gls, gq);
          }
        }
        float TS0[3], TS1[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
          TS0[k] = T0[0] * Sg[k] + T0[1] * Sg[3 + k] + T0[2] * Sg[6 + k];
          TS1[k] = T1[0] * Sg[k] + T1[1] * Sg[3 + k] + T1[2] * Sg[6 + k];
        }
        float GT0[3], GT1[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
          GT0[k] = 2.0f * (GS00 * TS0[k] + GS01 * TS1[k]);
          GT1[k] = 2.0f * (GS01 * TS0[k] + GS11 * TS1[k]);
        }
        // dl/dJ = dl/dT W^T (only the entries J00, J02, J11, J12 vary with t)
        const float GJ00 = GT0[0] * vw.R[0] + GT0[1] * vw.R[1] + GT0[2] * vw.R[2];
        const float GJ02 = GT0[0] * vw.R[6] + GT0[1] * vw.R[7] + GT0[2] * vw.R[8];
        const float GJ11 = GT1[0] * vw.R[3] + GT1[1] * vw.R[4] + GT1[2] * vw.R[5];
        const float GJ12 = GT1[0] * vw.R[6] + GT1[1] * vw.R[7] + GT1[2] * vw.R[8];
        float gt0 = GJ02 * (-vw.fx * iz2);
        float gt1 = GJ12 * (-vw.fy * iz2);
        float gt2 = GJ00 * (-vw.fx * iz2) + GJ02 * (2.0f * vw.fx * tx * iz2 * iz) +
                    GJ11 * (-vw.fy * iz2) + GJ12 * (2.0f * vw.fy * ty * iz2 * iz);
        gt0 += gmx * vw.fx * iz;
        gt1 += gmy * vw.fy * iz;
        gt2 += -gmx * vw.fx * tx * iz2 - gmy * vw.fy * ty * iz2;
#pragma unroll
        for (int k = 0; k < 3; k++) gS[k] = vw.R[k] * gt0 + vw.R[3 + k] * gt1 + vw.R[6 + k] * gt2;
      }
    }
    const bool per_prim_cov = p.attr_res == 1 && (out.log_scale || out.quat);
    // the Gaussian's record in its primitive's segment (the per-primitive sum
    // takes it to the control points, colour control points and opacity)
    if (active) {
      const unsigned peers = __match_any_sync(__activemask(), g);
      const int leader = __ffs(peers) - 1;
      int b0 = 0;
      if (lane == leader) b0 = atomicAdd(w.prim_gcnt + g, __popc(peers));
      b0 = __shfl_sync(peers, b0, leader);
      float4 *r = w.pg_rec + 4 * (w.prim_gseg[g] + b0 + __popc(peers & ((1u << lane) - 1u)));
      r[0] = make_float4(gS[0], gS[1], gS[2], gop);
      r[1] = make_float4(gcol[0], gcol[1], gcol[2], uv.x);
      r[2] = make_float4(uv.y, gc6[0], gc6[1], gc6[2]);
      r[3] = make_float4(gc6[3], gc6[4], gc6[5], __int_as_float(g));
    }
    if ((out.log_scale || out.quat) && !per_prim_cov) {
      // the map texels of the interpolation, with their weights; runs of equal
      // (primitive, texel) are summed before one atomic each
      const bool nm = active && (gls[0] != 0.f || gls[1] != 0.f || gls[2] != 0.f || gq[0] != 0.f ||
                                 gq[1] != 0.f || gq[2] != 0.f || gq[3] != 0.f);
#pragma unroll
      for (int e = 0; e < 3; e++) {
        const bool on = nm && tw[e] != 0.f;
        if (!__any_sync(0xffffffffu, on)) continue;
        const int t = g * p.ntex + tex[e];
        const Seg st = seg_info(on ? t : -1 - lane);
        if (out.log_scale)
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const float v = seg_sum(on ? tw[e] * gls[c] : 0.f, st);
            if (st.tail && on && v != 0.f) atomicAdd(out.log_scale + 3 * (size_t)t + c, v);
          }
        if (out.quat)
#pragma unroll
          for (int c = 0; c < 4; c++) {
            const float v = seg_sum(on ? tw[e] * gq[c] : 0.f, st);
            if (st.tail && on && v != 0.f) atomicAdd(out.quat + 4 * (size_t)t + c, v);
          }
      }
    }
  }
}

// View-dependent colour (SH bands 1..D, one coefficient set per primitive):
// dl/dk = Y(d) dl/dc summed per primitive, and the direction d = v / |v|,
// v = R^T t from the camera centre to S_q, moves with S_q:
// dl/dv = (I - d d^T) / |v| sum_k (sum_c dl/dc_c k_kc) grad Y_k(d), taken to
// the control points with the Bernstein weights (Eq. 3).
template <int N>
__global__ void __launch_bounds__(256) k_chain_sh(Params p, Scene s, Work w, Grads out) {
  __shared__ float s_rows[kChainWarps][32 * ((3 * SurfPoint<N>::M) | 1)];
  float *sw = s_rows[threadIdx.x >> 5];
  const int F = w.counters[kF];
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  constexpr int m = SurfPoint<N>::M;
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < F; base += warps_total * 32) {
    const int i = base + lane;
    const bool active = i < F;
    int g = -1;
    float gS[3] = {0.f, 0.f, 0.f}, gcol[3] = {0.f, 0.f, 0.f}, Y[15], B[m];
    if (active) {
      const float *gg = w.gg + 12 * (size_t)i;
      gcol[0] = gg[6];
      gcol[1] = gg[7];
      gcol[2] = gg[8];
      g = w.g_prim[i];
      const View vw = w.views[w.g_view[i]];
      const float2 uv = w.g_uv[i];
      float t[3], dv[3];
      camera_point_f32<N>(s.ctrl + (size_t)g * m * 3, uv.x, uv.y, vw, B, t);
#pragma unroll
      for (int k = 0; k < 3; k++) dv[k] = vw.R[k] * t[0] + vw.R[3 + k] * t[1] + vw.R[6 + k] * t[2];
      const float inv = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
      const float d0 = dv[0] * inv, d1 = dv[1] * inv, d2 = dv[2] * inv;
      sh_eval(p.sh_deg, d0, d1, d2, Y);
      const float *shp = s.sh + (size_t)g * p.sh_k * 3;
      float wk[15];
#pragma unroll
      for (int k = 0; k < 15; k++) {
        wk[k] = 0.f;
        if (k < p.sh_k)
          wk[k] = gcol[0] * __ldg(shp + 3 * k) + gcol[1] * __ldg(shp + 3 * k + 1) + gcol[2] * __ldg(shp + 3 * k + 2);
      }
      float gd[3];
      sh_grad(p.sh_deg, d0, d1, d2, wk, gd);
      const float dot = d0 * gd[0] + d1 * gd[1] + d2 * gd[2];
      gS[0] = (gd[0] - d0 * dot) * inv;
      gS[1] = (gd[1] - d1 * dot) * inv;
      gS[2] = (gd[2] - d2 * dot) * inv;
    }
    const bool nz = active && (gcol[0] != 0.f || gcol[1] != 0.f || gcol[2] != 0.f);
    if (!__any_sync(0xffffffffu, nz)) continue;
    {
      float v[3 * m];
#pragma unroll
      for (int a = 0; a < m; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[3 * a + c] = nz ? B[a] * gS[c] : 0.f;
      float *gctrl = out.ctrl;
      scatter_runs<3 * m>(sw, v, nz ? g : -1, [&](int gg, int j) { return gctrl + (size_t)gg * 3 * m + j; });
    }
    const Seg sg = seg_info(nz ? g : -1 - lane);
    if (out.sh) {
#pragma unroll
      for (int k = 0; k < 15; k++) {
        if (k >= p.sh_k) break;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const float v = seg_sum(nz ? Y[k] * gcol[c] : 0.f, sg);
          if (sg.tail && nz && v != 0.f) atomicAdd(out.sh + ((size_t)g * p.sh_k + k) * 3 + c, v);
        }
      }
    }
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_chain_bnd(Params p, Scene s, Work w, Grads out) {
  constexpr int m = SurfPoint<N>::M;
  __shared__ View s_views[kStagedViews];
  const int nsv = stage_views(p, w, s_views);
  const int Nb = w.counters[kNb];
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < Nb; base += warps_total * 32) {
    const int i = base + lane;
    if (i >= Nb) continue;
    const int g = w.b_prim[i];
    const float2 uv = w.b_uv[i];
    float gS[3] = {0.f, 0.f, 0.f}, grb = 0.f;
    const float4 gb = w.bg_grad[i];
    if (gb.x != 0.f || gb.y != 0.f || gb.z != 0.f) {
      const int vi = w.b_view[i];
      const View &vw = vi < nsv ? s_views[vi] : w.views[vi];
      float t[3], B[m];
      camera_point_f32<N>(s.ctrl + (size_t)g * m * 3, uv.x, uv.y, vw, B, t);
      const float tz = w.b_z[i], sigma = w.b_sigma[i];
      const float iz = 1.0f / tz, iz2 = iz * iz;
      const float gt0 = gb.x * vw.fx * iz;
      const float gt1 = gb.y * vw.fy * iz;
      const float gt2 = -gb.x * vw.fx * t[0] * iz2 - gb.y * vw.fy * t[1] * iz2 - gb.z * sigma * iz;
      grb = gb.z * p.k_b * vw.fx * iz;
#pragma unroll
      for (int k = 0; k < 3; k++) gS[k] = vw.R[k] * gt0 + vw.R[3 + k] * gt1 + vw.R[6 + k] * gt2;
    }
    // the boundary point's record in its primitive's segment
    const unsigned peers = __match_any_sync(__activemask(), g);
    const int leader = __ffs(peers) - 1;
    int b0 = 0;
    if (lane == leader) b0 = atomicAdd(w.prim_bcnt + g, __popc(peers));
    b0 = __shfl_sync(peers, b0, leader);
    float4 *r = w.pb_rec + 2 * (w.prim_bseg[g] + b0 + __popc(peers & ((1u << lane) - 1u)));
    r[0] = make_float4(gS[0], gS[1], gS[2], grb);
    r[1] = make_float4(uv.x, uv.y, __int_as_float(g), 0.f);
  }
}

// records per primitive: its Gaussians and its boundary points; the lanes of
// a warp with the same primitive add their count with one atomic
__global__ void k_prim_count(Work w) {
  const int F = w.counters[kF], Nb = w.counters[kNb];
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F + Nb; i += stride) {
    const bool gs = i < F;
    const int g = gs ? w.g_prim[i] : w.b_prim[i - F];
    const unsigned peers = __match_any_sync(__activemask(), gs ? g : -1 - g);
    if (lane == __ffs(peers) - 1) atomicAdd((gs ? w.prim_gcnt : w.prim_bcnt) + g, __popc(peers));
  }
}

constexpr int kSumCols = 15;   // staged row: dl/dS (3), dl/do, dl/dc (3), dl/dSigma3D (6), dl/dr_b, primitive
constexpr int kSumChunk = 256; // records per work item of the per-primitive sums

// Per-primitive sums of the records, which pass one left grouped by primitive:
// dl/dp_a = sum_q B_a(u_q, v_q) dl/dS_q over the primitive's Gaussians and
// boundary points (Eq. 3, supplementary), dl/dc_a = sum B_a dl/dc_q (Eq. 4),
// dl/do, dl/dr_b and dl/dSigma3D as plain sums. Warps take chunks of
// kSumChunk records (Gaussian records, then boundary records) and stage 32 at
// a time in shared memory with their Bernstein weights; lane j owns outputs
// j, j + 32, ... (3m control-point, 3m colour values, opacity, r_b, 6
// Sigma3D) and sums them along the run of the current primitive, adding the
// run's sum with one atomic when the primitive changes and at the chunk's end.
template <int N>
__global__ void __launch_bounds__(256) k_prim_sum(Params p, Work w, Grads out, int with_cov) {
  constexpr int m = SurfPoint<N>::M;
  constexpr int RS = (kSumCols + m) | 1;  // row stride (odd: conflict-free row writes)
  constexpr int NO = 6 * m + 8;           // outputs
  constexpr int NQ = (NO + 31) / 32;
  __shared__ float s_rows[kChainWarps][32 * RS];
  float *rows = s_rows[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int F = w.counters[kF], Nb = w.counters[kNb];
  // this lane's outputs: value column, Bernstein column (-1: weight 1) and destination
  int vcol[NQ], bcol[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    const int j = q * 32 + lane;
    vcol[q] = -1;
    bcol[q] = -1;
    if (j < 3 * m) {
      vcol[q] = j % 3;
      bcol[q] = kSumCols + j / 3;
    } else if (j < 6 * m) {
      vcol[q] = 4 + (j - 3 * m) % 3;
      bcol[q] = kSumCols + (j - 3 * m) / 3;
    } else if (j == 6 * m) {
      vcol[q] = 3;
    } else if (j == 6 * m + 1) {
      vcol[q] = 13;
    } else if (j < NO && with_cov) {
      vcol[q] = 7 + (j - 6 * m - 2);
    }
  }
  auto flush = [&](int g, const float *acc) {
#pragma unroll
    for (int q = 0; q < NQ; q++) {
      const int j = q * 32 + lane;
      if (vcol[q] < 0 || acc[q] == 0.f) continue;
      float *dst = j < 3 * m ? out.ctrl + (size_t)g * 3 * m + j
                   : j < 6 * m ? out.color + (size_t)g * 3 * m + (j - 3 * m)
                   : j == 6 * m ? out.opacity + g
                   : j == 6 * m + 1 ? out.r_b + g
                   : w.prim_gcov + 6 * (size_t)g + (j - 6 * m - 2);
      atomicAdd(dst, acc[q]);
    }
  };
  const long long ng = (F + kSumChunk - 1) / kSumChunk, nchunks = ng + (Nb + kSumChunk - 1) / kSumChunk;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (long long ck = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ck < nchunks; ck += warps_total) {
    const bool bnd = ck >= ng;
    const long long r0 = (bnd ? ck - ng : ck) * kSumChunk;
    const long long r1 = min(r0 + kSumChunk, (long long)(bnd ? Nb : F));
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] = 0.f;
    int gcur = -1;
    // this lane's record of the round, loaded one round ahead
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra, rd = ra;
    auto load = [&](long long c) {
      if (c + lane < r1) {
        if (!bnd) {
          const float4 *r = w.pg_rec + 4 * (c + lane);
          ra = r[0]; rb = r[1]; rc = r[2]; rd = r[3];
        } else {
          const float4 *r = w.pb_rec + 2 * (c + lane);
          ra = r[0]; rb = r[1];
        }
      }
    };
    load(r0);
    for (long long c0 = r0; c0 < r1; c0 += 32) {
      float *row = rows + lane * RS;
      float val[kSumCols];
#pragma unroll
      for (int k = 0; k < kSumCols; k++) val[k] = 0.f;
      float u = 0.f, v = 0.f;
      if (c0 + lane < r1) {
        if (!bnd) {
          val[0] = ra.x; val[1] = ra.y; val[2] = ra.z; val[3] = ra.w;
          val[4] = rb.x; val[5] = rb.y; val[6] = rb.z;
          val[7] = rc.y; val[8] = rc.z; val[9] = rc.w;
          val[10] = rd.x; val[11] = rd.y; val[12] = rd.z; val[14] = rd.w;
          u = rb.w;
          v = rc.x;
        } else {
          val[0] = ra.x; val[1] = ra.y; val[2] = ra.z; val[13] = ra.w; val[14] = rb.z;
          u = rb.x;
          v = rb.y;
        }
      }
      load(c0 + 32);
      float B[m];
      bernstein_f32<N>(u, v, B);
#pragma unroll
      for (int k = 0; k < kSumCols; k++) row[k] = val[k];
#pragma unroll
      for (int a = 0; a < m; a++) row[kSumCols + a] = B[a];
      const int nr = (int)min(32ll, r1 - c0);
      // the round's runs of equal primitive (rows are sorted by primitive):
      // each run is summed without a per-row test, the previous run flushed
      // when the primitive changes
      const int gl = __float_as_int(val[14]);
      const int gp = __shfl_up_sync(0xffffffffu, gl, 1);
      unsigned heads = __ballot_sync(0xffffffffu, lane < nr && (lane == 0 || gp != gl));
      __syncwarp();
      while (heads) {
        const int s0 = __ffs(heads) - 1;
        heads &= heads - 1;
        const int s1 = heads ? __ffs(heads) - 1 : nr;
        const int g = __float_as_int(rows[s0 * RS + 14]);
        if (g != gcur) {
          if (gcur >= 0) flush(gcur, acc);
#pragma unroll
          for (int q = 0; q < NQ; q++) acc[q] = 0.f;
          gcur = g;
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) {
          if (vcol[q] < 0) continue;
          float sum = acc[q];
          if (s1 - s0 == 32) {
            if (bcol[q] >= 0) {
#pragma unroll
              for (int r = 0; r < 32; r++) sum = fmaf(rows[r * RS + bcol[q]], rows[r * RS + vcol[q]], sum);
            } else {
#pragma unroll
              for (int r = 0; r < 32; r++) sum += rows[r * RS + vcol[q]];
            }
          } else if (bcol[q] >= 0) {
            for (int r = s0; r < s1; r++) sum = fmaf(rows[r * RS + bcol[q]], rows[r * RS + vcol[q]], sum);
          } else {
            for (int r = s0; r < s1; r++) sum += rows[r * RS + vcol[q]];
          }
          acc[q] = sum;
        }
      }
      __syncwarp();
    }
    if (gcur >= 0) flush(gcur, acc);
  }
}

// The per-primitive sums of k_prim_sum for degrees whose outputs fit in
// registers (6m + 8 <= 44 at degree 2): lane i owns record slot i of each
// round of 32 and adds its record's weighted values to its own 6m + 8
// accumulators over the rounds of a run of equal primitive; when the
// primitive changes (and at the chunk's end) a reduce-scatter over the warp
// (shuffle butterfly, 62 exchanges) leaves outputs 2i and 2i + 1 in lane i,
// which adds them with one atomic each. Same sums as k_prim_sum, with a
// shuffle exchange per run instead of a shared-memory pass per round.
template <int N>
__global__ void __launch_bounds__(256, 2) k_prim_sum_reg(Params p, Work w, Grads out) {
  constexpr int m = SurfPoint<N>::M;
  constexpr int NO = 6 * m + 8;
  static_assert(NO <= 64, "outputs beyond two per lane");
  const int lane = threadIdx.x & 31;
  const int F = w.counters[kF], Nb = w.counters[kNb];
  float acc[64];
  auto reduce_flush = [&](int g) {
#pragma unroll
    for (int off = 16, H = 32; off > 0; off >>= 1, H >>= 1) {
      const bool hb = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < H; i++) {
        const float send = hb ? acc[i] : acc[i + H];
        const float keep = hb ? acc[i + H] : acc[i];
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int j = 2 * lane + i;
      if (j < NO && acc[i] != 0.f) {
        float *dst = j < 3 * m ? out.ctrl + (size_t)g * 3 * m + j
                     : j < 6 * m ? out.color + (size_t)g * 3 * m + (j - 3 * m)
                     : j == 6 * m ? out.opacity + g
                     : j == 6 * m + 1 ? out.r_b + g
                     : w.prim_gcov + 6 * (size_t)g + (j - 6 * m - 2);
        atomicAdd(dst, acc[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 64; i++) acc[i] = 0.f;
  };
  const long long ng = (F + kSumChunk - 1) / kSumChunk, nchunks = ng + (Nb + kSumChunk - 1) / kSumChunk;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (long long ck = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ck < nchunks; ck += warps_total) {
    const bool bnd = ck >= ng;
    const long long r0 = (bnd ? ck - ng : ck) * kSumChunk;
    const long long r1 = min(r0 + kSumChunk, (long long)(bnd ? Nb : F));
#pragma unroll
    for (int i = 0; i < 64; i++) acc[i] = 0.f;
    int gcur = -1;
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra, rd = ra;
    auto load = [&](long long c) {
      if (c + lane < r1) {
        if (!bnd) {
          const float4 *r = w.pg_rec + 4 * (c + lane);
          ra = r[0]; rb = r[1]; rc = r[2]; rd = r[3];
        } else {
          const float4 *r = w.pb_rec + 2 * (c + lane);
          ra = r[0]; rb = r[1];
        }
      }
    };
    load(r0);
    for (long long c0 = r0; c0 < r1; c0 += 32) {
      const bool valid = c0 + lane < r1;
      // dl/dS, dl/do, dl/dc, dl/dSigma3D, dl/dr_b, u, v and the primitive
      float gS[3] = {ra.x, ra.y, ra.z}, gop = 0.f, gc[3] = {0.f, 0.f, 0.f}, gv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float grb = 0.f, u, v;
      int gl;
      if (!bnd) {
        gop = ra.w;
        gc[0] = rb.x; gc[1] = rb.y; gc[2] = rb.z;
        gv[0] = rc.y; gv[1] = rc.z; gv[2] = rc.w; gv[3] = rd.x; gv[4] = rd.y; gv[5] = rd.z;
        u = rb.w;
        v = rc.x;
        gl = __float_as_int(rd.w);
      } else {
        grb = ra.w;
        u = rb.x;
        v = rb.y;
        gl = __float_as_int(rb.z);
      }
      if (!valid) gl = -1;
      load(c0 + 32);
      float B[m];
      bernstein_f32<N>(u, v, B);
      bool consumed = !valid;
      for (;;) {
        if (!consumed && gl == gcur) {
#pragma unroll
          for (int a = 0; a < m; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
              acc[3 * a + c] = fmaf(B[a], gS[c], acc[3 * a + c]);
              acc[3 * m + 3 * a + c] = fmaf(B[a], gc[c], acc[3 * m + 3 * a + c]);
            }
          acc[6 * m] += gop;
          acc[6 * m + 1] += grb;
#pragma unroll
          for (int k = 0; k < 6; k++) acc[6 * m + 2 + k] += gv[k];
          consumed = true;
        }
        const unsigned rest = __ballot_sync(0xffffffffu, !consumed);
        if (!rest) break;
        // the round holds the start of the next primitive's run
        if (gcur >= 0) reduce_flush(gcur);
        gcur = __shfl_sync(0xffffffffu, gl, __ffs(rest) - 1);
      }
    }
    if (gcur >= 0) reduce_flush(gcur);
  }
}

__device__ __forceinline__ float l1_sign(float diff, float scale) {
  return diff > 0.f ? scale : (diff < 0.f ? -scale : 0.f);
}

// dl/dC = scale sign(C - target) and the loss scale |C - target| summed; four
// values per thread and load when the three arrays are 16-byte aligned (vec)
__global__ void k_l1_grad(const float *img, const float *tgt, long long n, float scale, float *d, float *loss,
                          int vec) {
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long done = 0;
  if (vec) {
    const long long n4 = n >> 2;
    const float4 *a4 = reinterpret_cast<const float4 *>(img), *b4 = reinterpret_cast<const float4 *>(tgt);
    float4 *d4 = reinterpret_cast<float4 *>(d);
    for (long long i = t0; i < n4; i += stride) {
      const float4 a = a4[i], b = b4[i];
      const float x = a.x - b.x, y = a.y - b.y, z = a.z - b.z, q = a.w - b.w;
      d4[i] = make_float4(l1_sign(x, scale), l1_sign(y, scale), l1_sign(z, scale), l1_sign(q, scale));
      acc += (fabsf(x) + fabsf(y)) + (fabsf(z) + fabsf(q));
    }
    done = n4 << 2;
  }
  for (long long i = done + t0; i < n; i += stride) {
    const float diff = img[i] - tgt[i];
    d[i] = l1_sign(diff, scale);
    acc += fabsf(diff);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc * scale);
}

}  // namespace

// maps of leg resolution 1: dl/dSigma3D summed over a primitive's Gaussians
// taken to its one rotation and scaling texel (linear in dl/dSigma3D, so the
// sum of the per-Gaussian terms)
__global__ void k_prim_attr_grad(Params p, Scene s, Work w, Grads out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= p.M) return;
  const float *gc = w.prim_gcov + 6 * (size_t)m;
  const float G3[9] = {gc[0], gc[1], gc[2], gc[1], gc[3], gc[4], gc[2], gc[4], gc[5]};
  float qa[4], ls[3], Rm[9], sc3[3], S3[6], gls[3], gq[4];
#pragma unroll
  for (int k = 0; k < 4; k++) qa[k] = s.quat[4 * (size_t)m + k];
#pragma unroll
  for (int k = 0; k < 3; k++) ls[k] = s.log_scale[3 * (size_t)m + k];
  cov3d_f32(qa, ls, S3, Rm, sc3);
  cov_grad_to_attrs(qa, G3, Rm, sc3, gls, gq);
  if (out.log_scale)
#pragma unroll
    for (int k = 0; k < 3; k++) out.log_scale[3 * (size_t)m + k] = gls[k];
  if (out.quat)
#pragma unroll
    for (int k = 0; k < 4; k++) out.quat[4 * (size_t)m + k] = gq[k];
}

int launch_chain(const Params &p, const Scene &s, const Work &w, const Grads &g, cudaStream_t st) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (sms > 0 ? sms : 152) * p.chain_bps;
  int k = 0;
  const int with_cov = p.attr_res == 1 && (g.log_scale || g.quat);
  if (p.M > 0) {
    // segments of the per-primitive records
    cudaMemsetAsync(w.prim_gcnt, 0, sizeof(int) * (size_t)p.M, st);
    cudaMemsetAsync(w.prim_bcnt, 0, sizeof(int) * (size_t)p.M, st);
    k_prim_count<<<(sms > 0 ? sms : 152) * 8, 256, 0, st>>>(w);
    k += 1 + launch_exclusive_scan(w.prim_gcnt, w.prim_gseg, p.M, w.scan_aux, st);
    k += launch_exclusive_scan(w.prim_bcnt, w.prim_bseg, p.M, w.scan_aux2, st);
    cudaMemsetAsync(w.prim_gcnt, 0, sizeof(int) * (size_t)p.M, st);  // now the fill counters
    cudaMemsetAsync(w.prim_bcnt, 0, sizeof(int) * (size_t)p.M, st);
    if (with_cov) cudaMemsetAsync(w.prim_gcov, 0, sizeof(float) * 6 * (size_t)p.M, st);
  }
  dispatch_degree(p.n, [&](auto d) {
    k_chain_gauss<decltype(d)::value><<<grid, 256, 0, st>>>(p, s, w, g);
    k_chain_bnd<decltype(d)::value><<<grid, 256, 0, st>>>(p, s, w, g);
    if (p.M > 0) {
      if constexpr (SurfPoint<decltype(d)::value>::M <= 6)
        k_prim_sum_reg<decltype(d)::value><<<(sms > 0 ? sms : 152) * 2, 256, 0, st>>>(p, w, g);
      else
        k_prim_sum<decltype(d)::value><<<(sms > 0 ? sms : 152) * 4, 256, 0, st>>>(p, w, g, with_cov);
    }
    if (p.sh_deg > 0) k_chain_sh<decltype(d)::value><<<grid, 256, 0, st>>>(p, s, w, g);
  });
  k += (p.sh_deg > 0 ? 3 : 2) + (p.M > 0 ? 1 : 0);
  if (p.attr_res == 1 && (g.log_scale || g.quat) && p.M > 0) {
    k_prim_attr_grad<<<(p.M + 255) / 256, 256, 0, st>>>(p, s, w, g);
    k++;
  }
  return k;
}

int launch_l1_grad(const float *img, const float *target, long long n, float scale, float *dimg, float *loss,
                   cudaStream_t st) {
  if (n <= 0) return 0;
  const int vec = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(target) |
                    reinterpret_cast<uintptr_t>(dimg)) & 15) == 0;
  long long blocks = ((vec ? n / 4 : n) + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_l1_grad<<<(int)blocks, 256, 0, st>>>(img, target, n, scale, dimg, loss, vec);
  return 1;
}

}  // namespace bgt
