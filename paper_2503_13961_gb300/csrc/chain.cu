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
// Control-point, colour and opacity gradients of consecutive Gaussians (which
// mostly share a primitive, being compacted in pixel order) are summed per
// run of equal primitive through shared memory before one atomic per run and
// value.
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

template <int N>
__global__ void __launch_bounds__(256) k_chain_gauss(Params p, Scene s, Work w, Grads out) {
  constexpr int m = SurfPoint<N>::M;
  __shared__ float s_rows[kChainWarps][32 * ((3 * m + 7) | 1)];
  float *sw = s_rows[threadIdx.x >> 5];
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
      g = __float_as_int(w.gC[i].w);
      const View vw = w.views[w.g_view[i]];
      const float2 uv = w.g_uv[i];
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
    const bool nz = active && (gS[0] != 0.f || gS[1] != 0.f || gS[2] != 0.f || gcol[0] != 0.f ||
                               gcol[1] != 0.f || gcol[2] != 0.f || gop != 0.f);
    if (!__any_sync(0xffffffffu, nz)) continue;
    const bool per_prim_cov = p.attr_res == 1 && (out.log_scale || out.quat);
    {
      // control points, opacity and (leg resolution 1) dl/dSigma3D, then colour
      // control points (Eq. 3, 4: dl/dp = sum B dl/dS)
      float v[3 * m + 7];
#pragma unroll
      for (int a = 0; a < m; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[3 * a + c] = nz ? B[a] * gS[c] : 0.f;
      v[3 * m] = nz ? gop : 0.f;
      float *gctrl = out.ctrl, *gopa = out.opacity, *gcov = w.prim_gcov;
      if (per_prim_cov) {
#pragma unroll
        for (int k = 0; k < 6; k++) v[3 * m + 1 + k] = nz ? gc6[k] : 0.f;
        scatter_runs<3 * m + 7>(sw, v, nz ? g : -1, [&](int gg, int j) {
          return j < 3 * m ? gctrl + (size_t)gg * 3 * m + j
                           : (j == 3 * m ? gopa + gg : gcov + 6 * (size_t)gg + (j - 3 * m - 1));
        });
      } else {
        scatter_runs<3 * m + 1>(sw, v, nz ? g : -1, [&](int gg, int j) {
          return j < 3 * m ? gctrl + (size_t)gg * 3 * m + j : gopa + gg;
        });
      }
#pragma unroll
      for (int a = 0; a < m; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[3 * a + c] = nz ? B[a] * gcol[c] : 0.f;
      float *gcolor = out.color;
      scatter_runs<3 * m>(sw, v, nz ? g : -1, [&](int gg, int j) { return gcolor + (size_t)gg * 3 * m + j; });
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
      g = __float_as_int(w.gC[i].w);
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
  __shared__ float s_rows[kChainWarps][32 * ((3 * m + 1) | 1)];
  float *sw = s_rows[threadIdx.x >> 5];
  const int Nb = w.counters[kNb];
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < Nb; base += warps_total * 32) {
    const int i = base + lane;
    bool nz = false;
    int g = -1;
    float gS[3] = {0.f, 0.f, 0.f}, grb = 0.f;
    float B[m];
    if (i < Nb) {
      const float4 gb = w.bg_grad[i];
      nz = gb.x != 0.f || gb.y != 0.f || gb.z != 0.f;
      if (nz) {
        g = w.b_prim[i];
        const View vw = w.views[w.b_view[i]];
        const float2 uv = w.b_uv[i];
        float t[3];
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
    }
    if (!__any_sync(0xffffffffu, nz)) continue;
    float v[3 * m + 1];
#pragma unroll
    for (int a = 0; a < m; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) v[3 * a + c] = nz ? B[a] * gS[c] : 0.f;
    v[3 * m] = nz ? grb : 0.f;
    float *gctrl = out.ctrl, *grbp = out.r_b;
    scatter_runs<3 * m + 1>(sw, v, nz ? g : -1, [&](int gg, int j) {
      return j < 3 * m ? gctrl + (size_t)gg * 3 * m + j : grbp + gg;
    });
  }
}

__global__ void k_l1_grad(const float *img, const float *tgt, long long n, float scale, float *d, float *loss) {
  float acc = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float diff = img[i] - tgt[i];
    d[i] = diff > 0.f ? scale : (diff < 0.f ? -scale : 0.f);
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
  dispatch_degree(p.n, [&](auto d) {
    k_chain_gauss<decltype(d)::value><<<grid, 256, 0, st>>>(p, s, w, g);
    k_chain_bnd<decltype(d)::value><<<grid, 256, 0, st>>>(p, s, w, g);
    if (p.sh_deg > 0) k_chain_sh<decltype(d)::value><<<grid, 256, 0, st>>>(p, s, w, g);
  });
  int k = p.sh_deg > 0 ? 3 : 2;
  if (p.attr_res == 1 && (g.log_scale || g.quat) && p.M > 0) {
    k_prim_attr_grad<<<(p.M + 255) / 256, 256, 0, st>>>(p, s, w, g);
    k++;
  }
  return k;
}

int launch_l1_grad(const float *img, const float *target, long long n, float scale, float *dimg, float *loss,
                   cudaStream_t st) {
  if (n <= 0) return 0;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_l1_grad<<<(int)blocks, 256, 0, st>>>(img, target, n, scale, dimg, loss);
  return 1;
}

}  // namespace bgt
