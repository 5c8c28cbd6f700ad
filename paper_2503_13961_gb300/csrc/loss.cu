// Photometric training loss of Sec. 3.3 (Eq. 9), L = (1 - lambda) L2 +
// lambda (1 - SSIM), and its gradient dL/dC with respect to the rendered
// image, in one fused kernel: the gradient lands in the layout the backward
// pass reads, and neither the windowed moments nor SSIM's partials ever
// leave shared memory.
//
// SSIM per channel: local moments under an 11 x 11 normalised Gaussian
// window (sigma 1.5, zero outside the image), C1 = 0.01^2, C2 = 0.03^2,
// averaged over pixels and channels; L2 is the mean of (C - C_gt)^2.
//
// One CTA owns a 32 x 32 output tile of one view (views of any size, the
// image layout of the renderer: concatenated [H][W][3] blocks). Its gradient needs SSIM's
// partials a = ds/dmu_x, b = ds/d(F x^2), c = ds/d(F xy) on the tile plus a
// 5-pixel halo (42 x 42), and those need the image on a 10-pixel halo
// (52 x 52). Per channel: image values to shared memory; separable window
// over the five moments (rows, then columns); SSIM and its partials (zero
// at pixels outside the image, which are not in the mean); separable window
// over the three partials; gradient = 2 w_l2 (x - y) - w_ssim (F a + 2 x F b
// + y F c) with the symmetric window as its own adjoint. The halo is
// recomputed by neighbouring CTAs instead of round-tripping the partials
// through HBM: HBM traffic is the two images read and the gradient written.
#include <cmath>
#include <cstring>

#include "bgt_internal.cuh"

namespace bgt {
namespace {

constexpr int kR = 5;
constexpr int kTaps = 2 * kR + 1;
constexpr int kTW = 32, kTH = 32;                       // output tile
constexpr int kAW = kTW + 2 * kR, kAH = kTH + 2 * kR;   // SSIM partials: 42 x 42
constexpr int kIW = kTW + 4 * kR, kIH = kTH + 4 * kR;   // image values: 52 x 52
// shared-memory row strides (in elements), odd so that threads walking down
// rows hit distinct banks
constexpr int kSI = kIW + 1, kSH1 = kAW + 1, kSA = kAW + 1, kSH2 = kTW + 1;
constexpr int kI = kIH * kSI, kH1 = kIH * kSH1, kA = kAH * kSA, kH2 = kAH * kSH2;
constexpr int kLossThreads = 256;
constexpr int kLoadRows = (kIH + kLossThreads / 32 - 1) / (kLossThreads / 32);
static_assert(kIW <= 64, "a region row is two loads per lane");
// (x, y) pairs; windowed rows as pairs (x, y), (x^2, y^2) and singles xy;
// partials as pairs (a, b) and singles c; second horizontal pass aliased on
// the first one's buffer
constexpr int kLossSmem = (int)(sizeof(float2) * (kI + 2 * kH1 + kA) + sizeof(float) * (kH1 + kA));
static_assert(sizeof(float2) * kH2 + sizeof(float) * kH2 <= sizeof(float2) * 2 * kH1, "aliasing");
static_assert(2 * kLossSmem + 2048 <= 232448, "two CTAs per SM");
// register blocking: each thread filters a run of consecutive outputs and
// loads every input of the run once (runs of 7 columns in the first
// horizontal pass, 7 rows in the first vertical one, 8 columns and 4 rows in
// the passes over the partials)
constexpr int kRunH1 = 7, kRunV1 = 7, kRunH2 = 8, kRunV2 = 4;
static_assert(kAW % kRunH1 == 0 && kAH % kRunV1 == 0 && kTW % kRunH2 == 0 && kTH % kRunV2 == 0, "runs tile");
static_assert((kAW / kRunH1) * kIH <= 2 * kLossThreads && (kAH / kRunV1) * kAW <= kLossThreads &&
              (kTW / kRunH2) * kAH <= kLossThreads && (kTH / kRunV2) * kTW <= kLossThreads, "work items");

constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

constexpr int kMaxLossViews = 112;  // views per launch: the table stays in 4 KB of parameters

// Two FP32 lanes in one 64-bit register: sm_100+ packed FMA / multiply, each
// lane rounded like fmaf / a single multiply.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ f32x2 pk(float2 v) { return pk(v.x, v.y); }
__device__ __forceinline__ float2 unpk(f32x2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

struct LossView {
  long long off;       // first pixel of the view in the concatenated images
  int W, H, tiles_x, tile0;
  float w_l2, w_ssim;  // scale (1 - lambda) / N and scale lambda / N, N = 3 W H
};

struct LossArgs {
  const float *img, *gt;
  float *dimg, *loss;
  int n_views;
  float g[kTaps];      // 1-D window weights
  f32x2 g2[kTaps];     // the same, each weight in both lanes
  LossView view[kMaxLossViews];
};
static_assert(sizeof(LossArgs) <= 4000, "kernel parameters");

__global__ void __launch_bounds__(kLossThreads, 2) k_l2_dssim_grad(const __grid_constant__ LossArgs a) {
  extern __shared__ float4 sm4[];
  float2 *sxy = reinterpret_cast<float2 *>(sm4);       // [kIH][kSI] (x, y)
  float2 *h1p = sxy + kI;                              // [2][kIH][kSH1] rows of (x, y), (x^2, y^2)
  float2 *pab = h1p + 2 * kH1;                         // [kAH][kSA] partials (a, b)
  float *h1s = reinterpret_cast<float *>(pab + kA);    // [kIH][kSH1] rows of xy
  float *pc = h1s + kH1;                               // [kAH][kSA] partial c
  float2 *h2p = h1p;                                   // [kAH][kSH2] rows of (a, b)
  float *h2s = reinterpret_cast<float *>(h1p + kH2);   // [kAH][kSH2] rows of c
  __shared__ float s_red[kLossThreads / 32];

  // the view this tile belongs to: last view whose first tile is <= blockIdx.x
  int lo = 0, hi = a.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.view[mid].tile0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const LossView &vw = a.view[lo];
  const int W = vw.W, H = vw.H;
  const int tile = blockIdx.x - vw.tile0;
  const int x0 = (tile % vw.tiles_x) * kTW, y0 = (tile / vw.tiles_x) * kTH;
  const size_t base = (size_t)vw.off;
  const float w_l2 = vw.w_l2, w_ssim = vw.w_ssim;
  const int tid = threadIdx.x;
  float acc = 0.f;

  for (int c = 0; c < 3; ++c) {
    {
      // warp w loads rows w, w + 8, ... of the region; every load in flight
      // at once, then the stores
      const int warp = tid >> 5, lane = tid & 31;
      float2 v[kLoadRows][2];
#pragma unroll
      for (int k = 0; k < kLoadRows; ++k) {
        const int r = warp + k * (kLossThreads / 32);
        const int gy = y0 - 2 * kR + r;
        const bool row_ok = r < kIH && gy >= 0 && gy < H;
        const size_t row = (base + (size_t)(row_ok ? gy : 0) * W) * 3 + c;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = lane + 32 * h;
          const int gx = x0 - 2 * kR + q;
          v[k][h] = make_float2(0.f, 0.f);
          if (row_ok && q < kIW && gx >= 0 && gx < W) {
            v[k][h].x = __ldg(a.img + row + 3 * (size_t)gx);
            v[k][h].y = __ldg(a.gt + row + 3 * (size_t)gx);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kLoadRows; ++k) {
        const int r = warp + k * (kLossThreads / 32);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = lane + 32 * h;
          if (r < kIH && q < kIW) sxy[r * kSI + q] = v[k][h];
        }
      }
    }
    __syncthreads();

    // rows: (x, y), (x^2, y^2) and xy under the 1-D window, runs of kRunH1 columns
    for (int it = tid; it < (kAW / kRunH1) * kIH; it += kLossThreads) {
      const int r = it % kIH, q0 = (it / kIH) * kRunH1;
      f32x2 m01[kRunH1], m23[kRunH1];
      float m4[kRunH1];
#pragma unroll
      for (int j = 0; j < kRunH1; ++j) {
        m01[j] = m23[j] = 0ull;
        m4[j] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < kRunH1 + 2 * kR; ++i) {
        const float2 v = sxy[r * kSI + q0 + i];
        const f32x2 xy2 = pk(v);
        const f32x2 sq2 = mul2(xy2, xy2);
        const float xy = v.x * v.y;
#pragma unroll
        for (int j = 0; j < kRunH1; ++j) {
          const int t = i - j;
          if (t >= 0 && t < kTaps) {
            m01[j] = fma2(a.g2[t], xy2, m01[j]);
            m23[j] = fma2(a.g2[t], sq2, m23[j]);
            m4[j] = fmaf(a.g[t], xy, m4[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kRunH1; ++j) {
        h1p[r * kSH1 + q0 + j] = unpk(m01[j]);
        h1p[kH1 + r * kSH1 + q0 + j] = unpk(m23[j]);
        h1s[r * kSH1 + q0 + j] = m4[j];
      }
    }
    __syncthreads();

    // columns, then SSIM and its partials, runs of kRunV1 rows
    if (tid < (kAH / kRunV1) * kAW) {
      const int q = tid % kAW, r0 = (tid / kAW) * kRunV1;
      f32x2 m01[kRunV1], m23[kRunV1];
      float m4[kRunV1];
#pragma unroll
      for (int j = 0; j < kRunV1; ++j) {
        m01[j] = m23[j] = 0ull;
        m4[j] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < kRunV1 + 2 * kR; ++i) {
        const int o = (r0 + i) * kSH1 + q;
        const f32x2 u = pk(h1p[o]), w = pk(h1p[kH1 + o]);
        const float z = h1s[o];
#pragma unroll
        for (int j = 0; j < kRunV1; ++j) {
          const int t = i - j;
          if (t >= 0 && t < kTaps) {
            m01[j] = fma2(a.g2[t], u, m01[j]);
            m23[j] = fma2(a.g2[t], w, m23[j]);
            m4[j] = fmaf(a.g[t], z, m4[j]);
          }
        }
      }
      const int gx = x0 - kR + q;
#pragma unroll
      for (int j = 0; j < kRunV1; ++j) {
        const int r = r0 + j, gy = y0 - kR + r;
        float2 dab = make_float2(0.f, 0.f);
        float dc = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
          const float2 mu = unpk(m01[j]), sq = unpk(m23[j]);
          const float mx = mu.x, my = mu.y;
          const float l1 = 2.f * mx * my + kC1;
          const float cs1 = 2.f * (m4[j] - mx * my) + kC2;
          const float l2 = mx * mx + my * my + kC1;
          const float cs2 = (sq.x - mx * mx) + (sq.y - my * my) + kC2;
          const float rD = __fdividef(1.f, l2 * cs2);  // D in [C1 C2, 4 (1 + C1) (2 + C2)]
          const float s = l1 * cs1 * rD;
          const float dN = 2.f * my * (cs1 - l1);
          const float dD = 2.f * mx * (cs2 - l2);
          dab.x = (dN - s * dD) * rD;
          dab.y = -s * l2 * rD;
          dc = 2.f * l1 * rD;
          if (r >= kR && r < kR + kTH && q >= kR && q < kR + kTW) {
            const float2 v = sxy[(r + kR) * kSI + q + kR];
            const float d = v.x - v.y;
            acc += w_l2 * d * d + w_ssim * (1.f - s);
          }
        }
        pab[r * kSA + q] = dab;
        pc[r * kSA + q] = dc;
      }
    }
    __syncthreads();

    // rows of the partials, runs of kRunH2 columns
    if (tid < (kTW / kRunH2) * kAH) {
      const int r = tid % kAH, q0 = (tid / kAH) * kRunH2;
      f32x2 fab[kRunH2];
      float fc[kRunH2];
#pragma unroll
      for (int j = 0; j < kRunH2; ++j) {
        fab[j] = 0ull;
        fc[j] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < kRunH2 + 2 * kR; ++i) {
        const f32x2 u = pk(pab[r * kSA + q0 + i]);
        const float z = pc[r * kSA + q0 + i];
#pragma unroll
        for (int j = 0; j < kRunH2; ++j) {
          const int t = i - j;
          if (t >= 0 && t < kTaps) {
            fab[j] = fma2(a.g2[t], u, fab[j]);
            fc[j] = fmaf(a.g[t], z, fc[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kRunH2; ++j) {
        h2p[r * kSH2 + q0 + j] = unpk(fab[j]);
        h2s[r * kSH2 + q0 + j] = fc[j];
      }
    }
    __syncthreads();

    // columns of the partials and the gradient, runs of kRunV2 rows
    if (tid < (kTH / kRunV2) * kTW) {
      const int q = tid % kTW, r0 = (tid / kTW) * kRunV2;
      f32x2 fab[kRunV2];
      float fc[kRunV2];
#pragma unroll
      for (int j = 0; j < kRunV2; ++j) {
        fab[j] = 0ull;
        fc[j] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < kRunV2 + 2 * kR; ++i) {
        const int o = (r0 + i) * kSH2 + q;
        const f32x2 u = pk(h2p[o]);
        const float z = h2s[o];
#pragma unroll
        for (int j = 0; j < kRunV2; ++j) {
          const int t = i - j;
          if (t >= 0 && t < kTaps) {
            fab[j] = fma2(a.g2[t], u, fab[j]);
            fc[j] = fmaf(a.g[t], z, fc[j]);
          }
        }
      }
      const int gx = x0 + q;
#pragma unroll
      for (int j = 0; j < kRunV2; ++j) {
        const int r = r0 + j, gy = y0 + r;
        if (gy < H && gx < W) {
          const float2 v = sxy[(r + 2 * kR) * kSI + q + 2 * kR];
          const float2 f = unpk(fab[j]);
          const float dssim = f.x + 2.f * v.x * f.y + v.y * fc[j];
          a.dimg[(base + (size_t)gy * W + gx) * 3 + c] = 2.f * w_l2 * (v.x - v.y) - w_ssim * dssim;
        }
      }
    }
    __syncthreads();
  }

  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0 && a.loss) {
    float t = 0.f;
    for (int k = 0; k < kLossThreads / 32; ++k) t += s_red[k];
    atomicAdd(a.loss, t);
  }
}

}  // namespace

int launch_l2_dssim_grad(const float *img, const float *gt, int n_views, const int *sizes, float lambda,
                         float scale, float *dimg, float *loss, cudaStream_t st) {
  LossArgs a;
  a.img = img;
  a.gt = gt;
  a.dimg = dimg;
  a.loss = loss;
  double g[kTaps], sum = 0.0;
  for (int t = 0; t < kTaps; ++t) {
    const double d = t - kR;
    g[t] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += g[t];
  }
  for (int t = 0; t < kTaps; ++t) {
    a.g[t] = (float)(g[t] / sum);
    unsigned int bits;
    std::memcpy(&bits, &a.g[t], sizeof(bits));
    a.g2[t] = ((unsigned long long)bits << 32) | bits;
  }
  cudaFuncSetAttribute(k_l2_dssim_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, kLossSmem);
  int launches = 0;
  long long off = 0;
  for (int v0 = 0; v0 < n_views; v0 += kMaxLossViews) {
    a.n_views = 0;
    int tiles = 0;
    for (int v = v0; v < n_views && v < v0 + kMaxLossViews; ++v) {
      const int W = sizes[2 * v], H = sizes[2 * v + 1];
      const long long npx = (long long)W * H;
      if (npx > 0) {
        LossView &r = a.view[a.n_views++];
        r.off = off;
        r.W = W;
        r.H = H;
        r.tiles_x = (W + kTW - 1) / kTW;
        r.tile0 = tiles;
        tiles += r.tiles_x * ((H + kTH - 1) / kTH);
        const double n = 3.0 * (double)npx;
        r.w_l2 = (float)((double)scale * (1.0 - (double)lambda) / n);
        r.w_ssim = (float)((double)scale * (double)lambda / n);
      }
      off += npx;
    }
    if (tiles == 0) continue;
    k_l2_dssim_grad<<<tiles, kLossThreads, kLossSmem, st>>>(a);
    ++launches;
  }
  return launches;
}

}  // namespace bgt
