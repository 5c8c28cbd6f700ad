// bgt_bin_sort_static: the binning + per-tile sort stage of bgt_bin_sort for
// callers that cannot allocate device memory. Its scratch lives in one
// file-scope static device array of fixed size (see include/bgt.h for the
// limits); inputs and outputs are the caller's buffers.
#include <cstring>
#include <mutex>

#include "../../include/bgt.h"
#include "bgt_internal.cuh"

namespace {

constexpr int kMaxGauss = 65536;
constexpr int kMaxTiles = 16384;
constexpr long long kMaxPairs = 262144;
constexpr int kThreads = 256;
constexpr int kSmemKeys = 4096;

// scratch layout (bytes): per-Gaussian tile rect (8) and depth key (8),
// per-tile counts and fill cursors, the pair total, and a sort buffer of
// 2 * kMaxPairs keys (a segment of n keys pads to at most 2n in it)
constexpr size_t kOffRect = 0;
constexpr size_t kOffDkey = kOffRect + sizeof(uint2) * kMaxGauss;
constexpr size_t kOffCount = kOffDkey + sizeof(unsigned long long) * kMaxGauss;
constexpr size_t kOffFill = kOffCount + sizeof(int) * (kMaxTiles + 1);
constexpr size_t kOffTotal = kOffFill + sizeof(int) * (kMaxTiles + 1);
constexpr size_t kOffTemp = (kOffTotal + sizeof(long long) + 255) & ~(size_t)255;
constexpr size_t kScratchBytes = kOffTemp + sizeof(unsigned long long) * 2 * kMaxPairs;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct Scratch {
  uint2 *rect;
  unsigned long long *dkey;
  int *count, *fill;
  long long *total;
  unsigned long long *temp;
};

Scratch carve(unsigned char *base) {
  Scratch s;
  s.rect = reinterpret_cast<uint2 *>(base + kOffRect);
  s.dkey = reinterpret_cast<unsigned long long *>(base + kOffDkey);
  s.count = reinterpret_cast<int *>(base + kOffCount);
  s.fill = reinterpret_cast<int *>(base + kOffFill);
  s.total = reinterpret_cast<long long *>(base + kOffTotal);
  s.temp = reinterpret_cast<unsigned long long *>(base + kOffTemp);
  return s;
}

__global__ void k_sb_zero(Scratch s, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s.count[i] = 0;
    s.fill[i] = 0;
  }
}

// support box of each Gaussian (o exp(-1/2 d^T K d) >= alpha_min), its tile
// rect and depth key; counts the Gaussian into every covered tile
__global__ void k_sb_load(Scratch s, int count, int W, int H, int t, int tiles_x, float alpha_min,
                          float log_alpha_min, const int *qxy, const float *off, const float *conic,
                          const float *opac, const float *depth) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const unsigned q = (unsigned)qxy[i];
  s.dkey[i] = bgt::plain_depth_key(depth[i]);
  const bgt::ConicBox box = bgt::conic_support_box(conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], opac[i],
                                                   (float)(q & 0xffffu) + off[2 * i], (float)(q >> 16) + off[2 * i + 1],
                                                   W, H, t, alpha_min, log_alpha_min);
  const uint2 rect = box.rect;
  const int x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff, y1 = rect.y >> 16;
  for (int ty = y0; ty <= y1; ty++)
    for (int tx = x0; tx <= x1; tx++) atomicAdd(s.count + ty * tiles_x + tx, 1);
  s.rect[i] = rect;
}

// exclusive scan of the tile counts (one block), total into the scratch
__global__ void __launch_bounds__(1024) k_sb_scan(Scratch s, int tiles, long long *ranges) {
  __shared__ long long s_warp[32];
  __shared__ long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int base = 0; base < tiles; base += 1024) {
    const int i = base + threadIdx.x;
    const long long v = i < tiles ? s.count[i] : 0;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wp] = x;
    __syncthreads();
    if (wp == 0) {
      long long a = s_warp[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, a, o);
        if (lane >= o) a += y;
      }
      s_warp[lane] = a;
    }
    __syncthreads();
    if (i < tiles) ranges[i] = s_carry + (wp ? s_warp[wp - 1] : 0) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_warp[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ranges[tiles] = s_carry;
    *s.total = s_carry;
  }
}

__global__ void k_sb_emit(Scratch s, int count, int tiles_x, const long long *ranges, unsigned long long *keys,
                          long long cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint2 r = s.rect[i];
  const int x0 = r.x & 0xffff, y0 = r.x >> 16, x1 = r.y & 0xffff, y1 = r.y >> 16;
  const unsigned long long hi = s.dkey[i] << bgt::kIndexBits;
  for (int ty = y0; ty <= y1; ty++)
    for (int tx = x0; tx <= x1; tx++) {
      const int tt = ty * tiles_x + tx;
      const long long pos = ranges[tt] + atomicAdd(s.fill + tt, 1);
      if (pos >= 0 && pos < cap) keys[pos] = hi | (unsigned long long)(unsigned)i;
    }
}

// bitonic sort of buf[0..N) (N a power of two) by one block; buf in shared or global memory
__device__ void sb_bitonic(unsigned long long *buf, int N) {
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = buf[i], b = buf[ixj];
          if ((a > b) == ((i & k) == 0)) {
            buf[i] = b;
            buf[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
}

// one block per tile: segments up to kSmemKeys keys sort in shared memory,
// longer ones in the scratch buffer at twice their offset (padded to 2^k)
__global__ void __launch_bounds__(kThreads) k_sb_sort(Scratch s, int tiles, const long long *ranges,
                                                      unsigned long long *keys) {
  __shared__ unsigned long long s_keys[kSmemKeys];
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const long long s0 = ranges[tt], s1 = ranges[tt + 1];
    const int n = (int)(s1 - s0);
    if (n > 1) {
      int N = 1;
      while (N < n) N <<= 1;
      unsigned long long *buf = (N <= kSmemKeys) ? s_keys : s.temp + 2 * s0;
      for (int i = threadIdx.x; i < N; i += kThreads) buf[i] = i < n ? keys[s0 + i] : ~0ull;
      __syncthreads();
      sb_bitonic(buf, N);
      for (int i = threadIdx.x; i < n; i += kThreads) keys[s0 + i] = buf[i];
    }
    __syncthreads();
  }
}

// Device address of the static scratch, looked up on the first call on each
// device and kept: the address stays valid while the CUDA context that loaded
// the module lives (a cudaDeviceReset destroys it; the library must not be
// used across one).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

}  // namespace

extern "C" bgt_status bgt_bin_sort_static(int width, int height, int tile_size, int count, const int *qxy,
                                          const float *off, const float *conic, const float *opacity,
                                          const float *depth, float alpha_min, long long *out_ranges,
                                          unsigned long long *out_keys, long long key_capacity, void *stream) {
  if (width < 1 || height < 1 || width > 32768 || height > 32768) return BGT_ERR_INVALID_ARG;
  if (tile_size != 8 && tile_size != 16 && tile_size != 32) return BGT_ERR_INVALID_ARG;
  if (!(alpha_min > 0.f && alpha_min < 1.f)) return BGT_ERR_INVALID_ARG;
  if (count < 0 || !out_ranges || key_capacity < 0 || (count > 0 && (!qxy || !off || !conic || !opacity || !depth)))
    return BGT_ERR_INVALID_ARG;
  const int tiles_x = (width + tile_size - 1) / tile_size, tiles_y = (height + tile_size - 1) / tile_size;
  const long long tiles = (long long)tiles_x * tiles_y;
  if (count > kMaxGauss || tiles > kMaxTiles) return BGT_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BGT_ERR_CUDA;
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return BGT_ERR_CUDA;
      g_addr[dev] = static_cast<unsigned char *>(ptr);
    }
    base = g_addr[dev];
  }
  const Scratch s = carve(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nt = (int)tiles;
  k_sb_zero<<<(nt + 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(s, nt + 1);
  if (count > 0)
    k_sb_load<<<(count + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        s, count, width, height, tile_size, tiles_x, alpha_min, logf(alpha_min), qxy, off, conic, opacity, depth);
  k_sb_scan<<<1, 1024, 0, st>>>(s, nt, out_ranges);
  long long total = 0;
  cudaError_t e = cudaMemcpyAsync(&total, s.total, sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return BGT_ERR_CUDA;
  if (total > key_capacity || total > kMaxPairs) return BGT_ERR_CAPACITY;
  if (total > 0 && !out_keys) return BGT_ERR_INVALID_ARG;
  if (count > 0) {
    k_sb_emit<<<(count + kThreads - 1) / kThreads, kThreads, 0, st>>>(s, count, tiles_x, out_ranges, out_keys,
                                                                       key_capacity);
    k_sb_sort<<<nt < 1024 ? nt : 1024, kThreads, 0, st>>>(s, nt, out_ranges, out_keys);
  }
  return cudaGetLastError() == cudaSuccess ? BGT_OK : BGT_ERR_CUDA;
}
