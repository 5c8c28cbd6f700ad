// Tile binning and the (tile, depth) sort of the Gaussians, and the per-tile
// boundary-point lists sorted by primitive id (Sec. 3.2, "Rendering
// Acceleration": precomputed tile range of each boundary point, per-tile
// lists sorted by ID so that a binary search finds a primitive's points).
//
// The sort is a most-significant-digit radix sort of the key (tile, depth,
// index): the first digit is the whole tile id (a counting sort: per-tile
// counts from the generation pass, an exclusive scan, one scatter), the
// remaining 64 bits (36-bit depth key = FP32 depth bits and 5 finer bits,
// 27-bit Gaussian index) are sorted inside each tile in shared memory. Keys
// are unique, so the order is fully determined.
// Boundary keys are (primitive, boundary index).
#include "bgt_internal.cuh"

namespace bgt {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

// block-wide exclusive scan of one value per thread; returns the block total
__device__ inline long long block_excl_scan(long long v, long long &total, long long *s_warp) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wp] = x;
  __syncthreads();
  if (wp == 0) {
    long long a = lane < nw ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, a, o);
      if (lane >= o) a += y;
    }
    s_warp[lane] = a;
  }
  __syncthreads();
  total = s_warp[nw - 1];
  const long long res = (wp ? s_warp[wp - 1] : 0) + x - v;
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *in, int n, long long *aux) {
  __shared__ long long s_warp[32];
  const int base = blockIdx.x * kScanChunk;
  long long sum = 0;
  for (int k = 0; k < kScanItems; k++) {
    const int i = base + k * kScanThreads + threadIdx.x;
    if (i < n) sum += in[i];
  }
  long long total;
  block_excl_scan(sum, total, s_warp);
  if (threadIdx.x == 0) aux[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(long long *aux, int nb) {
  __shared__ long long s_warp[32];
  __shared__ long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const long long v = i < nb ? aux[i] : 0;
    long long tot;
    const long long ex = block_excl_scan(v, tot, s_warp);
    if (i < nb) aux[i] = ex + s_carry;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int *in, long long *out, int n,
                                                            const long long *aux) {
  __shared__ long long s_warp[32];
  // each thread owns kScanItems consecutive elements
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
  int v[kScanItems];
  long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    sum += v[k];
  }
  long long total;
  long long run = block_excl_scan(sum, total, s_warp) + aux[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  // the thread holding element n - 1 also writes out[n] = grand total
  if (base < n && base + kScanItems >= n) out[n] = run;
}

// a slot in tile t's segment: the active lanes of the warp that want one in
// the same tile share one atomic (consecutive Gaussians mostly share tiles);
// the order inside a segment is set by the sort that follows
__device__ __forceinline__ int tile_slot(int *fill, int t) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(__activemask(), t);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(fill + t, __popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

__device__ inline void emit_rect(unsigned long long *keys, int *fill, const long long *start, long long cap,
                                 int tile_off, int tiles_x, uint2 rect, unsigned long long hi,
                                 unsigned lo) {
  const int x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff, y1 = rect.y >> 16;
  for (int ty = y0; ty <= y1; ty++)
    for (int tx = x0; tx <= x1; tx++) {
      const int t = tile_off + ty * tiles_x + tx;
      const long long pos = start[t] + tile_slot(fill, t);
      if (pos >= 0 && pos < cap) keys[pos] = hi | (unsigned long long)lo;
    }
}

__global__ void k_emit(Params p, Work w) {
  const int F = w.counters[kF], Nb = w.counters[kNb];
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F; i += stride) {
    const uint2 rect = w.g_rect[i];
    if ((rect.x & 0xffff) > (rect.y & 0xffff)) continue;
    const View *vw = w.views + w.g_view[i];
    const unsigned long long dkey =
        ((unsigned long long)__float_as_uint(w.g_depth[i]) << 5) | (unsigned long long)w.g_dsub[i];
    emit_rect(w.gkeys, w.g_tfill, w.g_tstart, p.max_pairs, __ldg(&vw->tile_off), __ldg(&vw->tiles_x),
              rect, dkey << kIndexBits, (unsigned)i);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Nb; i += stride) {
    const uint2 rect = w.b_rect[i];
    if ((rect.x & 0xffff) > (rect.y & 0xffff)) continue;
    const View *vw = w.views + w.b_view[i];
    emit_rect(w.bkeys, w.b_tfill, w.b_tstart, p.max_bpairs, __ldg(&vw->tile_off), __ldg(&vw->tiles_x),
              rect, (unsigned long long)(unsigned)w.b_prim[i] << 32, (unsigned)i);
  }
}

// per-tile descriptor, so that the blending kernels read two records instead
// of searching the view offsets and reading the list starts: [2t] geometry,
// [2t + 1] (Gaussian list start, length, boundary list start, length); an
// overflowed list (its slots were not all written) has length 0
__global__ void k_tile_desc(Params p, Work w) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.tiles) return;
  const int view = find_view(w.view_tile_off, p.V, t);
  const View &vw = w.views[view];
  const int lt = t - vw.tile_off;
  const int ty = lt / vw.tiles_x, tx = lt - ty * vw.tiles_x;
  w.tile_desc[2 * t] = make_int4(view, (int)((unsigned)(tx * p.tile) | ((unsigned)(ty * p.tile) << 16)),
                                 (int)((unsigned)vw.W | ((unsigned)vw.H << 16)), vw.pix_off);
  const bool g_over = w.g_tstart[p.tiles] > p.max_pairs, b_over = w.b_tstart[p.tiles] > p.max_bpairs;
  const long long gs = w.g_tstart[t], bs = w.b_tstart[t];
  w.tile_desc[2 * t + 1] = make_int4(g_over ? 0 : (int)gs, g_over ? 0 : (int)(w.g_tstart[t + 1] - gs),
                                     b_over ? 0 : (int)bs, b_over ? 0 : (int)(w.b_tstart[t + 1] - bs));
}

__global__ void k_check_capacity(Params p, Work w) {
  const long long K = w.g_tstart[p.tiles], Kb = w.b_tstart[p.tiles];
  w.counters[kK] = (int)(K < 0x7fffffffll ? K : 0x7fffffffll);
  w.counters[kKb] = (int)(Kb < 0x7fffffffll ? Kb : 0x7fffffffll);
  if (K > p.max_pairs) atomicOr(w.status, kStatusPairOverflow);
  if (Kb > p.max_bpairs) atomicOr(w.status, kStatusBoundaryOverflow);
}

// ---------------------------------------------------------------------------
// per-tile sort
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortCap = 4096;  // keys sorted in shared memory (32 KB)

__device__ void bitonic_smem(unsigned long long *s, int n) {
  int N = 1;
  while (N < n) N <<= 1;
  for (int i = n + threadIdx.x; i < N; i += blockDim.x) s[i] = ~0ull;
  __syncthreads();
  // every thread takes compare-exchange pairs (i, i + j): pair p has
  // i = (p with a zero bit inserted at j), so no thread idles on the
  // upper half of a pair
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = threadIdx.x; q < (N >> 1); q += blockDim.x) {
        const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
        const unsigned long long a = s[i], b = s[i + j];
        const bool up = (i & k) == 0;
        if ((a > b) == up) {
          s[i] = b;
          s[i + j] = a;
        }
      }
      __syncthreads();
    }
}

// Stable block-wide LSD radix sort (8-bit digits) of a segment in global
// memory, for segments larger than the shared-memory capacity. Digits that
// are equal across the whole segment are skipped.
__device__ void radix_global(unsigned long long *keys, unsigned long long *tmp, int n, int *s_hist,
                             int *s_base, int *s_wcnt, unsigned long long *s_red) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = kSortThreads / 32;
  // OR / AND over the segment to find constant digits
  unsigned long long vor = 0ull, vand = ~0ull;
  for (int i = threadIdx.x; i < n; i += kSortThreads) {
    vor |= keys[i];
    vand &= keys[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    vor |= __shfl_xor_sync(0xffffffffu, vor, o);
    vand &= __shfl_xor_sync(0xffffffffu, vand, o);
  }
  if (lane == 0) { s_red[wp] = vor; s_red[nw + wp] = vand; }
  __syncthreads();
  vor = 0ull; vand = ~0ull;
  for (int i = 0; i < nw; i++) { vor |= s_red[i]; vand &= s_red[nw + i]; }
  __syncthreads();
  const unsigned long long varying = vor ^ vand;
  unsigned long long *src = keys, *dst = tmp;
  for (int shift = 0; shift < 64; shift += 8) {
    if (((varying >> shift) & 0xffull) == 0ull) continue;
    for (int d = threadIdx.x; d < 256; d += kSortThreads) s_hist[d] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSortThreads) atomicAdd(&s_hist[(src[i] >> shift) & 0xff], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int d = 0; d < 256; d++) { s_base[d] = run; run += s_hist[d]; }
    }
    for (int d = threadIdx.x; d < nw * 256; d += kSortThreads) s_wcnt[d] = 0;
    __syncthreads();
    for (int chunk = 0; chunk < n; chunk += kSortThreads) {
      const int i = chunk + threadIdx.x;
      const bool valid = i < n;
      const unsigned long long key = valid ? src[i] : 0ull;
      const int dig = valid ? (int)((key >> shift) & 0xff) : 256 + wp;
      const unsigned peers = __match_any_sync(0xffffffffu, dig);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      if (valid && rank == 0) s_wcnt[wp * 256 + dig] = __popc(peers);
      __syncthreads();
      if (valid) {
        int pos = s_base[dig] + rank;
        for (int q = 0; q < wp; q++) pos += s_wcnt[q * 256 + dig];
        dst[pos] = key;
      }
      __syncthreads();
      for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        int add = 0;
        for (int q = 0; q < nw; q++) { add += s_wcnt[q * 256 + d]; s_wcnt[q * 256 + d] = 0; }
        s_base[d] += add;
      }
      __syncthreads();
    }
    unsigned long long *t = src; src = dst; dst = t;
  }
  if (src != keys)
    for (int i = threadIdx.x; i < n; i += kSortThreads) keys[i] = src[i];
  __syncthreads();
}

constexpr int kWarpSortCap = 512;  // keys a single warp sorts in its own shared memory (occupancy:
                                   // 16 keys per lane in registers, 36 KB of shared memory per block)
constexpr int kMidSortCap = 1024;  // longer segments up to this: one warp each in k_tile_sort_mid
                                   // (32 keys per lane, 72 KB of shared memory per block)
constexpr int kRadixMin = 129;     // segments from this length sort by radix, shorter ones by bitonic network
// per warp: the keys (kWarpSortCap) and 256 radix bins
constexpr int kTileSortSmem = (kSortThreads / 32) * (kWarpSortCap * (int)sizeof(unsigned long long) + 256 * 4);
constexpr int kTileSortMidSmem = (kSortThreads / 32) * (kMidSortCap * (int)sizeof(unsigned long long) + 256 * 4);

__device__ inline void segment_bounds(const Params &p, const Work &w, int item, bool &bnd, long long &s0,
                                      long long &s1) {
  bnd = item >= p.tiles;
  const int tile = bnd ? item - p.tiles : item;
  const long long *start = bnd ? w.b_tstart : w.g_tstart;
  const long long cap = bnd ? p.max_bpairs : p.max_pairs;
  s0 = start[tile];
  s1 = start[tile + 1];
  s0 = s0 < 0 ? 0 : (s0 > cap ? cap : s0);
  s1 = s1 < s0 ? s0 : (s1 > cap ? cap : s1);
}

__device__ inline void gather_boundary(const Work &w, long long s0, long long s1, int lane, int step) {
  for (long long i = s0 + lane; i < s1; i += step) {
    const unsigned long long k = w.bkeys[i];
    w.bl_prim[i] = (int)(k >> 32);
    w.bl_rec[i] = w.bR[(unsigned)(k & 0xffffffffu)];
  }
}

// Bitonic sort of sk[0, N) (N a power of two, 64..kWarpSortCap) by one warp:
// every stage is N / 2 independent compare-exchanges, 1 / 32 of them per lane.
__device__ __forceinline__ void warp_bitonic_smem(unsigned long long *sk, int N, int lane) {
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < (N >> 1); t += 32) {
        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // i has bit j clear; its partner is i + j
        const unsigned long long a = sk[i], b = sk[i + j];
        if ((a > b) == ((i & k) == 0)) {
          sk[i] = b;
          sk[i + j] = a;
        }
      }
      __syncwarp();
    }
}

// Stable LSD radix sort (8-bit digits) of sk[0, n) (n <= 32 R) by
// one warp on the key bits from lo_shift up: the keys sit in registers, key i
// in lane i % 32, slot i / 32; each pass histograms the digit into `bins`,
// scans it and scatters the keys back to sk in order, ranking equal digits of
// a round with a match; digits that are equal over the whole segment are
// skipped. Keys equal above lo_shift keep their input order.
template <int R>  // n <= 32 R
__device__ __forceinline__ void warp_radix_smem(unsigned long long *sk, unsigned *bins, int n, int lane,
                                                int lo_shift) {
  const int rounds = (n + 31) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long key[R];
  unsigned long long vor = 0ull, vand = ~0ull;
#pragma unroll
  for (int r = 0; r < R; r++) {
    key[r] = 0ull;
    if (r < rounds && r * 32 + lane < n) {
      key[r] = sk[r * 32 + lane];
      vor |= key[r];
      vand &= key[r];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vor |= __shfl_xor_sync(0xffffffffu, vor, o);
    vand &= __shfl_xor_sync(0xffffffffu, vand, o);
  }
  const unsigned long long varying = vor ^ vand;
  for (int shift = lo_shift; shift < 64; shift += 8) {
    if (((varying >> shift) & 0xffull) == 0ull) continue;
    for (int d = lane; d < 256; d += 32) bins[d] = 0u;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; r++)
      if (r < rounds && r * 32 + lane < n) atomicAdd(&bins[(unsigned)(key[r] >> shift) & 0xffu], 1u);
    __syncwarp();
    // exclusive scan of the 256 bins: 8 consecutive bins per lane
    unsigned c[8], tot = 0u;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      c[q] = bins[lane * 8 + q];
      tot += c[q];
    }
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    unsigned run = inc - tot;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      bins[lane * 8 + q] = run;
      run += c[q];
    }
    __syncwarp();
    // stable scatter, one round of 32 keys at a time
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r >= rounds) break;
      const bool valid = r * 32 + lane < n;
      const unsigned d = valid ? ((unsigned)(key[r] >> shift) & 0xffu) : 0x100u + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const unsigned base = valid ? bins[d] : 0u;
      if (valid) sk[base + __popc(peers & lt)] = key[r];
      __syncwarp();
      if (valid && lane == 31 - __clz(peers)) bins[d] = base + __popc(peers);
      __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; r++)
      if (r < rounds && r * 32 + lane < n) key[r] = sk[r * 32 + lane];
    __syncwarp();
  }
}

// A segment staged in sk[0, n) (padded with ~0 to the power of two N) sorted
// by one warp: boundary keys by radix on all bits; Gaussian keys by their
// depth bits only (the index below them just breaks ties), and when a tie is
// left in emission order (rare) the full keys go through the bitonic network,
// so the order is the (tile, depth, index) order either way.
template <int R>
__device__ __forceinline__ void warp_sort_segment(unsigned long long *sk, unsigned *bins, int n, int N, bool bnd,
                                                  int lane) {
  if (bnd) {
    warp_radix_smem<R>(sk, bins, n, lane, 0);
    return;
  }
  warp_radix_smem<R>(sk, bins, n, lane, kIndexBits);
  bool tie = false;
  for (int i = lane; i + 1 < n; i += 32) tie |= ((sk[i] ^ sk[i + 1]) >> kIndexBits) == 0ull;
  if (__any_sync(0xffffffffu, tie)) warp_bitonic_smem(sk, N, lane);
}

// Warps take segments from a queue. Up to 32 keys: bitonic sort across the
// lanes' registers; up to kWarpSortCap: bitonic sort (up to 128 keys) or
// radix sort in the warp's shared memory; longer segments are listed for
// k_tile_sort_mid (up to kMidSortCap keys) or k_tile_sort_big.
__global__ void __launch_bounds__(kSortThreads, 3) k_tile_sort(Params p, Work w, int *big_list) {
  extern __shared__ __align__(16) unsigned long long s_sort[];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const bool g_over = w.g_tstart[p.tiles] > p.max_pairs, b_over = w.b_tstart[p.tiles] > p.max_bpairs;
  const int items = 2 * p.tiles;
  unsigned long long *sk = s_sort + wp * kWarpSortCap;
  unsigned *bins = reinterpret_cast<unsigned *>(s_sort + (kSortThreads / 32) * kWarpSortCap) + wp * 256;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(w.counters + kQueueSort, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= items) break;
    bool bnd;
    long long s0, s1;
    segment_bounds(p, w, item, bnd, s0, s1);
    if (bnd ? b_over : g_over) continue;  // unwritten slots: nothing to sort
    const int n = (int)(s1 - s0);
    unsigned long long *keys = (bnd ? w.bkeys : w.gkeys) + s0;
    if (n > kWarpSortCap) {  // listed for k_tile_sort_mid (from the top of the list) or k_tile_sort_big
      if (lane == 0) {
        if (n <= kMidSortCap) big_list[2 * p.tiles + 1 - atomicAdd(w.counters + kMidCount, 1)] = item;
        else big_list[atomicAdd(w.counters + kQueueSort + 1, 1)] = item;
      }
      continue;
    }
    if (n > 1 && n <= 32) {
      unsigned long long key = lane < n ? keys[lane] : ~0ull;
      for (int k = 2; k <= 32; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, j);
          const bool up = (lane & k) == 0;
          const bool lower = (lane & j) == 0;
          key = (lower == up) ? (key < other ? key : other) : (key < other ? other : key);
        }
      if (lane < n) keys[lane] = key;
    } else if (n > 32) {
      int N = 64;
      while (N < n) N <<= 1;
      for (int i = lane; i < N; i += 32) sk[i] = i < n ? keys[i] : ~0ull;
      __syncwarp();
      if (n < kRadixMin) warp_bitonic_smem(sk, N, lane);
      else warp_sort_segment<kWarpSortCap / 32>(sk, bins, n, N, bnd, lane);
      for (int i = lane; i < n; i += 32) keys[i] = sk[i];
      __syncwarp();
    }
    if (bnd) {
      __syncwarp();
      gather_boundary(w, s0, s1, lane, 32);
    }
  }
}

// Segments of kWarpSortCap + 1 .. kMidSortCap keys (listed from the top of
// big_list): one warp each, as in k_tile_sort with 32 keys per lane.
__global__ void __launch_bounds__(kSortThreads, 2) k_tile_sort_mid(Params p, Work w, const int *big_list) {
  extern __shared__ __align__(16) unsigned long long s_mid[];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  unsigned long long *sk = s_mid + wp * kMidSortCap;
  unsigned *bins = reinterpret_cast<unsigned *>(s_mid + (kSortThreads / 32) * kMidSortCap) + wp * 256;
  const int nmid = w.counters[kMidCount];
  for (int it = blockIdx.x * (kSortThreads / 32) + wp; it < nmid; it += gridDim.x * (kSortThreads / 32)) {
    bool bnd;
    long long s0, s1;
    segment_bounds(p, w, big_list[2 * p.tiles + 1 - it], bnd, s0, s1);
    const int n = (int)(s1 - s0);
    unsigned long long *keys = (bnd ? w.bkeys : w.gkeys) + s0;
    int N = 64;
    while (N < n) N <<= 1;
    for (int i = lane; i < N; i += 32) sk[i] = i < n ? keys[i] : ~0ull;
    __syncwarp();
    warp_sort_segment<kMidSortCap / 32>(sk, bins, n, N, bnd, lane);
    for (int i = lane; i < n; i += 32) keys[i] = sk[i];
    __syncwarp();
    if (bnd) gather_boundary(w, s0, s1, lane, 32);
  }
}

// Segments longer than kMidSortCap: one block each (bitonic in shared memory
// up to kSortCap keys, stable radix sort in global memory beyond; a block
// radix sort in shared memory measured slower on dense tiles).
__global__ void __launch_bounds__(kSortThreads) k_tile_sort_big(Params p, Work w, const int *big_list,
                                                               unsigned long long *gtmp, unsigned long long *btmp) {
  __shared__ unsigned long long s_keys[kSortCap];
  __shared__ int s_hist[256], s_base[256];
  __shared__ int s_wcnt[(kSortThreads / 32) * 256];
  __shared__ unsigned long long s_red[2 * (kSortThreads / 32)];
  const int nbig = w.counters[kQueueSort + 1];
  for (int b = blockIdx.x; b < nbig; b += gridDim.x) {
    bool bnd;
    long long s0, s1;
    segment_bounds(p, w, big_list[b], bnd, s0, s1);
    const int n = (int)(s1 - s0);
    unsigned long long *keys = (bnd ? w.bkeys : w.gkeys) + s0;
    unsigned long long *tmp = (bnd ? btmp : gtmp) + s0;
    if (n <= kSortCap) {
      for (int i = threadIdx.x; i < n; i += kSortThreads) s_keys[i] = keys[i];
      __syncthreads();
      bitonic_smem(s_keys, n);
      for (int i = threadIdx.x; i < n; i += kSortThreads) keys[i] = s_keys[i];
    } else {
      radix_global(keys, tmp, n, s_hist, s_base, s_wcnt, s_red);
    }
    __syncthreads();
    if (bnd) gather_boundary(w, s0, s1, threadIdx.x, kSortThreads);
    __syncthreads();
  }
}

}  // namespace

int launch_exclusive_scan(const int *in, long long *out, int n, long long *aux, cudaStream_t st) {
  // out[0..n) = exclusive prefix sums of in, out[n] = total
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(long long), st);
    return 0;
  }
  const int nb = (n + kScanChunk - 1) / kScanChunk;
  k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, aux);
  k_scan_top<<<1, kScanThreads, 0, st>>>(aux, nb);
  k_scan_down<<<nb, kScanThreads, 0, st>>>(in, out, n, aux);
  return 3;
}

cudaError_t configure_binning() {
  cudaError_t e = cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSortSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tile_sort_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSortMidSmem);
  return e;
}

int launch_bin_sort_only(const Params &p, const Work &w, cudaStream_t st) {
  k_emit<<<16 * 152, 256, 0, st>>>(p, w);
  if (p.tiles <= 0) return 1;
  cudaMemsetAsync(w.counters + kQueueSort, 0, 2 * sizeof(int), st);
  cudaMemsetAsync(w.counters + kMidCount, 0, sizeof(int), st);
  k_tile_sort<<<3 * 152, kSortThreads, kTileSortSmem, st>>>(p, w, w.big_list);
  k_tile_sort_mid<<<2 * 152, kSortThreads, kTileSortMidSmem, st>>>(p, w, w.big_list);
  k_tile_sort_big<<<4 * 152, kSortThreads, 0, st>>>(p, w, w.big_list, w.gkeys + p.max_pairs, w.bkeys + p.max_bpairs);
  return 4;
}

int launch_binning(const Params &p, const Work &w, cudaStream_t st) {
  int k = launch_exclusive_scan(w.g_tcount, w.g_tstart, p.tiles, w.scan_aux, st);
  k += launch_exclusive_scan(w.b_tcount, w.b_tstart, p.tiles, w.scan_aux2, st);
  k_check_capacity<<<1, 1, 0, st>>>(p, w);
  k += 2;
  if (p.tiles > 0) {
    k_tile_desc<<<(p.tiles + 255) / 256, 256, 0, st>>>(p, w);
    k++;
  }
  return k + launch_bin_sort_only(p, w, st);
}

}  // namespace bgt
