// C ABI of the BG-Triangle rasterizer: handle, workspace, launch sequences,
// CUDA-graph capture, autotuner and stage access. See include/bgt.h.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bgt.h"
#include "bgt_internal.cuh"

namespace bgt {
// split.cu (its arguments are the C-ABI structs)
int launch_subdivide(int degree, const bgt_scene &sc, const int *sel, int n_sel, const bgt_prims &out,
                     cudaStream_t st);
}  // namespace bgt

using bgt::View;

struct bgt_handle {
  bgt_config cfg;
  int device = 0;
  long long Pcap = 0, Fcap = 0, Kcap = 0, Kbcap = 0, Bcap = 0;
  int Tcap = 0, Vcap = 0, Mcap = 0, nblk_cap = 0;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  bgt::Work w{};
  View *d_views = nullptr;
  int *d_offs = nullptr;
  View *h_views = nullptr;  // pinned staging
  int *h_offs = nullptr;    // pinned staging
  int *h_status = nullptr;  // pinned
  cudaEvent_t staged = nullptr;
  int tile = 16;
  // scheduling knobs of bgt_tuning other than the tile size
  int raster_prims = 8, bwd_dequeue = 1, chain_bps = 8;
  // last forward
  bool fwd_valid = false;
  bgt::Params last{};
  const float *fwd_ctrl = nullptr;
  int fwd_views = 0;
  std::vector<int> fwd_shapes;
  // graphs
  cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;
  std::string g_fwd_key, g_bwd_key;
  // profiling: events between stages, kernels enqueued per pass; count_units:
  // the blending kernels also count their work units (their counting build)
  bool profiling = false, count_units = false;
  cudaEvent_t prof[12] = {};
  int kernels_fwd = 0, kernels_bwd = 0;
  std::string err;
};

namespace {

bgt_status fail(bgt_handle *h, bgt_status s, const char *msg) {
  if (h) h->err = msg;
  return s;
}

bgt_status cuda_fail(bgt_handle *h, cudaError_t e, const char *where) {
  if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return BGT_ERR_CUDA;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(long long count) {
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += align_up(sizeof(T) * (size_t)(count > 0 ? count : 1));
    return p;
  }
};

void carve(bgt_handle *h, char *base, size_t *total) {
  Carver c{base};
  bgt::Work &w = h->w;
  const long long P = h->Pcap, F = h->Fcap, K = h->Kcap, Kb = h->Kbcap;
  const int T = h->Tcap;
  h->d_views = c.take<View>(h->Vcap);
  h->d_offs = c.take<int>(2 * (h->Vcap + 1));
  w.zbuf = c.take<unsigned long long>(P);
  w.pid = c.take<int>(P);
  w.vis_seen = c.take<unsigned long long>(h->Mcap);
  w.puv = c.take<float2>(P);
  w.pix_gidx = c.take<int>(P);
  w.T_final = c.take<float>(P);
  w.n_contrib = c.take<int>(P);
  w.blk_cnt = c.take<int>(2 * (long long)h->nblk_cap);
  w.blk_off = c.take<long long>(2 * ((long long)h->nblk_cap + 1));
  w.counters = c.take<int>(16);
  w.stats = c.take<unsigned long long>(8);
  w.status = c.take<int>(1);
  w.gA = c.take<float4>(F);
  w.gB = c.take<float4>(F);
  w.gC = c.take<float4>(F);
  w.g_pix = c.take<int>(F);
  w.g_view = c.take<int>(F);
  w.g_bidx = c.take<int>(F);
  w.g_prim = c.take<int>(F);
  w.g_uv = c.take<float2>(F);
  w.g_rect = c.take<uint2>(F);
  w.g_depth = c.take<float>(F);
  w.g_dsub = c.take<unsigned char>(F);
  w.bR = c.take<float4>(F);
  w.b_pix = c.take<int>(F);
  w.b_prim = c.take<int>(F);
  w.b_view = c.take<int>(F);
  w.b_uv = c.take<float2>(F);
  w.b_sigma = c.take<float>(F);
  w.b_z = c.take<float>(F);
  w.b_rect = c.take<uint2>(F);
  w.g_tcount = c.take<int>(T + 1);
  w.g_tstart = c.take<long long>(T + 1);
  w.g_tfill = c.take<int>(T + 1);
  w.b_tcount = c.take<int>(T + 1);
  w.b_tstart = c.take<long long>(T + 1);
  w.b_tfill = c.take<int>(T + 1);
  const long long naux = std::max<long long>(std::max<long long>(T, h->nblk_cap), h->Mcap) / 4096 + 4;
  w.scan_aux = c.take<long long>(2 * naux);
  w.scan_aux2 = w.scan_aux ? w.scan_aux + naux : nullptr;
  w.big_list = c.take<int>(2 * (long long)T + 2);
  w.tile_desc = c.take<int4>(2 * (long long)T + 2);
  // headers 3/4 of the capacity, fill units 1/64 (fills are per primitive-cache miss: ~1 in 13
  // headers on the 64-view scene, ~1 in 200 on dense tiles)
  w.rec_chunk_cap = (int)(h->Bcap / 4 * 3 / bgt::kRecChunk + 1);
  w.fill_unit_cap = (int)(h->Bcap / 64 + bgt::kFillChunk * 4 * 1024);
  w.rec_hdr = c.take<uint4>((long long)w.rec_chunk_cap * bgt::kRecChunk);
  w.rec_prev = c.take<int>(w.rec_chunk_cap);
  w.rec_fill = c.take<int>((long long)w.fill_unit_cap * 32);
  w.blk_rec = c.take<int2>(8 * (long long)T + 8);  // warp blocks: at most 8 per tile at any tile size
  w.walk_list = c.take<int>(8 * (long long)T + 8);
  w.gkeys = c.take<unsigned long long>(2 * K);   // second half: sort scratch
  w.bkeys = c.take<unsigned long long>(2 * Kb);  // second half: sort scratch
  w.bl_prim = c.take<int>(Kb);
  w.bl_rec = c.take<float4>(Kb);
  w.prim_cov = c.take<float>(6 * (long long)h->Mcap);
  w.prim_gcov = c.take<float>(6 * (long long)h->Mcap);
  w.gg = c.take<float>(12 * F);
  w.bg_grad = c.take<float4>(F);
  w.prim_gcnt = c.take<int>(h->Mcap);
  w.prim_bcnt = c.take<int>(h->Mcap);
  w.prim_gseg = c.take<long long>((long long)h->Mcap + 1);
  w.prim_bseg = c.take<long long>((long long)h->Mcap + 1);
  w.pg_rec = c.take<float4>(4 * F);
  w.pb_rec = c.take<float4>(2 * F);
  w.Fcap = F;
  w.nblk = h->nblk_cap;
  w.views = h->d_views;
  w.view_pix_off = h->d_offs;
  w.view_tile_off = h->d_offs + (h->Vcap + 1);
  *total = c.off;
}

bool cfg_ok(const bgt_config *c, const char **why) {
  if (c->degree < 1 || c->degree > bgt::kMaxDegree) return *why = "degree must be 1..4", false;
  if (c->max_prims < 0 || c->max_views < 1 || c->max_views > bgt::kMaxViews) return *why = "max_views must be 1..4096", false;
  if (c->max_pixels < 1 || c->max_pixels > (1ll << bgt::kIndexBits)) return *why = "max_pixels must be 1..2^27", false;
  if (c->max_pairs < 1 || c->max_pairs > (1ll << 31) - 1) return *why = "max_pairs must be 1..2^31-1", false;
  if (c->max_boundary_pairs < 1 || c->max_boundary_pairs > (1ll << 31) - 1) return *why = "max_boundary_pairs must be 1..2^31-1", false;
  if (c->max_blend_pairs < 0 || c->max_blend_pairs > (1ll << 31) - 1) return *why = "max_blend_pairs must be 0..2^31-1", false;
  if (c->tess_level < 1 || c->tess_level > bgt::kMaxTess) return *why = "tess_level must be 1..16", false;
  if (c->tile_size != 8 && c->tile_size != 16 && c->tile_size != 32) return *why = "tile_size must be 8, 16 or 32", false;
  if ((long long)c->max_prims * 2 * c->tess_level * c->tess_level > 0xffffffffll) return *why = "max_prims * 2 L^2 must fit 32 bits", false;
  if (!(c->alpha_min > 0.f && c->alpha_min < c->alpha_max && c->alpha_max <= 1.f)) return *why = "need 0 < alpha_min < alpha_max <= 1", false;
  if (!(c->t_stop >= 0.f && c->t_stop < 1.f) || !(c->dilation >= 0.f) || !(c->k_b > 0.f) || !(c->near_z > 0.f))
    return *why = "bad t_stop / dilation / k_b / near_z", false;
  return true;
}

// Upload the view table of this call and fill the per-call parameters.
bgt_status setup_call(bgt_handle *h, const bgt_scene *sc, const bgt_camera *cams, int n, cudaStream_t st,
                      bgt::Params &p) {
  if (!sc || !cams || n < 1) return fail(h, BGT_ERR_INVALID_ARG, "null scene / cameras or n_views < 1");
  if (n > h->Vcap) return fail(h, BGT_ERR_CAPACITY, "n_views exceeds max_views");
  if (sc->num_prims < 0 || sc->num_prims > h->Mcap) return fail(h, BGT_ERR_CAPACITY, "num_prims exceeds max_prims");
  if (sc->num_prims > 0 && (!sc->ctrl || !sc->color || !sc->opacity || !sc->r_b || !sc->log_scale || !sc->quat))
    return fail(h, BGT_ERR_INVALID_ARG, "null scene array");
  const int R = sc->attr_res == 0 ? 1 : sc->attr_res;
  if (R < 1 || R > 16) return fail(h, BGT_ERR_INVALID_ARG, "attr_res must be 0..16");
  if (sc->sh_degree < 0 || sc->sh_degree > 3) return fail(h, BGT_ERR_INVALID_ARG, "sh_degree must be 0..3");
  if (sc->sh_degree > 0 && sc->num_prims > 0 && !sc->sh) return fail(h, BGT_ERR_INVALID_ARG, "null sh array");
  const int t = h->tile;
  cudaError_t e = cudaEventSynchronize(h->staged);  // previous upload has left the staging buffer
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
  long long P = 0, tiles = 0;
  for (int v = 0; v < n; v++) {
    const bgt_camera &c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768)
      return fail(h, BGT_ERR_INVALID_ARG, "view size must be 1..32768");
    bool finite = std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy);
    for (int k = 0; k < 9; k++) finite = finite && std::isfinite(c.R[k]);
    for (int k = 0; k < 3; k++) finite = finite && std::isfinite(c.t[k]);
    if (!finite || c.fx <= 0.f || c.fy <= 0.f) return fail(h, BGT_ERR_INVALID_ARG, "non-finite camera or fx, fy <= 0");
    View &vw = h->h_views[v];
    memset(&vw, 0, sizeof(View));
    memcpy(vw.R, c.R, sizeof(vw.R));
    memcpy(vw.t, c.t, sizeof(vw.t));
    vw.fx = c.fx; vw.fy = c.fy; vw.cx = c.cx; vw.cy = c.cy;
    vw.W = c.width; vw.H = c.height;
    vw.tiles_x = (c.width + t - 1) / t;
    vw.tiles_y = (c.height + t - 1) / t;
    vw.pix_off = (int)P;
    vw.tile_off = (int)tiles;
    h->h_offs[v] = (int)P;
    h->h_offs[h->Vcap + 1 + v] = (int)tiles;
    P += (long long)c.width * c.height;
    tiles += (long long)vw.tiles_x * vw.tiles_y;
    if (P > h->Pcap) return fail(h, BGT_ERR_CAPACITY, "total pixels exceed max_pixels");
    if (tiles > h->Tcap) return fail(h, BGT_ERR_CAPACITY, "total tiles exceed capacity");
  }
  h->h_offs[n] = (int)P;
  h->h_offs[h->Vcap + 1 + n] = (int)tiles;
  e = cudaMemcpyAsync(h->d_views, h->h_views, sizeof(View) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_offs, h->h_offs, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_offs + h->Vcap + 1, h->h_offs + h->Vcap + 1, sizeof(int) * (n + 1),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(h->staged, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "view upload");
  const bgt_config &c = h->cfg;
  p.n = c.degree;
  p.ncp = bgt::ncp_of(c.degree);
  p.M = sc->num_prims;
  p.L = c.tess_level;
  p.near_z = c.near_z;
  p.k_b = c.k_b;
  p.alpha_min = c.alpha_min;
  p.alpha_max = c.alpha_max;
  p.t_stop = c.t_stop;
  p.dilation = c.dilation;
  p.log_alpha_min = logf(c.alpha_min);
  p.use_boundary = (c.flags & BGT_FLAG_NO_BOUNDARY) ? 0 : 1;
  p.tile = t;
  p.V = n;
  p.P = (int)P;
  p.tiles = (int)tiles;
  p.bg[0] = sc->bg[0]; p.bg[1] = sc->bg[1]; p.bg[2] = sc->bg[2];
  p.max_pairs = h->Kcap;
  p.max_bpairs = h->Kbcap;
  p.stats = h->count_units ? 1 : 0;
  p.attr_res = R;
  p.ntex = R * (R + 1) / 2;
  p.sh_deg = sc->sh_degree;
  p.sh_k = (sc->sh_degree + 1) * (sc->sh_degree + 1) - 1;
  p.raster_prims = h->raster_prims;
  p.bwd_dequeue = h->bwd_dequeue;
  p.chain_bps = h->chain_bps;
  return BGT_OK;
}

bgt::Scene to_scene(const bgt_scene *s) {
  return bgt::Scene{s->ctrl, s->color, s->opacity, s->r_b, s->log_scale, s->quat, s->sh_degree > 0 ? s->sh : nullptr};
}

// stage boundaries recorded when profiling: 0 fwd start, 1 after prep, 2 raster,
// 3 resolve, 4 generate, 5 binning, 6 composite fwd; 7 bwd start, 8 composite
// bwd, 9 chain
void mark(bgt_handle *h, int i, cudaStream_t st) {
  if (!h->profiling) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(h->prof[i], st, cudaEventRecordExternal);
  else cudaEventRecord(h->prof[i], st);
}

cudaError_t enqueue_fwd(bgt_handle *h, const bgt::Params &p, const bgt::Scene &s, float *images, cudaStream_t st) {
  const bgt::Work &w = h->w;
  const size_t tb = sizeof(int) * (size_t)(p.tiles + 1);
  mark(h, 0, st);
  if (p.stats) cudaMemsetAsync(w.stats, 0, 8 * sizeof(unsigned long long), st);
  cudaMemsetAsync(w.zbuf, 0xff, sizeof(unsigned long long) * (size_t)p.P, st);
  cudaMemsetAsync(w.g_tcount, 0, tb, st);
  cudaMemsetAsync(w.g_tfill, 0, tb, st);
  cudaMemsetAsync(w.b_tcount, 0, tb, st);
  cudaMemsetAsync(w.b_tfill, 0, tb, st);
  cudaMemsetAsync(w.counters, 0, 16 * sizeof(int), st);
  int k = 0;
  mark(h, 1, st);
  k += bgt::launch_raster(p, s, w, st);
  mark(h, 2, st);
  k += bgt::launch_resolve(p, s, w, st);
  mark(h, 3, st);
  k += bgt::launch_prim_cov(p, s, w, st);
  k += bgt::launch_generate(p, s, w, st);
  mark(h, 4, st);
  k += bgt::launch_binning(p, w, st);
  mark(h, 5, st);
  k += bgt::launch_composite_fwd(p, w, images, st);
  mark(h, 6, st);
  h->kernels_fwd = k;
  return cudaGetLastError();
}

cudaError_t enqueue_bwd(bgt_handle *h, const bgt::Params &p, const bgt::Scene &s, const float *dimg,
                        const bgt::Grads &g, cudaStream_t st) {
  const bgt::Work &w = h->w;
  const size_t cp = sizeof(float) * (size_t)p.M * p.ncp * 3;
  mark(h, 7, st);
  if (p.M > 0) {
    cudaMemsetAsync(g.ctrl, 0, cp, st);
    cudaMemsetAsync(g.color, 0, cp, st);
    cudaMemsetAsync(g.opacity, 0, sizeof(float) * (size_t)p.M, st);
    cudaMemsetAsync(g.r_b, 0, sizeof(float) * (size_t)p.M, st);
    if (g.log_scale) cudaMemsetAsync(g.log_scale, 0, sizeof(float) * 3 * (size_t)p.M * p.ntex, st);
    if (g.quat) cudaMemsetAsync(g.quat, 0, sizeof(float) * 4 * (size_t)p.M * p.ntex, st);
    if (g.sh && p.sh_k > 0) cudaMemsetAsync(g.sh, 0, sizeof(float) * 3 * (size_t)p.M * p.sh_k, st);
  }
  int k = bgt::launch_composite_bwd(p, w, dimg, st);
  mark(h, 8, st);
  k += bgt::launch_chain(p, s, w, g, st);
  mark(h, 9, st);
  h->kernels_bwd = k;
  return cudaGetLastError();
}

std::string graph_key(const bgt::Params &p, const void *a, const void *b, const void *c, const void *d,
                      const void *e, const bgt_camera *cams, int n) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%p|%p|%p|%p|%p|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|", a, b, c, d, e, p.M, p.V, p.P,
           p.tiles, p.tile, p.use_boundary, p.attr_res, p.sh_deg, p.raster_prims, p.bwd_dequeue, p.chain_bps);
  std::string k(buf);
  for (int v = 0; v < n; v++) k += std::to_string(cams[v].width) + "x" + std::to_string(cams[v].height) + ",";
  // the parameters passed by value to kernels are part of the graph
  k.append(reinterpret_cast<const char *>(&p.bg[0]), sizeof(float) * 3);
  return k;
}

template <class F>
cudaError_t run_graph(cudaGraphExec_t *exec, std::string *key_slot, const std::string &key, cudaStream_t st, F body) {
  if (*exec && *key_slot == key) return cudaGraphLaunch(*exec, st);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = body();
  e = cudaStreamEndCapture(st, &graph);
  if (eb != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return eb; }
  if (e != cudaSuccess) return e;
  if (*exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(*exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(*exec);
      *exec = nullptr;
    }
  }
  if (!*exec) e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { *exec = nullptr; return e; }
  *key_slot = key;
  return cudaGraphLaunch(*exec, st);
}

}  // namespace

extern "C" {

bgt_status bgt_default_config(bgt_config *c) {
  if (!c) return BGT_ERR_INVALID_ARG;
  memset(c, 0, sizeof(*c));
  c->degree = 2;
  c->max_prims = 100000;
  c->max_views = 64;
  c->max_pixels = 1024 * 1024;
  c->max_pairs = 8ll * 1024 * 1024;
  c->max_boundary_pairs = 8ll * 1024 * 1024;
  c->tess_level = 8;
  c->tile_size = 16;
  c->k_b = 3.0f;
  c->alpha_min = 1.0f / 255.0f;
  c->alpha_max = 0.99f;
  c->t_stop = 1e-4f;
  c->dilation = 0.3f;
  c->near_z = 0.2f;
  c->flags = 0;
  return BGT_OK;
}

bgt_status bgt_create(const bgt_config *cfg, bgt_handle **out) {
  if (!cfg || !out) return BGT_ERR_INVALID_ARG;
  *out = nullptr;
  const char *why = nullptr;
  if (!cfg_ok(cfg, &why)) return BGT_ERR_INVALID_ARG;
  bgt_handle *h = new bgt_handle();
  h->cfg = *cfg;
  h->tile = cfg->tile_size;
  cudaGetDevice(&h->device);
  h->Pcap = cfg->max_pixels;
  h->Fcap = cfg->max_pixels;
  h->Kcap = cfg->max_pairs;
  h->Kbcap = cfg->max_boundary_pairs;
  // default 8 per pixel, at least 4M (every resident warp holds a partly used fill chunk); warp
  // blocks whose records do not fit are differentiated by re-walking their tile lists
  h->Bcap = cfg->max_blend_pairs > 0 ? cfg->max_blend_pairs : std::max(8 * cfg->max_pixels, 1ll << 22);
  if (h->Bcap > (1ll << 31) - 1024) h->Bcap = (1ll << 31) - 1024;
  h->Vcap = cfg->max_views;
  h->Mcap = cfg->max_prims;
  // tiles of all views at the smallest tile size: sum (W/8+1)(H/8+1) <= P (1/64 + 1/8) + 2 V
  h->Tcap = (int)(h->Pcap * 9 / 64 + 2ll * h->Vcap + 1);
  h->nblk_cap = (int)((h->Pcap + 127) / 128);  // warp chunks of 128 pixels (sub-primitive generation)
  size_t total = 0;
  carve(h, nullptr, &total);
  cudaError_t e = cudaMalloc(&h->arena, total);
  if (e != cudaSuccess) {
    cuda_fail(h, e, "cudaMalloc workspace");
    delete h;
    return BGT_ERR_CUDA;
  }
  h->arena_bytes = total;
  carve(h, static_cast<char *>(h->arena), &total);
  e = cudaMallocHost(&h->h_views, sizeof(View) * h->Vcap);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_offs, sizeof(int) * 2 * (h->Vcap + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_status, sizeof(int) * 16);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->staged, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(h->w.status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->w.counters, 0, 16 * sizeof(int));
  if (e == cudaSuccess) e = bgt::configure_composite();
  if (e == cudaSuccess) e = bgt::configure_binning();
  if (e != cudaSuccess) {
    bgt_destroy(h);
    return BGT_ERR_CUDA;
  }
  *out = h;
  return BGT_OK;
}

void bgt_destroy(bgt_handle *h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t ev : h->prof)
    if (ev) cudaEventDestroy(ev);
  if (h->g_fwd) cudaGraphExecDestroy(h->g_fwd);
  if (h->g_bwd) cudaGraphExecDestroy(h->g_bwd);
  if (h->staged) cudaEventDestroy(h->staged);
  if (h->h_views) cudaFreeHost(h->h_views);
  if (h->h_offs) cudaFreeHost(h->h_offs);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->arena) cudaFree(h->arena);
  delete h;
}

bgt_status bgt_render_fwd(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views,
                          float *images, void *stream) {
  if (!h) return BGT_ERR_INVALID_ARG;
  if (!images) return fail(h, BGT_ERR_INVALID_ARG, "null images");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bgt::Params p;
  bgt_status s = setup_call(h, scene, cams, n_views, st, p);
  if (s != BGT_OK) return s;
  const bgt::Scene sc = to_scene(scene);
  cudaError_t e;
  if ((h->cfg.flags & BGT_FLAG_GRAPH) && st != nullptr) {
    const std::string key = graph_key(p, scene->ctrl, scene->color, scene->opacity, scene->r_b, images, cams, n_views) +
                            std::to_string((size_t)scene->quat) + std::to_string((size_t)scene->log_scale) +
                            std::to_string((size_t)scene->sh) + (h->profiling ? "P" : "-") + (h->count_units ? "U" : "-");
    e = run_graph(&h->g_fwd, &h->g_fwd_key, key, st, [&]() { return enqueue_fwd(h, p, sc, images, st); });
  } else {
    e = enqueue_fwd(h, p, sc, images, st);
  }
  if (e != cudaSuccess) {
    h->fwd_valid = false;
    return cuda_fail(h, e, "forward launch");
  }
  h->fwd_valid = true;
  h->last = p;
  h->fwd_ctrl = scene->ctrl;
  h->fwd_views = n_views;
  h->fwd_shapes.assign(2 * n_views, 0);
  for (int v = 0; v < n_views; v++) {
    h->fwd_shapes[2 * v] = cams[v].width;
    h->fwd_shapes[2 * v + 1] = cams[v].height;
  }
  return BGT_OK;
}

bgt_status bgt_render_bwd(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views,
                          const float *d_images, const bgt_grads *grads, void *stream) {
  if (!h) return BGT_ERR_INVALID_ARG;
  if (!d_images || !grads || !scene || !cams) return fail(h, BGT_ERR_INVALID_ARG, "null argument");
  if (scene->num_prims > 0 && (!grads->ctrl || !grads->color || !grads->opacity || !grads->r_b))
    return fail(h, BGT_ERR_INVALID_ARG, "null gradient array");
  if (!h->fwd_valid) return fail(h, BGT_ERR_STATE, "backward without a forward");
  bool same = scene->ctrl == h->fwd_ctrl && n_views == h->fwd_views && scene->num_prims == h->last.M;
  for (int v = 0; same && v < n_views; v++)
    same = cams[v].width == h->fwd_shapes[2 * v] && cams[v].height == h->fwd_shapes[2 * v + 1];
  if (!same) return fail(h, BGT_ERR_STATE, "backward scene / views differ from the forward");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bgt::Params p = h->last;
  const bgt::Scene sc = to_scene(scene);
  const bgt::Grads g{grads->ctrl, grads->color, grads->opacity, grads->r_b, grads->log_scale, grads->quat,
                     scene->sh_degree > 0 ? grads->sh : nullptr};
  cudaError_t e;
  if ((h->cfg.flags & BGT_FLAG_GRAPH) && st != nullptr) {
    const std::string key = graph_key(p, scene->ctrl, d_images, grads->ctrl, grads->color, grads->opacity, cams,
                                      n_views) + std::to_string((size_t)grads->r_b) +
                            std::to_string((size_t)grads->log_scale) + std::to_string((size_t)grads->quat) +
                            std::to_string((size_t)grads->sh) + (h->profiling ? "P" : "-") + (h->count_units ? "U" : "-");
    e = run_graph(&h->g_bwd, &h->g_bwd_key, key, st, [&]() { return enqueue_bwd(h, p, sc, d_images, g, st); });
  } else {
    e = enqueue_bwd(h, p, sc, d_images, g, st);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "backward launch");
  return BGT_OK;
}

bgt_status bgt_sync_status(bgt_handle *h, void *stream) {
  if (!h) return BGT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h->h_status, h->w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  const int s = h->h_status[0];
  cudaMemsetAsync(h->w.status, 0, sizeof(int), st);
  if (s & (bgt::kStatusPairOverflow | bgt::kStatusBoundaryOverflow | bgt::kStatusTileOverflow))
    return fail(h, BGT_ERR_CAPACITY, "device-side pair count exceeded its capacity");
  if (s & bgt::kStatusNonFinite) return fail(h, BGT_ERR_NONFINITE, "non-finite projected Gaussian");
  if (s & bgt::kStatusBadPrim) return fail(h, BGT_ERR_STATE, "depth buffer held an invalid primitive id");
  return BGT_OK;
}

const char *bgt_last_error(const bgt_handle *h) { return h ? h->err.c_str() : ""; }

bgt_status bgt_get_counts(bgt_handle *h, long long out[8], void *stream) {
  if (!h || !out) return BGT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(h->h_status + 4, h->w.counters, 11 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "counter read");
  for (int i = 0; i < 4; i++) out[i] = h->h_status[4 + i];
  out[4] = h->last.tiles;
  const int ppt = h->last.tile == 32 ? 4 : 1;
  out[5] = (long long)h->h_status[4 + bgt::kRecChunks] * bgt::kRecChunk;
  out[6] = (long long)h->h_status[4 + bgt::kFillChunks] * bgt::kFillChunk * ppt;
  out[7] = h->h_status[4 + bgt::kWalkCount];
  return BGT_OK;
}

bgt_status bgt_set_tile_size(bgt_handle *h, int t) {
  if (!h || (t != 8 && t != 16 && t != 32)) return BGT_ERR_INVALID_ARG;
  h->tile = t;
  h->fwd_valid = false;
  return BGT_OK;
}

int bgt_get_tile_size(const bgt_handle *h) { return h ? h->tile : 0; }

bgt_status bgt_set_profiling(bgt_handle *h, int on) {
  if (!h) return BGT_ERR_INVALID_ARG;
  if (on && !h->prof[0]) {
    for (cudaEvent_t &ev : h->prof) {
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
    }
  }
  if (on < 0 || on > 2) return fail(h, BGT_ERR_INVALID_ARG, "profiling mode must be 0, 1 or 2");
  h->profiling = on != 0;
  h->count_units = on == 1;
  return BGT_OK;
}

bgt_status bgt_get_profile(bgt_handle *h, float ms[8], int *kernels_fwd, int *kernels_bwd,
                           unsigned long long units[8]) {
  if (!h || !ms) return BGT_ERR_INVALID_ARG;
  if (!h->profiling) return fail(h, BGT_ERR_STATE, "profiling is off");
  cudaError_t e = cudaEventSynchronize(h->prof[9]);
  if (e != cudaSuccess) return cuda_fail(h, e, "profile events");
  const int a[8] = {0, 1, 2, 3, 4, 5, 7, 8}, b[8] = {1, 2, 3, 4, 5, 6, 8, 9};
  for (int i = 0; i < 8; i++) {
    ms[i] = 0.f;
    if (cudaEventElapsedTime(&ms[i], h->prof[a[i]], h->prof[b[i]]) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, BGT_ERR_STATE, "no profiled forward + backward yet");
    }
  }
  if (kernels_fwd) *kernels_fwd = h->kernels_fwd;
  if (kernels_bwd) *kernels_bwd = h->kernels_bwd;
  if (units) {
    e = cudaMemcpy(units, h->w.stats, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "profile units");
  }
  return BGT_OK;
}

bgt_status bgt_get_tuning(const bgt_handle *h, bgt_tuning *out) {
  if (!h || !out) return BGT_ERR_INVALID_ARG;
  out->tile_size = h->tile;
  out->raster_prims = h->raster_prims;
  out->bwd_dequeue = h->bwd_dequeue;
  out->chain_blocks_per_sm = h->chain_bps;
  return BGT_OK;
}

bgt_status bgt_set_tuning(bgt_handle *h, const bgt_tuning *t) {
  if (!h || !t) return BGT_ERR_INVALID_ARG;
  if ((t->tile_size != 8 && t->tile_size != 16 && t->tile_size != 32) || t->raster_prims < 1 ||
      t->raster_prims > 64 || t->bwd_dequeue < 1 || t->bwd_dequeue > 8 || t->chain_blocks_per_sm < 1 ||
      t->chain_blocks_per_sm > 32)
    return fail(h, BGT_ERR_INVALID_ARG, "tuning value out of range");
  if (t->tile_size != h->tile) h->fwd_valid = false;
  h->tile = t->tile_size;
  h->raster_prims = t->raster_prims;
  h->bwd_dequeue = t->bwd_dequeue;
  h->chain_bps = t->chain_blocks_per_sm;
  return BGT_OK;
}

namespace {

// ms per forward + backward pass of the handle's current scheduling (one
// untimed pass first), timed with CUDA events on the stream
bgt_status time_passes(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views, float *images,
                       const float *d_images, const bgt_grads *grads, int iters, void *stream, cudaEvent_t a,
                       cudaEvent_t b, float *ms) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->fwd_valid = false;
  bgt_status s = bgt_render_fwd(h, scene, cams, n_views, images, stream);
  if (s == BGT_OK) s = bgt_render_bwd(h, scene, cams, n_views, d_images, grads, stream);
  if (s != BGT_OK) return s;
  cudaEventRecord(a, st);
  for (int i = 0; i < iters && s == BGT_OK; i++) {
    s = bgt_render_fwd(h, scene, cams, n_views, images, stream);
    if (s == BGT_OK) s = bgt_render_bwd(h, scene, cams, n_views, d_images, grads, stream);
  }
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  *ms = 0.f;
  cudaEventElapsedTime(ms, a, b);
  *ms /= iters;
  if (s == BGT_OK) s = bgt_sync_status(h, stream);
  return s;
}

}  // namespace

bgt_status bgt_autotune(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views, float *images,
                        const float *d_images, const bgt_grads *grads, int iters, int *best, float *ms_out,
                        void *stream) {
  if (!h || iters < 1) return BGT_ERR_INVALID_ARG;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  bgt_status s = BGT_OK;
  // Each knob's candidates are timed in two interleaved rounds (a b c a b c) and
  // each keeps its faster time, so that a drift of the clock during tuning
  // does not decide between candidates a few per cent apart.
  constexpr int kRounds = 2;
  // 1. tile size
  const int sizes[3] = {8, 16, 32};
  float tile_ms[3] = {3e38f, 3e38f, 3e38f};
  for (int r = 0; r < kRounds && s == BGT_OK; r++)
    for (int k = 0; k < 3 && s == BGT_OK; k++) {
      h->tile = sizes[k];
      float ms = 0.f;
      s = time_passes(h, scene, cams, n_views, images, d_images, grads, iters, stream, a, b, &ms);
      if (s == BGT_OK) tile_ms[k] = std::min(tile_ms[k], ms);
    }
  int best_t = sizes[0];
  float best_ms = tile_ms[0];
  for (int k = 1; k < 3; k++)
    if (tile_ms[k] < best_ms) { best_ms = tile_ms[k]; best_t = sizes[k]; }
  if (ms_out)
    for (int k = 0; k < 3; k++) ms_out[k] = tile_ms[k];
  h->tile = best_t;
  // 2. the work-queue knobs, one at a time at that tile size
  int *knob[3] = {&h->raster_prims, &h->bwd_dequeue, &h->chain_bps};
  const int values[3][3] = {{4, 8, 16}, {1, 2, 4}, {4, 8, 16}};
  for (int q = 0; q < 3 && s == BGT_OK; q++) {
    const int keep = *knob[q];
    float knob_ms[3] = {3e38f, 3e38f, 3e38f};
    for (int r = 0; r < kRounds && s == BGT_OK; r++)
      for (int k = 0; k < 3 && s == BGT_OK; k++) {
        *knob[q] = values[q][k];
        float ms = 0.f;
        s = time_passes(h, scene, cams, n_views, images, d_images, grads, iters, stream, a, b, &ms);
        if (s == BGT_OK) knob_ms[k] = std::min(knob_ms[k], ms);
      }
    int best_v = keep;
    float bm = 3e38f;
    for (int k = 0; k < 3; k++)
      if (knob_ms[k] < bm) { bm = knob_ms[k]; best_v = values[q][k]; }
    *knob[q] = s == BGT_OK ? best_v : keep;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->fwd_valid = false;
  if (best) *best = best_t;
  return s;
}

bgt_status bgt_l1_loss_grad(const float *images, const float *target, long long n, float scale, float *d_images,
                            float *loss, void *stream) {
  if (n < 0 || (n > 0 && (!images || !target || !d_images))) return BGT_ERR_INVALID_ARG;
  bgt::launch_l1_grad(images, target, n, scale, d_images, loss, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? BGT_OK : BGT_ERR_CUDA;
}

bgt_status bgt_l2_dssim_loss_grad(const float *images, const float *target, int n_views, const int *sizes,
                                  float lambda, float scale, float *d_images, float *loss, void *stream) {
  if (n_views < 0 || (n_views > 0 && !sizes)) return BGT_ERR_INVALID_ARG;
  if (!(lambda >= 0.f && lambda <= 1.f) || !std::isfinite(scale)) return BGT_ERR_INVALID_ARG;
  long long n = 0;
  for (int v = 0; v < n_views; ++v) {
    const int W = sizes[2 * v], H = sizes[2 * v + 1];
    if (W < 0 || H < 0 || (long long)W * H > (1LL << 31) / 3) return BGT_ERR_INVALID_ARG;
    n += 3LL * W * H;
  }
  if (n > 0 && (!images || !target || !d_images)) return BGT_ERR_INVALID_ARG;
  if (n > 0 && (d_images == images || d_images == target)) return BGT_ERR_INVALID_ARG;
  bgt::launch_l2_dssim_grad(images, target, n_views, sizes, lambda, scale, d_images, loss,
                            static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? BGT_OK : BGT_ERR_CUDA;
}

bgt_status bgt_prim_metrics(int degree, const bgt_scene *scene, const float *g_ctrl, float tau_a, float tau_s,
                            float tau_g, const float *edge_sum, const int *edge_count, float tau_b,
                            const int *view_count, int n_views, const unsigned long long *cell_mask, int tess_level,
                            float tau_v, float tau_r, float *area, float *aspect, float *grad, unsigned char *flags,
                            void *stream) {
  if (degree < 1 || degree > bgt::kMaxDegree || !scene || scene->num_prims < 0) return BGT_ERR_INVALID_ARG;
  if (scene->num_prims > 0 && !scene->ctrl) return BGT_ERR_INVALID_ARG;
  if (n_views < 0 || (cell_mask && (tess_level < 1 || tess_level > bgt::kMaxTess))) return BGT_ERR_INVALID_ARG;
  if ((edge_sum == nullptr) != (edge_count == nullptr)) return BGT_ERR_INVALID_ARG;
  bgt::launch_prim_metrics(degree, scene->ctrl, scene->num_prims, g_ctrl, tau_a, tau_s, tau_g, edge_sum, edge_count,
                           tau_b, view_count, n_views, cell_mask, cell_mask ? tess_level : 1, tau_v, tau_r, area,
                           aspect, grad, flags, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? BGT_OK : BGT_ERR_CUDA;
}

bgt_status bgt_edge_magnitude(const float *images, int n_views, const int *sizes, float *edges, void *stream) {
  if (n_views < 0 || (n_views > 0 && !sizes)) return BGT_ERR_INVALID_ARG;
  long long n = 0;
  for (int v = 0; v < n_views; ++v) {
    if (sizes[2 * v] < 0 || sizes[2 * v + 1] < 0) return BGT_ERR_INVALID_ARG;
    n += (long long)sizes[2 * v] * sizes[2 * v + 1];
  }
  if (n > (1LL << 31) / 3) return BGT_ERR_INVALID_ARG;
  if (n > 0 && (!images || !edges)) return BGT_ERR_INVALID_ARG;
  bgt::launch_edge_magnitude(images, n_views, sizes, edges, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? BGT_OK : BGT_ERR_CUDA;
}

bgt_status bgt_edge_prior(bgt_handle *h, const float *edges, float *edge_sum, int *edge_count, void *stream) {
  if (!h) return BGT_ERR_INVALID_ARG;
  if (!h->fwd_valid) return fail(h, BGT_ERR_STATE, "edge prior without a forward");
  if (h->last.P > 0 && !edges) return fail(h, BGT_ERR_INVALID_ARG, "null edges");
  bgt::launch_edge_prior(h->last, h->w, edges, edge_sum, edge_count, static_cast<cudaStream_t>(stream));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BGT_OK : cuda_fail(h, e, "edge prior");
}

bgt_status bgt_visibility(bgt_handle *h, int *view_count, unsigned long long *cell_mask, void *stream) {
  if (!h) return BGT_ERR_INVALID_ARG;
  if (!h->fwd_valid) return fail(h, BGT_ERR_STATE, "visibility without a forward");
  const bgt::Params &p = h->last;
  std::vector<int> off(p.V + 1, 0);
  for (int v = 0; v < p.V; v++) off[v + 1] = off[v] + h->fwd_shapes[2 * v] * h->fwd_shapes[2 * v + 1];
  bgt::launch_visibility(p, h->w, off.data(), view_count, cell_mask, static_cast<cudaStream_t>(stream));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BGT_OK : cuda_fail(h, e, "visibility");
}

bgt_status bgt_subdivide(int degree, const bgt_scene *scene, const int *sel, int n_sel, const bgt_prims *out,
                         void *stream) {
  if (degree < 1 || degree > bgt::kMaxDegree || !scene || scene->num_prims < 0) return BGT_ERR_INVALID_ARG;
  if (n_sel < 0 || n_sel > (1 << 28)) return BGT_ERR_INVALID_ARG;
  if (n_sel == 0) return BGT_OK;
  const int R = scene->attr_res <= 0 ? 1 : scene->attr_res;
  if (R > 16 || scene->sh_degree < 0 || scene->sh_degree > 3) return BGT_ERR_INVALID_ARG;
  if (!sel || !out || !out->ctrl || !out->color || !out->opacity || !out->r_b || !out->log_scale || !out->quat)
    return BGT_ERR_INVALID_ARG;
  if (scene->sh_degree > 0 && !out->sh) return BGT_ERR_INVALID_ARG;
  if (scene->num_prims > 0 && (!scene->ctrl || !scene->color || !scene->opacity || !scene->r_b ||
                               !scene->log_scale || !scene->quat || (scene->sh_degree > 0 && !scene->sh)))
    return BGT_ERR_INVALID_ARG;
  if (out->ctrl == scene->ctrl || out->color == scene->color || out->log_scale == scene->log_scale ||
      out->quat == scene->quat)
    return BGT_ERR_INVALID_ARG;
  bgt::launch_subdivide(degree, *scene, sel, n_sel, *out, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? BGT_OK : BGT_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// stage access
// ---------------------------------------------------------------------------
namespace {

__global__ void k_pack_gauss(bgt::Work w, int F, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  const float4 A = w.gA[i], B = w.gB[i], C = w.gC[i];
  float *o = out + 12 * (size_t)i;
  o[0] = A.x; o[1] = A.y; o[2] = B.x; o[3] = B.y;
  o[4] = B.z; o[5] = B.w; o[6] = A.z; o[7] = C.w;
  o[8] = C.x; o[9] = C.y; o[10] = C.z; o[11] = w.g_depth[i];
}

__global__ void k_pack_ggrad(bgt::Work w, int F, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  float gd[9];
  bgt::gauss_grad_from_sums(w.gg + 12 * (size_t)i, w.gB[i], gd);
  float *o = out + 12 * (size_t)i;
  for (int k = 0; k < 9; k++) o[k] = gd[k];
  o[9] = o[10] = o[11] = 0.f;
}

__global__ void k_pack_bnd(bgt::Work w, int Nb, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nb) return;
  const float4 R = w.bR[i];
  float *o = out + 8 * (size_t)i;
  o[0] = __int_as_float(w.b_pix[i]);
  o[1] = __int_as_float(w.b_prim[i]);
  o[2] = R.y; o[3] = R.z;
  o[4] = w.b_sigma[i];
  o[5] = w.b_z[i];
  o[6] = 0.f; o[7] = 0.f;
}

// synthetic Gaussians for the binning / sort stage on its own
__global__ void k_load_gaussians(bgt::Params p, bgt::Work w, int count, const int *qxy, const float *off,
                                 const float *conic, const float *opac, const float *depth) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const View vw = w.views[0];
  const float Ka = conic[3 * i], Kb = conic[3 * i + 1], Kc = conic[3 * i + 2];
  const float o = opac[i];
  const unsigned q = (unsigned)qxy[i];
  w.gA[i] = make_float4(off[2 * i], off[2 * i + 1], __uint_as_float(q), -1.0f);
  w.gB[i] = make_float4(Ka, Kb, Kc, o);
  w.gC[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(0));
  w.g_depth[i] = depth[i];
  w.g_view[i] = 0;
  w.g_dsub[i] = (unsigned char)(bgt::plain_depth_key(depth[i]) & 31ull);
  const bgt::ConicBox box = bgt::conic_support_box(Ka, Kb, Kc, o, (float)(q & 0xffffu) + off[2 * i],
                                                   (float)(q >> 16) + off[2 * i + 1], vw.W, vw.H, p.tile,
                                                   p.alpha_min, p.log_alpha_min);
  const uint2 rect = box.rect;
  w.gA[i].w = box.r;
  const int x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff, y1 = rect.y >> 16;
  for (int ty = y0; ty <= y1; ty++)
    for (int tx = x0; tx <= x1; tx++) atomicAdd(w.g_tcount + ty * vw.tiles_x + tx, 1);
  w.g_rect[i] = rect;
}

}  // namespace

extern "C" {

bgt_status bgt_get_stage(bgt_handle *h, int which, void *dst, long long bytes, long long *written, void *stream) {
  if (!h || !dst || bytes < 0) return BGT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long cnt[8];
  bgt_status s = bgt_get_counts(h, cnt, stream);
  if (s != BGT_OK) return s;
  const bgt::Params &p = h->last;
  const long long P = p.P, F = cnt[0], Nb = cnt[1];
  const long long K = cnt[2] < h->Kcap ? cnt[2] : h->Kcap, Kb = cnt[3] < h->Kbcap ? cnt[3] : h->Kbcap;
  const void *src = nullptr;
  long long need = 0;
  float *tmp = nullptr;
  switch (which) {
    case 0: src = h->w.pid; need = 4 * P; break;
    case 1: src = h->w.puv; need = 8 * P; break;
    case 2:
    case 3:
    case 10: {
      const long long items = which == 3 ? Nb : F;
      need = (which == 3 ? 32 : 48) * items;
      if (need > bytes) return fail(h, BGT_ERR_CAPACITY, "destination too small");
      // pack through the (unused between calls) sort scratch of the Gaussian keys
      tmp = reinterpret_cast<float *>(h->w.gkeys + h->Kcap);
      if (need > 8 * h->Kcap) return fail(h, BGT_ERR_CAPACITY, "stage larger than scratch");
      if (items > 0) {
        if (which == 2) k_pack_gauss<<<(int)((items + 255) / 256), 256, 0, st>>>(h->w, (int)items, tmp);
        else if (which == 10) k_pack_ggrad<<<(int)((items + 255) / 256), 256, 0, st>>>(h->w, (int)items, tmp);
        else k_pack_bnd<<<(int)((items + 255) / 256), 256, 0, st>>>(h->w, (int)items, tmp);
      }
      src = tmp;
      break;
    }
    case 4: src = h->w.g_tstart; need = 8 * (long long)(p.tiles + 1); break;
    case 5: src = h->w.gkeys; need = 8 * K; break;
    case 6: src = h->w.b_tstart; need = 8 * (long long)(p.tiles + 1); break;
    case 7: src = h->w.bkeys; need = 8 * Kb; break;
    case 8: src = h->w.T_final; need = 4 * P; break;
    case 9: src = h->w.n_contrib; need = 4 * P; break;
    case 11: src = h->w.bg_grad; need = 16 * Nb; break;
    default: return fail(h, BGT_ERR_INVALID_ARG, "unknown stage");
  }
  if (need > bytes) return fail(h, BGT_ERR_CAPACITY, "destination too small");
  cudaError_t e = cudaSuccess;
  if (need > 0) e = cudaMemcpyAsync(dst, src, (size_t)need, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage copy");
  if (written) *written = need;
  return BGT_OK;
}

bgt_status bgt_bin_sort(bgt_handle *h, int width, int height, int count, const int *qxy, const float *off,
                        const float *conic, const float *opacity, const float *depth, void *stream) {
  if (!h || count < 0 || (count > 0 && (!qxy || !off || !conic || !opacity || !depth)))
    return BGT_ERR_INVALID_ARG;
  if (count > h->Fcap) return fail(h, BGT_ERR_CAPACITY, "count exceeds max_pixels");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bgt_camera cam;
  memset(&cam, 0, sizeof(cam));
  cam.R[0] = cam.R[4] = cam.R[8] = 1.f;
  cam.fx = cam.fy = 1.f;
  cam.width = width;
  cam.height = height;
  bgt_scene sc;
  memset(&sc, 0, sizeof(sc));
  bgt::Params p;
  bgt_status s = setup_call(h, &sc, &cam, 1, st, p);
  if (s != BGT_OK) return s;
  const bgt::Work &w = h->w;
  const size_t tb = sizeof(int) * (size_t)(p.tiles + 1);
  cudaMemsetAsync(w.g_tcount, 0, tb, st);
  cudaMemsetAsync(w.g_tfill, 0, tb, st);
  cudaMemsetAsync(w.b_tcount, 0, tb, st);
  cudaMemsetAsync(w.b_tfill, 0, tb, st);
  cudaMemsetAsync(w.counters, 0, 16 * sizeof(int), st);
  if (count > 0)
    k_load_gaussians<<<(count + 255) / 256, 256, 0, st>>>(p, w, count, qxy, off, conic, opacity, depth);
  cudaMemcpyAsync(w.counters + bgt::kF, &count, sizeof(int), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  bgt::launch_binning(p, w, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "bin_sort launch");
  h->last = p;
  h->fwd_valid = false;
  return BGT_OK;
}

}  // extern "C"
