// C ABI of the scorer (declared in include/nbvgs.h): context, memory, and the
// per-view launch sequence
//   project -> scan -> duplicate -> radix sort -> ranges -> composite(+IG)
//   -> per-Gaussian log-det gains -> reduction -> scores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "nbv_internal.cuh"

namespace nbv {
size_t scan_scratch_elems(int64_t n);
size_t radix_hist_elems(int64_t count);

int device_sm_count() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
    cudaGetLastError();
    nsm = 1;
  }
  cache[dev] = nsm;
  return nsm;
}
}  // namespace nbv

namespace {
// Entries of one binning pass are offset and ranged in 32-bit integers.
constexpr int64_t kMaxPassEntries = int64_t(0xFFFFFFFF) - 4096;
// Internal return code of batched_setup: the pass would hold more entries
// than the limit (the caller splits the candidates).
constexpr int kTooManyEntries = 1;
}  // namespace

using namespace nbv;

struct nbv_ctx {
  // capacity of every buffer alloc() manages, keyed by the address of its pointer
  std::unordered_map<const void*, size_t> alloc_caps;
  nbv_config cfg;
  Consts c;
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;   // private stream on which graphs are captured
  int tw = 16, th = 16;            // screen tile (16 x 16 or 32 x 8)
  int stage = 32;                  // Gaussians staged per round in the compositing kernel
  int device = 0;
  std::string err;
  bool cuda_dead = false;
  int64_t launches = 0;
  int nB = 0, nBp = 0;

  // scene
  int64_t n = 0;
  bool scene_ok = false;        // the last load passed the input check
  float *mu = nullptr, *logs = nullptr, *q = nullptr, *rho = nullptr, *sh = nullptr, *obj = nullptr;
  float4 *mu_sig = nullptr, *scale_skip = nullptr, *qn = nullptr, *aux = nullptr;
  float* p = nullptr;
  int prepared_target = -2;
  // active set of the last prepare (Gaussians with c_g > 0): blocks, factors
  // and gains are kept for these only, in slot order
  int* slot = nullptr;            // [n]
  int* act = nullptr;             // [n]
  int64_t n_act = 0;
  int last_target = -2;           // target of the active set above

  // cameras
  std::vector<nbv_camera> train, cand;
  DevCam* d_train_cams = nullptr;

  // per-view projection
  DevProj pr{};
  // sort
  SortBuffers sb{};
  // per-view binning in depth order: the slots with entries compacted with
  // their depth keys and sorted, their entry counts gathered and scanned in
  // that order, the view's camera and tile base on the device
  struct ViewBin {
    uint32_t* flags = nullptr;
    uint32_t* pos = nullptr;        // [n + 1]
    uint32_t* scan_tmp = nullptr;
    SortBuffers db{};               // depth keys of the slots with entries
    uint32_t* tcount = nullptr;     // [n]
    uint32_t* doffsets = nullptr;   // [n + 1]
    DevCam* d_cam = nullptr;        // [1]
    uint32_t* d_tbase = nullptr;    // [1] = 0
  } vb;
  uint4* fwd = nullptr;           // per-view scoring: forward results per (tile, pixel)
  uint32_t* tile_first = nullptr; // and each tile's first active entry
  size_t fwd_cap = 0, tile_first_cap = 0;
  uint32_t* h_total = nullptr;   // pinned [2]: entries of the last per-view pass, its slots with entries
  unsigned long long* h_total64 = nullptr;   // pinned: 64-bit entry count of the last pass
  unsigned long long* d_total64 = nullptr;
  int64_t entry_limit = kMaxPassEntries;     // entries one binning pass may hold
  int nsm = 1;                               // SMs of the context's device
  size_t ranges_cap = 0;

  // blocks and factors
  float* blocks = nullptr;        // [n][nBp]
  float* train_blocks = nullptr;  // [n_train][n][nBp]
  size_t train_blocks_cap = 0;
  Factors F{};
  bool prepared = false;

  // gains and scores
  double* partial = nullptr;
  int partial_cap = 0;
  double* ig_train = nullptr;   // [n_train][3]
  double* ig_cand = nullptr;    // [n_cand][3]
  size_t ig_train_cap = 0, ig_cand_cap = 0;
  float* out4 = nullptr;
  size_t out4_cap = 0;
  int* d_flags = nullptr;       // [0] best, [1] empty flag, [2] input check, [3] a staging wait gave up
  float* d_best_score = nullptr;
  bool scored = false;
  int* d_err = nullptr;

  // profiling: CUDA events bracketing each phase on the context stream
  struct PhaseRec { int phase; cudaEvent_t a, b; int launches; };
  bool prof = false;
  std::vector<PhaseRec> recs;
  std::vector<cudaEvent_t> pool;
  double acc_ms[NBV_NUM_PHASES] = {0};
  int64_t acc_launch[NBV_NUM_PHASES] = {0};
  unsigned long long* d_stats = nullptr;   // composite work counters: [0..3] candidates, [4..7] training
  int64_t composite_launches[2] = {0, 0};
  int64_t binned_entries[2] = {0, 0};      // (view, tile, Gaussian) entries of the binning passes

  // batched multi-view scoring (cfg.batched): buffers sized once per
  // (scene, candidate set), the whole score captured in a CUDA graph
  float* gacc = nullptr;           // backward: per-Gaussian gradients of the projected quantities
  size_t gacc_cap = 0;
  DevCam* d_desc_cams = nullptr;  // candidate cameras for the descriptors
  float* desc_raw = nullptr;
  float* desc = nullptr;
  float* d_pred = nullptr;
  size_t desc_cap = 0;             // candidates the descriptor buffers hold
  struct Batched {
    bool ready = false;             // buffers sized for the current scene / candidates
    int v0 = 0;                     // first candidate of the views this state covers
    int nv = 0, ntiles = 0;
    int64_t total = 0;              // (view, tile, Gaussian) entries
    DevCam* cams = nullptr;
    uint32_t* tile_base = nullptr;  // [nv]
    int* tile_view = nullptr;       // [ntiles]
    DevProj pr{};                   // [nv][n] records
    uint8_t* mark = nullptr;        // [ntiles] tiles an active splat reaches (active subset only)
    int4* bbox = nullptr;           // [nv] each view's bounding box of marked tiles
    uint32_t* flags = nullptr;      // [nv n] slots that emit entries
    int64_t m = 0;                  // how many slots emit entries
    uint32_t* offsets = nullptr;    // [nv n + 1] their positions
    uint32_t* scan_tmp = nullptr;
    SortBuffers db{};               // depth order of the (view, Gaussian) slots
    uint32_t* tcount = nullptr;     // [nv n] tiles touched, in depth order
    const uint32_t* svals = nullptr;  // sorted Gaussian ids of the last multi-view pass
    std::vector<uint32_t> h_base;     // first global tile of each view
    uint32_t* doffsets = nullptr;   // [nv n + 1] their exclusive scan
    SortBuffers sb{};               // entries (32-bit tile keys, stored in the 64-bit arrays)
    SortBuffers qb{};               // work queue
    uint2* ranges = nullptr;        // [ntiles]
    uint4* fwd = nullptr;           // [ntiles][256] forward results
    uint32_t* tile_first = nullptr; // [ntiles]
    int* counter = nullptr;         // [2] work-queue heads of the forward and information passes
    float* blocks = nullptr;        // [nv][n][nBp]
    double* partial = nullptr;
    int parts_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_replay = 0;
    int forced_chunk = 0;           // > 0: the full set was found over the entry limit; views per pass
  } bt;
};

namespace {

int fail(nbv_ctx* x, int code, const std::string& msg) {
  x->err = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ctx->cuda_dead = true;                                                           \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? NBV_ERR_OOM : NBV_ERR_CUDA,   \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                  \
  } while (0)

#define CKR(expr)                  \
  do {                             \
    int r_ = (expr);               \
    if (r_ != NBV_OK) return r_;   \
  } while (0)

template <class T>
int grow(nbv_ctx* ctx, T** ptr, size_t* cap, size_t count) {
  if (*ptr && *cap >= count) return NBV_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  size_t bytes = sizeof(T) * (count > 0 ? count : 1);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(ctx, NBV_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  *cap = count;
  return NBV_OK;
}

template <class T>
int alloc(nbv_ctx* ctx, T** ptr, size_t count) {
  // keeps a buffer that is large enough (re-setting a multi-view path of the
  // same size frees and maps nothing: cudaFree synchronises the device, and
  // mapping gigabytes takes milliseconds)
  size_t& cap = ctx->alloc_caps[static_cast<const void*>(ptr)];
  if (!*ptr) cap = 0;
  return grow(ctx, ptr, &cap, count);
}

bool finite_cam(const nbv_camera& c) {
  for (float v : c.R) if (!std::isfinite(v)) return false;
  for (float v : c.t) if (!std::isfinite(v)) return false;
  return std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy) &&
         c.fx > 0.0f && c.fy > 0.0f && c.width >= 1 && c.height >= 1 && c.width <= 16384 &&
         c.height <= 16384;
}

DevCam to_dev(const nbv_camera& c, int tw, int th) {
  DevCam d;
  for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
  d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
  for (int i = 0; i < 3; ++i)   // camera centre -R^T t, in double then rounded
    d.campos[i] = (float)(-((double)c.R[i] * c.t[0] + (double)c.R[3 + i] * c.t[1] +
                            (double)c.R[6 + i] * c.t[2]));
  d.W = c.width; d.H = c.height;
  d.TW = tw; d.TH = th;
  d.GX = (c.width + d.TW - 1) / d.TW;
  d.GY = (c.height + d.TH - 1) / d.TH;
  return d;
}

DevScene dev_scene(nbv_ctx* ctx) {
  DevScene s;
  s.n = ctx->n;
  s.mu_raw = ctx->mu; s.logs_raw = ctx->logs; s.q_raw = ctx->q; s.rho_raw = ctx->rho;
  s.sh = ctx->sh; s.obj_raw = ctx->obj;
  s.mu_sig = ctx->mu_sig; s.scale_skip = ctx->scale_skip; s.qn = ctx->qn; s.aux = ctx->aux;
  s.p = ctx->p;
  s.slot = ctx->slot;
  s.act = ctx->act;
  s.n_act = ctx->n_act;
  return s;
}

int check_launch(nbv_ctx* ctx, int nl) {
  ctx->launches += nl;
  CK(cudaGetLastError());
  return NBV_OK;
}

cudaEvent_t take_event(nbv_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one phase with CUDA events on the context stream while profiling.
struct Phase {
  nbv_ctx* ctx;
  int ph;
  cudaEvent_t a = nullptr;
  int64_t l0;
  Phase(nbv_ctx* c, int p) : ctx(c), ph(p), l0(c->launches) {
    if (ctx->prof) {
      a = take_event(ctx);
      cudaEventRecord(a, ctx->st);
    }
  }
  ~Phase() {
    if (ctx->prof && a) {
      cudaEvent_t b = take_event(ctx);
      cudaEventRecord(b, ctx->st);
      ctx->recs.push_back({ph, a, b, (int)(ctx->launches - l0)});
    }
  }
};

int bits_for(int64_t n);

// Project, bin and sort one view; composite it (images and/or IG blocks).
int render_view(nbv_ctx* ctx, const nbv_camera& cam, float* blocks, float* rgb, float* depth,
                float* alpha, float* obj, bool compensated = false, bool training = false) {
  cudaStream_t st = ctx->st;
  const DevCam dc = to_dev(cam, ctx->tw, ctx->th);
  const int ntiles = dc.GX * dc.GY;
  DevScene s = dev_scene(ctx);
  {
    Phase ph(ctx, NBV_PHASE_PROJECT);
    CKR(check_launch(ctx, launch_project(s, ctx->c, dc, ctx->pr, st)));
  }
  auto& V = ctx->vb;
  {
    Phase ph(ctx, NBV_PHASE_SORT);
    CKR(check_launch(ctx, launch_scan_u32(ctx->pr.touched, ctx->sb.offsets, ctx->n, ctx->sb.scan_tmp, st)));
    CKR(check_launch(ctx, launch_sum_u64(ctx->pr.touched, ctx->n, ctx->d_total64, st)));
    // the slots with entries and their depth keys (0 << 31 | z bits), in Gaussian order
    CKR(check_launch(ctx, launch_compact_depth_keys(ctx->pr.touched, ctx->n, V.flags, V.pos, V.scan_tmp,
                                                    ctx->pr.zbits, ctx->n, V.db.keys[0], V.db.vals[0], st)));
    CK(cudaMemcpyAsync(ctx->h_total, ctx->sb.offsets + ctx->n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_total + 1, V.pos + ctx->n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_total64, ctx->d_total64, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(V.d_cam, &dc, sizeof(DevCam), cudaMemcpyHostToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
  // the 64-bit count decides: the 32-bit scan (and every offset after the
  // wrap) is only valid below the limit
  if ((int64_t)*ctx->h_total64 > ctx->entry_limit)
    return fail(ctx, NBV_ERR_ARG, "a view has " + std::to_string(*ctx->h_total64) +
                                      " (tile, Gaussian) entries, more than one binning pass holds (" +
                                      std::to_string(ctx->entry_limit) + ")");
  const int64_t total = (int64_t)ctx->h_total[0];
  const int64_t m = (int64_t)ctx->h_total[1];
  if (ctx->prof) ctx->binned_entries[training ? 1 : 0] += total;
  if ((size_t)total > ctx->sb.cap) {
    size_t cap = ctx->sb.cap;
    size_t want = (size_t)(total * 1.25) + 1024;
    size_t c0 = cap, c1 = cap, c2 = cap, c3 = cap;
    CKR(grow(ctx, &ctx->sb.keys[0], &c0, want));
    CKR(grow(ctx, &ctx->sb.keys[1], &c1, want));
    CKR(grow(ctx, &ctx->sb.vals[0], &c2, want));
    CKR(grow(ctx, &ctx->sb.vals[1], &c3, want));
    ctx->sb.cap = want;
    CKR(grow(ctx, &ctx->sb.hist, &ctx->sb.hist_cap, radix_hist_elems((int64_t)want)));
  }
  CKR(grow(ctx, &ctx->sb.ranges, &ctx->ranges_cap, (size_t)ntiles));
  {
    // the slots in depth order (a stable sort of the compacted slots: ties in
    // Gaussian order), their entries emitted in that order with 32-bit tile
    // ids, and a stable sort on the tile id alone: every tile's list in
    // (depth bits, Gaussian index) order
    Phase ph(ctx, NBV_PHASE_SORT);
    int dw = 0;
    CKR(check_launch(ctx, launch_radix_sort(V.db, m, 31, &dw, st)));
    const uint32_t* order = V.db.vals[dw];
    CKR(check_launch(ctx, launch_gather_touched(ctx->pr.touched, order, m, V.tcount, st)));
    CKR(check_launch(ctx, launch_scan_u32(V.tcount, V.doffsets, m, V.scan_tmp, st)));
    uint32_t* k32[2] = {reinterpret_cast<uint32_t*>(ctx->sb.keys[0]), reinterpret_cast<uint32_t*>(ctx->sb.keys[1])};
    CKR(check_launch(ctx, launch_duplicate_sorted(ctx->pr.rect, ctx->pr.r0, ctx->pr.r1, order, ctx->n, m, V.d_cam,
                                                  V.d_tbase, nullptr, nullptr, V.doffsets, k32[0],
                                                  ctx->sb.vals[0], st)));
    int which = 0;
    CKR(check_launch(ctx, launch_radix_sort32(k32, ctx->sb.vals, ctx->sb.hist, total, bits_for(ntiles), &which, st)));
    if (which != 0) {
      // keep the sorted result in buffer 0
      std::swap(ctx->sb.keys[0], ctx->sb.keys[1]);
      std::swap(ctx->sb.vals[0], ctx->sb.vals[1]);
    }
    CKR(check_launch(ctx, launch_ranges32(reinterpret_cast<uint32_t*>(ctx->sb.keys[0]), total, ctx->sb.ranges,
                                          ntiles, st)));
  }
  CompositeArgs a{};
  a.cam = dc;
  a.r0 = ctx->pr.r0; a.r1 = ctx->pr.r1; a.r2 = ctx->pr.r2;
  a.p = ctx->p;
  a.vals = ctx->sb.vals[0];
  a.ranges = ctx->sb.ranges;
  a.blocks = blocks;
  a.rgb = rgb; a.depth = depth; a.alpha = alpha; a.obj = obj;
  a.nB = ctx->nB;
  a.n = ctx->n;
  a.slot = ctx->slot;
  a.n_act = ctx->n_act;
  a.err = ctx->d_flags + 3;
  a.stats = ctx->prof ? ctx->d_stats + (training ? 4 : 0) : nullptr;
  const bool scoring = blocks && !rgb && !depth && !alpha && !obj;
  if (scoring) {
    // forward pass on its own (lean, high occupancy), then the information pass
    CKR(grow(ctx, &ctx->fwd, &ctx->fwd_cap, (size_t)ntiles * kTilePix));
    CKR(grow(ctx, &ctx->tile_first, &ctx->tile_first_cap, (size_t)ntiles));
    a.fwd = ctx->fwd;
    a.tile_first = ctx->tile_first;
  }
  if (blocks || rgb || depth || alpha || obj) {
    Consts cc = ctx->c;
    if (compensated) cc.tf32 = 0;
    if (scoring) {
      Phase ph(ctx, training ? NBV_PHASE_TRAIN_COMPOSITE : NBV_PHASE_FORWARD);
      CKR(check_launch(ctx, launch_forward(a, cc, st)));
    }
    Phase ph(ctx, training ? NBV_PHASE_TRAIN_COMPOSITE : NBV_PHASE_COMPOSITE);
    CKR(check_launch(ctx, launch_composite(a, cc, st, ctx->stage)));
    if (ctx->prof) ctx->composite_launches[training ? 1 : 0]++;
  }
  return NBV_OK;
}

// Gains of one view from its blocks: per-Gaussian deltas (optional) and the
// double-precision sum into out3 (device).
int view_gains(nbv_ctx* ctx, const nbv_camera& cam, const float* blocks, float* delta, double* out3) {
  Phase ph(ctx, NBV_PHASE_GAINS);
  int used = 0;
  CKR(check_launch(ctx, launch_view_gains(dev_scene(ctx), ctx->c, to_dev(cam, ctx->tw, ctx->th), blocks, ctx->F, delta,
                                          ctx->partial, ctx->partial_cap, &used, ctx->st)));
  CKR(check_launch(ctx, launch_reduce_gains(ctx->partial, used, out3, ctx->st)));
  return NBV_OK;
}

int resolve_phases(nbv_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->st));

  for (auto& r : ctx->recs) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->acc_ms[r.phase] += ms;
    ctx->acc_launch[r.phase] += r.launches;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->recs.clear();
  return NBV_OK;
}

int bits_for(int64_t n) {
  int b = 1;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

void batched_drop_graph(nbv_ctx* ctx) {
  auto& B = ctx->bt;
  if (B.exec) cudaGraphExecDestroy(B.exec);
  if (B.graph) cudaGraphDestroy(B.graph);
  B.exec = nullptr;
  B.graph = nullptr;
}

void batched_invalidate(nbv_ctx* ctx) {
  batched_drop_graph(ctx);
  ctx->bt.ready = false;
  ctx->bt.svals = nullptr;
  ctx->bt.forced_chunk = 0;
}

// Projection of every (view, Gaussian) slot, the tile mark of the active
// subset (when only part of the scene carries a confidence, Eq. 12), every
// slot's entry count, and the depth keys of the slots that emit entries, in
// slot order (positions in B.offsets; how many at B.offsets[nv n]).
int binning_counts(nbv_ctx* ctx, cudaStream_t st) {
  auto& B = ctx->bt;
  const int64_t n = ctx->n;
  const int64_t slots = (int64_t)B.nv * n;
  const DevScene s = dev_scene(ctx);
  int l = 0;
  const bool target = ctx->n_act < n;
  {
    Phase ph(ctx, NBV_PHASE_PROJECT);
    if (target)   // marks, boxes and per-slot counts in the projection itself
      l += launch_project_target(s, ctx->c, B.cams, B.nv, B.pr, B.mark, B.ntiles, B.bbox, B.tile_base, st);
    else
      l += launch_project_views(s, ctx->c, B.cams, B.nv, B.pr, st);
  }
  Phase ph(ctx, NBV_PHASE_SORT);
  if (!target)
    l += launch_count_tiles(B.pr.rect, B.pr.r0, B.pr.r1, n, B.nv, B.cams, B.tile_base, nullptr, nullptr,
                            B.pr.touched, st);
  l += launch_compact_depth_keys(B.pr.touched, slots, B.flags, B.offsets, B.scan_tmp, B.pr.zbits, n, B.db.keys[0],
                                 B.db.vals[0], st);
  return l;
}

// Size every buffer of the multi-view path: camera tables, records, and the
// entry count (one eager binning count, one host read-back).
int batched_setup(nbv_ctx* ctx, int v0, int nv) {
  auto& B = ctx->bt;
  cudaStream_t st = ctx->st;
  const int64_t n = ctx->n;
  const int nc = (int)ctx->cand.size();
  B.v0 = v0;
  B.nv = nv;
  std::vector<DevCam> hc(nv);
  std::vector<uint32_t> base(nv);
  int64_t nt = 0;
  for (int v = 0; v < nv; ++v) {
    hc[v] = to_dev(ctx->cand[v0 + v], ctx->tw, ctx->th);
    base[v] = (uint32_t)nt;
    nt += (int64_t)hc[v].GX * hc[v].GY;
  }
  if (nt >= (int64_t(1) << 31)) return fail(ctx, NBV_ERR_ARG, "too many tiles in the candidate set");
  B.ntiles = (int)nt;
  B.h_base = base;
  B.svals = nullptr;
  std::vector<int> tv((size_t)nt);
  for (int v = 0; v < nv; ++v)
    for (int64_t t = 0; t < (int64_t)hc[v].GX * hc[v].GY; ++t) tv[base[v] + t] = v;
  CKR(alloc(ctx, &B.cams, (size_t)nv));
  CKR(alloc(ctx, &B.tile_base, (size_t)nv));
  CKR(alloc(ctx, &B.tile_view, (size_t)nt));
  CK(cudaMemcpyAsync(B.cams, hc.data(), sizeof(DevCam) * nv, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(B.tile_base, base.data(), sizeof(uint32_t) * nv, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(B.tile_view, tv.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st));
  const size_t slots = (size_t)nv * n;
  CKR(alloc(ctx, &B.pr.r0, slots)); CKR(alloc(ctx, &B.pr.r1, slots)); CKR(alloc(ctx, &B.pr.r2, slots));
  CKR(alloc(ctx, &B.pr.rect, slots)); CKR(alloc(ctx, &B.pr.zbits, slots));
  CKR(alloc(ctx, &B.pr.touched, slots));
  CKR(alloc(ctx, &B.flags, slots));
  CKR(alloc(ctx, &B.mark, (size_t)nt));
  CKR(alloc(ctx, &B.bbox, (size_t)nv));
  CKR(alloc(ctx, &B.offsets, slots + 1));
  CKR(alloc(ctx, &B.scan_tmp, scan_scratch_elems((int64_t)slots + 1)));
  CKR(alloc(ctx, &B.db.keys[0], slots)); CKR(alloc(ctx, &B.db.keys[1], slots));
  CKR(alloc(ctx, &B.db.vals[0], slots)); CKR(alloc(ctx, &B.db.vals[1], slots));
  CKR(alloc(ctx, &B.db.hist, radix_hist_elems((int64_t)slots)));
  B.db.cap = slots;
  CKR(alloc(ctx, &B.tcount, slots));
  CKR(alloc(ctx, &B.doffsets, slots + 1));
  CKR(alloc(ctx, &B.ranges, (size_t)nt));
  CKR(alloc(ctx, &B.fwd, (size_t)nt * kTilePix));
  CKR(alloc(ctx, &B.tile_first, (size_t)nt));
  CKR(alloc(ctx, &B.counter, 2));
  CKR(alloc(ctx, &B.blocks, (size_t)nv * ctx->n_act * ctx->nBp));
  B.parts_cap = ctx->nsm * 64;      // >= the multi-view gains launch's warps (a few blocks of <= 8 per SM)
  CKR(alloc(ctx, &B.partial, (size_t)nv * B.parts_cap * 3));
  CKR(grow(ctx, &ctx->ig_cand, &ctx->ig_cand_cap, (size_t)(nc > 0 ? nc : 1) * 3));
  CKR(grow(ctx, &ctx->out4, &ctx->out4_cap, (size_t)(nc > 0 ? nc : 1) * 4));
  // queue sort buffers
  CKR(alloc(ctx, &B.qb.keys[0], (size_t)nt)); CKR(alloc(ctx, &B.qb.keys[1], (size_t)nt));
  CKR(alloc(ctx, &B.qb.vals[0], (size_t)nt)); CKR(alloc(ctx, &B.qb.vals[1], (size_t)nt));
  CKR(alloc(ctx, &B.qb.hist, radix_hist_elems(nt)));
  B.qb.cap = (size_t)nt;
  // entry count and the number of slots that emit entries (the same on every
  // replay of the captured pass: they depend only on the scene, the cameras
  // and the active set, any change of which drops this state)
  CKR(check_launch(ctx, binning_counts(ctx, st)));
  CKR(check_launch(ctx, launch_sum_u64(B.pr.touched, (int64_t)slots, ctx->d_total64, st)));
  CK(cudaMemcpyAsync(ctx->h_total, B.offsets + slots, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_total64, ctx->d_total64, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if ((int64_t)*ctx->h_total64 > ctx->entry_limit) {
    if (nv == 1)
      return fail(ctx, NBV_ERR_ARG, "candidate " + std::to_string(v0) + " has " + std::to_string(*ctx->h_total64) +
                                        " (tile, Gaussian) entries, more than one binning pass holds (" +
                                        std::to_string(ctx->entry_limit) + ")");
    return kTooManyEntries;      // nothing was duplicated; the caller splits the views
  }
  B.m = (int64_t)*ctx->h_total;
  B.total = (int64_t)*ctx->h_total64;
  const size_t cap = (size_t)B.total + 1024;
  CKR(alloc(ctx, &B.sb.keys[0], cap)); CKR(alloc(ctx, &B.sb.keys[1], cap));
  CKR(alloc(ctx, &B.sb.vals[0], cap)); CKR(alloc(ctx, &B.sb.vals[1], cap));
  CKR(alloc(ctx, &B.sb.hist, radix_hist_elems((int64_t)cap)));
  B.sb.cap = cap;
  B.ready = true;
  return NBV_OK;
}

// The whole multi-view score, enqueued on the context stream (captured into
// a graph by batched_score).
int batched_sequence(nbv_ctx* ctx, bool final_scores) {
  auto& B = ctx->bt;
  cudaStream_t st = ctx->st;
  const int nv = B.nv;
  const int64_t n = ctx->n;
  DevScene s = dev_scene(ctx);
  CK(cudaMemsetAsync(B.blocks, 0, sizeof(float) * (size_t)nv * ctx->n_act * ctx->nBp, st));
  CKR(check_launch(ctx, binning_counts(ctx, st)));
  uint32_t* qv = nullptr;
  const uint32_t* svals = nullptr;
  {
    Phase ph(ctx, NBV_PHASE_SORT);
    // (view, depth bits) order of the slots that emit entries (compacted in
    // view-major, Gaussian-index order; every pass is stable), then the
    // entries duplicated in that order and sorted stably on the tile id
    // alone: each tile's list comes out in (depth bits, Gaussian index) order
    int dw = 0;
    CKR(check_launch(ctx, launch_radix_sort(B.db, B.m, 31 + bits_for(nv), &dw, st)));
    const uint32_t* order = B.db.vals[dw];
    CKR(check_launch(ctx, launch_gather_touched(B.pr.touched, order, B.m, B.tcount, st)));
    CKR(check_launch(ctx, launch_scan_u32(B.tcount, B.doffsets, B.m, B.scan_tmp, st)));
    uint32_t* k32[2] = {reinterpret_cast<uint32_t*>(B.sb.keys[0]), reinterpret_cast<uint32_t*>(B.sb.keys[1])};
    CKR(check_launch(ctx, launch_duplicate_sorted(B.pr.rect, B.pr.r0, B.pr.r1, order, n, B.m, B.cams, B.tile_base,
                                                  ctx->n_act < n ? B.mark : nullptr,
                                                  ctx->n_act < n ? B.bbox : nullptr, B.doffsets, k32[0],
                                                  B.sb.vals[0], st)));
    int which = 0;
    CKR(check_launch(ctx, launch_radix_sort32(k32, B.sb.vals, B.sb.hist, B.total, bits_for(B.ntiles), &which, st)));
    svals = B.sb.vals[which];
    B.svals = svals;
    CKR(check_launch(ctx, launch_ranges32(k32[which], B.total, B.ranges, B.ntiles, st)));
    CKR(check_launch(ctx, launch_queue_keys(B.ranges, B.ntiles, B.qb.keys[0], B.qb.vals[0], st)));
    int qw = 0;
    CKR(check_launch(ctx, launch_radix_sort(B.qb, B.ntiles, 32 + bits_for(B.ntiles), &qw, st)));
    qv = B.qb.vals[qw];
  }
  {
    CK(cudaMemsetAsync(B.counter, 0, 2 * sizeof(int), st));
    if (ctx->prof) {
      ctx->composite_launches[0]++;
      ctx->binned_entries[0] += B.total;
    }
    CompositeArgs a{};
    a.cam = B.nv > 0 ? to_dev(ctx->cand[B.v0], ctx->tw, ctx->th) : DevCam{};
    a.r0 = B.pr.r0; a.r1 = B.pr.r1; a.r2 = B.pr.r2;
    a.p = ctx->p;
    a.vals = svals;
    a.ranges = B.ranges;
    a.blocks = B.blocks;
    a.stats = ctx->prof ? ctx->d_stats : nullptr;
    a.nB = ctx->nB;
    a.queue = qv;
    a.counter = B.counter;
    a.n_items = B.ntiles;
    a.tile_view = B.tile_view;
    a.tile_base = B.tile_base;
    a.cams = B.cams;
    a.n = n;
    a.slot = ctx->slot;
    a.n_act = ctx->n_act;
    a.err = ctx->d_flags + 3;
    a.fwd = B.fwd;
    a.tile_first = B.tile_first;
    {
      Phase ph(ctx, NBV_PHASE_FORWARD);
      CKR(check_launch(ctx, launch_forward(a, ctx->c, st)));   // records of view v start at slot v n
    }
    Phase ph(ctx, NBV_PHASE_COMPOSITE);
    a.counter = B.counter + 1;
    CKR(check_launch(ctx, launch_composite(a, ctx->c, st, ctx->stage)));
  }
  {
    Phase ph(ctx, NBV_PHASE_GAINS);
    int nparts = 0;
    int r = launch_views_gains_gm(s, ctx->c, B.cams, nv, B.blocks, ctx->F, B.partial, B.parts_cap, &nparts, st);
    if (r < 0)
      r = launch_views_gains(s, ctx->c, B.cams, nv, B.blocks, ctx->F, B.partial, B.parts_cap, &nparts, st);
    CKR(check_launch(ctx, r));
    CKR(check_launch(ctx, launch_reduce_gains_views(B.partial, nparts, nv, ctx->ig_cand + 3 * (size_t)B.v0, st)));
  }
  if (final_scores) {
    Phase ph(ctx, NBV_PHASE_SCORE);
    CKR(check_launch(ctx, launch_final_scores(ctx->ig_cand, ctx->ig_train, (int)ctx->cand.size(),
                                              (int)ctx->train.size(), ctx->c, ctx->out4, ctx->d_flags,
                                              ctx->d_best_score, ctx->d_flags + 1, st)));
  }
  return NBV_OK;
}

// Candidates per multi-view pass: all of them unless their per-(view,
// Gaussian) state (blocks, records, binning slots) would take more than 45%
// of the device memory free now (at least 4 GB; the rest is left for the
// entries of the binning, which scale with the views too), or the
// configuration caps it.
int batched_chunk(const nbv_ctx* ctx) {
  const int nc = (int)ctx->cand.size();
  const double per_view = (double)ctx->n * 128.0 + (double)ctx->n_act * (double)ctx->nBp * 4.0;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  const double budget = std::max(4.0e9, 0.45 * (double)free_b);
  int chunk = (int)std::max(1.0, std::floor(budget / std::max(per_view, 1.0)));
  // slot ids (view n + Gaussian) and the depth keys' view field are 31-bit
  chunk = (int)std::min<int64_t>(chunk, std::max<int64_t>(1, ((int64_t(1) << 31) - 1) / std::max<int64_t>(ctx->n, 1)));
  if (ctx->cfg.max_batch_views > 0) chunk = std::min(chunk, ctx->cfg.max_batch_views);
  return std::max(1, std::min(chunk, std::max(nc, 1)));
}

// Candidates [v0, v0 + *nv) as one multi-view pass, set up and run eagerly;
// *nv is halved until the pass's entries fit the limit.
int batched_eager_chunk(nbv_ctx* ctx, int v0, int* nv) {
  auto& B = ctx->bt;
  for (;;) {
    B.ready = false;
    const int r = batched_setup(ctx, v0, *nv);
    if (r == kTooManyEntries) {
      *nv = std::max(1, *nv / 2);
      continue;
    }
    CKR(r);
    return batched_sequence(ctx, false);
  }
}

int batched_score(nbv_ctx* ctx) {
  auto& B = ctx->bt;
  cudaStream_t st = ctx->st;
  const int nc = (int)ctx->cand.size();
  int chunk = batched_chunk(ctx);
  if (B.forced_chunk > 0) chunk = std::min(chunk, B.forced_chunk);
  if (nc <= chunk && (!B.ready || B.v0 != 0 || B.nv != nc)) {
    batched_drop_graph(ctx);
    const int r = batched_setup(ctx, 0, nc);
    if (r == kTooManyEntries) {
      B.ready = false;
      chunk = B.forced_chunk = std::max(1, nc / 2);
    } else {
      CKR(r);
    }
  }
  if (nc > chunk) {
    // candidate chunks one after the other, each set up and run eagerly; the
    // final normalisation over all of them at the end
    batched_drop_graph(ctx);
    for (int v0 = 0; v0 < nc;) {
      int nv = std::min(chunk, nc - v0);
      CKR(batched_eager_chunk(ctx, v0, &nv));
      v0 += nv;
    }
    B.ready = false;
    Phase ph(ctx, NBV_PHASE_SCORE);
    CKR(check_launch(ctx, launch_final_scores(ctx->ig_cand, ctx->ig_train, nc, (int)ctx->train.size(), ctx->c,
                                              ctx->out4, ctx->d_flags, ctx->d_best_score, ctx->d_flags + 1, st)));
    return NBV_OK;
  }
  if (ctx->prof) return batched_sequence(ctx, true);   // timed phase by phase, not replayed
  if (!B.exec) {
    // capture on the private stream (the caller's stream may be the legacy
    // default stream, which cannot be captured)
    struct StreamSwap {
      nbv_ctx* c;
      cudaStream_t keep;
      ~StreamSwap() { c->st = keep; }
    } swap{ctx, ctx->st};
    ctx->st = ctx->cap_st;
    const int64_t l0 = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    const int rc = batched_sequence(ctx, true);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->st, &g);
    if (rc != NBV_OK) { if (g) cudaGraphDestroy(g); return rc; }
    CK(ec);
    B.graph = g;
    CK(cudaGraphInstantiate(&B.exec, B.graph, 0));
    B.launches_per_replay = ctx->launches - l0;
    ctx->launches = l0;
  }
  CK(cudaGraphLaunch(B.exec, st));
  ctx->launches += B.launches_per_replay;
  return NBV_OK;
}

int ensure_scene_buffers(nbv_ctx* ctx, int64_t n) {
  const int KC = ctx->c.KC, nb = ctx->c.nb;
  CKR(alloc(ctx, &ctx->mu, 3 * n)); CKR(alloc(ctx, &ctx->logs, 3 * n)); CKR(alloc(ctx, &ctx->q, 4 * n));
  CKR(alloc(ctx, &ctx->rho, n)); CKR(alloc(ctx, &ctx->sh, (size_t)n * nb * 3));
  CKR(alloc(ctx, &ctx->obj, (size_t)n * KC));
  CKR(alloc(ctx, &ctx->mu_sig, n)); CKR(alloc(ctx, &ctx->scale_skip, n)); CKR(alloc(ctx, &ctx->qn, n));
  CKR(alloc(ctx, &ctx->aux, n)); CKR(alloc(ctx, &ctx->p, (size_t)n * KC));
  CKR(alloc(ctx, &ctx->slot, n)); CKR(alloc(ctx, &ctx->act, n));
  CKR(alloc(ctx, &ctx->pr.r0, n)); CKR(alloc(ctx, &ctx->pr.r1, n)); CKR(alloc(ctx, &ctx->pr.r2, n));
  CKR(alloc(ctx, &ctx->pr.rect, n)); CKR(alloc(ctx, &ctx->pr.zbits, n));
  CKR(alloc(ctx, &ctx->pr.touched, n)); CKR(alloc(ctx, &ctx->pr.radius, n));
  CKR(alloc(ctx, &ctx->sb.offsets, n + 1));
  CKR(alloc(ctx, &ctx->sb.scan_tmp, scan_scratch_elems(n + 1)));
  {
    auto& V = ctx->vb;
    CKR(alloc(ctx, &V.flags, n)); CKR(alloc(ctx, &V.pos, n + 1));
    CKR(alloc(ctx, &V.scan_tmp, scan_scratch_elems(n + 1)));
    CKR(alloc(ctx, &V.db.keys[0], n)); CKR(alloc(ctx, &V.db.keys[1], n));
    CKR(alloc(ctx, &V.db.vals[0], n)); CKR(alloc(ctx, &V.db.vals[1], n));
    CKR(alloc(ctx, &V.db.hist, radix_hist_elems(n)));
    V.db.cap = (size_t)n;
    CKR(alloc(ctx, &V.tcount, n)); CKR(alloc(ctx, &V.doffsets, n + 1));
    CKR(alloc(ctx, &V.d_cam, 1)); CKR(alloc(ctx, &V.d_tbase, 1));
    CK(cudaMemsetAsync(V.d_tbase, 0, sizeof(uint32_t), ctx->st));
  }
  CKR(alloc(ctx, &ctx->blocks, (size_t)n * ctx->nBp));
  for (int f = 0; f < 3; ++f) {
    const int l = f == 0 ? kNG + 3 * nb : (f == 1 ? kNG : kNG + KC);
    ctx->F.l[f] = l;
    const size_t per = f == 0 ? (size_t)rgb_L_size(nb) : (size_t)l * (l + 1) / 2;
    CKR(alloc(ctx, &ctx->F.L[f], (size_t)n * per));
  }
  ctx->partial_cap = ctx->nsm * 16;    // blocks; up to 8 warp partial sums each
  CKR(alloc(ctx, &ctx->partial, (size_t)ctx->partial_cap * 8 * 3));
  return NBV_OK;
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

void nbv_config_default(nbv_config* cfg, int K, int sh_degree) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->K = K;
  cfg->sh_degree = sh_degree;
  cfg->alpha_obj = 0.3f;
  cfg->alpha_opa = 0.3f;
  cfg->beta_d = 10.0f;
  cfg->beta_o = 1.0f;
  cfg->lambda_damp = 0.1f;
  cfg->near_z = 0.2f;
  cfg->alpha_min = 1.0f / 255.0f;
  cfg->alpha_max = 0.99f;
  cfg->t_min = 1e-4f;
  cfg->dilation = 0.3f;
  cfg->guard = 1.3f;
  cfg->tile_w = 16;
  cfg->tile_h = 16;
  cfg->batched = 0;
  cfg->stage = 32;
  cfg->max_batch_views = 0;
  cfg->criterion = 0;
  cfg->tf32_contraction = 0;
}

int nbv_create(const nbv_config* cfg, void* cuda_stream, nbv_ctx** out) {
  if (!cfg || !out) return NBV_ERR_ARG;
  *out = nullptr;
  const bool tile_ok = (cfg->tile_w == 16 && cfg->tile_h == 16) || (cfg->tile_w == 32 && cfg->tile_h == 8) ||
                       (cfg->tile_w == 0 && cfg->tile_h == 0);
  if (cfg->K < 1 || cfg->K > kMaxK || cfg->sh_degree < 0 || cfg->sh_degree > 3 || !tile_ok) return NBV_ERR_ARG;
  if (cfg->stage != 16 && cfg->stage != 32) return NBV_ERR_ARG;
  if (cfg->max_batch_views < 0) return NBV_ERR_ARG;
  if (cfg->criterion < 0 || cfg->criterion > 2) return NBV_ERR_ARG;
  if (cfg->tf32_contraction < 0 || cfg->tf32_contraction > 2) return NBV_ERR_ARG;
  const float fl[] = {cfg->alpha_obj, cfg->alpha_opa, cfg->beta_d, cfg->beta_o, cfg->lambda_damp,
                      cfg->near_z, cfg->alpha_min, cfg->alpha_max, cfg->t_min, cfg->dilation, cfg->guard};
  for (float v : fl)
    if (!std::isfinite(v)) return NBV_ERR_ARG;
  if (!(cfg->lambda_damp > 0.0f) || !(cfg->alpha_min > 0.0f) || !(cfg->alpha_max < 1.0f) ||
      !(cfg->alpha_max > cfg->alpha_min) || !(cfg->t_min > 0.0f) || !(cfg->near_z > 0.0f) ||
      !(cfg->guard > 0.0f) || cfg->dilation < 0.0f)
    return NBV_ERR_ARG;
  nbv_ctx* ctx = new nbv_ctx();
  ctx->cfg = *cfg;
  Consts& c = ctx->c;
  c.K = cfg->K; c.KC = cfg->K + 1; c.deg = cfg->sh_degree; c.nb = (cfg->sh_degree + 1) * (cfg->sh_degree + 1);
  c.alpha_obj = cfg->alpha_obj; c.alpha_opa = cfg->alpha_opa; c.beta_d = cfg->beta_d; c.beta_o = cfg->beta_o;
  c.lam = cfg->lambda_damp; c.near_z = cfg->near_z; c.alpha_min = cfg->alpha_min;
  c.alpha_max = cfg->alpha_max; c.t_min = cfg->t_min; c.dilation = cfg->dilation; c.guard = cfg->guard;
  c.crit = cfg->criterion;
  // automatic: single TF32 products for the log-det criterion (the logarithm
  // compresses their rounding), error-compensated for the linear trace criteria
  c.tf32 = cfg->tf32_contraction == 1 || (cfg->tf32_contraction == 0 && cfg->criterion == 0);
  ctx->nB = block_floats(c.K);
  if (cfg->tile_w != 0) { ctx->tw = cfg->tile_w; ctx->th = cfg->tile_h; }
  ctx->stage = cfg->stage;
  ctx->nBp = (ctx->nB + 3) & ~3;
  ctx->st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&ctx->h_total), 2 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&ctx->h_total64), sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_total64), sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_flags), 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_best_score), sizeof(float)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_err), sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    nbv_destroy(ctx);
    return NBV_ERR_CUDA;
  }
  ctx->nsm = device_sm_count();
  cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int), ctx->st);
  launch_tri_table_init(ctx->st);
  if (cudaGetLastError() != cudaSuccess) {
    nbv_destroy(ctx);
    return NBV_ERR_CUDA;
  }
  *out = ctx;
  return NBV_OK;
}

void nbv_destroy(nbv_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st || true) cudaStreamSynchronize(ctx->st);
  void* ptrs[] = {ctx->mu, ctx->logs, ctx->q, ctx->rho, ctx->sh, ctx->obj, ctx->mu_sig, ctx->scale_skip,
                  ctx->qn, ctx->aux, ctx->p, ctx->d_train_cams, ctx->pr.r0, ctx->pr.r1, ctx->pr.r2,
                  ctx->pr.rect, ctx->pr.zbits, ctx->pr.touched, ctx->pr.radius, ctx->sb.keys[0],
                  ctx->sb.keys[1], ctx->sb.vals[0], ctx->sb.vals[1], ctx->sb.offsets, ctx->sb.scan_tmp,
                  ctx->sb.hist, ctx->sb.ranges, ctx->blocks, ctx->train_blocks, ctx->partial,
                  ctx->ig_train, ctx->ig_cand, ctx->out4, ctx->d_flags, ctx->d_best_score, ctx->d_err,
                  ctx->F.L[0], ctx->F.L[1], ctx->F.L[2], ctx->slot, ctx->act, ctx->vb.flags, ctx->vb.pos,
                  ctx->vb.scan_tmp, ctx->vb.db.keys[0], ctx->vb.db.keys[1], ctx->vb.db.vals[0],
                  ctx->vb.db.vals[1], ctx->vb.db.hist, ctx->vb.tcount, ctx->vb.doffsets, ctx->vb.d_cam,
                  ctx->vb.d_tbase};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->d_stats) cudaFree(ctx->d_stats);
  batched_drop_graph(ctx);
  {
    auto& B = ctx->bt;
    void* bp[] = {B.cams, B.tile_base, B.tile_view, B.pr.r0, B.pr.r1, B.pr.r2, B.pr.rect, B.pr.zbits,
                  B.pr.touched, B.mark, B.bbox, B.flags, B.offsets, B.scan_tmp, B.sb.keys[0], B.sb.keys[1], B.sb.vals[0],
                  B.sb.vals[1], B.sb.hist, B.qb.keys[0], B.qb.keys[1], B.qb.vals[0], B.qb.vals[1], B.qb.hist,
                  B.ranges, B.fwd, B.tile_first, B.counter, B.blocks, B.partial, B.db.keys[0], B.db.keys[1], B.db.vals[0],
                  B.db.vals[1], B.db.hist, B.tcount, B.doffsets};
    for (void* q : bp)
      if (q) cudaFree(q);
  }
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  if (ctx->h_total) cudaFreeHost(ctx->h_total);
  if (ctx->h_total64) cudaFreeHost(ctx->h_total64);
  if (ctx->d_total64) cudaFree(ctx->d_total64);
  for (void* p : {(void*)ctx->d_desc_cams, (void*)ctx->desc_raw, (void*)ctx->desc, (void*)ctx->d_pred,
                  (void*)ctx->gacc, (void*)ctx->fwd, (void*)ctx->tile_first})
    if (p) cudaFree(p);
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  delete ctx;
}

int nbv_load_gaussians(nbv_ctx* ctx, int64_t n, const float* means, const float* log_scales,
                       const float* quats, const float* opacity, const float* sh,
                       const float* obj_logits, int ptrs_on_device) {
  if (!ctx) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (n < 1 || n > (int64_t)1 << 31 || !means || !log_scales || !quats || !opacity || !sh || !obj_logits)
    return fail(ctx, NBV_ERR_ARG, "nbv_load_gaussians: bad size or NULL pointer");
  const int KC = ctx->c.KC, nb = ctx->c.nb;
  const size_t sizes[6] = {(size_t)3 * n, (size_t)3 * n, (size_t)4 * n, (size_t)n, (size_t)n * nb * 3,
                           (size_t)n * KC};
  const float* src[6] = {means, log_scales, quats, opacity, sh, obj_logits};
  if (n != ctx->n) {
    CKR(ensure_scene_buffers(ctx, n));
    ctx->n = n;
  }
  ctx->scene_ok = false;
  ctx->prepared = false;
  ctx->scored = false;
  ctx->prepared_target = -2;
  batched_invalidate(ctx);
  float* dst[6] = {ctx->mu, ctx->logs, ctx->q, ctx->rho, ctx->sh, ctx->obj};
  for (int i = 0; i < 6; ++i)
    CK(cudaMemcpyAsync(dst[i], src[i], sizes[i] * 4,
                       ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->st));
  // validation on the device, after the copy; one synchronisation (after which
  // the caller may also reuse its host memory)
  int bad = 0;
  CK(cudaMemsetAsync(ctx->d_flags + 2, 0, sizeof(int), ctx->st));
  CKR(check_launch(ctx, launch_check_inputs(ctx->mu, ctx->logs, ctx->q, ctx->rho, ctx->sh, ctx->obj, n, nb * 3, KC,
                                            ctx->d_flags + 2, ctx->st)));
  CK(cudaMemcpyAsync(&bad, ctx->d_flags + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (bad & 2) return fail(ctx, NBV_ERR_ARG, "zero quaternion");
  if (bad) return fail(ctx, NBV_ERR_ARG, "non-finite Gaussian parameter");
  ctx->scene_ok = true;
  CKR(check_launch(ctx, launch_scene_prep(dev_scene(ctx), ctx->c, -1, ctx->st)));
  return NBV_OK;
}

static int set_views(nbv_ctx* ctx, int n, const nbv_camera* cams, std::vector<nbv_camera>& dst) {
  if (!ctx) return NBV_ERR_ARG;
  if (n < 0 || n > 65535 || (n > 0 && !cams)) return fail(ctx, NBV_ERR_ARG, "bad view count");
  for (int i = 0; i < n; ++i)
    if (!finite_cam(cams[i])) return fail(ctx, NBV_ERR_ARG, "bad camera " + std::to_string(i));
  dst.assign(cams, cams + n);
  return NBV_OK;
}

static bool same_views(const std::vector<nbv_camera>& a, int n, const nbv_camera* cams) {
  return (int)a.size() == n && (n == 0 || std::memcmp(a.data(), cams, sizeof(nbv_camera) * n) == 0);
}

int nbv_set_train_views(nbv_ctx* ctx, int n, const nbv_camera* cams) {
  if (ctx && same_views(ctx->train, n, cams)) return NBV_OK;
  CKR(set_views(ctx, n, cams, ctx->train));
  batched_drop_graph(ctx);     // the graph reads the training gains buffer
  ctx->prepared = false;
  ctx->scored = false;
  return NBV_OK;
}

int nbv_set_candidates(nbv_ctx* ctx, int n, const nbv_camera* cams) {
  if (ctx && same_views(ctx->cand, n, cams)) return NBV_OK;   // keeps the captured multi-view graph
  CKR(set_views(ctx, n, cams, ctx->cand));
  batched_invalidate(ctx);
  ctx->scored = false;
  return NBV_OK;
}

int nbv_prepare(nbv_ctx* ctx, int target_obj) {
  if (!ctx) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (ctx->n < 1 || !ctx->scene_ok || ctx->train.empty())
    return fail(ctx, NBV_ERR_STATE, "nbv_prepare: no Gaussians or no training views");
  if (target_obj < -1 || target_obj > ctx->c.K) return fail(ctx, NBV_ERR_ARG, "target_obj out of range");
  cudaStream_t st = ctx->st;
  const int nt = (int)ctx->train.size();
  ctx->prepared = false;
  ctx->scored = false;
  CK(cudaMemsetAsync(ctx->d_flags + 3, 0, sizeof(int), st));
  {
    Phase ph(ctx, NBV_PHASE_PREP);
    CKR(check_launch(ctx, launch_scene_prep(dev_scene(ctx), ctx->c, target_obj, st)));
    // the active set (c_g > 0) in Gaussian-index order; the per-view scratch
    // (touched counts, their scan) holds the flags and slots meanwhile
    CKR(check_launch(ctx, launch_active_flags(dev_scene(ctx), ctx->pr.touched, st)));
    CKR(check_launch(ctx, launch_scan_u32(ctx->pr.touched, ctx->sb.offsets, ctx->n, ctx->sb.scan_tmp, st)));
    CKR(check_launch(ctx, launch_active_scatter(dev_scene(ctx), ctx->pr.touched, ctx->sb.offsets, ctx->slot, ctx->act,
                                                st)));
    CK(cudaMemcpyAsync(ctx->h_total, ctx->sb.offsets + ctx->n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  const int64_t n_act = (int64_t)*ctx->h_total;
  // the multi-view blocks are [view][active slot], and the captured pass's
  // entry counts depend on the active set
  if (n_act != ctx->n_act || target_obj != ctx->last_target) batched_invalidate(ctx);
  ctx->last_target = target_obj;
  ctx->n_act = n_act;
  CKR(alloc(ctx, &ctx->d_train_cams, (size_t)nt));
  std::vector<DevCam> hc(nt);
  for (int t = 0; t < nt; ++t) hc[t] = to_dev(ctx->train[t], ctx->tw, ctx->th);
  CK(cudaMemcpyAsync(ctx->d_train_cams, hc.data(), sizeof(DevCam) * nt, cudaMemcpyHostToDevice, st));
  CKR(grow(ctx, &ctx->train_blocks, &ctx->train_blocks_cap, (size_t)nt * ctx->n_act * ctx->nBp));
  CK(cudaMemsetAsync(ctx->train_blocks, 0, sizeof(float) * (size_t)nt * ctx->n_act * ctx->nBp, st));
  for (int t = 0; t < nt; ++t)
    CKR(render_view(ctx, ctx->train[t], ctx->train_blocks + (size_t)t * ctx->n_act * ctx->nBp, nullptr,
                    nullptr, nullptr, nullptr, true, true));   // the factors' sums: error-compensated always
  CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  {
    Phase ph(ctx, NBV_PHASE_FACTORS);
    CKR(check_launch(ctx, launch_build_factors(dev_scene(ctx), ctx->c, ctx->d_train_cams, ctx->train_blocks,
                                               nt, ctx->F, ctx->d_err, st)));
  }
  CKR(grow(ctx, &ctx->ig_train, &ctx->ig_train_cap, (size_t)nt * 3));
  {
    // training gains (the normalisers of Eq. 10): all training views in one
    // multi-view gains launch when its shared memory fits, else view by view
    Phase ph(ctx, NBV_PHASE_GAINS);
    const int parts_cap = (ctx->partial_cap * 8) / std::max(nt, 1);
    int nparts = 0;
    const int r = parts_cap >= 8
                      ? launch_views_gains_gm(dev_scene(ctx), ctx->c, ctx->d_train_cams, nt, ctx->train_blocks, ctx->F,
                                              ctx->partial, parts_cap, &nparts, st)
                      : -1;
    if (r >= 0) {
      CKR(check_launch(ctx, r));
      CKR(check_launch(ctx, launch_reduce_gains_views(ctx->partial, nparts, nt, ctx->ig_train, st)));
    }
    if (r < 0) {
      for (int t = 0; t < nt; ++t)
        CKR(view_gains(ctx, ctx->train[t], ctx->train_blocks + (size_t)t * ctx->n_act * ctx->nBp, nullptr,
                       ctx->ig_train + 3 * t));
    }
  }
  int herr = 0, hto = 0;
  CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hto, ctx->d_flags + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hto) return fail(ctx, NBV_ERR_TIMEOUT, "a bounded wait for staged splat records gave up");
  if (herr) return fail(ctx, NBV_ERR_CUDA, "non-finite training Hessian");
  ctx->prepared = true;
  ctx->prepared_target = target_obj;
  return NBV_OK;
}

int nbv_render(nbv_ctx* ctx, int cand, float* rgb, float* depth, float* alpha, float* obj) {
  if (!ctx) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (ctx->n < 1 || !ctx->scene_ok) return fail(ctx, NBV_ERR_STATE, "nbv_render: no Gaussians");
  if (cand < 0 || cand >= (int)ctx->cand.size()) return fail(ctx, NBV_ERR_ARG, "candidate out of range");
  return render_view(ctx, ctx->cand[cand], nullptr, rgb, depth, alpha, obj);
}

int nbv_score(nbv_ctx* ctx, float* ig_out, int out_on_device) {
  if (!ctx) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (!ctx->prepared) return fail(ctx, NBV_ERR_STATE, "nbv_score before nbv_prepare");
  cudaStream_t st = ctx->st;
  const int nc = (int)ctx->cand.size();
  if (ctx->cfg.batched && nc > 0) {
    CKR(batched_score(ctx));
  } else {
    CKR(grow(ctx, &ctx->ig_cand, &ctx->ig_cand_cap, (size_t)(nc > 0 ? nc : 1) * 3));
    CKR(grow(ctx, &ctx->out4, &ctx->out4_cap, (size_t)(nc > 0 ? nc : 1) * 4));
    for (int v = 0; v < nc; ++v) {
      CK(cudaMemsetAsync(ctx->blocks, 0, sizeof(float) * (size_t)ctx->n_act * ctx->nBp, st));
      CKR(render_view(ctx, ctx->cand[v], ctx->blocks, nullptr, nullptr, nullptr, nullptr));
      CKR(view_gains(ctx, ctx->cand[v], ctx->blocks, nullptr, ctx->ig_cand + 3 * v));
    }
    Phase ph(ctx, NBV_PHASE_SCORE);
    CKR(check_launch(ctx, launch_final_scores(ctx->ig_cand, ctx->ig_train, nc, (int)ctx->train.size(),
                                              ctx->c, ctx->out4, ctx->d_flags, ctx->d_best_score,
                                              ctx->d_flags + 1, st)));
  }
  ctx->scored = true;
  int fl[3] = {0, 0, 0};
  if (ig_out) {
    if (out_on_device) {
      CK(cudaMemcpyAsync(ig_out, ctx->out4, sizeof(float) * 4 * nc, cudaMemcpyDeviceToDevice, st));
    } else {
      CK(cudaMemcpyAsync(ig_out, ctx->out4, sizeof(float) * 4 * nc, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(fl, ctx->d_flags + 1, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (fl[2]) return fail(ctx, NBV_ERR_TIMEOUT, "a bounded wait for staged splat records gave up");
      if (fl[0]) return fail(ctx, NBV_ERR_EMPTY, "a training normaliser is zero");
    }
  }
  return NBV_OK;
}

int nbv_argmax(nbv_ctx* ctx, int* best_view, float* best_score) {
  if (!ctx) return NBV_ERR_ARG;
  if (!ctx->scored) return fail(ctx, NBV_ERR_STATE, "nbv_argmax before nbv_score");
  int flags[4] = {0, 0, 0, 0};
  float bs = 0.0f;
  CK(cudaMemcpyAsync(flags, ctx->d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(&bs, ctx->d_best_score, sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (best_view) *best_view = flags[0];
  if (best_score) *best_score = bs;
  if (flags[3]) return fail(ctx, NBV_ERR_TIMEOUT, "a bounded wait for staged splat records gave up");
  if (flags[1]) return fail(ctx, NBV_ERR_EMPTY, "a training normaliser is zero");
  return NBV_OK;
}

int nbv_train_gains(nbv_ctx* ctx, float* out) {
  if (!ctx || !out) return NBV_ERR_ARG;
  if (!ctx->prepared) return fail(ctx, NBV_ERR_STATE, "nbv_train_gains before nbv_prepare");
  const int nt = (int)ctx->train.size();
  std::vector<double> h((size_t)nt * 3);
  CK(cudaMemcpyAsync(h.data(), ctx->ig_train, sizeof(double) * 3 * nt, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int i = 0; i < 3 * nt; ++i) out[i] = (float)h[i];
  return NBV_OK;
}

int nbv_gaussian_gains(nbv_ctx* ctx, int cand, float* delta) {
  if (!ctx || !delta) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (!ctx->prepared) return fail(ctx, NBV_ERR_STATE, "nbv_gaussian_gains before nbv_prepare");
  if (cand < 0 || cand >= (int)ctx->cand.size()) return fail(ctx, NBV_ERR_ARG, "candidate out of range");
  cudaStream_t st = ctx->st;
  CKR(grow(ctx, &ctx->ig_cand, &ctx->ig_cand_cap, (size_t)ctx->cand.size() * 3));
  CK(cudaMemsetAsync(ctx->blocks, 0, sizeof(float) * (size_t)ctx->n_act * ctx->nBp, st));
  CK(cudaMemsetAsync(delta, 0, sizeof(float) * 3 * (size_t)ctx->n, st));   // c_g = 0: no gain
  // single terms are inspected here: error-compensated contraction whatever the mode
  CKR(render_view(ctx, ctx->cand[cand], ctx->blocks, nullptr, nullptr, nullptr, nullptr, true));
  CKR(view_gains(ctx, ctx->cand[cand], ctx->blocks, delta, ctx->ig_cand + 3 * cand));
  return NBV_OK;
}

int nbv_debug_project(nbv_ctx* ctx, int view_set, int view, int32_t* rect, float* radius,
                      uint32_t* zbits, float* mean2d, float* conic) {
  if (!ctx) return NBV_ERR_ARG;
  if (ctx->n < 1 || !ctx->scene_ok) return fail(ctx, NBV_ERR_STATE, "no Gaussians");
  const std::vector<nbv_camera>& vs = view_set ? ctx->train : ctx->cand;
  if (view < 0 || view >= (int)vs.size()) return fail(ctx, NBV_ERR_ARG, "view out of range");
  cudaStream_t st = ctx->st;
  CKR(check_launch(ctx, launch_project(dev_scene(ctx), ctx->c, to_dev(vs[view], ctx->tw, ctx->th), ctx->pr, st)));
  const size_t n = (size_t)ctx->n;
  if (rect) CK(cudaMemcpyAsync(rect, ctx->pr.rect, n * sizeof(int4), cudaMemcpyDeviceToDevice, st));
  if (radius) CK(cudaMemcpyAsync(radius, ctx->pr.radius, n * 4, cudaMemcpyDeviceToDevice, st));
  if (zbits) CK(cudaMemcpyAsync(zbits, ctx->pr.zbits, n * 4, cudaMemcpyDeviceToDevice, st));
  if (mean2d) CK(cudaMemcpy2DAsync(mean2d, 8, ctx->pr.r0, sizeof(float4), 8, n, cudaMemcpyDeviceToDevice, st));
  if (conic) CK(cudaMemcpy2DAsync(conic, 12, ctx->pr.r1, sizeof(float4), 12, n, cudaMemcpyDeviceToDevice, st));
  return NBV_OK;
}

namespace {
// Tile lists of candidate `view` as the last multi-view pass binned them.
int debug_batched_lists(nbv_ctx* ctx, int view, int64_t* offsets, int32_t* ids, int64_t cap, int64_t* count) {
  auto& B = ctx->bt;
  if (!B.svals || B.nv < 1) return fail(ctx, NBV_ERR_STATE, "no multi-view pass since the last change");
  if (view < 0 || view >= (int)ctx->cand.size()) return fail(ctx, NBV_ERR_ARG, "view out of range");
  const int lv = view - B.v0;
  if (lv < 0 || lv >= B.nv) return fail(ctx, NBV_ERR_STATE, "view not in the last multi-view chunk");
  cudaStream_t st = ctx->st;
  const DevCam dc = to_dev(ctx->cand[view], ctx->tw, ctx->th);
  const int ntiles = dc.GX * dc.GY;
  std::vector<uint2> hr(ntiles);
  CK(cudaMemcpyAsync(hr.data(), B.ranges + B.h_base[lv], sizeof(uint2) * ntiles, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int64_t> ho(ntiles + 1);
  int64_t run = 0, first = -1;
  for (int t = 0; t < ntiles; ++t) {
    ho[t] = run;
    if (hr[t].y > hr[t].x) {
      if (first < 0) first = hr[t].x;
      if ((int64_t)hr[t].x != first + run) return fail(ctx, NBV_ERR_CUDA, "tile ranges of a view are not contiguous");
    }
    run += (int64_t)(hr[t].y - hr[t].x);
  }
  ho[ntiles] = run;
  *count = run;
  if (run > cap || !offsets || !ids) return NBV_OK;
  CK(cudaMemcpyAsync(offsets, ho.data(), sizeof(int64_t) * (ntiles + 1), cudaMemcpyHostToDevice, st));
  if (run > 0) CK(cudaMemcpyAsync(ids, B.svals + first, sizeof(int32_t) * run, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return NBV_OK;
}
}  // namespace

int nbv_debug_tile_lists(nbv_ctx* ctx, int view_set, int view, int64_t* offsets, int32_t* ids,
                         int64_t cap, int64_t* count) {
  if (!ctx || !count) return NBV_ERR_ARG;
  if (ctx->n < 1 || !ctx->scene_ok) return fail(ctx, NBV_ERR_STATE, "no Gaussians");
  if (view_set == 2) return debug_batched_lists(ctx, view, offsets, ids, cap, count);
  const std::vector<nbv_camera>& vs = view_set ? ctx->train : ctx->cand;
  if (view < 0 || view >= (int)vs.size()) return fail(ctx, NBV_ERR_ARG, "view out of range");
  CKR(render_view(ctx, vs[view], nullptr, nullptr, nullptr, nullptr, nullptr));
  cudaStream_t st = ctx->st;
  const int64_t total = (int64_t)*ctx->h_total;
  *count = total;
  if (total > cap || !offsets || !ids) return NBV_OK;
  const DevCam dc = to_dev(vs[view], ctx->tw, ctx->th);
  const int ntiles = dc.GX * dc.GY;
  std::vector<uint2> hr(ntiles);
  CK(cudaMemcpyAsync(hr.data(), ctx->sb.ranges, sizeof(uint2) * ntiles, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int64_t> ho(ntiles + 1);
  int64_t run = 0;
  for (int t = 0; t < ntiles; ++t) {
    ho[t] = run;
    run += (int64_t)(hr[t].y - hr[t].x);
  }
  ho[ntiles] = run;
  if (run != total) return fail(ctx, NBV_ERR_CUDA, "tile ranges do not cover the sorted list");
  CK(cudaMemcpyAsync(offsets, ho.data(), sizeof(int64_t) * (ntiles + 1), cudaMemcpyHostToDevice, st));
  if (total > 0)
    CK(cudaMemcpyAsync(ids, ctx->sb.vals[0], sizeof(int32_t) * total, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return NBV_OK;
}

int nbv_set_profiling(nbv_ctx* ctx, int on) {
  if (!ctx) return NBV_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  for (auto& r : ctx->recs) { ctx->pool.push_back(r.a); ctx->pool.push_back(r.b); }
  ctx->recs.clear();
  for (int i = 0; i < NBV_NUM_PHASES; ++i) { ctx->acc_ms[i] = 0.0; ctx->acc_launch[i] = 0; }
  ctx->composite_launches[0] = ctx->composite_launches[1] = 0;
  ctx->binned_entries[0] = ctx->binned_entries[1] = 0;
  if (!ctx->d_stats) CK(cudaMalloc(reinterpret_cast<void**>(&ctx->d_stats), 8 * sizeof(unsigned long long)));
  // the batched path runs eagerly while profiling, from its graph otherwise
  CK(cudaMemsetAsync(ctx->d_stats, 0, 8 * sizeof(unsigned long long), ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->prof = on != 0;
  return NBV_OK;
}

int nbv_phase_times(nbv_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx) return NBV_ERR_ARG;
  CKR(resolve_phases(ctx));
  for (int i = 0; i < NBV_NUM_PHASES; ++i) {
    if (ms) ms[i] = ctx->acc_ms[i];
    if (launches) launches[i] = ctx->acc_launch[i];
  }
  return NBV_OK;
}

int nbv_work_stats(nbv_ctx* ctx, int which, int64_t* out6) {
  if (!ctx || !out6 || which < 0 || which > 1) return NBV_ERR_ARG;
  unsigned long long h[4] = {0, 0, 0, 0};
  if (ctx->d_stats) {
    CK(cudaMemcpyAsync(h, ctx->d_stats + 4 * which, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  for (int i = 0; i < 4; ++i) out6[i] = (int64_t)h[i];
  out6[4] = ctx->composite_launches[which];
  out6[5] = ctx->binned_entries[which];
  return NBV_OK;
}


namespace {
int ensure_desc(nbv_ctx* ctx, int nc) {
  if ((size_t)nc <= ctx->desc_cap) return NBV_OK;
  for (void* p : {(void*)ctx->d_desc_cams, (void*)ctx->desc_raw, (void*)ctx->desc, (void*)ctx->d_pred})
    if (p) cudaFree(p);
  ctx->d_desc_cams = nullptr; ctx->desc_raw = nullptr; ctx->desc = nullptr; ctx->d_pred = nullptr;
  ctx->desc_cap = 0;
  CKR(alloc(ctx, &ctx->d_desc_cams, (size_t)nc));
  CKR(alloc(ctx, &ctx->desc_raw, (size_t)nc * NBV_DESC_DIM));
  CKR(alloc(ctx, &ctx->desc, (size_t)nc * NBV_DESC_DIM));
  CKR(alloc(ctx, &ctx->d_pred, (size_t)nc));
  ctx->desc_cap = (size_t)nc;
  return NBV_OK;
}
}  // namespace

int nbv_descriptors(nbv_ctx* ctx, float* out) {
  if (!ctx || !out) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (!ctx->prepared) return fail(ctx, NBV_ERR_STATE, "nbv_descriptors before nbv_prepare");
  const int nc = (int)ctx->cand.size();
  if (nc == 0) return NBV_OK;
  CKR(ensure_desc(ctx, nc));
  std::vector<DevCam> hc(nc);
  for (int v = 0; v < nc; ++v) hc[v] = to_dev(ctx->cand[v], ctx->tw, ctx->th);
  CK(cudaMemcpyAsync(ctx->d_desc_cams, hc.data(), sizeof(DevCam) * nc, cudaMemcpyHostToDevice, ctx->st));
  CKR(check_launch(ctx, launch_descriptors(dev_scene(ctx), ctx->c, ctx->d_desc_cams, nc, ctx->d_train_cams,
                                           (int)ctx->train.size(), ctx->train_blocks, ctx->nBp, ctx->desc_raw,
                                           out, ctx->st)));
  CK(cudaStreamSynchronize(ctx->st));   // the host copy of the cameras above
  return NBV_OK;
}

int nbv_score_pruned(nbv_ctx* ctx, nbv_mlp* mlp, int keep, float* pred, int* kept, float* exact, int* best,
                     float* best_score) {
  if (!ctx || !mlp || keep < 1 || !kept || !best || !best_score) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (!ctx->prepared) return fail(ctx, NBV_ERR_STATE, "nbv_score_pruned before nbv_prepare");
  const int nc = (int)ctx->cand.size();
  if (nc == 0) return fail(ctx, NBV_ERR_STATE, "no candidates");
  if (keep > nc) keep = nc;
  CKR(ensure_desc(ctx, nc));
  CKR(nbv_descriptors(ctx, ctx->desc));
  const int rc = nbv_mlp_forward(mlp, ctx->desc, nc, ctx->d_pred);
  if (rc != NBV_OK) return fail(ctx, rc, "MLP forward failed (input size must be NBV_DESC_DIM)");
  std::vector<float> hp(nc);
  CK(cudaMemcpy(hp.data(), ctx->d_pred, sizeof(float) * nc, cudaMemcpyDeviceToHost));
  if (pred) CK(cudaMemcpy(pred, ctx->d_pred, sizeof(float) * nc, cudaMemcpyDeviceToDevice));
  std::vector<int> order(nc);
  for (int i = 0; i < nc; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hp[a] > hp[b]; });
  std::vector<nbv_camera> full = ctx->cand, sub(keep);
  for (int i = 0; i < keep; ++i) {
    kept[i] = order[i];
    sub[i] = full[order[i]];
  }
  CKR(nbv_set_candidates(ctx, keep, sub.data()));
  std::vector<float> h4((size_t)keep * 4);
  int src = nbv_score(ctx, h4.data(), 0);
  const int rs = nbv_set_candidates(ctx, nc, full.data());
  if (src != NBV_OK) return src;
  if (rs != NBV_OK) return rs;
  int bi = -1;
  float bs = 0.0f;
  for (int i = 0; i < keep; ++i) {
    const float v = h4[(size_t)4 * i + 3];
    if (bi < 0 || v > bs || (v == bs && kept[i] < bi)) { bi = kept[i]; bs = v; }
  }
  if (exact) std::memcpy(exact, h4.data(), sizeof(float) * 4 * keep);
  *best = bi;
  *best_score = bs;
  return NBV_OK;
}


int nbv_render_view(nbv_ctx* ctx, const nbv_camera* cam, float* rgb, float* depth, float* alpha, float* obj) {
  if (!ctx || !cam) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (ctx->n < 1 || !ctx->scene_ok) return fail(ctx, NBV_ERR_STATE, "nbv_render_view: no Gaussians");
  if (!finite_cam(*cam)) return fail(ctx, NBV_ERR_ARG, "bad camera");
  return render_view(ctx, *cam, nullptr, rgb, depth, alpha, obj);
}

int nbv_render_backward(nbv_ctx* ctx, const nbv_camera* cam, const float* g_rgb, const float* g_depth,
                        const float* g_alpha, const float* g_obj, float* g_means, float* g_log_scales,
                        float* g_quats, float* g_opacity, float* g_sh, float* g_obj_logits) {
  if (!ctx || !cam || !g_means || !g_log_scales || !g_quats || !g_opacity || !g_sh || !g_obj_logits)
    return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (ctx->n < 1 || !ctx->scene_ok) return fail(ctx, NBV_ERR_STATE, "nbv_render_backward: no Gaussians");
  if (!finite_cam(*cam)) return fail(ctx, NBV_ERR_ARG, "bad camera");
  // projection and binning of the view (the lists the backward pass walks)
  CKR(render_view(ctx, *cam, nullptr, nullptr, nullptr, nullptr, nullptr));
  const int gw = backward_width(ctx->c);
  CKR(grow(ctx, &ctx->gacc, &ctx->gacc_cap, (size_t)ctx->n * gw));
  cudaStream_t st = ctx->st;
  CK(cudaMemsetAsync(ctx->gacc, 0, sizeof(float) * (size_t)ctx->n * gw, st));
  BackwardArgs a{};
  a.cam = to_dev(*cam, ctx->tw, ctx->th);
  a.r0 = ctx->pr.r0; a.r1 = ctx->pr.r1; a.r2 = ctx->pr.r2;
  a.p = ctx->p;
  a.vals = ctx->sb.vals[0];
  a.ranges = ctx->sb.ranges;
  a.g_rgb = g_rgb; a.g_depth = g_depth; a.g_alpha = g_alpha; a.g_obj = g_obj;
  a.gacc = ctx->gacc;
  a.gw = gw;
  CKR(check_launch(ctx, launch_render_backward(a, ctx->c, st)));
  CKR(check_launch(ctx, launch_project_backward(dev_scene(ctx), ctx->c, a.cam, ctx->gacc, gw, ctx->pr.rect, g_means,
                                                g_log_scales, g_quats, g_opacity, g_sh, g_obj_logits, st)));
  return NBV_OK;
}

int nbv_get_tiling(const nbv_ctx* ctx, int* tile_w, int* tile_h, int* stage) {
  if (!ctx) return NBV_ERR_ARG;
  if (tile_w) *tile_w = ctx->tw;
  if (tile_h) *tile_h = ctx->th;
  if (stage) *stage = ctx->stage;
  return NBV_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<std::vector<int>, std::tuple<int, int, int>> g_tune_cache;   // (K, deg, W, H, ...) -> choice
}  // namespace

int nbv_autotune(nbv_ctx* ctx, int* tile_w, int* tile_h, int* stage) {
  if (!ctx) return NBV_ERR_ARG;
  if (ctx->cuda_dead) return fail(ctx, NBV_ERR_CUDA, "context unusable after a CUDA error");
  if (ctx->n < 1 || !ctx->scene_ok || ctx->train.empty() || ctx->cand.empty())
    return fail(ctx, NBV_ERR_STATE, "nbv_autotune needs Gaussians, training and candidate views");
  std::vector<int> key = {ctx->c.K, ctx->c.deg};
  for (auto& cm : ctx->cand) { key.push_back(cm.width); key.push_back(cm.height); }
  const int target = ctx->prepared ? ctx->prepared_target : -1;
  const bool was_batched = ctx->cfg.batched != 0;
  int bw = 16, bh = 16, bs = 32;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) { std::tie(bw, bh, bs) = it->second; cached = true; }
  }
  if (!cached) {
    ctx->cfg.batched = 1;
    const bool prof = ctx->prof;
    ctx->prof = false;
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    float best = 1e30f;
    const int shapes[2][2] = {{16, 16}, {32, 8}};
    const int stages[2] = {32, 16};
    int rc = NBV_OK;
    for (int si = 0; si < 2 && rc == NBV_OK; ++si)
      for (int gi = 0; gi < 2 && rc == NBV_OK; ++gi) {
        ctx->tw = shapes[si][0]; ctx->th = shapes[si][1]; ctx->stage = stages[gi];
        batched_invalidate(ctx);
        rc = nbv_prepare(ctx, target);
        if (rc == NBV_OK) rc = batched_score(ctx);      // set-up and capture
        if (rc == NBV_OK) rc = batched_score(ctx);      // warm replay
        if (rc != NBV_OK) break;
        cudaEventRecord(e0, ctx->st);
        rc = batched_score(ctx);
        cudaEventRecord(e1, ctx->st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(ctx, NBV_ERR_CUDA, "autotune timing"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bw = ctx->tw; bh = ctx->th; bs = ctx->stage; }
      }
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    ctx->prof = prof;
    ctx->cfg.batched = was_batched ? 1 : 0;
    if (rc != NBV_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = std::make_tuple(bw, bh, bs);
  }
  ctx->tw = bw; ctx->th = bh; ctx->stage = bs;
  batched_invalidate(ctx);
  ctx->prepared = false;
  ctx->scored = false;
  if (tile_w) *tile_w = bw;
  if (tile_h) *tile_h = bh;
  if (stage) *stage = bs;
  return nbv_prepare(ctx, target);
}

int nbv_set_entry_limit(nbv_ctx* ctx, int64_t max_entries) {
  if (!ctx) return NBV_ERR_ARG;
  if (max_entries < 0 || max_entries > kMaxPassEntries)
    return fail(ctx, NBV_ERR_ARG, "entry limit outside 0 .. 2^32 - 4097");
  ctx->entry_limit = max_entries == 0 ? kMaxPassEntries : max_entries;
  batched_invalidate(ctx);
  return NBV_OK;
}

const char* nbv_last_error(const nbv_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int64_t nbv_launch_count(const nbv_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
