// Internal declarations shared by the translation units of libnbvgs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "nbvgs.h"

namespace nbv {

constexpr int kTile = 16;           // 16x16 screen tiles, one thread per pixel
constexpr int kTilePix = kTile * kTile;
constexpr int kMaxK = 98;           // the view-major gains kernel's object workspace (2 l u + 3 u^2 floats, u = 6 + K) fits one block's shared memory
constexpr int kNG = 11;             // geometric parameters: mu(3) log-scale(3) quat(4) opacity logit(1)

// Structured per-(view, Gaussian) 2D block layout (floats). With
// a = d alpha / d(mx, my, A, B, C, sigma), s_X = d X / d alpha and the
// blend weight w = alpha T, every pixel adds:
//   Q_rgb += (sum_c s_c^2) a a^T      Q_d += s_D^2 a a^T
//   Q_o   += (sum_k s_k^2) a a^T      (k over the K+1 object channels)
//   X_rgb[c] += w s_c a               X_d += w s_D a
//   X_o[j]   += w (s_j - s_0) a  (j = 1..K)
//   W2 += w^2
// which is everything the rgb / depth / object Gauss-Newton blocks in the
// 2D splat parameters need (their colour, depth and probability blocks are
// W2 I_3, W2 and W2 (I_K + 1 1^T)).
constexpr int kOffQrgb = 0;
constexpr int kOffQd = 21;
constexpr int kOffQo = 42;
constexpr int kOffXrgb = 63;
constexpr int kOffXd = 81;
constexpr int kOffW2 = 87;
constexpr int kOffXo = 88;
__host__ __device__ constexpr int block_floats(int K) { return kOffXo + 6 * K; }
// packed lower-triangle index of (i, j), i >= j
__host__ __device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

struct DevCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];
  int W, H, GX, GY;
  int TW, TH;          // screen tile size (16 x 16 by default)
};

struct Consts {
  int K, KC, deg, nb;
  float alpha_obj, alpha_opa, beta_d, beta_o, lam;
  float near_z, alpha_min, alpha_max, t_min, dilation, guard;
  int crit;   // 0: log det (Eq. 6); 1: tr(H_T^-1 c A); 2: tr(c A) (T-optimality)
  int tf32;   // 1: single TF32 products in the information contraction; 0: error-compensated (3 x TF32)
};

// Scene on the device (structure of arrays).
struct DevScene {
  int64_t n;
  const float* mu_raw;       // [n][3]
  const float* logs_raw;     // [n][3]
  const float* q_raw;        // [n][4]
  const float* rho_raw;      // [n]
  const float* sh;           // [n][nb][3]
  const float* obj_raw;      // [n][KC]
  float4* mu_sig;            // {mu, sigma}
  float4* scale_skip;        // {s, power threshold of alpha_min}
  float4* qn;                // normalised quaternion (w,x,y,z)
  float4* aux;               // {power threshold of alpha_max, c_g, |q|, argmax id}
  float* p;                  // softmax(o) [n][KC]
  // Active set: the Gaussians with c_g > 0 (all of them without a target;
  // those of the target object under Eq. 12). Information blocks, training
  // factors and gains exist only for these, in slot order: a Gaussian with
  // c_g = 0 adds log det(H + 0) - log det H = 0 to every gain.
  const int* slot;           // [n] slot of Gaussian g, or -1
  const int* act;            // [n_act] Gaussian of slot s
  int64_t n_act;
};

// Per-view projection (structure of arrays).
struct DevProj {
  float4* r0;                // {mx, my, power threshold skip, power threshold clamp}
  float4* r1;                // {A, B, C, sigma}
  float4* r2;                // {r, g, b, z}
  int4* rect;                // {x0, x1, y0, y1}
  uint32_t* zbits;
  uint32_t* touched;         // tiles of the rectangle that pass tile_hit (0 = culled)
  float* radius;
};

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device); every grid and partial-sum capacity is sized from it.
int device_sm_count();

// ------------------------------------------------------------ kernels (host wrappers)
// Each wrapper launches on `st` and returns the number of launches issued.
int launch_scene_prep(const DevScene& s, const Consts& c, int target, cudaStream_t st);
// Active-set flags (c_g > 0) of the n Gaussians into flags; after their
// exclusive scan `offsets` [n + 1], launch_active_scatter writes slot / act.
int launch_active_flags(const DevScene& s, uint32_t* flags, cudaStream_t st);
int launch_active_scatter(const DevScene& s, const uint32_t* flags, const uint32_t* offsets, int* slot, int* act,
                          cudaStream_t st);
// Non-finite parameters (bit 0) and zero quaternions (bit 1) of loaded Gaussians, OR-ed into *flag.
int launch_check_inputs(const float* mu, const float* logs, const float* q, const float* rho, const float* sh,
                        const float* obj, int64_t n, int nsh, int KC, int* flag, cudaStream_t st);
int launch_project(const DevScene& s, const Consts& c, const DevCam& cam, const DevProj& pr,
                   cudaStream_t st);
// Projection of every Gaussian into nv views (device camera array); slot v n + g.
int launch_project_views(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const DevProj& pr,
                         cudaStream_t st);
// The same with an active subset (s.n_act < s.n): the active slots are
// projected first and their tiles marked (mark [ntiles], zeroed here; bb [nv]
// each view's box of marked tiles), then every slot gets pr.touched = its
// marked tiles inside the box that pass tile_hit, and records only if that is
// not zero (no other slot's records are read).
int launch_project_target(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const DevProj& pr,
                          uint8_t* mark, int64_t ntiles, int4* bb, const uint32_t* tile_base, cudaStream_t st);

struct SortBuffers {
  uint64_t* keys[2];
  uint32_t* vals[2];
  uint32_t* offsets;     // [n+1] exclusive scan of touched
  uint32_t* scan_tmp;    // scan scratch
  uint32_t* hist;        // radix histograms
  uint2* ranges;         // [ntiles]
  size_t cap;            // capacity of keys / vals
  size_t scan_tmp_cap, hist_cap;
};
// 64-bit sum of n 32-bit counts into *out (device; zeroed on the stream first).
int launch_sum_u64(const uint32_t* in, int64_t n, unsigned long long* out, cudaStream_t st);
// Exclusive scan of touched into offsets; total written to *d_total (device).
int launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t st);
// Candidate descriptors [nv][448] (raw: scratch of the same size); tcams: the
// training cameras; tblocks: their blocks [n_train][n][nBp] (W2 entries read).
int launch_descriptors(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const DevCam* tcams,
                       int n_train, const float* tblocks, int nBp, float* raw, float* out, cudaStream_t st);
// Stable LSD radix sort of 32-bit keys (8-bit digits, 9-bit where that takes fewer passes) over `bits` bits,
// ping-ponging between keys[0/1], vals[0/1]; *which = the buffer holding the result.
int launch_radix_sort32(uint32_t* keys[2], uint32_t* vals[2], uint32_t* hist, int64_t count, int bits, int* which,
                        cudaStream_t st);
// Entry counts of the m slots in `order` (touched[order[i]]), for their scan in that order.
int launch_gather_touched(const uint32_t* touched, const uint32_t* order, int64_t m, uint32_t* out, cudaStream_t st);
// Entries of the m slots in `order` (n Gaussians per view): 32-bit global
// tile keys and Gaussian indices; with a tile mark, only marked tiles.
int launch_duplicate_sorted(const int4* rect, const float4* r0, const float4* r1, const uint32_t* order, int64_t n,
                            int64_t m, const DevCam* cams, const uint32_t* tile_base, const uint8_t* mark,
                            const int4* bb, const uint32_t* offsets, uint32_t* keys, uint32_t* vals,
                            cudaStream_t st);
// touched [nv n] = entries of every slot (rectangle tiles passing tile_hit,
// marked ones inside the view's box bb only when mark != NULL).
int launch_count_tiles(const int4* rect, const float4* r0, const float4* r1, int64_t n, int nv, const DevCam* cams,
                       const uint32_t* tile_base, const uint8_t* mark, const int4* bb, uint32_t* touched,
                       cudaStream_t st);
// Depth keys (view << 31 | z bits) and slot values of the slots with
// touched > 0, in slot order (flags / pos / scan_tmp: scratch of m words).
int launch_compact_depth_keys(const uint32_t* touched, int64_t m, uint32_t* flags, uint32_t* pos, uint32_t* scan_tmp,
                              const uint32_t* zbits, int64_t n, uint64_t* keys, uint32_t* vals, cudaStream_t st);
int launch_ranges32(const uint32_t* keys, int64_t count, uint2* ranges, int ntiles, cudaStream_t st);
// Stable LSD radix sort of 64-bit keys with 32-bit values on their low `bits`
// bits (8 a pass); *which = the buffer holding the result.
int launch_radix_sort(SortBuffers& b, int64_t count, int bits, int* which, cudaStream_t st);

// Work-queue keys: longest tile lists first.
int launch_queue_keys(const uint2* ranges, int ntiles, uint64_t* keys, uint32_t* vals, cudaStream_t st);
size_t scan_scratch_elems(int64_t n);
size_t radix_hist_elems(int64_t count);

// Whether a splat can pass its alpha cut-off at some pixel centre of tile
// (tx, ty): the minimum over the rectangle of the tile's pixel centres of
// q(d) = A dx^2 + 2 B dx dy + C dy^2 (d = pixel centre - mean2D; zero when
// the mean lies inside, else on an edge at the clamped stationary point, at
// dy = bc dx on a vertical edge and dx = ba dy on a horizontal one, with the
// ratios bc = -B / C and ba = -B / A rounded once per splat) against -2 thr
// (thr = log(alpha_min / sigma), the exponent of the skip test), widened by
// 2^-8 relative, 2^-8 absolute and 2^-18 of M = A max(dx^2) + C max(dy^2)
// over the tile. q along an edge is a parabola about its minimum, so the
// rounded ratio (off by a relative 2^-23) moves the evaluated point by a
// second-order amount, C (2^-23 dy)^2 <= 2^-46 M; with the rounding of q here
// and of the per-pixel exponent (at most about 24 units of 2^-24 times M: the
// cross term is at most M/2 for a positive-definite conic) the widening
// covers it, so no tile with a pixel that passes the skip test is dropped,
// however elongated the splat.
__device__ __forceinline__ bool tile_hit(float A, float B, float C, float mx, float my, float thr, float bc, float ba,
                                         int tx, int ty, int TW, int TH) {
  const float xl = __fsub_rn(__fadd_rn((float)(tx * TW), 0.5f), mx);
  const float xh = __fsub_rn(__fsub_rn((float)((tx + 1) * TW), 0.5f), mx);
  const float yl = __fsub_rn(__fadd_rn((float)(ty * TH), 0.5f), my);
  const float yh = __fsub_rn(__fsub_rn((float)((ty + 1) * TH), 0.5f), my);
  if (xl <= 0.0f && xh >= 0.0f && yl <= 0.0f && yh >= 0.0f) return true;
  const float mxx = fmaxf(__fmul_rn(xl, xl), __fmul_rn(xh, xh)), myy = fmaxf(__fmul_rn(yl, yl), __fmul_rn(yh, yh));
  const float M = __fadd_rn(__fmul_rn(A, mxx), __fmul_rn(C, myy));
  const float lim = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(-2.0f, thr), 1.00390625f), 0.00390625f),
                              __fmul_rn(M, 3.814697265625e-06f));
  const float B2 = __fmul_rn(2.0f, B);
  float best = __int_as_float(0x7f800000);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float dx, dy;
    if (e < 2) {
      dx = e == 0 ? xl : xh;
      dy = fminf(fmaxf(__fmul_rn(bc, dx), yl), yh);
    } else {
      dy = e == 2 ? yl : yh;
      dx = fminf(fmaxf(__fmul_rn(ba, dy), xl), xh);
    }
    const float q = __fadd_rn(__fadd_rn(__fmul_rn(A, __fmul_rn(dx, dx)), __fmul_rn(B2, __fmul_rn(dx, dy))),
                              __fmul_rn(C, __fmul_rn(dy, dy)));
    best = fminf(best, q);
  }
  return best <= lim;
}

// One slot's tile walk: its tile rectangle {x0, x1, y0, y1} (x0 < 0: none),
// the splat's mean, conic and skip exponent, the stationary-point ratios of
// tile_hit, and the view's tile grid. The warp kernels below load one slot
// per lane and walk the tiles of all 32 rectangles together (packed_walk).
struct SlotTiles {
  int4 r;
  float mx, my, thr, A, B, C, bc, ba;
  uint32_t base;
  int gx, tw, th;
};

__device__ __forceinline__ SlotTiles slot_tiles(int4 r, float4 a0, float4 a1, uint32_t base, const DevCam& cam) {
  SlotTiles t;
  t.r = r;
  t.mx = a0.x; t.my = a0.y; t.thr = a0.z;
  t.A = a1.x; t.B = a1.y; t.C = a1.z;
  t.bc = -__fdiv_rn(a1.y, a1.z);
  t.ba = -__fdiv_rn(a1.y, a1.x);
  t.base = base;
  t.gx = cam.GX; t.tw = cam.TW; t.th = cam.TH;
  return t;
}

__device__ __forceinline__ SlotTiles no_tiles() {
  SlotTiles t{};
  t.r = make_int4(-1, -1, -1, -1);
  t.tw = t.th = 1;
  return t;
}

constexpr int kDupThreads = 256;   // blocks of the tile-walking kernels

// The tiles of a warp's 32 slots (lane l holds slot l; an empty rectangle
// has x0 < 0) walked as one sequence: slot order, then row order within a
// rectangle, numbered by an inclusive scan of the areas, 32 tiles per round,
// each lane finding its slot by a binary search of the scan. Small
// rectangles share rounds, and the sequence order is the order of walking
// the rectangles one after the other. fn(s, q, tx, ty, hit) is called by every
// lane each round (s = the lane's slot, hit false past the end), so fn may
// use warp collectives; keep(q, tx, ty) filters tiles before tile_hit.
// s_st / s_incl: 32 entries of this warp's shared memory.
template <class Keep, class Fn>
__device__ __forceinline__ void packed_walk(const SlotTiles& st, SlotTiles* s_st, int* s_incl, int lane, Keep keep,
                                            Fn fn) {
  const int area = st.r.x >= 0 ? (st.r.y - st.r.x) * (st.r.w - st.r.z) : 0;
  int incl = area;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  s_st[lane] = st;
  s_incl[lane] = incl;
  __syncwarp();
  for (int t0 = 0; t0 < total; t0 += 32) {
    const int t = t0 + lane;
    int lo = 0, tx = 0, ty = 0;
    bool hit = false;
    if (t < total) {
      // the first slot whose inclusive end passes t: it lies in [0, 31]
      // (t < total = incl[31]), so five halvings of [lo, hi] end on it
      int hi = 31;
#pragma unroll
      for (int it = 0; it < 5; ++it) {
        const int mid = (lo + hi) >> 1;
        if (s_incl[mid] > t) hi = mid; else lo = mid + 1;
      }
      const SlotTiles& q = s_st[lo];
      const int idx = t - (lo > 0 ? s_incl[lo - 1] : 0);
      const int w = q.r.y - q.r.x;
      const int qy = idx / w, qx = idx - qy * w;
      tx = q.r.x + qx;
      ty = q.r.z + qy;
      hit = keep(q, tx, ty) && tile_hit(q.A, q.B, q.C, q.mx, q.my, q.thr, q.bc, q.ba, tx, ty, q.tw, q.th);
    }
    fn(lo, s_st[lo], tx, ty, hit);
  }
}

// A slot's tile rectangle {x0, x1, y0, y1} (exclusive ends) cut to the view's
// bounding box of marked tiles {min x, min y, max x, max y} (inclusive);
// x0 = -1 when nothing is left. No tile outside the box is marked.
__device__ __forceinline__ int4 clip_rect(int4 r, int4 b) {
  const int4 c = make_int4(max(r.x, b.x), min(r.y, b.z + 1), max(r.z, b.y), min(r.w, b.w + 1));
  return (c.x < c.y && c.z < c.w) ? c : make_int4(-1, -1, -1, -1);
}

// (dx, dy) = mean2D - pixel centre: the quantity the alpha decisions compare,
// computed by correctly rounded operations in one fixed order (shared by the
// forward pass and the backward pass's recomputation).
__device__ __forceinline__ float splat_power(float mx, float my, float A, float B, float C, float pxc, float pyc) {
  const float dx = __fsub_rn(mx, pxc), dy = __fsub_rn(my, pyc);
  const float dxx = __fmul_rn(dx, dx), dyy = __fmul_rn(dy, dy), dxy = __fmul_rn(dx, dy);
  const float q = __fadd_rn(__fmul_rn(A, dxx), __fmul_rn(C, dyy));
  return __fsub_rn(__fmul_rn(-0.5f, q), __fmul_rn(B, dxy));
}

struct CompositeArgs {
  DevCam cam;
  const float4* r0;
  const float4* r1;
  const float4* r2;
  const float* p;          // [n][KC]
  const uint32_t* vals;    // sorted Gaussian ids
  const uint2* ranges;     // per tile
  float* blocks;           // [n][nB] structured blocks (IG pass), or NULL
  float* rgb;              // optional images
  float* depth;
  float* alpha;
  float* obj;
  unsigned long long* stats;   // optional work counters (evaluated, blended, flushes)
  int nB;
  // persistent multi-view form (queue != NULL): items are global tile ids
  const uint32_t* queue;       // work items, longest lists first
  int* counter;                // next item (zeroed before the launch)
  int n_items;
  const int* tile_view;        // global tile -> view
  const uint32_t* tile_base;   // view -> first global tile
  const DevCam* cams;          // per view
  int64_t n;                   // Gaussians (stride of the per-view record arrays)
  const int* slot;             // Gaussian -> block slot or -1 (no information block)
  int64_t n_act;               // active Gaussians (stride of the per-view block arrays)
  int* err;                    // set to 1 when a bounded wait for staged records gave up (may be NULL)
  // Scoring launches run as two kernels: the forward pass (launch_forward)
  // writes every pixel's final transmittance, one past its last blended
  // list index and the list index of the first splat with an information
  // block that it blended (kNoEntry if none), fwd[tile * 256 + pixel] =
  // {float bits of T, last, first, 0}, and each tile's first list entry with
  // an information block (its list end when it has none); the information
  // pass (launch_composite with fwd != NULL) reads them instead of
  // compositing again, and a warp's walk back to front ends at its pixels'
  // earliest such splat. Tiles are global tile ids in the persistent form,
  // the view's tile index otherwise.
  uint4* fwd;
  uint32_t* tile_first;
};
constexpr uint32_t kNoEntry = 0xffffffffu;
// stage = Gaussians staged in shared memory per round (16 or 32).
int launch_composite(const CompositeArgs& a, const Consts& c, cudaStream_t st, int stage = 32);
// The forward pass of a scoring launch (no images): per pixel T, the last
// blended index and the first blended index with an information block into a.fwd, per tile the first active entry into a.tile_first;
// a.counter (persistent form) must be zeroed first.
int launch_forward(const CompositeArgs& a, const Consts& c, cudaStream_t st);

// Backward pass of the rasterizer for one view (backward.cu): per-pixel
// output gradients in, per-Gaussian gradients of the projected quantities
// out, gacc[g][gw] += {u (mean2D, A, B, C, sigma), rgb (3), z, p_0..p_K}.
struct BackwardArgs {
  DevCam cam;
  const float4* r0;
  const float4* r1;
  const float4* r2;
  const float* p;
  const uint32_t* vals;
  const uint2* ranges;
  const float* g_rgb;      // [H][W][3] or NULL
  const float* g_depth;    // [H][W] or NULL
  const float* g_alpha;    // [H][W] or NULL
  const float* g_obj;      // [H][W][K+1] or NULL
  float* gacc;             // [n][gw]
  int gw;
};
int backward_width(const Consts& c);
int launch_render_backward(const BackwardArgs& a, const Consts& c, cudaStream_t st);
// Chain rule through the projection (logdet.cu): gradients of the raw
// parameters += M^T gacc for every projected Gaussian of the view.
int launch_project_backward(const DevScene& s, const Consts& c, const DevCam& cam, const float* gacc, int gw,
                            const int4* rect, float* g_means, float* g_logs, float* g_quats, float* g_rho,
                            float* g_sh, float* g_obj, cudaStream_t st);

struct Factors {
  // per output, L~ = L^-1 D^-1/2, where D = diag(H) and D^-1/2 H D^-1/2 =
  // L L^T; hence H^-1 = L~^T L~. Depth and object: packed lower triangle.
  // Colour: the SH coefficients of different channels never meet in H (the
  // colour-colour part of the 2D block is W2 I_3), so with the parameters
  // ordered [SH of channel 0, 1, 2 | the 11 geometric ones] L^-1 is
  //   [[A_0, 0, 0, 0], [0, A_1, 0, 0], [0, 0, A_2, 0], [C_0, C_1, C_2, E]]
  // and is stored as A_0..A_2 (packed nb-triangles), C (11 x 3 nb, row-major,
  // column c nb + k), E (packed 11-triangle); see rgb_L_size.
  float* L[3];
  int l[3];
};
__host__ __device__ inline int rgb_tri_nb(int nb) { return nb * (nb + 1) / 2; }
__host__ __device__ inline int rgb_off_C(int nb) { return 3 * rgb_tri_nb(nb); }
__host__ __device__ inline int rgb_off_E(int nb) { return 3 * rgb_tri_nb(nb) + kNG * 3 * nb; }
__host__ __device__ inline int rgb_L_size(int nb) { return rgb_off_E(nb) + kNG * (kNG + 1) / 2; }
// Training Hessians: H^f_g = lambda I + c_g sum_t M_t^T B_t M_t, scaled and factorised.
// Decode table of packed lower-triangle indices used by the factor and gains
// kernels; launched once when a context is created.
int launch_tri_table_init(cudaStream_t st);
int launch_build_factors(const DevScene& s, const Consts& c, const DevCam* cams, const float* blocks,
                         int n_train, const Factors& f, int* d_err, cudaStream_t st);
// Per-Gaussian log-det gains of one view: delta [n][3]; per-block partial sums
// into partial [nblocks][3] (double).
int launch_view_gains(const DevScene& s, const Consts& c, const DevCam& cam, const float* blocks,
                      const Factors& f, float* delta, double* partial, int nblocks_cap,
                      int* nblocks_used, cudaStream_t st);
int launch_reduce_gains(const double* partial, int nblocks, double* out3, cudaStream_t st);
// All views at once: blocks [nv][n][nBp]; partial sums [nv][nparts][3] with
// nparts returned; out3 [nv][3].
int launch_views_gains(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const float* blocks,
                       const Factors& f, double* partial, int parts_cap, int* nparts, cudaStream_t st);
// Multi-view gains, Gaussian-major (one warp per Gaussian, lane = view,
// 32 views per grid row). Writes partial[(v * nparts + slot) * 3 + f].
// Returns -1 (nothing launched) when its shared memory does not fit.
int launch_views_gains_gm(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const float* blocks,
                          const Factors& f, double* partial, int parts_cap, int* nparts, cudaStream_t st);
int launch_reduce_gains_views(const double* partial, int nparts, int nv, double* out3, cudaStream_t st);
int launch_final_scores(const double* ig_cand, const double* ig_train, int n_cand, int n_train,
                        const Consts& c, float* out4, int* best, float* best_score, int* err,
                        cudaStream_t st);

}  // namespace nbv
