// Tile binning and depth sort (the rasterizer's second stage).
//
// Every projected Gaussian is duplicated once per screen tile of its 3-sigma
// rectangle in which it can pass its alpha cut-off at some pixel centre
// (tile_hit), keyed (tile << 32 | float bits of camera z). A stable
// LSD radix sort over the used key bits then orders each tile's entries
// front to back, ties going to the lower Gaussian index (duplication emits
// in index order and every pass is stable). Per-tile [start, end) ranges
// are read off the sorted keys.
#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of kScanTile elements; writes the block total.
__global__ void k_scan_tile(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                            uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
  uint32_t v[kScanItems];
  uint32_t t = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    t += v[k];
  }
  // inclusive warp scan of per-thread totals
  uint32_t x = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  uint32_t run = x - t + (wid > 0 ? warp_tot[wid - 1] : 0u);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (tid == kScanThreads - 1 && sums) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ sums) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const uint32_t add = sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t j = i + (int64_t)k * kScanThreads;
    if (j < n) out[j] += add;
  }
}

__global__ void k_set_total(const uint32_t* in, uint32_t* out, int64_t n) {
  // out[n] = out[n-1] + in[n-1]
  if (threadIdx.x == 0 && blockIdx.x == 0) out[n] = n > 0 ? out[n - 1] + in[n - 1] : 0u;
}

int scan_rec(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t st) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  int launches = 0;
  if (nb <= 1) {
    k_scan_tile<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
    return 1;
  }
  k_scan_tile<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, tmp);
  ++launches;
  launches += scan_rec(tmp, tmp, nb, tmp + nb, st);
  k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, tmp);
  return launches + 1;
}

// One slot's tile walk: its tile rectangle {x0, x1, y0, y1} (x0 < 0: none),
// the splat's mean, conic and skip exponent, the stationary-point ratios of
// tile_hit, and the view's tile grid. The warp kernels below load one slot
// per lane and then walk the non-empty rectangles one after the other with
// all 32 lanes, each lane's fields broadcast by shuffles.
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

__device__ __forceinline__ SlotTiles shfl_tiles(const SlotTiles& t, int s) {
  SlotTiles o;
  o.r = make_int4(__shfl_sync(0xffffffffu, t.r.x, s), __shfl_sync(0xffffffffu, t.r.y, s),
                  __shfl_sync(0xffffffffu, t.r.z, s), __shfl_sync(0xffffffffu, t.r.w, s));
  o.mx = __shfl_sync(0xffffffffu, t.mx, s); o.my = __shfl_sync(0xffffffffu, t.my, s);
  o.thr = __shfl_sync(0xffffffffu, t.thr, s);
  o.A = __shfl_sync(0xffffffffu, t.A, s); o.B = __shfl_sync(0xffffffffu, t.B, s);
  o.C = __shfl_sync(0xffffffffu, t.C, s);
  o.bc = __shfl_sync(0xffffffffu, t.bc, s); o.ba = __shfl_sync(0xffffffffu, t.ba, s);
  o.base = __shfl_sync(0xffffffffu, t.base, s);
  o.gx = __shfl_sync(0xffffffffu, t.gx, s);
  o.tw = __shfl_sync(0xffffffffu, t.tw, s); o.th = __shfl_sync(0xffffffffu, t.th, s);
  return o;
}

// Walks rectangle q with the warp, 32 tiles at a time in row order; fn(tx,
// ty, hit) is called by every lane each round (hit false past the end), so
// that fn may use warp collectives. keep(tx, ty): a tile filter checked
// before tile_hit (e.g. a mark).
template <class Keep, class Fn>
__device__ __forceinline__ void walk_tiles(const SlotTiles& q, int lane, Keep keep, Fn fn) {
  const int w = q.r.y - q.r.x, cnt = w * (q.r.w - q.r.z);
  // entry t = (ty - y0) w + (tx - x0); lane starts at t = lane, steps by 32
  int qy = lane / w, qx = lane - qy * w;
  const int dq = 32 / w, dr = 32 - dq * w;
  for (int t0 = 0; t0 < cnt; t0 += 32) {
    const int tx = q.r.x + qx, ty = q.r.z + qy;
    const bool hit = t0 + lane < cnt && keep(tx, ty) &&
                     tile_hit(q.A, q.B, q.C, q.mx, q.my, q.thr, q.bc, q.ba, tx, ty, q.tw, q.th);
    fn(tx, ty, hit);
    qy += dq;
    qx += dr;
    if (qx >= w) {
      qx -= w;
      ++qy;
    }
  }
}

// A slot's tile rectangle {x0, x1, y0, y1} (exclusive ends) cut to the view's
// bounding box of marked tiles {min x, min y, max x, max y} (inclusive);
// x0 = -1 when nothing is left. No tile outside the box is marked.
__device__ __forceinline__ int4 clip_rect(int4 r, int4 b) {
  const int4 c = make_int4(max(r.x, b.x), min(r.y, b.z + 1), max(r.z, b.y), min(r.w, b.w + 1));
  return (c.x < c.y && c.z < c.w) ? c : make_int4(-1, -1, -1, -1);
}

// Every Gaussian's entries for the tiles of its rectangle that pass
// tile_hit, in row order: a lane per Gaussian, then each Gaussian's
// rectangle walked by the whole warp (32 tiles at a time, the passing ones
// compacted by a ballot), so that the stores of a run are contiguous.
__global__ void k_duplicate(DevProj pr, int64_t n, DevCam cam, const uint32_t* __restrict__ offsets,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  SlotTiles st = no_tiles();
  uint32_t o = 0, zb = 0;
  if (g < n) {
    const int4 r = pr.rect[g];
    if (r.x >= 0) {
      st = slot_tiles(r, pr.r0[g], pr.r1[g], 0u, cam);
      o = offsets[g];
      zb = pr.zbits[g];
    }
  }
  const int64_t g0 = g - lane;
  for (unsigned todo = __ballot_sync(0xffffffffu, st.r.x >= 0); todo; todo &= todo - 1) {
    const int s = __ffs(todo) - 1;
    const SlotTiles q = shfl_tiles(st, s);
    const uint32_t zs = __shfl_sync(0xffffffffu, zb, s);
    uint32_t wo = __shfl_sync(0xffffffffu, o, s);
    walk_tiles(q, lane, [](int, int) { return true; }, [&](int tx, int ty, bool hit) {
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const uint32_t at = wo + (uint32_t)__popc(m & ((1u << lane) - 1u));
        keys[at] = ((uint64_t)(ty * q.gx + tx) << 32) | (uint64_t)zs;
        vals[at] = (uint32_t)(g0 + s);
      }
      wo += (uint32_t)__popc(m);
    });
  }
}

// Work-queue keys: longest tile list first, ties by tile id.
__global__ void k_queue_keys(const uint2* __restrict__ ranges, int ntiles, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const uint2 r = ranges[t];
  keys[t] = ((uint64_t)(0xFFFFFFFFu - (r.y - r.x)) << 32) | (uint32_t)t;
  vals[t] = (uint32_t)t;
}

constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 11;   // tile of 2816 keys: the staging fits the 48 KB of static shared memory
constexpr int kRadixTile = kRadixThreads * kRadixRounds;

template <typename K>
__global__ void k_radix_hist(const K* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ ghist,
                             int nblocks) {
  __shared__ uint32_t h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    const int64_t i = base + r * kRadixThreads + tid;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  ghist[(int64_t)tid * nblocks + blockIdx.x] = h[tid];
}

// One stable counting pass over a tile of kRadixTile keys: every element's
// place among the tile's elements of its digit (in input order) is ranked
// round by round (warp match + per-warp counts), the tile is rearranged by
// digit in shared memory, and written out in that order, so that each
// digit's elements leave as one contiguous run.
template <typename K>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const K* __restrict__ kin,
                                                                 const uint32_t* __restrict__ vin,
                                                                 K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                 int64_t n, int shift,
                                                                 const uint32_t* __restrict__ ghist,
                                                                 const uint32_t* __restrict__ gscan, int nblocks) {
  __shared__ uint32_t cnt[kRadixThreads / 32][256];
  __shared__ uint32_t run[256], lstart[256], gbase[256], wsum[kRadixThreads / 32];
  __shared__ K sk[kRadixTile];
  __shared__ uint32_t sv[kRadixTile];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // tile-local start of each digit: exclusive scan of this tile's counts
  const uint32_t myc = ghist[(int64_t)tid * nblocks + blockIdx.x];
  uint32_t x = myc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int w = 0; w < wid; ++w) pre += wsum[w];
  lstart[tid] = pre + x - myc;
  gbase[tid] = gscan[(int64_t)tid * nblocks + blockIdx.x];
  run[tid] = 0;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  const int tile_n = (int)((n - base) < kRadixTile ? (n - base) : kRadixTile);
  for (int r = 0; r < kRadixRounds; ++r) {
#pragma unroll
    for (int w = 0; w < kRadixThreads / 32; ++w) cnt[w][tid] = 0;
    __syncthreads();
    const int li = r * kRadixThreads + tid;
    const bool valid = li < tile_n;
    K key = 0;
    uint32_t val = 0;
    int digit = 256;
    if (valid) {
      key = kin[base + li];
      val = vin[base + li];
      digit = (int)((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int lrank = __popc(peers & lt);
    if (valid && lrank == 0) cnt[wid][digit] = (uint32_t)__popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = lstart[digit] + run[digit] + (uint32_t)lrank;
      for (int w = 0; w < wid; ++w) pos += cnt[w][digit];
      sk[pos] = key;
      sv[pos] = val;
    }
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int w = 0; w < kRadixThreads / 32; ++w) add += cnt[w][tid];
    run[tid] += add;
  }
  __syncthreads();
  for (int i = tid; i < tile_n; i += kRadixThreads) {
    const K key = sk[i];
    const int d = (int)((key >> shift) & 255u);
    const uint32_t o = gbase[d] + (uint32_t)i - lstart[d];
    kout[o] = key;
    vout[o] = sv[i];
  }
}

// Depth keys of every (view, Gaussian) slot: (view << 31) | the low 31 bits
// of the float bits of camera z (z > near > 0, so the sign bit is clear for
// every slot that has entries); value = the slot.
__global__ void k_depth_keys(const uint32_t* __restrict__ zbits, int64_t n, int nv, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (slot >= n * nv) return;
  const uint64_t v = (uint64_t)(slot / n);
  keys[slot] = (v << 31) | (uint64_t)(zbits[slot] & 0x7FFFFFFFu);
  vals[slot] = (uint32_t)slot;
}

__global__ void k_gather_touched(const uint32_t* __restrict__ touched, const uint32_t* __restrict__ order,
                                 int64_t m, uint32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = touched[order[i]];
}

// Slots in depth order (per view): each emits its tiles that pass tile_hit
// (global tile id, 32-bit key) and its Gaussian index, so that a stable sort
// on the tile id alone leaves every tile's entries in (depth bits, Gaussian
// index) order. A warp takes 32 consecutive slots (one per lane) and then
// walks their rectangles one slot after the other, 32 tiles at a time, the
// passing ones compacted by a ballot, so that the stores are contiguous.
// With a mark, only marked tiles (inside the view's box bb) are emitted.
__global__ void k_duplicate_sorted(const int4* __restrict__ rect, const float4* __restrict__ r0,
                                   const float4* __restrict__ r1, const uint32_t* __restrict__ order, int64_t n,
                                   int64_t m, const DevCam* __restrict__ cams,
                                   const uint32_t* __restrict__ tile_base, const uint8_t* __restrict__ mark,
                                   const int4* __restrict__ bb, const uint32_t* __restrict__ offsets,
                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  SlotTiles st = no_tiles();
  uint32_t g = 0, o = 0;
  if (i < m) {
    const uint32_t slot = order[i];
    const int v = (int)(slot / (uint64_t)n);
    int4 r = rect[slot];
    if (r.x >= 0 && bb != nullptr) r = clip_rect(r, bb[v]);
    if (r.x >= 0) {
      g = (uint32_t)(slot - (uint64_t)v * n);
      st = slot_tiles(r, r0[slot], r1[slot], tile_base[v], cams[v]);
      o = offsets[i];
    }
  }
  for (unsigned todo = __ballot_sync(0xffffffffu, st.r.x >= 0); todo; todo &= todo - 1) {
    const int s = __ffs(todo) - 1;
    const SlotTiles q = shfl_tiles(st, s);
    const uint32_t gs = __shfl_sync(0xffffffffu, g, s);
    uint32_t wo = __shfl_sync(0xffffffffu, o, s);
    walk_tiles(
        q, lane, [&](int tx, int ty) { return mark == nullptr || mark[q.base + (uint32_t)(ty * q.gx + tx)] != 0; },
        [&](int tx, int ty, bool hit) {
          const unsigned mk = __ballot_sync(0xffffffffu, hit);
          if (hit) {
            const uint32_t at = wo + (uint32_t)__popc(mk & ((1u << lane) - 1u));
            keys[at] = q.base + (uint32_t)(ty * q.gx + tx);
            vals[at] = gs;
          }
          wo += (uint32_t)__popc(mk);
        });
  }
}

// Entries every (view, Gaussian) slot will emit: its rectangle's tiles that
// pass tile_hit (and, with a mark, that a splat of the active set reaches,
// all inside the view's box bb). A lane per slot, then each non-empty
// rectangle walked by the whole warp, the passing tiles counted by a ballot.
__global__ void k_count_tiles(const int4* __restrict__ rect, const float4* __restrict__ r0,
                              const float4* __restrict__ r1, int64_t n, int nv, const DevCam* __restrict__ cams,
                              const uint32_t* __restrict__ tile_base, const uint8_t* __restrict__ mark,
                              const int4* __restrict__ bb, uint32_t* __restrict__ touched) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  SlotTiles st = no_tiles();
  if (i < n * nv) {
    const int v = (int)(i / n);
    int4 r = rect[i];
    if (r.x >= 0 && bb != nullptr) r = clip_rect(r, bb[v]);
    if (r.x >= 0) st = slot_tiles(r, r0[i], r1[i], tile_base[v], cams[v]);
  }
  uint32_t mine = 0;
  for (unsigned todo = __ballot_sync(0xffffffffu, st.r.x >= 0); todo; todo &= todo - 1) {
    const int s = __ffs(todo) - 1;
    const SlotTiles q = shfl_tiles(st, s);
    uint32_t tot = 0;
    walk_tiles(
        q, lane, [&](int tx, int ty) { return mark == nullptr || mark[q.base + (uint32_t)(ty * q.gx + tx)] != 0; },
        [&](int, int, bool hit) { tot += (uint32_t)__popc(__ballot_sync(0xffffffffu, hit)); });
    if (lane == s) mine = tot;
  }
  if (i < n * nv) touched[i] = mine;
}

// Multi-view depth order of the slots that emit entries: for every slot
// with touched > 0, at its place in the exclusive scan `pos` of those flags,
// the key (view << 31) | the low 31 bits of the float bits of camera z
// (z > near > 0: the sign bit is clear) and the slot as the value.
__global__ void k_compact_depth_keys(const uint32_t* __restrict__ touched, const uint32_t* __restrict__ pos,
                                     const uint32_t* __restrict__ zbits, int64_t n, int64_t m,
                                     uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (slot >= m || touched[slot] == 0u) return;
  const uint32_t at = pos[slot];
  keys[at] = ((uint64_t)(slot / n) << 31) | (uint64_t)(zbits[slot] & 0x7FFFFFFFu);
  vals[at] = (uint32_t)slot;
}

__global__ void k_flags_nonzero(const uint32_t* __restrict__ in, int64_t m, uint32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = in[i] != 0u ? 1u : 0u;
}

__global__ void k_ranges32(const uint32_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = keys[i];
  if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
  if (i == n - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

template <typename K>
int radix_passes(K* keys[2], uint32_t* vals[2], uint32_t* hist, int64_t count, int bits, int* which,
                 cudaStream_t st) {
  *which = 0;
  if (count <= 1) return 0;
  const int nblocks = (int)((count + kRadixTile - 1) / kRadixTile);
  int l = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    const int src = *which, dst = 1 - src;
    k_radix_hist<K><<<nblocks, kRadixThreads, 0, st>>>(keys[src], count, shift, hist, nblocks);
    const int64_t hn = 256LL * nblocks;
    l += 1 + scan_rec(hist, hist + hn, hn, hist + 2 * hn, st);
    k_radix_scatter<K><<<nblocks, kRadixThreads, 0, st>>>(keys[src], vals[src], keys[dst], vals[dst], count, shift,
                                                          hist, hist + hn, nblocks);
    ++l;
    *which = dst;
  }
  return l;
}

__global__ void k_ranges(const uint64_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = (uint32_t)(keys[i] >> 32);
  if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
}

// 64-bit sum of n 32-bit counts into *out (zeroed by the caller): the entry
// count of a binning pass without the wrap of the 32-bit scan.
__global__ void k_sum_u64(const uint32_t* __restrict__ in, int64_t n, unsigned long long* __restrict__ out) {
  unsigned long long acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) acc += in[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0) atomicAdd(out, acc);
}

}  // namespace

int launch_sum_u64(const uint32_t* in, int64_t n, unsigned long long* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (n <= 0) return 0;
  int64_t nb = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 8;
  if (nb > cap) nb = cap;
  k_sum_u64<<<(unsigned)nb, 256, 0, st>>>(in, n, out);
  return 1;
}

int launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t st) {
  int l = 0;
  if (n > 0) l += scan_rec(in, out, n, tmp, st);
  k_set_total<<<1, 1, 0, st>>>(in, out, n);
  return l + 1;
}

int launch_duplicate(const DevProj& pr, int64_t n, const DevCam& cam, const uint32_t* offsets, uint64_t* keys,
                     uint32_t* vals, cudaStream_t st) {
  if (n <= 0) return 0;
  k_duplicate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pr, n, cam, offsets, keys, vals);
  return 1;
}

int launch_radix_sort(SortBuffers& b, int64_t count, int bits, int* which, cudaStream_t st) {
  return radix_passes<uint64_t>(b.keys, b.vals, b.hist, count, bits, which, st);
}

int launch_radix_sort32(uint32_t* keys[2], uint32_t* vals[2], uint32_t* hist, int64_t count, int bits, int* which,
                        cudaStream_t st) {
  return radix_passes<uint32_t>(keys, vals, hist, count, bits, which, st);
}

int launch_depth_keys(const uint32_t* zbits, int64_t n, int nv, uint64_t* keys, uint32_t* vals, cudaStream_t st) {
  const int64_t m = n * nv;
  if (m <= 0) return 0;
  k_depth_keys<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(zbits, n, nv, keys, vals);
  return 1;
}

int launch_gather_touched(const uint32_t* touched, const uint32_t* order, int64_t m, uint32_t* out,
                          cudaStream_t st) {
  if (m <= 0) return 0;
  k_gather_touched<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(touched, order, m, out);
  return 1;
}

int launch_duplicate_sorted(const int4* rect, const float4* r0, const float4* r1, const uint32_t* order, int64_t n,
                            int64_t m, const DevCam* cams, const uint32_t* tile_base, const uint8_t* mark,
                            const int4* bb, const uint32_t* offsets, uint32_t* keys, uint32_t* vals,
                            cudaStream_t st) {
  if (m <= 0) return 0;
  k_duplicate_sorted<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(rect, r0, r1, order, n, m, cams, tile_base, mark,
                                                                  bb, offsets, keys, vals);
  return 1;
}

int launch_count_tiles(const int4* rect, const float4* r0, const float4* r1, int64_t n, int nv, const DevCam* cams,
                       const uint32_t* tile_base, const uint8_t* mark, const int4* bb, uint32_t* touched,
                       cudaStream_t st) {
  const int64_t m = n * nv;
  if (m <= 0) return 0;
  k_count_tiles<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(rect, r0, r1, n, nv, cams, tile_base, mark, bb, touched);
  return 1;
}

int launch_compact_depth_keys(const uint32_t* touched, int64_t m, uint32_t* flags, uint32_t* pos, uint32_t* scan_tmp,
                              const uint32_t* zbits, int64_t n, uint64_t* keys, uint32_t* vals, cudaStream_t st) {
  if (m <= 0) return 0;
  k_flags_nonzero<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(touched, m, flags);
  int l = 1 + launch_scan_u32(flags, pos, m, scan_tmp, st);
  k_compact_depth_keys<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(touched, pos, zbits, n, m, keys, vals);
  return l + 1;
}

int launch_ranges32(const uint32_t* keys, int64_t count, uint2* ranges, int ntiles, cudaStream_t st) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, st);
  if (count <= 0) return 0;
  k_ranges32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(keys, count, ranges);
  return 1;
}

// One stable radix pass on the 8 key bits at `shift`, from (kin, vin) to
// (kout, vout); `hist` holds radix_hist_elems(count) words of scratch.
int launch_radix_pass(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                      int64_t count, int shift, uint32_t* hist, cudaStream_t st) {
  if (count <= 0) return 0;
  const int nblocks = (int)((count + kRadixTile - 1) / kRadixTile);
  const int64_t hn = 256LL * nblocks;
  k_radix_hist<uint64_t><<<nblocks, kRadixThreads, 0, st>>>(kin, count, shift, hist, nblocks);
  int l = 1 + scan_rec(hist, hist + hn, hn, hist + 2 * hn, st);
  k_radix_scatter<uint64_t><<<nblocks, kRadixThreads, 0, st>>>(kin, vin, kout, vout, count, shift, hist, hist + hn,
                                                               nblocks);
  return l + 1;
}

int launch_ranges(const uint64_t* keys, int64_t count, uint2* ranges, int ntiles, cudaStream_t st) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, st);
  if (count <= 0) return 0;
  k_ranges<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(keys, count, ranges);
  return 1;
}

int launch_queue_keys(const uint2* ranges, int ntiles, uint64_t* keys, uint32_t* vals, cudaStream_t st) {
  if (ntiles <= 0) return 0;
  k_queue_keys<<<(ntiles + 255) / 256, 256, 0, st>>>(ranges, ntiles, keys, vals);
  return 1;
}

// Scratch needed by launch_scan_u32 / launch_radix_sort for n elements.
size_t scan_scratch_elems(int64_t n) {
  size_t tot = 0;
  int64_t m = n;
  while (m > kScanTile) {
    m = (m + kScanTile - 1) / kScanTile;
    tot += (size_t)m;
  }
  return tot + 64;
}

size_t radix_hist_elems(int64_t count) {
  const int64_t nblocks = (count + kRadixTile - 1) / kRadixTile;
  const int64_t hn = 256 * nblocks;
  return (size_t)(2 * hn) + scan_scratch_elems(hn);
}

}  // namespace nbv
