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
constexpr int kRadixItems = 4;     // keys a thread ranks per round
constexpr int kRadixRounds = 4;
constexpr int kRadixTile = kRadixThreads * kRadixItems * kRadixRounds;   // 4096 keys per block
constexpr int kRadixWarps = kRadixThreads / 32;

// Digits of RB bits (8, or 9 for 32-bit keys where that saves a pass);
// each of the 256 threads owns DPT = 2^RB / 256 consecutive digits.
template <typename K, int RB>
__global__ void k_radix_hist(const K* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ ghist,
                             int nblocks) {
  constexpr int D = 1 << RB, DPT = D / kRadixThreads;
  constexpr unsigned kMask = (unsigned)D - 1u;
  __shared__ uint32_t h[D];
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < DPT; ++q) h[tid + q * kRadixThreads] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
  for (int r = 0; r < kRadixTile / kRadixThreads; ++r) {
    const int64_t i = base + r * kRadixThreads + tid;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & kMask], 1u);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int d = tid + q * kRadixThreads;
    ghist[(int64_t)d * nblocks + blockIdx.x] = h[d];
  }
}

// Dynamic shared memory of k_radix_scatter<K, RB>: two sets of per-warp
// digit counts, the per-digit round base, run, tile start and global base,
// the warp sums, and the tile's keys and values.
template <typename K, int RB>
constexpr size_t radix_scatter_smem() {
  return sizeof(uint32_t) * (2 * kRadixWarps * (1 << RB) + 4 * (1 << RB) + kRadixWarps) +
         (sizeof(K) + sizeof(uint32_t)) * kRadixTile;
}

// One stable counting pass over a tile of kRadixTile keys, in rounds of
// 1024: warp w ranks the round's keys [128 w, 128 w + 128) four at a time
// (warp match on the digit; the lowest lane of each digit group reads and
// advances the warp's running count of that digit), so that a key's rank
// in its warp follows its input order; the digits' owners then turn the
// warps' counts into exclusive prefixes in place and advance each digit's
// run, and every key goes to lstart + run + (earlier warps) + (its rank)
// in shared memory. The two count sets alternate between rounds (the owners
// clear the next one), so two barriers a round suffice. The tile leaves
// rearranged by digit, each digit's keys as one contiguous run.
template <typename K, int RB>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const K* __restrict__ kin,
                                                                 const uint32_t* __restrict__ vin,
                                                                 K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                 int64_t n, int shift,
                                                                 const uint32_t* __restrict__ ghist,
                                                                 const uint32_t* __restrict__ gscan, int nblocks) {
  constexpr int D = 1 << RB, DPT = D / kRadixThreads;
  constexpr unsigned kMask = (unsigned)D - 1u;
  extern __shared__ __align__(16) unsigned char rsm[];
  uint32_t* cnt = reinterpret_cast<uint32_t*>(rsm);            // [2][kRadixWarps][D]
  uint32_t* rbase = cnt + 2 * kRadixWarps * D;                  // [D]
  uint32_t* run = rbase + D;                                    // [D]
  uint32_t* lstart = run + D;                                   // [D]
  uint32_t* gbase = lstart + D;                                 // [D]
  uint32_t* wsum = gbase + D;                                   // [kRadixWarps]
  K* sk = reinterpret_cast<K*>(rsm + sizeof(uint32_t) * (2 * kRadixWarps * D + 4 * D + kRadixWarps));
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + kRadixTile);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // tile-local start of each digit: exclusive scan of this tile's counts
  // (thread t holds digits DPT t .. DPT t + DPT - 1)
  uint32_t myc[DPT], mysum = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    myc[q] = ghist[(int64_t)(DPT * tid + q) * nblocks + blockIdx.x];
    mysum += myc[q];
  }
  uint32_t x = mysum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  for (int i = tid; i < 2 * kRadixWarps * D; i += kRadixThreads) cnt[i] = 0;
  __syncthreads();
  uint32_t pre = 0;
  for (int w = 0; w < wid; ++w) pre += wsum[w];
  uint32_t s = pre + x - mysum;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int d = DPT * tid + q;
    lstart[d] = s;
    s += myc[q];
    gbase[d] = gscan[(int64_t)d * nblocks + blockIdx.x];
    run[d] = 0;
  }
  const unsigned lt = (1u << lane) - 1u;
  const int64_t tbase = (int64_t)blockIdx.x * kRadixTile;
  const int tile_n = (int)((n - tbase) < kRadixTile ? (n - tbase) : kRadixTile);
  __syncthreads();
  for (int r = 0; r < kRadixRounds; ++r) {
    uint32_t* c = cnt + (r & 1) * kRadixWarps * D;
    uint32_t* cw = c + wid * D;
    K key[kRadixItems];
    uint32_t val[kRadixItems], rk[kRadixItems];
    int dig[kRadixItems];
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
      const int li = r * (kRadixThreads * kRadixItems) + wid * (32 * kRadixItems) + it * 32 + lane;
      const bool valid = li < tile_n;
      key[it] = valid ? kin[tbase + li] : K(0);
      val[it] = valid ? vin[tbase + li] : 0u;
      const int d = valid ? (int)((key[it] >> shift) & kMask) : D;   // D: no digit, never counted
      dig[it] = d;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (valid && lane == leader) before = cw[d];
      before = __shfl_sync(0xffffffffu, before, leader);
      rk[it] = before + (uint32_t)__popc(peers & lt);
      if (valid && lane == leader) cw[d] = before + (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();            // every warp's counts of this round
    uint32_t* cn = cnt + ((r + 1) & 1) * kRadixWarps * D;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid + q * kRadixThreads;
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < kRadixWarps; ++w) {
        const uint32_t v = c[w * D + d];
        c[w * D + d] = acc;     // keys of digit d in the round's earlier warps
        acc += v;
        cn[w * D + d] = 0u;     // the next round's counts start at zero
      }
      rbase[d] = lstart[d] + run[d];
      run[d] += acc;
    }
    __syncthreads();            // prefixes, bases and the cleared set are published
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
      const int d = dig[it];
      if (d < D) {
        const uint32_t pos = rbase[d] + c[wid * D + d] + rk[it];
        sk[pos] = key[it];
        sv[pos] = val[it];
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < tile_n; i += kRadixThreads) {
    const K key = sk[i];
    const int d = (int)((key >> shift) & kMask);
    const uint32_t o = gbase[d] + (uint32_t)i - lstart[d];
    kout[o] = key;
    vout[o] = sv[i];
  }
}

// Opts k_radix_scatter<K, RB> into its dynamic shared memory on the current
// device (a host-side attribute, set before every launch).
template <typename K, int RB>
void radix_scatter_attr() {
  cudaFuncSetAttribute(k_radix_scatter<K, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)radix_scatter_smem<K, RB>());
}

__global__ void k_gather_touched(const uint32_t* __restrict__ touched, const uint32_t* __restrict__ order,
                                 int64_t m, uint32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = touched[order[i]];
}

// Slots in depth order (per view): each emits its tiles that pass tile_hit
// (global tile id, 32-bit key) and its Gaussian index, so that a stable sort
// on the tile id alone leaves every tile's entries in (depth bits, Gaussian
// index) order. A warp takes 32 consecutive slots (one per lane), numbers
// the tiles of their rectangles one after the other (slot order, then row
// order within a rectangle: an exclusive scan of the areas) and walks that
// sequence 32 tiles per round, each lane finding its slot by a binary search
// of the scan, so that small rectangles share rounds; the passing tiles of a
// round are compacted by a ballot. The warp's slots are consecutive in the
// scan of their entry counts, so its entries form one contiguous run from
// the first slot's offset. With a mark, only marked tiles (inside the view's
// box bb) are emitted.
__global__ void __launch_bounds__(kDupThreads) k_duplicate_sorted(
    const int4* __restrict__ rect, const float4* __restrict__ r0, const float4* __restrict__ r1,
    const uint32_t* __restrict__ order, int64_t n, int64_t m, const DevCam* __restrict__ cams,
    const uint32_t* __restrict__ tile_base, const uint8_t* __restrict__ mark, const int4* __restrict__ bb,
    const uint32_t* __restrict__ offsets, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  __shared__ SlotTiles s_st[kDupThreads / 32][32];
  __shared__ int s_incl[kDupThreads / 32][32];
  __shared__ uint32_t s_g[kDupThreads / 32][32];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i0 = i - lane;                   // the warp's first slot
  if (i0 >= m) return;                           // warp-uniform; no block-wide barrier below
  SlotTiles st = no_tiles();
  uint32_t g = 0;
  if (i < m) {
    const uint32_t slot = order[i];
    const int v = (int)(slot / (uint64_t)n);
    int4 r = rect[slot];
    if (r.x >= 0 && bb != nullptr) r = clip_rect(r, bb[v]);
    if (r.x >= 0) {
      g = (uint32_t)(slot - (uint64_t)v * n);
      st = slot_tiles(r, r0[slot], r1[slot], tile_base[v], cams[v]);
    }
  }
  s_g[wid][lane] = g;                            // published by packed_walk's __syncwarp
  uint32_t wo = offsets[i0];
  const unsigned lt = (1u << lane) - 1u;
  packed_walk(
      st, s_st[wid], s_incl[wid], lane,
      [&](const SlotTiles& q, int tx, int ty) {
        return mark == nullptr || mark[q.base + (uint32_t)(ty * q.gx + tx)] != 0;
      },
      [&](int sl, const SlotTiles& q, int tx, int ty, bool hit) {
        const unsigned mk = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const uint32_t at = wo + (uint32_t)__popc(mk & lt);
          keys[at] = q.base + (uint32_t)(ty * q.gx + tx);
          vals[at] = s_g[wid][sl];
        }
        wo += (uint32_t)__popc(mk);
      });
}

// Entries every (view, Gaussian) slot will emit: its rectangle's tiles that
// pass tile_hit (and, with a mark, that a splat of the active set reaches,
// all inside the view's box bb). A lane per slot, the warp's rectangles
// walked together (packed_walk), each passing tile counted for its slot.
__global__ void __launch_bounds__(kDupThreads) k_count_tiles(
    const int4* __restrict__ rect, const float4* __restrict__ r0, const float4* __restrict__ r1, int64_t n, int nv,
    const DevCam* __restrict__ cams, const uint32_t* __restrict__ tile_base, const uint8_t* __restrict__ mark,
    const int4* __restrict__ bb, uint32_t* __restrict__ touched) {
  __shared__ SlotTiles s_st[kDupThreads / 32][32];
  __shared__ int s_incl[kDupThreads / 32][32];
  __shared__ uint32_t s_cnt[kDupThreads / 32][32];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (i - lane >= n * nv) return;                // warp-uniform; no block-wide barrier below
  SlotTiles st = no_tiles();
  if (i < n * nv) {
    const int v = (int)(i / n);
    int4 r = rect[i];
    if (r.x >= 0 && bb != nullptr) r = clip_rect(r, bb[v]);
    if (r.x >= 0) st = slot_tiles(r, r0[i], r1[i], tile_base[v], cams[v]);
  }
  s_cnt[wid][lane] = 0u;
  packed_walk(
      st, s_st[wid], s_incl[wid], lane,
      [&](const SlotTiles& q, int tx, int ty) {
        return mark == nullptr || mark[q.base + (uint32_t)(ty * q.gx + tx)] != 0;
      },
      [&](int sl, const SlotTiles&, int, int, bool hit) {
        if (hit) atomicAdd(&s_cnt[wid][sl], 1u);
      });
  __syncwarp();
  if (i < n * nv) touched[i] = s_cnt[wid][lane];
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

// Tile ranges of the sorted 32-bit tile keys: four consecutive keys per
// thread in one 16-byte load (the key arrays are 256-byte aligned), and
// their neighbours on either side; no valid tile id is ~0u.
__global__ void k_ranges32(const uint32_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges) {
  const int64_t i0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (i0 >= n) return;
  uint32_t k[4];
  if (i0 + 4 <= n) {
    const uint4 v = *reinterpret_cast<const uint4*>(keys + i0);
    k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? keys[i0 + j] : ~0u;
  }
  const uint32_t prev = i0 > 0 ? keys[i0 - 1] : ~0u;
  const uint32_t next = i0 + 4 < n ? keys[i0 + 4] : ~0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t i = i0 + j;
    if (i >= n) break;
    const uint32_t t = k[j];
    const uint32_t before = j == 0 ? prev : k[j - 1];
    const uint32_t after = j == 3 ? next : k[j + 1];
    if (before != t) ranges[t].x = (uint32_t)i;
    if (after != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

template <typename K, int RB>
int radix_passes(K* keys[2], uint32_t* vals[2], uint32_t* hist, int64_t count, int bits, int* which,
                 cudaStream_t st) {
  *which = 0;
  if (count <= 1) return 0;
  const int nblocks = (int)((count + kRadixTile - 1) / kRadixTile);
  int l = 0;
  for (int shift = 0; shift < bits; shift += RB) {
    const int src = *which, dst = 1 - src;
    k_radix_hist<K, RB><<<nblocks, kRadixThreads, 0, st>>>(keys[src], count, shift, hist, nblocks);
    const int64_t hn = (int64_t)(1 << RB) * nblocks;
    l += 1 + scan_rec(hist, hist + hn, hn, hist + 2 * hn, st);
    radix_scatter_attr<K, RB>();
    k_radix_scatter<K, RB><<<nblocks, kRadixThreads, radix_scatter_smem<K, RB>(), st>>>(keys[src], vals[src],
                                                                                          keys[dst], vals[dst], count,
                                                              shift, hist, hist + hn, nblocks);
    ++l;
    *which = dst;
  }
  return l;
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


int launch_radix_sort(SortBuffers& b, int64_t count, int bits, int* which, cudaStream_t st) {
  return radix_passes<uint64_t, 8>(b.keys, b.vals, b.hist, count, bits, which, st);
}

int launch_radix_sort32(uint32_t* keys[2], uint32_t* vals[2], uint32_t* hist, int64_t count, int bits, int* which,
                        cudaStream_t st) {
  // 9-bit digits where they take fewer passes (e.g. 18 bits: 2 instead of 3)
  if ((bits + 8) / 9 < (bits + 7) / 8) return radix_passes<uint32_t, 9>(keys, vals, hist, count, bits, which, st);
  return radix_passes<uint32_t, 8>(keys, vals, hist, count, bits, which, st);
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
  const int64_t quads = (count + 3) / 4;
  k_ranges32<<<(unsigned)((quads + 255) / 256), 256, 0, st>>>(keys, count, ranges);
  return 1;
}

// One stable radix pass on the 8 key bits at `shift`, from (kin, vin) to
// (kout, vout); `hist` holds radix_hist_elems(count) words of scratch.
int launch_radix_pass(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                      int64_t count, int shift, uint32_t* hist, cudaStream_t st) {
  if (count <= 0) return 0;
  const int nblocks = (int)((count + kRadixTile - 1) / kRadixTile);
  const int64_t hn = 256LL * nblocks;
  k_radix_hist<uint64_t, 8><<<nblocks, kRadixThreads, 0, st>>>(kin, count, shift, hist, nblocks);
  int l = 1 + scan_rec(hist, hist + hn, hn, hist + 2 * hn, st);
  radix_scatter_attr<uint64_t, 8>();
  k_radix_scatter<uint64_t, 8><<<nblocks, kRadixThreads, radix_scatter_smem<uint64_t, 8>(), st>>>(
      kin, vin, kout, vout, count, shift, hist,
                                                                  hist + hn, nblocks);
  return l + 1;
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
  const int64_t hn = 512 * nblocks;      // digits of up to 9 bits
  return (size_t)(2 * hn) + scan_scratch_elems(hn);
}

}  // namespace nbv
