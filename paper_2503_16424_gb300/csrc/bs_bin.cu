// Tile binning (Section 3.4): per-Gaussian tile rectangles, (tile, depth)
// keys in ascending order, and per-tile ranges.  The order comes from one of
// two sorts with the same result: on one canvas with 32-bit keys and at most
// 512 x 512 tiles, a two-level stable counting sort over the rectangles
// (rows, then columns; see "two-level binning" below); otherwise (wider
// grids, 64-bit keys, batches, the fixed scratch of bs_bin_tiles_static) a
// hand-written stable LSD radix sort of the tile bits:
//
// The keys are emitted Gaussian by Gaussian, so the emitted array is already
// ordered by the Gaussian index (the depth, since the table is in draw
// order).  A stable sort on the tile bits alone therefore orders the keys by
// (tile, depth): ceil(tile_bits / 8) passes instead of one per key byte.
//
// Per-tile pair counts come from a 2D difference array: each Gaussian adds
// +1/-1 at the four corners of its rectangle, and a row scan then a column
// scan turn the array into the number of rectangles covering each tile.
// Their exclusive scan over tile ids is the tile ranges, and their sums by
// digit are the histograms the sort passes need.
//
// Sort pass (per digit, reduce then scan then scatter): the keys are cut into
// partitions of 4096; upsweep_kernel counts each partition's digits,
// scan_parts_kernel turns the counts into each partition's first output index
// per digit (the digit's global start, from the tile counts, plus the counts
// of the partitions before it), and downsweep_kernel ranks each partition's
// keys stably (peer lanes of a digit from one ballot per digit bit) and
// writes them there.  Nothing waits on
// another CTA.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kCountThreads = 256;   // Gaussians per count CTA
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;        // keys per emit thread
constexpr int kEmitTile = kEmitThreads * kEmitItems;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per partition
constexpr int kMaxPasses = 4;
constexpr int64_t kMaxPairs = (1ll << 30) - 1;
constexpr int kScanThreads = 1024;

// Header of the binning workspace: status bits (kDevErr*), the pairs the
// Gaussians' rectangles hold, and the pairs sorted (n_pairs, or 0 when they
// exceed the capacity: then nothing is emitted or sorted and every tile
// range is empty).
struct Hdr {
  uint32_t status;
  uint32_t pad;
  unsigned long long n_pairs;
  unsigned long long n_sorted;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// ---- the tile rectangle of one Gaussian (float32, fixed operation order) ----
struct Rect {
  int tx0, tx1, ty0, ty1;
};

__device__ __forceinline__ bool tile_rect(const float *gauss, int64_t g, int W, int H, int tile, Rect *r) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(gauss + g * BS_GAUSS_FLOATS));
  const float4 c = __ldg(reinterpret_cast<const float4 *>(gauss + g * BS_GAUSS_FLOATS + 8));
  const float mx = a.x, my = a.y, ex = c.z, ey = c.w;
  if (!(ex >= 0.f) || !(ey >= 0.f)) return false;
  const float xlo = __fsub_rn(__fsub_rn(mx, ex), 0.5f);
  const float xhi = __fsub_rn(__fadd_rn(mx, ex), 0.5f);
  const float ylo = __fsub_rn(__fsub_rn(my, ey), 0.5f);
  const float yhi = __fsub_rn(__fadd_rn(my, ey), 0.5f);
  if (!isfinite(xlo) || !isfinite(xhi) || !isfinite(ylo) || !isfinite(yhi)) return false;
  const float i0 = fmaxf(ceilf(xlo), 0.f), i1 = fminf(floorf(xhi), (float)(W - 1));
  const float j0 = fmaxf(ceilf(ylo), 0.f), j1 = fminf(floorf(yhi), (float)(H - 1));
  if (!(i0 <= i1) || !(j0 <= j1)) return false;
  r->tx0 = (int)i0 / tile;
  r->tx1 = (int)i1 / tile;
  r->ty0 = (int)j0 / tile;
  r->ty1 = (int)j1 / tile;
  return true;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// The four corner updates of a rectangle [tx0, tx1] x [ty0, ty1] in a 2D
// difference array of row stride `stride`; the lanes of `active` (all
// calling, with this warp's other lanes not) that update the same cell add
// once, through the lowest of them.
__device__ __forceinline__ void add_corners(unsigned active, int *d, int stride, const Rect &r) {
  const int lane = threadIdx.x & 31;
  int *const cell[4] = {d + r.ty0 * stride + r.tx0, d + r.ty0 * stride + r.tx1 + 1, d + (r.ty1 + 1) * stride + r.tx0,
                        d + (r.ty1 + 1) * stride + r.tx1 + 1};
  const int sign[4] = {1, -1, -1, 1};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned peers = __match_any_sync(active, (unsigned long long)(uintptr_t)cell[k]);
    if (lane == __ffs(peers) - 1) atomicAdd(cell[k], sign[k] * __popc(peers));
  }
}

__global__ void zero_kernel(uint32_t *a, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = 0u;
}

// Per Gaussian: its pair count, its block-local exclusive offset, its
// rectangle packed as {tx0 | ty0 << 16, width | height << 16}, and the four
// corner updates of the tile difference array (row stride tiles_x + 1).
__global__ void __launch_bounds__(kCountThreads) count_kernel(const float *gauss, int64_t n_gauss, int W, int H,
                                                              int tile, int tiles_x, uint32_t *local,
                                                              unsigned long long *partial, uint2 *rects,
                                                              int *diff) {
  __shared__ uint32_t s_warp[kCountThreads / 32];
  const int64_t g = (int64_t)blockIdx.x * kCountThreads + threadIdx.x;
  uint32_t cnt = 0;
  Rect r;
  bool ok = false;
  if (g < n_gauss) {
    uint2 packed = make_uint2(0u, 0u);
    ok = tile_rect(gauss, g, W, H, tile, &r);
    if (ok) {
      const uint32_t w = (uint32_t)(r.tx1 - r.tx0 + 1), h = (uint32_t)(r.ty1 - r.ty0 + 1);
      cnt = w * h;
      packed = make_uint2((uint32_t)r.tx0 | ((uint32_t)r.ty0 << 16), w | (h << 16));
    }
    rects[g] = packed;
  }
  const unsigned active = __ballot_sync(0xffffffffu, ok);
  if (ok) add_corners(active, diff, tiles_x + 1, r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(cnt, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < kCountThreads / 32 ? s_warp[lane] : 0u;
    v = warp_incl_scan(v, lane);
    if (lane < kCountThreads / 32) s_warp[lane] = v;
  }
  __syncthreads();
  const uint32_t warp_excl = warp == 0 ? 0u : s_warp[warp - 1];
  if (g < n_gauss) local[g] = warp_excl + incl - cnt;
  if (threadIdx.x == kCountThreads - 1) partial[blockIdx.x] = warp_excl + incl;
}

// Exclusive scan of the per-CTA totals (one CTA); writes the pair count P,
// the sentinel partial[n] = P, and with a header (one canvas) the count to
// sort: P, or 0 with the capacity bit of the status word when P exceeds the
// capacity.
__global__ void __launch_bounds__(1024) scan_partials_kernel(unsigned long long *partial, int64_t n,
                                                             unsigned long long *total_out, Hdr *hdr,
                                                             int64_t capacity) {
  __shared__ unsigned long long s[1024];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const unsigned long long v = i < n ? partial[i] : 0ull;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const unsigned long long t = threadIdx.x >= o ? s[threadIdx.x - o] : 0ull;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) partial[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total_out = carry;
    if (hdr) {
      const bool over = carry > (unsigned long long)capacity;
      hdr->n_sorted = over ? 0ull : carry;
      if (over) hdr->status |= kDevErrCapacity;
    }
    partial[n] = carry;
  }
}

// ---- per-tile counts from the difference array ----
// Row scan: one warp per row, 32 columns at a time, in place.
__global__ void diff_rows_kernel(int *diff, int rows, int cols) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  int *d = diff + (size_t)row * cols;
  int carry = 0;
  for (int c0 = 0; c0 < cols; c0 += 32) {
    const int c = c0 + lane;
    int v = c < cols ? d[c] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (c < cols) d[c] = carry + v;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
}

// Column scan: one warp per column, 32 rows at a time, in place.
__global__ void diff_cols_kernel(int *diff, int rows, int cols) {
  const int col = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= cols) return;
  int carry = 0;
  for (int r0 = 0; r0 < rows; r0 += 32) {
    const int r = r0 + lane;
    int v = r < rows ? diff[(size_t)r * cols + col] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (r < rows) diff[(size_t)r * cols + col] = carry + v;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
}

// Exclusive scan of the per-tile counts in tile-id order (one CTA): writes
// the tile ranges ((0, 0) for an empty tile) and, per sort pass, where the
// keys of each digit start (the exclusive scan of the digit histogram).  Each thread owns a run of consecutive tiles: a local running
// sum, one block scan of the run totals, then the ranges.
__device__ __forceinline__ uint32_t block_excl_scan1024(uint32_t v, uint32_t *s_warp, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(v, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = warp_incl_scan(s_warp[lane], lane);
    s_warp[lane] = w;
  }
  __syncthreads();
  *total = s_warp[31];
  return (warp ? s_warp[warp - 1] : 0u) + incl - v;
}

__global__ void __launch_bounds__(1024) tile_scan_kernel(const int *counts, int tiles_x, int tiles_y, int passes,
                                                         int digit_bits, const Hdr *hdr, uint2 *ranges,
                                                         uint32_t *hist) {
  __shared__ uint32_t s_hist[kMaxPasses * 256];
  __shared__ uint32_t s_warp[32];
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) s_hist[i] = 0u;
  __syncthreads();
  const int n = tiles_x * tiles_y;
  const int stride = tiles_x + 1;
  const uint32_t dmask = (1u << digit_bits) - 1;
  const int run = (n + 1023) / 1024;
  const int t0 = threadIdx.x * run, t1 = min(n, t0 + run);
  uint32_t sum = 0;
  for (int t = t0; t < t1; ++t) {
    const int ty = t / tiles_x, tx = t - ty * tiles_x;
    const uint32_t v = (uint32_t)counts[ty * stride + tx];
    sum += v;
    if (v)
      for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p * 256 + (((uint32_t)t >> (p * digit_bits)) & dmask)], v);
  }
  uint32_t total;
  uint32_t start = block_excl_scan1024(sum, s_warp, &total);
  const bool over = (hdr->status & kDevErrCapacity) != 0u;  // nothing sorted: every range empty
  for (int t = t0; t < t1; ++t) {
    const int ty = t / tiles_x, tx = t - ty * tiles_x;
    const uint32_t v = (uint32_t)counts[ty * stride + tx];
    ranges[t] = (v && !over) ? make_uint2(start, start + v) : make_uint2(0u, 0u);
    start += v;
  }
  __syncthreads();
  // per pass, the exclusive prefix over digits: where each digit's keys start
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < passes) {
    uint32_t carry = 0;
    for (int d0 = 0; d0 < 256; d0 += 32) {
      const uint32_t v = s_hist[warp * 256 + d0 + lane];
      const uint32_t incl = warp_incl_scan(v, lane);
      hist[warp * 256 + d0 + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// The difference array's scans, the tile ranges and the digit starts in one
// CTA of 1024 threads, with the per-tile counts in shared memory (used when
// they fit; at most two sort passes).  Only the tiles' own part of the
// difference array matters (a count sums the array above and left of its
// tile), so shared memory holds tiles_y rows of ldc = tiles_x rounded up to
// 4 ints, read and written 16 bytes a lane:
//   1. row scans, one warp per row, 4 consecutive entries a lane, fused with
//      the load from global memory;
//   2. column scans in row blocks: a thread sums its column over its block,
//      then adds the blocks above and rewrites the block as running sums;
//   3. per row the total, a block scan of the totals (each row's first
//      pair), then per row an exclusive scan of its counts, written as the
//      ranges of its tiles.
// Digit counts: pass 0 (digit t mod 2^digit_bits) by shared-memory adds
// from consecutive tiles, which hit distinct digits; the last pass's digit
// d covers the tile range [d 2^shift, (d + 1) 2^shift), whose count is the
// difference of the prefixes at its two ends (kept as marks).
constexpr int kFusedMaxWords = 48 * 1024;   // ints of dynamic shared memory
__host__ __device__ constexpr int fused_ldc(int tiles_x) { return (tiles_x + 3) & ~3; }
// row blocks of the column scans: about one column block per thread, at most 64 blocks
__host__ __device__ constexpr int fused_row_blocks(int tiles_x, int tiles_y) {
  return tiles_x >= 1024 ? 1 : ((1024 / tiles_x < 64 ? 1024 / tiles_x : 64) < tiles_y
                                    ? (1024 / tiles_x < 64 ? 1024 / tiles_x : 64) : tiles_y);
}
// ints of dynamic shared memory: the counts, the column block totals, the row starts
__host__ __device__ constexpr int64_t fused_words(int tiles_x, int tiles_y) {
  return (int64_t)tiles_y * fused_ldc(tiles_x) + (int64_t)fused_row_blocks(tiles_x, tiles_y) * tiles_x + tiles_y;
}

__global__ void __launch_bounds__(1024) fused_tile_scan_kernel(const int *__restrict__ diff, int tiles_x,
                                                               int tiles_y, int passes, int digit_bits,
                                                               const Hdr *hdr, uint2 *__restrict__ ranges,
                                                               uint32_t *__restrict__ hist) {
  extern __shared__ __align__(16) int s_dyn[];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_dig[kMaxPasses * 256];
  __shared__ uint32_t s_mark[257];
  const int W = tiles_x, H = tiles_y, cols = tiles_x + 1;
  const int ldc = fused_ldc(W), nb = fused_row_blocks(W, H);
  int *s_c = s_dyn;                              // [H][ldc]
  int *s_bt = s_dyn + (size_t)H * ldc;           // [nb][W]
  uint32_t *s_row = reinterpret_cast<uint32_t *>(s_bt + (size_t)nb * W);  // [H]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kMaxPasses * 256; i += blockDim.x) s_dig[i] = 0u;
  // 1. row scans, four rows of a warp (rg + 32 j) at a time, their loads issued together
  for (int rg = warp; rg < H; rg += 128) {
    int carry[4] = {0, 0, 0, 0};
    for (int c0 = 0; c0 < W; c0 += 128) {
      const int c = c0 + 4 * lane;
      int v[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = rg + 32 * j;
        const int *src = diff + (size_t)r * cols;
#pragma unroll
        for (int i = 0; i < 4; ++i) v[j][i] = (r < H && c + i < W) ? src[c + i] : 0;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = rg + 32 * j;
        v[j][1] += v[j][0];
        v[j][2] += v[j][1];
        v[j][3] += v[j][2];
        const int incl = (int)warp_incl_scan((uint32_t)v[j][3], lane);
        const int off = carry[j] + incl - v[j][3];
        if (r < H && c < ldc)
          *reinterpret_cast<int4 *>(s_c + (size_t)r * ldc + c) =
              make_int4(off + v[j][0], off + v[j][1], off + v[j][2], off + v[j][3]);
        carry[j] += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
  }
  __syncthreads();
  // 2. column scans: thread (b, x) owns rows [b rb, (b + 1) rb) of column x
  const int rb = (H + nb - 1) / nb;
  for (int task = tid; task < nb * W; task += blockDim.x) {
    const int b = task / W, x = task - b * W;
    const int r1 = min(H, (b + 1) * rb);
    int s = 0;
    for (int r = b * rb; r < r1; ++r) s += s_c[(size_t)r * ldc + x];
    s_bt[task] = s;
  }
  __syncthreads();
  for (int task = tid; task < nb * W; task += blockDim.x) {
    const int b = task / W, x = task - b * W;
    const int r1 = min(H, (b + 1) * rb);
    int s = 0;
    for (int q = 0; q < b; ++q) s += s_bt[q * W + x];
    for (int r = b * rb; r < r1; ++r) {
      s += s_c[(size_t)r * ldc + x];
      s_c[(size_t)r * ldc + x] = s;
    }
  }
  __syncthreads();
  // 3a. row totals (counts of the columns x < W only: the padding holds partial sums)
  for (int r = warp; r < H; r += 32) {
    uint32_t s = 0;
    for (int c0 = 0; c0 < W; c0 += 128) {
      const int c = c0 + 4 * lane;
      if (c < W) {
        const int4 v = *reinterpret_cast<const int4 *>(s_c + (size_t)r * ldc + c);
        s += (uint32_t)v.x + (c + 1 < W ? (uint32_t)v.y : 0u) + (c + 2 < W ? (uint32_t)v.z : 0u) +
             (c + 3 < W ? (uint32_t)v.w : 0u);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_row[r] = s;
  }
  __syncthreads();
  // 3b. each row's first pair: thread i sums rows [i run, (i + 1) run)
  uint32_t total;
  {
    const int run = (H + 1023) / 1024;
    const int r0 = min(H, tid * run), r1 = min(H, r0 + run);
    uint32_t sum = 0;
    for (int r = r0; r < r1; ++r) sum += s_row[r];
    uint32_t start = block_excl_scan1024(sum, s_warp, &total);
    for (int r = r0; r < r1; ++r) {
      const uint32_t v = s_row[r];
      s_row[r] = start;
      start += v;
    }
  }
  __syncthreads();
  // 3c. per row: the exclusive scan of its counts, the ranges, the digit counts
  const uint32_t dmask = (1u << digit_bits) - 1;
  const int hshift = digit_bits * (passes - 1);
  const uint32_t hmask = (1u << hshift) - 1;
  const bool over = (hdr->status & kDevErrCapacity) != 0u;  // nothing sorted: every range empty
  for (int r = warp; r < H; r += 32) {
    uint32_t carry = s_row[r];
    for (int c0 = 0; c0 < W; c0 += 128) {
      const int c = c0 + 4 * lane;
      uint32_t v[4] = {0u, 0u, 0u, 0u};
      if (c < W) {
        const int4 q = *reinterpret_cast<const int4 *>(s_c + (size_t)r * ldc + c);
        v[0] = (uint32_t)q.x;
        v[1] = c + 1 < W ? (uint32_t)q.y : 0u;
        v[2] = c + 2 < W ? (uint32_t)q.z : 0u;
        v[3] = c + 3 < W ? (uint32_t)q.w : 0u;
      }
      const uint32_t lsum = v[0] + v[1] + v[2] + v[3];
      const uint32_t incl = warp_incl_scan(lsum, lane);
      uint32_t pre = carry + incl - lsum;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (c + i < W) {
          const uint32_t t = (uint32_t)r * (uint32_t)W + (uint32_t)(c + i);
          ranges[t] = (v[i] && !over) ? make_uint2(pre, pre + v[i]) : make_uint2(0u, 0u);
          if (passes > 1 && v[i]) atomicAdd(&s_dig[t & dmask], v[i]);
          if ((t & hmask) == 0u) s_mark[t >> hshift] = pre;
        }
        pre += v[i];
      }
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();
  // the last pass's digit counts: prefix differences between marks
  const int n = W * H;
  const int nmark = (n + (1 << hshift) - 1) >> hshift;
  for (int d = tid; d < nmark; d += blockDim.x)
    s_dig[(passes - 1) * 256 + d] = (d + 1 < nmark ? s_mark[d + 1] : total) - s_mark[d];
  __syncthreads();
  if (warp < passes) {  // per pass, the exclusive prefix over digits
    uint32_t carry = 0;
    for (int d0 = 0; d0 < 256; d0 += 32) {
      const uint32_t v = s_dig[warp * 256 + d0 + lane];
      const uint32_t incl = warp_incl_scan(v, lane);
      hist[warp * 256 + d0 + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// ---- emit keys ----
// CTA b writes keys [b T, (b+1) T), T = 2048.  One binary search over the
// CTA offsets and the offsets inside a count CTA finds the owner of the
// first key; the offsets of the following Gaussians are then staged in
// shared memory, where every thread finds the owners of its keys.  Keys are
// written coalesced whatever the sizes of the rectangles.
__device__ __forceinline__ uint32_t global_offset(const unsigned long long *partial, const uint32_t *local,
                                                  int64_t g) {
  return (uint32_t)partial[g / kCountThreads] + local[g];
}

__device__ __forceinline__ int64_t pair_owner(const unsigned long long *__restrict__ partial, int64_t nb,
                                              const uint32_t *__restrict__ local, int64_t n_gauss, uint32_t i) {
  int64_t lo = 0, hi = nb;  // first count CTA whose offset exceeds i
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (partial[mid] <= i) lo = mid + 1;
    else hi = mid;
  }
  const int64_t b = lo - 1;
  const uint32_t i2 = i - (uint32_t)partial[b];
  lo = b * kCountThreads;
  hi = min(lo + kCountThreads, n_gauss);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (local[mid] <= i2) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// owner[c] = the Gaussian whose pairs contain key c * kEmitTile, for every
// emit CTA c below the capacity.  One thread per Gaussian; a range covers
// floor((off + cnt - 1) / T) - ceil(off / T) + 1 chunk starts (usually 0 or 1).
// Pairs of a packed rectangle: {tx0 | ty0 << 16, w | h << 16} (one canvas)
// or {first tile, tiles_x, w, h} (a batch).
__device__ __forceinline__ uint32_t rect_pairs(const uint2 &rc) { return (rc.y & 0xffffu) * (rc.y >> 16); }
__device__ __forceinline__ uint32_t rect_pairs(const uint4 &rc) { return rc.z * rc.w; }

template <typename Rect>
__global__ void chunk_owner_kernel(const uint32_t *__restrict__ local, const unsigned long long *__restrict__ partial,
                                   const Rect *__restrict__ rects, int64_t n_gauss, uint32_t n_chunks,
                                   uint32_t *__restrict__ owner) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_gauss) return;
  const uint32_t cnt = rect_pairs(rects[g]);
  if (!cnt) return;
  const unsigned long long off = partial[g / kCountThreads] + local[g];
  const unsigned long long c0 = (off + kEmitTile - 1) / kEmitTile, c1 = (off + cnt - 1) / kEmitTile;
  for (unsigned long long c = c0; c <= c1 && c < n_chunks; ++c) owner[c] = (uint32_t)g;
}

// Owner of key i: a binary search over the CTA's window of offsets in
// shared memory, or over the global offsets when the window is too short
// (runs of Gaussians without pairs).
__device__ __forceinline__ int64_t window_owner(const uint32_t *s_off, int win, int64_t g0,
                                                const unsigned long long *partial, int64_t nb,
                                                const uint32_t *local, int64_t n_gauss, uint32_t i) {
  if (s_off[win - 1] <= i) return pair_owner(partial, nb, local, n_gauss, i);
  int lo = 0, hi = win;  // first window entry whose offset exceeds i
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s_off[mid] <= i) lo = mid + 1;
    else hi = mid;
  }
  return g0 + lo - 1;
}

// CTA b writes keys [b T, (b+1) T), T = 2048; thread t makes the keys
// 8t .. 8t+7 of that range: one owner search, then a walk along the owner's
// rectangle row by row (a new search only when the walk leaves the owner's
// pairs).  The keys are staged in shared memory and written coalesced.
// The CTA's keys belong to Gaussians owner[b] .. owner[b+1], so only their
// offsets are staged.  It also adds the digit counts of its keys for the
// sort's first pass to hist1 (digit-major, partition b / 2).
// K = uint32_t: key = tile << gbits | g; K = unsigned long long (wide keys,
// tile bits + gbits > 32): key = tile << 32 | g.
static_assert(2 * kEmitTile == kSortTile, "a sort partition is two emit chunks");
template <typename K>
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(const uint32_t *__restrict__ local,
                                                            const unsigned long long *__restrict__ partial,
                                                            int64_t nb, const uint2 *__restrict__ rects,
                                                            int64_t n_gauss, const unsigned long long *count,
                                                            int tiles_x, int gbits,
                                                            const uint32_t *__restrict__ owner,
                                                            K *__restrict__ keys, int bits1,
                                                            uint32_t *__restrict__ hist1, uint32_t parts) {
  constexpr int kWin = kEmitTile + 1;
  __shared__ uint32_t s_off[kWin];
  __shared__ K s_keys[kEmitTile];
  __shared__ uint32_t s_h[256];
  const uint32_t n = (uint32_t)*count;
  const uint32_t k0 = blockIdx.x * (uint32_t)kEmitTile;
  if (k0 >= n) return;
  const int64_t g0 = owner[blockIdx.x];
  // the window ends one past the owner of the next chunk's first key (the
  // last chunk: capped; an owner outside the window is found globally)
  const bool last_chunk = k0 + (uint32_t)kEmitTile >= n;
  const int64_t win_need = last_chunk ? n_gauss - g0 + 1 : (int64_t)owner[blockIdx.x + 1] - g0 + 2;
  const int win = (int)(win_need < kWin ? win_need : kWin);
  for (int k = threadIdx.x; k < 256; k += kEmitThreads) s_h[k] = 0u;
  // offsets of Gaussians g0, g0+1, ...; beyond the table: +infinity
  for (int k = threadIdx.x; k < win; k += kEmitThreads) {
    const int64_t g = g0 + k;
    s_off[k] = g < n_gauss ? global_offset(partial, local, g) : 0xffffffffu;
  }
  __syncthreads();
  const uint32_t i0 = k0 + (uint32_t)threadIdx.x * kEmitItems;
  const uint32_t dmask = (1u << bits1) - 1;
  if (i0 < n) {
    int64_t g = window_owner(s_off, win, g0, partial, nb, local, n_gauss, i0);
    uint32_t off = global_offset(partial, local, g);
    uint2 rc = rects[g];
    uint32_t w = rc.y & 0xffffu, cnt = w * (rc.y >> 16);
    uint32_t l = i0 - off;
    uint32_t ry = l / w, rx = l - ry * w;
#pragma unroll
    for (int it = 0; it < kEmitItems; ++it) {
      const uint32_t i = i0 + (uint32_t)it;
      if (i >= n) break;
      if (i - off >= cnt) {  // left the owner's pairs
        g = window_owner(s_off, win, g0, partial, nb, local, n_gauss, i);
        off = global_offset(partial, local, g);
        rc = rects[g];
        w = rc.y & 0xffffu;
        cnt = w * (rc.y >> 16);
        l = i - off;
        ry = l / w;
        rx = l - ry * w;
      }
      const uint32_t tid = ((rc.x >> 16) + ry) * (uint32_t)tiles_x + (rc.x & 0xffffu) + rx;
      if constexpr (sizeof(K) == 8)
        s_keys[threadIdx.x * kEmitItems + it] = ((K)tid << 32) | (K)g;
      else
        s_keys[threadIdx.x * kEmitItems + it] = (tid << gbits) | (uint32_t)g;
      atomicAdd(&s_h[tid & dmask], 1u);
      if (++rx == w) {
        rx = 0;
        ++ry;
      }
    }
  }
  __syncthreads();
  const uint32_t m = min((uint32_t)kEmitTile, n - k0);
  for (uint32_t j = threadIdx.x; j < m; j += kEmitThreads) keys[k0 + j] = s_keys[j];
  for (uint32_t d = threadIdx.x; d <= dmask; d += kEmitThreads)
    if (s_h[d]) atomicAdd(&hist1[(size_t)d * parts + (blockIdx.x >> 1)], s_h[d]);
}

// ---- sort passes ----

// Digit counts of partition blockIdx.x, stored digit-major:
// hist[d * parts + partition].
template <typename K>
__global__ void __launch_bounds__(kSortThreads) upsweep_kernel(const K *__restrict__ in,
                                                               const unsigned long long *count, int shift, int bits,
                                                               uint32_t *__restrict__ hist, uint32_t parts) {
  __shared__ uint32_t s_h[kSortWarps][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&s_h[0][0])[i] = 0u;
  const uint32_t n = (uint32_t)*count, nbins = 1u << bits, dmask = nbins - 1;
  const uint32_t base = blockIdx.x * (uint32_t)kSortTile;
  // all of a thread's keys in flight at once, 16 bytes a load when the key
  // array is 16-byte aligned (partitions start on multiples of kSortTile
  // keys); the counts do not depend on the order
  constexpr int kVec = 16 / (int)sizeof(K), kLoads = kSortTile / (kSortThreads * kVec);
  const bool vec = (reinterpret_cast<uintptr_t>(in) & 15u) == 0u;
  K key[kLoads][kVec];
#pragma unroll
  for (int j = 0; j < kLoads; ++j) {
    const uint32_t idx = base + (uint32_t)(j * kSortThreads + tid) * kVec;
    if (vec && idx + kVec <= n) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in + idx));
      memcpy(&key[j][0], &v, sizeof(v));
    } else {
#pragma unroll
      for (int e = 0; e < kVec; ++e) key[j][e] = idx + e < n ? in[idx + e] : K(0);
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kLoads; ++j) {
    const uint32_t idx = base + (uint32_t)(j * kSortThreads + tid) * kVec;
#pragma unroll
    for (int e = 0; e < kVec; ++e)
      if (idx + e < n) atomicAdd(&s_h[warp][(uint32_t)(key[j][e] >> shift) & dmask], 1u);
  }
  __syncthreads();
  for (uint32_t d = tid; d < nbins; d += kSortThreads) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) c += s_h[w][d];
    hist[(size_t)d * parts + blockIdx.x] = c;
  }
}

// Digit blockIdx.x: in place, the exclusive prefix over partitions of its
// counts plus the digit's global start = each partition's first output index
// for its keys of this digit.
__global__ void __launch_bounds__(kScanThreads) scan_parts_kernel(uint32_t *__restrict__ hist, uint32_t parts,
                                                                  const uint32_t *__restrict__ digit_start) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *row = hist + (size_t)blockIdx.x * parts;
  if (threadIdx.x == 0) s_carry = digit_start[blockIdx.x];
  constexpr int kPer = 4;
  for (uint32_t base = 0; base < parts; base += kScanThreads * kPer) {
    uint32_t v[kPer], sum = 0;
    const uint32_t i0 = base + threadIdx.x * kPer;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      v[k] = i0 + k < parts ? row[i0 + k] : 0u;
      sum += v[k];
    }
    const uint32_t incl = warp_incl_scan(sum, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) s_warp[lane] = warp_incl_scan(s_warp[lane], lane);
    __syncthreads();
    uint32_t run = s_carry + (warp ? s_warp[warp - 1] : 0u) + incl - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (i0 + k < parts) row[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_warp[31];
    __syncthreads();
  }
}

// Partition blockIdx.x: stable rank of each key among the partition's keys
// with the same digit (peer lanes from ballots, then per-warp running counts), keys
// gathered by digit in shared memory, then written at the partition's first
// output index for the digit (from scan_parts_kernel) plus their rank.
// K: the key type; O: the output type (the last pass of a batch writes the
// key's low 32 bits, the Gaussian index, only).  A partition past the count
// has nothing to write.
template <typename K, typename O>
__global__ void __launch_bounds__(kSortThreads, 4) downsweep_kernel(const K *__restrict__ in,
                                                                 O *__restrict__ out,
                                                                 const unsigned long long *count,
                                                                 int shift, int bits,
                                                                 const uint32_t *__restrict__ offs, uint32_t parts) {
  __shared__ K s_keys[kSortTile];
  __shared__ uint32_t s_whist[kSortWarps][256];
  __shared__ uint32_t s_bexcl[256];
  __shared__ uint32_t s_dst[256];
  __shared__ uint32_t s_wtot[kSortWarps];
  const uint32_t n = (uint32_t)*count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nbins = 1u << bits, dmask = nbins - 1;
  const uint32_t part = blockIdx.x;
  if (part * (uint32_t)kSortTile >= n) return;
  for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t base = part * (uint32_t)kSortTile + (uint32_t)warp * (32u * kSortItems);
  const unsigned lt_mask = (1u << lane) - 1;

  // a key's rank among its warp's keys of the same digit is < 512: two
  // ranks share a register
  K keys[kSortItems];
  uint32_t rank2[kSortItems / 2];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + (uint32_t)i * 32u + (uint32_t)lane;
    keys[i] = idx < n ? in[idx] : K(0);
  }
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + (uint32_t)i * 32u + (uint32_t)lane;
    const bool valid = idx < n;
    const uint32_t d = (uint32_t)(keys[i] >> shift) & dmask;
    // lanes with the same digit: the AND of one ballot per digit bit
    unsigned peers = __ballot_sync(0xffffffffu, valid);
    for (int b = 0; b < bits; ++b) {
      const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? bb : ~bb;
    }
    const uint32_t cnt = valid ? s_whist[warp][d] : 0u;
    const uint32_t rk = cnt + __popc(peers & lt_mask);
    rank2[i >> 1] = (i & 1) ? (rank2[i >> 1] | (rk << 16)) : rk;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_whist[warp][d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // per digit (one thread each): warp offsets within the partition
  uint32_t bcount = 0;
  if (tid < (int)nbins) {
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = bcount;
      bcount += c;
    }
  }
  // exclusive prefix of the partition's digit counts (warp scans, then totals)
  const uint32_t incl = warp_incl_scan(bcount, lane);
  if (lane == 31) s_wtot[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wbase += w < warp ? s_wtot[w] : 0u;
  const uint32_t bexcl = wbase + incl - bcount;
  s_bexcl[tid] = bexcl;
  if (tid < (int)nbins) s_dst[tid] = offs[(size_t)tid * parts + part] - bexcl;
  __syncthreads();
  // gather in shared memory by (digit, input order)
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + (uint32_t)i * 32u + (uint32_t)lane;
    if (idx < n) {
      const uint32_t d = (uint32_t)(keys[i] >> shift) & dmask;
      s_keys[s_bexcl[d] + s_whist[warp][d] + ((rank2[i >> 1] >> (16 * (i & 1))) & 0xffffu)] = keys[i];
    }
  }
  __syncthreads();
  const uint32_t pstart = part * (uint32_t)kSortTile;
  const uint32_t n_here = n > pstart ? min((uint32_t)kSortTile, n - pstart) : 0u;
  for (uint32_t j = tid; j < n_here; j += kSortThreads) {
    const K k = s_keys[j];
    out[s_dst[(uint32_t)(k >> shift) & dmask] + j] = (O)k;
  }
}


// ---- batches of images ----

// Per Gaussian of a batch: its image's tile rectangle (the rule of
// tile_rect on the image's canvas), packed as {first tile (global), tiles_x,
// w, h}; its pair count and block-local offset; the four corner updates of
// its image's difference array.
__global__ void __launch_bounds__(kCountThreads) batch_count_kernel(const float *gauss, int64_t n_gauss,
                                                                    const BatchImage *__restrict__ tab, int n_images,
                                                                    int tile, uint32_t *local,
                                                                    unsigned long long *partial, uint4 *rects,
                                                                    int *diff) {
  __shared__ uint32_t s_warp[kCountThreads / 32];
  const int64_t g = (int64_t)blockIdx.x * kCountThreads + threadIdx.x;
  uint32_t cnt = 0;
  Rect r;
  bool ok = false;
  int *d = nullptr;
  int stride = 0;
  if (g < n_gauss) {
    const BatchImage &im = tab[last_image_le<&BatchImage::gauss0>(tab, n_images, g)];
    uint4 packed = make_uint4(0u, 0u, 0u, 0u);
    ok = tile_rect(gauss, g, im.W, im.H, tile, &r);
    if (ok) {
      const uint32_t w = (uint32_t)(r.tx1 - r.tx0 + 1), h = (uint32_t)(r.ty1 - r.ty0 + 1);
      cnt = w * h;
      packed = make_uint4((uint32_t)(im.tile0 + (int64_t)r.ty0 * im.tiles_x + r.tx0), (uint32_t)im.tiles_x, w, h);
      stride = im.tiles_x + 1;
      d = diff + im.diff0;
    }
    rects[g] = packed;
  }
  const unsigned active = __ballot_sync(0xffffffffu, ok);
  if (ok) add_corners(active, d, stride, r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(cnt, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < kCountThreads / 32 ? s_warp[lane] : 0u;
    v = warp_incl_scan(v, lane);
    if (lane < kCountThreads / 32) s_warp[lane] = v;
  }
  __syncthreads();
  const uint32_t warp_excl = warp == 0 ? 0u : s_warp[warp - 1];
  if (g < n_gauss) local[g] = warp_excl + incl - cnt;
  if (threadIdx.x == kCountThreads - 1) partial[blockIdx.x] = warp_excl + incl;
}

// Row scans of every image's difference array: one warp per row.
__global__ void batch_diff_rows_kernel(int *diff, const BatchImage *__restrict__ tab, int n_images, int64_t n_rows) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const BatchImage &im = tab[last_image_le<&BatchImage::row0>(tab, n_images, row)];
  const int cols = im.tiles_x + 1;
  int *d = diff + im.diff0 + (row - im.row0) * cols;
  int carry = 0;
  for (int c0 = 0; c0 < cols; c0 += 32) {
    const int c = c0 + lane;
    int v = c < cols ? d[c] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (c < cols) d[c] = carry + v;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
}

// Column scans of every image's difference array: one warp per column.
__global__ void batch_diff_cols_kernel(int *diff, const BatchImage *__restrict__ tab, int n_images, int64_t n_cols) {
  const int64_t col = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= n_cols) return;
  const BatchImage &im = tab[last_image_le<&BatchImage::col0>(tab, n_images, col)];
  const int cols = im.tiles_x + 1, rows = im.tiles_y + 1;
  int *d = diff + im.diff0 + (col - im.col0);
  int carry = 0;
  for (int r0 = 0; r0 < rows; r0 += 32) {
    const int r = r0 + lane;
    int v = r < rows ? d[(size_t)r * cols] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (r < rows) d[(size_t)r * cols] = carry + v;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
}

// Per-tile counts of a batch in tile order: thread i of CTA c walks tiles
// [(c 256 + i) 8, +8), which may cross into the next image.
constexpr int kTileThreads = 256;
constexpr int kTileItems = 8;

struct TileWalk {
  int b, tiles_x, tx, ty;
  int64_t next0, diff0;
};

__device__ __forceinline__ TileWalk tile_walk_start(const BatchImage *__restrict__ tab, int n_images, int64_t t) {
  TileWalk w;
  w.b = last_image_le<&BatchImage::tile0>(tab, n_images, t);
  const BatchImage &im = tab[w.b];
  const int local = (int)(t - im.tile0);
  w.tiles_x = im.tiles_x;
  w.ty = local / im.tiles_x;
  w.tx = local - w.ty * im.tiles_x;
  w.diff0 = im.diff0;
  w.next0 = w.b + 1 < n_images ? tab[w.b + 1].tile0 : INT64_MAX;
  return w;
}

// The count of tile t (the walk's current tile), then the walk moves on.
__device__ __forceinline__ uint32_t tile_walk_next(TileWalk &w, const BatchImage *__restrict__ tab, int n_images,
                                                   const int *__restrict__ diff, int64_t t) {
  if (t == w.next0) {  // the next image starts at its tile (0, 0)
    ++w.b;
    w.tiles_x = tab[w.b].tiles_x;
    w.diff0 = tab[w.b].diff0;
    w.next0 = w.b + 1 < n_images ? tab[w.b + 1].tile0 : INT64_MAX;
    w.tx = w.ty = 0;
  }
  const uint32_t v = (uint32_t)diff[w.diff0 + (int64_t)w.ty * (w.tiles_x + 1) + w.tx];
  if (++w.tx == w.tiles_x) {
    w.tx = 0;
    ++w.ty;
  }
  return v;
}

// Sum of each CTA's tiles (tsum) and, per sort pass, the digit totals of the
// tile ids weighted by their counts (hist, added atomically).
__global__ void __launch_bounds__(kTileThreads) batch_tile_reduce_kernel(const int *__restrict__ diff,
                                                                         const BatchImage *__restrict__ tab,
                                                                         int n_images, int64_t n_tiles, int passes,
                                                                         int digit_bits,
                                                                         unsigned long long *__restrict__ tsum,
                                                                         uint32_t *__restrict__ hist) {
  __shared__ uint32_t s_h[kMaxPasses * 256];
  __shared__ unsigned long long s_w[kTileThreads / 32];
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += kTileThreads) s_h[i] = 0u;
  __syncthreads();
  const uint32_t dmask = (1u << digit_bits) - 1;
  const int64_t t0 = ((int64_t)blockIdx.x * kTileThreads + threadIdx.x) * kTileItems;
  unsigned long long sum = 0;
  if (t0 < n_tiles) {
    TileWalk w = tile_walk_start(tab, n_images, t0);
    for (int k = 0; k < kTileItems; ++k) {
      const int64_t t = t0 + k;
      if (t >= n_tiles) break;
      const uint32_t v = tile_walk_next(w, tab, n_images, diff, t);
      sum += v;
      if (v)
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p * 256 + (((uint32_t)t >> (p * digit_bits)) & dmask)], v);
    }
  }
  unsigned long long x = sum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kTileThreads / 32; ++w) t += s_w[w];
    tsum[blockIdx.x] = t;
  }
  for (int i = threadIdx.x; i < passes * 256; i += kTileThreads)
    if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

// The pair count against the capacity (status and the count to sort), and
// per pass the exclusive prefix of the digit totals: where each digit's
// keys start.  One warp per pass.
// The sort trusts that the digit starts (from the tile counts) and the keys
// (from the Gaussians' rectangles) agree; both totals are compared and
// nothing is sorted if they differ.
__global__ void batch_digits_kernel(BatchHdr *hdr, int64_t capacity, int passes, uint32_t *hist) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long P = hdr->n_pairs;
  const bool over = P > (unsigned long long)capacity;
  const bool mismatch = hdr->tile_total != P;
  if (threadIdx.x == 0) {
    hdr->n_sorted = (over || mismatch) ? 0ull : P;
    if (over) hdr->status |= kDevErrCapacity;
    if (mismatch) hdr->status |= kDevErrCounts;
  }
  if (warp < passes) {
    uint32_t carry = 0;
    for (int d0 = 0; d0 < 256; d0 += 32) {
      const uint32_t v = hist[warp * 256 + d0 + lane];
      const uint32_t incl = warp_incl_scan(v, lane);
      hist[warp * 256 + d0 + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// Tile ranges of a batch: tsum holds each CTA's first output index (the
// exclusive scan of the CTA sums).  Every range is (0, 0) after an overflow.
__global__ void __launch_bounds__(kTileThreads) batch_tile_ranges_kernel(const int *__restrict__ diff,
                                                                         const BatchImage *__restrict__ tab,
                                                                         int n_images, int64_t n_tiles,
                                                                         const unsigned long long *__restrict__ tsum,
                                                                         const BatchHdr *hdr, uint2 *__restrict__ ranges) {
  __shared__ unsigned long long s_w[kTileThreads / 32];
  const int64_t t0 = ((int64_t)blockIdx.x * kTileThreads + threadIdx.x) * kTileItems;
  uint32_t cnt[kTileItems];
  unsigned long long sum = 0;
  TileWalk w;
  if (t0 < n_tiles) {
    w = tile_walk_start(tab, n_images, t0);
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) {
      const int64_t t = t0 + k;
      cnt[k] = t < n_tiles ? tile_walk_next(w, tab, n_images, diff, t) : 0u;
      sum += cnt[k];
    }
  }
  // block-exclusive prefix of the thread sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  unsigned long long base = tsum[blockIdx.x];
  for (int k = 0; k < warp; ++k) base += s_w[k];
  if (t0 >= n_tiles) return;
  const bool over = (hdr->status & (kDevErrCapacity | kDevErrCounts)) != 0u;
  unsigned long long start = base + incl - sum;
#pragma unroll
  for (int k = 0; k < kTileItems; ++k) {
    const int64_t t = t0 + k;
    if (t >= n_tiles) break;
    ranges[t] = (!over && cnt[k]) ? make_uint2((uint32_t)start, (uint32_t)(start + cnt[k])) : make_uint2(0u, 0u);
    start += cnt[k];
  }
}

// emit_kernel for a batch: 64-bit keys (global tile << 32 | g) from the
// packed rectangles {first tile, tiles_x, w, h}; the first sort pass's digit
// counts go to hist1 as in emit_kernel.
__global__ void __launch_bounds__(kEmitThreads) batch_emit_kernel(const uint32_t *__restrict__ local,
                                                                  const unsigned long long *__restrict__ partial,
                                                                  int64_t nb, const uint4 *__restrict__ rects,
                                                                  int64_t n_gauss, const unsigned long long *count,
                                                                  const uint32_t *__restrict__ owner,
                                                                  unsigned long long *__restrict__ keys, int bits1,
                                                                  uint32_t *__restrict__ hist1, uint32_t parts) {
  constexpr int kWin = kEmitTile + 1;
  __shared__ uint32_t s_off[kWin];
  __shared__ unsigned long long s_keys[kEmitTile];
  __shared__ uint32_t s_h[256];
  const uint32_t n = (uint32_t)*count;
  const uint32_t k0 = blockIdx.x * (uint32_t)kEmitTile;
  if (k0 >= n) return;
  const int64_t g0 = owner[blockIdx.x];
  const bool last_chunk = k0 + (uint32_t)kEmitTile >= n;
  const int64_t win_need = last_chunk ? n_gauss - g0 + 1 : (int64_t)owner[blockIdx.x + 1] - g0 + 2;
  const int win = (int)(win_need < kWin ? win_need : kWin);
  for (int k = threadIdx.x; k < 256; k += kEmitThreads) s_h[k] = 0u;
  for (int k = threadIdx.x; k < win; k += kEmitThreads) {
    const int64_t g = g0 + k;
    s_off[k] = g < n_gauss ? global_offset(partial, local, g) : 0xffffffffu;
  }
  __syncthreads();
  const uint32_t i0 = k0 + (uint32_t)threadIdx.x * kEmitItems;
  const uint32_t dmask = (1u << bits1) - 1;
  if (i0 < n) {
    int64_t g = window_owner(s_off, win, g0, partial, nb, local, n_gauss, i0);
    uint32_t off = global_offset(partial, local, g);
    uint4 rc = rects[g];
    uint32_t cnt = rc.z * rc.w;
    uint32_t l = i0 - off;
    uint32_t ry = l / rc.z, rx = l - ry * rc.z;
#pragma unroll
    for (int it = 0; it < kEmitItems; ++it) {
      const uint32_t i = i0 + (uint32_t)it;
      if (i >= n) break;
      if (i - off >= cnt) {  // left the owner's pairs
        g = window_owner(s_off, win, g0, partial, nb, local, n_gauss, i);
        off = global_offset(partial, local, g);
        rc = rects[g];
        cnt = rc.z * rc.w;
        l = i - off;
        ry = l / rc.z;
        rx = l - ry * rc.z;
      }
      const uint32_t tid = rc.x + ry * rc.y + rx;
      s_keys[threadIdx.x * kEmitItems + it] = ((unsigned long long)tid << 32) | (unsigned long long)g;
      atomicAdd(&s_h[tid & dmask], 1u);
      if (++rx == rc.z) {
        rx = 0;
        ++ry;
      }
    }
  }
  __syncthreads();
  const uint32_t m = min((uint32_t)kEmitTile, n - k0);
  for (uint32_t j = threadIdx.x; j < m; j += kEmitThreads) keys[k0 + j] = s_keys[j];
  for (uint32_t d = threadIdx.x; d <= dmask; d += kEmitThreads)
    if (s_h[d]) atomicAdd(&hist1[(size_t)d * parts + (blockIdx.x >> 1)], s_h[d]);
}

// ---- two-level binning (one canvas, 32-bit keys) ----
// A stable counting sort that uses the rectangles' shape instead of sorting
// the keys.  Level 1 puts every Gaussian into the list of each tile row its
// rectangle covers, in ascending index.  Per chunk of 256 Gaussians: a bit
// per (row, Gaussian), one 32-bit ballot per warp and row, gives the chunk's
// count per row (row_count_kernel); their exclusive scan over the chunks of
// each row (row_scan_kernel) and the rows' starts (row_starts_kernel) give
// where each chunk's Gaussians of a row begin; a Gaussian's rank among them
// is the population count of the row's bits below its own
// (row_scatter_kernel).  Level 2 does the same for the columns of each
// row's list, cut into chunks of 128 entries (col_count_kernel with a
// difference array per chunk, col_scan_kernel, col_scatter_kernel): a pair's
// place is its tile's first pair, plus the tile's pairs in the row's earlier
// chunks, plus its rank among the chunk's entries covering the tile.  The
// keys come out as the radix sort writes them, (tile << gbits) | g in
// (tile, g) order.
constexpr int kRowChunk = 256;   // Gaussians per level-1 chunk (8 words of bits per row)
constexpr int kColChunk = 128;   // row-list entries per level-2 chunk (one 32-bit word of bits per warp and column)
constexpr int kColWords = kColChunk / 32;
constexpr int kRowsMax = 512, kColsMax = 512;
constexpr int kColGrid = 152 * (2048 / kColChunk);  // CTAs of the level-2 kernels (2,048 threads per SM)
static_assert(kRowChunk == 256, "eight 32-bit words of bits per row");
static_assert(kColChunk % 32 == 0 && kColChunk <= 1024, "whole warps per level-2 chunk");

// The 32 items of a warp (item = lane) over lines [a, b] (valid items only):
// bm[l * 8 + warp] = the ballot of the items covering line l, for every line
// some item of the warp covers.  Lines no item covers are left as they are.
__device__ __forceinline__ void warp_line_bits(uint32_t *bm, bool valid, int a, int b, int warp) {
  const unsigned lo = __reduce_min_sync(0xffffffffu, valid ? (unsigned)a : 0xffffffffu);
  const unsigned hi = __reduce_max_sync(0xffffffffu, valid ? (unsigned)b : 0u);
  for (unsigned l = lo; l <= hi && lo != 0xffffffffu; ++l) {
    const unsigned bits = __ballot_sync(0xffffffffu, valid && (int)l >= a && (int)l <= b);
    if ((threadIdx.x & 31) == 0) bm[l * 8 + warp] = bits;
  }
}

__device__ __forceinline__ uint32_t line_count(const uint32_t *bm, int l) {
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) c += __popc(bm[l * 8 + w]);
  return c;
}

// Exclusive scan of one value per thread over a CTA of kThreads (a multiple
// of 32, at most 1024); *total gets the sum.  Starts and ends with a barrier
// crossed by every thread, so s_warp can be reused right after.
template <int kThreads>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
  constexpr int kWarps = kThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  const uint32_t incl = warp_incl_scan(v, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = warp_incl_scan(lane < kWarps ? s_warp[lane] : 0u, lane);
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  *total = s_warp[kWarps - 1];
  const uint32_t ex = (warp ? s_warp[warp - 1] : 0u) + incl - v;
  __syncthreads();
  return ex;
}

// Level 1: the bits of chunk blockIdx.x's Gaussians over the rows.
__device__ __forceinline__ void gauss_row_bits(const uint2 *__restrict__ rects, int64_t n_gauss, int H, uint32_t *s_bm) {
  for (int i = threadIdx.x; i < H * 8; i += kRowChunk) s_bm[i] = 0u;
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * kRowChunk + threadIdx.x;
  const uint2 rc = g < n_gauss ? rects[g] : make_uint2(0u, 0u);
  const int h = (int)(rc.y >> 16), ty0 = (int)(rc.x >> 16);
  warp_line_bits(s_bm, (rc.y & 0xffffu) != 0u && h != 0, ty0, ty0 + h - 1, threadIdx.x >> 5);
  __syncthreads();
}

// t1[row][chunk] = the chunk's Gaussians covering the row.  Dynamic shared
// memory: 8 H words.
__global__ void __launch_bounds__(kRowChunk) row_count_kernel(const uint2 *__restrict__ rects, int64_t n_gauss,
                                                              int H, int n_g1, const unsigned long long *count,
                                                              uint32_t *__restrict__ t1) {
  extern __shared__ uint32_t s_rows[];
  if (*count == 0) return;  // nothing to sort (no pairs, or more than the capacity)
  gauss_row_bits(rects, n_gauss, H, s_rows);
  for (int r = threadIdx.x; r < H; r += kRowChunk) t1[(size_t)r * n_g1 + blockIdx.x] = line_count(s_rows, r);
}

// One CTA per row: t1[row][.] becomes its exclusive scan over the chunks,
// rowcnt[row] the row's total.
__global__ void __launch_bounds__(1024) row_scan_kernel(uint32_t *__restrict__ t1, int n_g1,
                                                        const unsigned long long *count,
                                                        uint32_t *__restrict__ rowcnt) {
  __shared__ uint32_t s_warp[32];
  if (*count == 0) return;
  uint32_t *row = t1 + (size_t)blockIdx.x * n_g1;
  uint32_t carry = 0;
  for (int base = 0; base < n_g1; base += 1024) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < n_g1 ? row[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan<1024>(v, s_warp, &total);
    if (i < n_g1) row[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) rowcnt[blockIdx.x] = carry;
}

// One CTA: rowstart[r] = the list entries of rows < r (rowstart[H] = all),
// chstart[r] = the level-2 chunks of rows < r (chstart[H] = all), and
// chrow[ch] = the row of level-2 chunk ch (at most n_ch_max chunks).
__global__ void __launch_bounds__(1024) row_starts_kernel(const uint32_t *__restrict__ rowcnt, int H,
                                                          const unsigned long long *count,
                                                          uint32_t *__restrict__ rowstart,
                                                          uint32_t *__restrict__ chstart,
                                                          uint32_t *__restrict__ chrow, uint32_t n_ch_max) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_ch[kRowsMax + 1];
  if (*count == 0) return;
  const int run = (H + 1023) / 1024;
  const int r0 = min(H, (int)threadIdx.x * run), r1 = min(H, r0 + run);
  uint32_t s = 0, c = 0;
  for (int r = r0; r < r1; ++r) {
    s += rowcnt[r];
    c += (rowcnt[r] + kColChunk - 1) / kColChunk;
  }
  uint32_t tot_s, tot_c;
  uint32_t ps = block_excl_scan<1024>(s, s_warp, &tot_s);
  uint32_t pc = block_excl_scan<1024>(c, s_warp, &tot_c);
  for (int r = r0; r < r1; ++r) {
    rowstart[r] = ps;
    chstart[r] = pc;
    s_ch[r] = pc;
    ps += rowcnt[r];
    pc += (rowcnt[r] + kColChunk - 1) / kColChunk;
  }
  if (threadIdx.x == 0) {
    rowstart[H] = tot_s;
    chstart[H] = tot_c;
    s_ch[H] = tot_c;
  }
  __syncthreads();
  // the row of every chunk: the last row whose first chunk is <= it
  for (uint32_t ch = threadIdx.x; ch < tot_c && ch < n_ch_max; ch += blockDim.x) {
    int lo = 0, hi = H;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_ch[mid] <= ch) lo = mid + 1;
      else hi = mid;
    }
    chrow[ch] = (uint32_t)(lo - 1);
  }
}

// Per line of a CTA's bits (kWords words, one per warp of 32 items): the set
// bits of its earlier words, pre[l * kWords + w].
template <int kWords>
__device__ __forceinline__ void word_prefixes(const uint32_t *bm, int n, uint32_t *pre, int threads) {
  for (int l = threadIdx.x; l < n; l += threads) {
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kWords; ++w) {
      pre[l * kWords + w] = acc;
      acc += __popc(bm[l * kWords + w]);
    }
  }
}

// Item e (= threadIdx.x, valid, covering lines [a, b]) writes v (kTileKey:
// ((tile0 + l) << gbits) | v) to out[base[l] + its rank among the items
// covering l] for each of its lines l.  A warp whose lines span at most 64
// walks them in step, so each store instruction writes one line's
// consecutive ranks; a wider warp walks each item's own lines.
template <bool kTileKey, int kWords>
__device__ __forceinline__ void scatter_ranks(const uint32_t *bm, const uint32_t *pre, const uint32_t *base,
                                              bool valid, int a, int b, uint32_t v, uint32_t tile0, int gbits,
                                              uint32_t *__restrict__ out, uint32_t cap) {
  const int e = threadIdx.x, we = e >> 5;
  const uint32_t below = (1u << (e & 31)) - 1u;
  const unsigned lo = __reduce_min_sync(0xffffffffu, valid ? (unsigned)a : 0xffffffffu);
  const unsigned hi = __reduce_max_sync(0xffffffffu, valid ? (unsigned)b : 0u);
  if (lo == 0xffffffffu) return;
  const bool step = hi - lo < 64u;
  const int l0 = step ? (int)lo : a, l1 = step ? (int)hi : (valid ? b : a - 1);
  for (int l = l0; l <= l1; ++l) {
    if (valid && l >= a && l <= b) {
      const uint32_t pos = base[l] + pre[l * kWords + we] + (uint32_t)__popc(bm[l * kWords + we] & below);
      if (pos < cap) out[pos] = kTileKey ? ((tile0 + (uint32_t)l) << gbits) | v : v;
    }
  }
}

// The chunk's Gaussians into the row lists: Gaussian g of the chunk goes to
// rowlist[rowstart[row] + t1[row][chunk] + its rank among the chunk's
// Gaussians covering the row] for each row it covers.  Dynamic shared
// memory: 17 H words.
__global__ void __launch_bounds__(kRowChunk) row_scatter_kernel(const uint2 *__restrict__ rects, int64_t n_gauss,
                                                                int H, int n_g1, const unsigned long long *count,
                                                                const uint32_t *__restrict__ t1,
                                                                const uint32_t *__restrict__ rowstart,
                                                                uint32_t *__restrict__ rowlist, uint32_t cap) {
  extern __shared__ uint32_t s_rows[];  // [H][8] bits, [H][8] word prefixes, [H] bases
  if (*count == 0) return;
  uint32_t *s_pre = s_rows + H * 8, *s_base = s_pre + H * 8;
  for (int r = threadIdx.x; r < H; r += kRowChunk) s_base[r] = rowstart[r] + t1[(size_t)r * n_g1 + blockIdx.x];
  gauss_row_bits(rects, n_gauss, H, s_rows);
  word_prefixes<8>(s_rows, H, s_pre, kRowChunk);
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * kRowChunk + threadIdx.x;
  const uint2 rc = g < n_gauss ? rects[g] : make_uint2(0u, 0u);
  const int h = (int)(rc.y >> 16), ty0 = (int)(rc.x >> 16);
  scatter_ranks<false, 8>(s_rows, s_pre, s_base, (rc.y & 0xffffu) != 0u && h != 0, ty0, ty0 + h - 1, (uint32_t)g, 0u,
                       0, rowlist, cap);
}

// Level 2: chunk ch of the row lists (its row, its first entry and its
// entries m).  The level-2 kernels loop over the chunks (CTA b takes b, b +
// gridDim.x, ...: their number is known only on the device, below
// chstart[H]); thread e holds entry e of the chunk.
struct ColChunk {
  int row;
  uint32_t e0, m;
};

__device__ __forceinline__ void col_chunk(const uint32_t *__restrict__ rowcnt, const uint32_t *__restrict__ chstart,
                                          const uint32_t *__restrict__ chrow, uint32_t ch, ColChunk *c) {
  c->row = (int)chrow[ch];
  c->e0 = (ch - chstart[c->row]) * kColChunk;
  c->m = min((uint32_t)kColChunk, rowcnt[c->row] - c->e0);
}

// t2[chunk][tx] = the chunk's entries covering column tx: each entry adds
// +1 / -1 at the ends of its columns in a difference array, then a scan.
// Dynamic shared memory: W + 1 words.
__global__ void __launch_bounds__(kColChunk) col_count_kernel(const uint2 *__restrict__ rects,
                                                              const uint32_t *__restrict__ rowlist,
                                                              const uint32_t *__restrict__ rowcnt,
                                                              const uint32_t *__restrict__ rowstart,
                                                              const uint32_t *__restrict__ chstart,
                                                              const uint32_t *__restrict__ chrow, int H, int W,
                                                              const unsigned long long *count,
                                                              uint32_t *__restrict__ t2) {
  extern __shared__ int s_diff[];
  __shared__ uint32_t s_warp[32];
  if (*count == 0) return;
  const uint32_t n_ch = chstart[H];
  const int run = (W + kColChunk - 1) / kColChunk;
  const int x0 = min(W, (int)threadIdx.x * run), x1 = min(W, x0 + run);
  for (uint32_t ch = blockIdx.x; ch < n_ch; ch += gridDim.x) {
    ColChunk c;
    col_chunk(rowcnt, chstart, chrow, ch, &c);
    for (int i = threadIdx.x; i <= W; i += kColChunk) s_diff[i] = 0;
    __syncthreads();
    if (threadIdx.x < c.m) {
      const uint2 rc = rects[rowlist[rowstart[c.row] + c.e0 + threadIdx.x]];
      const int tx0 = (int)(rc.x & 0xffffu), w = (int)(rc.y & 0xffffu);
      atomicAdd(&s_diff[tx0], 1);
      atomicSub(&s_diff[tx0 + w], 1);
    }
    __syncthreads();
    int sum = 0;
    for (int x = x0; x < x1; ++x) sum += s_diff[x];
    uint32_t total;
    int acc = (int)block_excl_scan<kColChunk>((uint32_t)sum, s_warp, &total);
    for (int x = x0; x < x1; ++x) {
      acc += s_diff[x];
      t2[(size_t)ch * W + x] = (uint32_t)acc;
    }
    __syncthreads();  // before the next chunk clears s_diff
  }
}

// One CTA of 1024 threads per row: t2[.][tx] over the row's chunks becomes
// its exclusive scan.  Thread (seg, tx) owns segment seg of the row's chunks
// (1024 / W segments): it sums its segment, then adds the segments before it
// and rewrites its segment as running sums (eight chunks' counts loaded at a
// time).
__global__ void __launch_bounds__(1024) col_scan_kernel(uint32_t *__restrict__ t2,
                                                        const uint32_t *__restrict__ chstart, int W,
                                                        const unsigned long long *count) {
  __shared__ uint32_t s_tot[1024];
  if (*count == 0) return;
  const int row = blockIdx.x, n_seg = 1024 / W;
  const int seg = threadIdx.x / W, tx = threadIdx.x - seg * W;
  const uint32_t c0 = chstart[row], c1 = chstart[row + 1];
  const uint32_t per = (c1 - c0 + n_seg - 1) / n_seg;
  const uint32_t a = min(c1, c0 + (uint32_t)seg * per), b = min(c1, a + per);
  const bool mine = seg < n_seg;
  uint32_t s = 0;
  if (mine)
    for (uint32_t c = a; c < b; c += 8) {
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = c + k < b ? t2[(size_t)(c + k) * W + tx] : 0u;
#pragma unroll
      for (int k = 0; k < 8; ++k) s += v[k];
    }
  s_tot[threadIdx.x] = s;
  __syncthreads();
  if (!mine) return;
  uint32_t off = 0;
  for (int q = 0; q < seg; ++q) off += s_tot[q * W + tx];
  for (uint32_t c = a; c < b; c += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = c + k < b ? t2[(size_t)(c + k) * W + tx] : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c + k < b) {
        t2[(size_t)(c + k) * W + tx] = off;
        off += v[k];
      }
  }
}

// Each entry of the chunk writes its pairs: in column tx, its rank is the
// chunk's entries before it covering tx (a bit per (column, entry), the
// population counts of the column's earlier words kept as prefixes), and
// its key (tile << gbits) | g goes to ranges[tile].x + t2[chunk][tx] + rank
// (the sum of the first two kept per column).  Dynamic shared memory:
// (2 kColWords + 1) W words.
__global__ void __launch_bounds__(kColChunk) col_scatter_kernel(const uint2 *__restrict__ rects,
                                                                const uint32_t *__restrict__ rowlist,
                                                                const uint32_t *__restrict__ rowcnt,
                                                                const uint32_t *__restrict__ rowstart,
                                                                const uint32_t *__restrict__ chstart,
                                                                const uint32_t *__restrict__ chrow, int H, int W,
                                                                const unsigned long long *count,
                                                                const uint32_t *__restrict__ t2,
                                                                const uint2 *__restrict__ ranges, int gbits,
                                                                uint32_t *__restrict__ keys, uint32_t cap) {
  extern __shared__ uint32_t s_cols[];  // [W][8] bits, [W][8] word prefixes, [W] bases
  if (*count == 0) return;
  uint32_t *s_wpre = s_cols + W * kColWords, *s_base = s_wpre + W * kColWords;
  const uint32_t n_ch = chstart[H];
  const int e = threadIdx.x, we = e >> 5;
  for (uint32_t ch = blockIdx.x; ch < n_ch; ch += gridDim.x) {
    ColChunk c;
    col_chunk(rowcnt, chstart, chrow, ch, &c);
    for (int i = threadIdx.x; i < W * kColWords; i += kColChunk) s_cols[i] = 0u;
    for (int tx = threadIdx.x; tx < W; tx += kColChunk)
      s_base[tx] = ranges[c.row * W + tx].x + t2[(size_t)ch * W + tx];
    __syncthreads();
    const bool valid = (uint32_t)e < c.m;
    uint32_t g = 0;
    int tx0 = 0, tx1 = -1;
    if (valid) {
      g = rowlist[rowstart[c.row] + c.e0 + e];
      const uint2 rc = rects[g];
      tx0 = (int)(rc.x & 0xffffu);
      tx1 = tx0 + (int)(rc.y & 0xffffu) - 1;
      for (int tx = tx0; tx <= tx1; ++tx) atomicOr(&s_cols[tx * kColWords + we], 1u << (e & 31));
    }
    __syncthreads();
    word_prefixes<kColWords>(s_cols, W, s_wpre, kColChunk);
    __syncthreads();
    scatter_ranks<true, kColWords>(s_cols, s_wpre, s_base, valid, tx0, tx1, g, (uint32_t)c.row * (uint32_t)W, gbits, keys, cap);
    __syncthreads();  // before the next chunk rewrites the shared tables
  }
}

}  // namespace

bs_status plan_binning(int64_t n_gauss, const bs_canvas &cv, int64_t capacity, BinPlan *p, bool allow_rows) {
  if (n_gauss < 0 || n_gauss > (1ll << 31) - 1) {
    set_error("n_gauss %lld out of range", (long long)n_gauss);
    return BS_ERR_INVALID_ARG;
  }
  if (cv.width < 1 || cv.height < 1 || cv.width > 32768 || cv.height > 32768) {
    set_error("canvas %dx%d out of range", cv.width, cv.height);
    return BS_ERR_INVALID_ARG;
  }
  if (cv.tile != 8 && cv.tile != 16 && cv.tile != 32) {
    set_error("tile side %d not supported (8, 16, 32)", cv.tile);
    return BS_ERR_UNSUPPORTED;
  }
  if (capacity < 0 || capacity > kMaxPairs) {
    set_error("pair_capacity %lld out of range [0, 2^30)", (long long)capacity);
    return BS_ERR_INVALID_ARG;
  }
  p->n_gauss = n_gauss;
  p->tiles_x = div_up(cv.width, cv.tile);
  p->tiles_y = div_up(cv.height, cv.tile);
  p->n_tiles = p->tiles_x * p->tiles_y;
  p->gbits = gauss_bits(n_gauss);
  p->tbits = p->n_tiles > 1 ? bit_length((uint64_t)(p->n_tiles - 1)) : 1;
  p->wide = p->gbits + p->tbits > 32;
  p->passes = div_up(p->tbits, 8);
  p->digit_bits = div_up(p->tbits, p->passes);
  p->capacity = capacity;
  p->count_blocks = div_up64(n_gauss > 0 ? n_gauss : 1, kCountThreads);
  p->parts = div_up64(capacity > 0 ? capacity : 1, kSortTile);
  // zeroed at the start of every call: [hdr, hist, diff]
  size_t o = 0;
  p->off_hdr = o;        o = align256(o + sizeof(Hdr));
  p->off_hist = o;       o = align256(o + sizeof(uint32_t) * kMaxPasses * 256);
  p->off_diff = o;       o = align256(o + sizeof(int) * (size_t)(p->tiles_x + 1) * (size_t)(p->tiles_y + 1));
  p->zero_bytes = o;
  // per-partition digit counts of one pass, then its output offsets (in place)
  p->off_parts = o;      o = align256(o + sizeof(uint32_t) * (size_t)p->parts * 256);
  p->off_local = o;      o = align256(o + sizeof(uint32_t) * (size_t)(n_gauss > 0 ? n_gauss : 1));
  p->off_partial = o;    o = align256(o + sizeof(unsigned long long) * (size_t)(p->count_blocks + 1));
  p->off_rects = o;      o = align256(o + sizeof(uint2) * (size_t)(n_gauss > 0 ? n_gauss : 1));
  p->off_owner = o;      o = align256(o + sizeof(uint32_t) * (size_t)(div_up64(capacity, kEmitTile) + 1));
  p->off_keys_tmp = o;
  o = align256(o + (p->wide ? 2 * sizeof(unsigned long long) : sizeof(uint32_t)) * (size_t)(capacity > 0 ? capacity : 1));
  // the two-level counting sort (32-bit keys, up to 512 tile rows and 512
  // tile columns); its row lists use keys_tmp
  p->n_g1 = (int)div_up64(n_gauss > 0 ? n_gauss : 1, kRowChunk);
  p->rows = allow_rows && !p->wide && p->tiles_y <= kRowsMax && p->tiles_x <= kColsMax &&
            (int64_t)p->tiles_y * p->n_g1 <= (int64_t(1) << 24);
  p->n_ch_max = div_up64(capacity > 0 ? capacity : 1, kColChunk) + p->tiles_y;
  p->off_t1 = p->off_rowcnt = p->off_rowstart = p->off_chstart = p->off_t2 = p->off_chrow = 0;
  if (p->rows) {
    p->off_t1 = o;       o = align256(o + sizeof(uint32_t) * (size_t)p->tiles_y * (size_t)p->n_g1);
    p->off_rowcnt = o;   o = align256(o + sizeof(uint32_t) * (size_t)(p->tiles_y + 1));
    p->off_rowstart = o; o = align256(o + sizeof(uint32_t) * (size_t)(p->tiles_y + 1));
    p->off_chstart = o;  o = align256(o + sizeof(uint32_t) * (size_t)(p->tiles_y + 1));
    p->off_t2 = o;       o = align256(o + sizeof(uint32_t) * (size_t)p->n_ch_max * (size_t)p->tiles_x);
    p->off_chrow = o;    o = align256(o + sizeof(uint32_t) * (size_t)p->n_ch_max);
  }
  p->bytes = o;
  return BS_OK;
}

// sync: read the pair count back (one stream synchronisation) and size the
// sort's grids by it; otherwise size them by the capacity and let the
// kernels read the count to sort from the workspace header (no host
// dependency, so the binning can be captured in a CUDA graph).
bs_status run_binning(const BinPlan &p, const float *gauss, const bs_canvas &cv, void *ws, int64_t *n_pairs,
                      uint32_t *tile_keys, uint32_t *tile_ranges, cudaStream_t s, bool sync,
                      int64_t *n_pairs_dev) {
  char *base = static_cast<char *>(ws);
  Hdr *hdr = reinterpret_cast<Hdr *>(base + p.off_hdr);
  uint32_t *local = reinterpret_cast<uint32_t *>(base + p.off_local);
  auto *partial = reinterpret_cast<unsigned long long *>(base + p.off_partial);
  uint2 *rects = reinterpret_cast<uint2 *>(base + p.off_rects);
  uint32_t *owner = reinterpret_cast<uint32_t *>(base + p.off_owner);
  int *diff = reinterpret_cast<int *>(base + p.off_diff);
  uint32_t *keys_tmp = reinterpret_cast<uint32_t *>(base + p.off_keys_tmp);
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + p.off_hist);
  uint32_t *part_offs = reinterpret_cast<uint32_t *>(base + p.off_parts);
  uint2 *ranges = reinterpret_cast<uint2 *>(tile_ranges);
  const int rows = p.tiles_y + 1, cols = p.tiles_x + 1;
  const unsigned long long *count = &hdr->n_sorted;

  {
    const size_t nz = p.zero_bytes / sizeof(uint32_t);
    const int blocks = (int)std::min<int64_t>(div_up64((int64_t)nz, 256), 152 * 8);
    zero_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<uint32_t *>(base), nz);
    BS_LAUNCHED("zero_kernel");
  }
  if (p.n_gauss > 0) {
    count_kernel<<<(unsigned)p.count_blocks, kCountThreads, 0, s>>>(gauss, p.n_gauss, cv.width, cv.height,
                                                                    cv.tile, p.tiles_x, local, partial, rects, diff);
    BS_LAUNCHED("count_kernel");
    scan_partials_kernel<<<1, 1024, 0, s>>>(partial, p.count_blocks, &hdr->n_pairs, hdr, p.capacity);
    BS_LAUNCHED("scan_partials_kernel");
    if (!p.rows) {
      chunk_owner_kernel<uint2><<<(unsigned)p.count_blocks, kCountThreads, 0, s>>>(
          local, partial, rects, p.n_gauss, (uint32_t)div_up64(p.capacity, kEmitTile), owner);
      BS_LAUNCHED("chunk_owner_kernel");
    }
  }
  if (fused_words(p.tiles_x, p.tiles_y) <= kFusedMaxWords && p.passes <= 2) {
    const size_t smem = sizeof(int) * (size_t)fused_words(p.tiles_x, p.tiles_y);
    static bool attr_set[64] = {};  // per device, under attr_mu
    static std::mutex attr_mu;
    int dev = 0;
    BS_CUDA(cudaGetDevice(&dev));
    {
      std::lock_guard<std::mutex> lock(attr_mu);
      if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        BS_CUDA(cudaFuncSetAttribute(fused_tile_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(int) * kFusedMaxWords)));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
      }
    }
    fused_tile_scan_kernel<<<1, 1024, smem, s>>>(diff, p.tiles_x, p.tiles_y, p.passes, p.digit_bits, hdr, ranges,
                                                 hist);
    BS_LAUNCHED("fused_tile_scan_kernel");
  } else {
    diff_rows_kernel<<<div_up(rows, 8), 256, 0, s>>>(diff, rows, cols);
    BS_LAUNCHED("diff_rows_kernel");
    diff_cols_kernel<<<div_up(cols, 8), 256, 0, s>>>(diff, rows, cols);
    BS_LAUNCHED("diff_cols_kernel");
    tile_scan_kernel<<<1, 1024, 0, s>>>(diff, p.tiles_x, p.tiles_y, p.passes, p.digit_bits, hdr, ranges, hist);
    BS_LAUNCHED("tile_scan_kernel");
  }
  if (n_pairs_dev) {
    BS_CUDA(cudaMemcpyAsync(n_pairs_dev, &hdr->n_pairs, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  }
  // the number of keys the grids below cover: P (read back) or the capacity
  int64_t P;
  if (sync) {
    Hdr h;
    BS_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, s));
    BS_CUDA(cudaStreamSynchronize(s));
    *n_pairs = (int64_t)h.n_pairs;
    if ((int64_t)h.n_pairs > p.capacity) {
      set_error("%lld pairs exceed pair_capacity %lld", (long long)h.n_pairs, (long long)p.capacity);
      return BS_ERR_CAPACITY;
    }
    P = (int64_t)h.n_pairs;
  } else {
    P = p.capacity;
  }
  if (P == 0 || p.n_gauss == 0) return BS_OK;
  if (p.rows) {
    const int H = p.tiles_y, W = p.tiles_x;
    uint32_t *t1 = reinterpret_cast<uint32_t *>(base + p.off_t1);
    uint32_t *rowcnt = reinterpret_cast<uint32_t *>(base + p.off_rowcnt);
    uint32_t *rowstart = reinterpret_cast<uint32_t *>(base + p.off_rowstart);
    uint32_t *chstart = reinterpret_cast<uint32_t *>(base + p.off_chstart);
    uint32_t *t2 = reinterpret_cast<uint32_t *>(base + p.off_t2);
    uint32_t *chrow = reinterpret_cast<uint32_t *>(base + p.off_chrow);
    uint32_t *rowlist = keys_tmp;
    const uint32_t cap = (uint32_t)p.capacity;
    row_count_kernel<<<(unsigned)p.n_g1, kRowChunk, sizeof(uint32_t) * 8 * H, s>>>(rects, p.n_gauss, H, p.n_g1,
                                                                                   count, t1);
    BS_LAUNCHED("row_count_kernel");
    row_scan_kernel<<<(unsigned)H, 1024, 0, s>>>(t1, p.n_g1, count, rowcnt);
    BS_LAUNCHED("row_scan_kernel");
    row_starts_kernel<<<1, 1024, 0, s>>>(rowcnt, H, count, rowstart, chstart, chrow, (uint32_t)p.n_ch_max);
    BS_LAUNCHED("row_starts_kernel");
    row_scatter_kernel<<<(unsigned)p.n_g1, kRowChunk, sizeof(uint32_t) * 17 * (size_t)H, s>>>(
        rects, p.n_gauss, H, p.n_g1, count, t1, rowstart, rowlist, cap);
    BS_LAUNCHED("row_scatter_kernel");
    // the row lists hold at most P entries, so at most P / 256 + H chunks;
    // the level-2 kernels loop over the chunks there are
    const int64_t n_ch = std::min<int64_t>(std::min(p.n_ch_max, div_up64(P, kColChunk) + H), kColGrid);
    col_count_kernel<<<(unsigned)n_ch, kColChunk, sizeof(int) * ((size_t)W + 1), s>>>(rects, rowlist, rowcnt, rowstart,
                                                                                 chstart, chrow, H, W, count, t2);
    BS_LAUNCHED("col_count_kernel");
    col_scan_kernel<<<(unsigned)H, 1024, 0, s>>>(t2, chstart, W, count);
    BS_LAUNCHED("col_scan_kernel");
    col_scatter_kernel<<<(unsigned)n_ch, kColChunk, sizeof(uint32_t) * (2 * kColWords + 1) * (size_t)W, s>>>(
        rects, rowlist, rowcnt, rowstart, chstart, chrow, H, W, count, t2, ranges, p.gbits, tile_keys, cap);
    BS_LAUNCHED("col_scatter_kernel");
    return BS_OK;
  }
  const int64_t parts = div_up64(P, kSortTile);
  const int bits0 = std::min(p.digit_bits, p.tbits);
  BS_CUDA(cudaMemsetAsync(part_offs, 0, sizeof(uint32_t) * ((size_t)1 << bits0) * (size_t)parts, s));
  if (p.wide) {
    // 64-bit keys in the workspace; the last pass writes g alone to tile_keys
    auto *k64 = reinterpret_cast<unsigned long long *>(base + p.off_keys_tmp);
    unsigned long long *kb[2] = {k64, k64 + p.capacity};
    emit_kernel<unsigned long long><<<(unsigned)div_up64(P, kEmitTile), kEmitThreads, 0, s>>>(
        local, partial, p.count_blocks, rects, p.n_gauss, count, p.tiles_x, p.gbits, owner, kb[0], bits0,
        part_offs, (uint32_t)parts);
    BS_LAUNCHED("emit_kernel");
    int cur = 0;
    for (int pass = 0; pass < p.passes; ++pass) {
      const int shift = 32 + pass * p.digit_bits;
      const int bits = std::min(p.digit_bits, p.tbits - pass * p.digit_bits);
      if (pass > 0) {
        upsweep_kernel<unsigned long long><<<(unsigned)parts, kSortThreads, 0, s>>>(kb[cur], count, shift, bits,
                                                                                   part_offs, (uint32_t)parts);
        BS_LAUNCHED("upsweep_kernel");
      }
      scan_parts_kernel<<<1u << bits, kScanThreads, 0, s>>>(part_offs, (uint32_t)parts, hist + pass * 256);
      BS_LAUNCHED("scan_parts_kernel");
      if (pass + 1 < p.passes) {
        downsweep_kernel<unsigned long long, unsigned long long><<<(unsigned)parts, kSortThreads, 0, s>>>(
            kb[cur], kb[1 - cur], count, shift, bits, part_offs, (uint32_t)parts);
        cur = 1 - cur;
      } else {
        downsweep_kernel<unsigned long long, uint32_t><<<(unsigned)parts, kSortThreads, 0, s>>>(
            kb[cur], tile_keys, count, shift, bits, part_offs, (uint32_t)parts);
      }
      BS_LAUNCHED("downsweep_kernel");
    }
    return BS_OK;
  }
  // emit into the buffer that makes the last pass land in tile_keys
  uint32_t *bufs[2] = {tile_keys, keys_tmp};
  uint32_t *src = (p.passes % 2 == 0) ? tile_keys : keys_tmp;
  emit_kernel<uint32_t><<<(unsigned)div_up64(P, kEmitTile), kEmitThreads, 0, s>>>(local, partial, p.count_blocks, rects,
                                                                                 p.n_gauss, count, p.tiles_x,
                                                                                 p.gbits, owner, src, bits0, part_offs,
                                                                                 (uint32_t)parts);
  BS_LAUNCHED("emit_kernel");
  for (int pass = 0; pass < p.passes; ++pass) {
    uint32_t *dst = (src == bufs[0]) ? bufs[1] : bufs[0];
    const int shift = p.gbits + pass * p.digit_bits;
    const int bits = std::min(p.digit_bits, p.tbits - pass * p.digit_bits);
    if (pass > 0) {  // the first pass's counts come from emit_kernel
      upsweep_kernel<uint32_t><<<(unsigned)parts, kSortThreads, 0, s>>>(src, count, shift, bits, part_offs,
                                                                        (uint32_t)parts);
      BS_LAUNCHED("upsweep_kernel");
    }
    scan_parts_kernel<<<1u << bits, kScanThreads, 0, s>>>(part_offs, (uint32_t)parts, hist + pass * 256);
    BS_LAUNCHED("scan_parts_kernel");
    downsweep_kernel<uint32_t, uint32_t><<<(unsigned)parts, kSortThreads, 0, s>>>(src, dst, count, shift,
                                                                                   bits, part_offs, (uint32_t)parts);
    BS_LAUNCHED("downsweep_kernel");
    src = dst;
  }
  return BS_OK;
}

bs_status run_batch_binning(const BatchPlan &p, void *ws, const float *gauss, uint32_t *tile_vals,
                            uint32_t *tile_ranges, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  BatchHdr *hdr = reinterpret_cast<BatchHdr *>(base + p.off_hdr);
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + p.off_hist);
  int *diff = reinterpret_cast<int *>(base + p.off_diff);
  const BatchImage *tab = reinterpret_cast<const BatchImage *>(base + p.off_images);
  uint32_t *part_offs = reinterpret_cast<uint32_t *>(base + p.off_parts);
  uint32_t *local = reinterpret_cast<uint32_t *>(base + p.off_local);
  auto *partial = reinterpret_cast<unsigned long long *>(base + p.off_partial);
  uint4 *rects = reinterpret_cast<uint4 *>(base + p.off_rects);
  uint32_t *owner = reinterpret_cast<uint32_t *>(base + p.off_owner);
  auto *tsum = reinterpret_cast<unsigned long long *>(base + p.off_tsum);
  auto *keys0 = reinterpret_cast<unsigned long long *>(base + p.off_keys0);
  auto *keys1 = reinterpret_cast<unsigned long long *>(base + p.off_keys1);
  uint2 *ranges = reinterpret_cast<uint2 *>(tile_ranges);
  {
    const size_t nz = p.zero_bytes / sizeof(uint32_t);
    const int blocks = (int)std::min<int64_t>(div_up64((int64_t)nz, 256), 152 * 8);
    zero_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<uint32_t *>(base), nz);
    BS_LAUNCHED("zero_kernel");
  }
  if (p.n_gauss > 0) {
    batch_count_kernel<<<(unsigned)p.count_blocks, kCountThreads, 0, s>>>(gauss, p.n_gauss, tab, p.n_images,
                                                                          p.tile, local, partial, rects, diff);
    BS_LAUNCHED("batch_count_kernel");
    scan_partials_kernel<<<1, 1024, 0, s>>>(partial, p.count_blocks, &hdr->n_pairs, nullptr, 0);
    BS_LAUNCHED("scan_partials_kernel");
    chunk_owner_kernel<uint4><<<(unsigned)p.count_blocks, kCountThreads, 0, s>>>(
        local, partial, rects, p.n_gauss, (uint32_t)div_up64(p.capacity, kEmitTile), owner);
    BS_LAUNCHED("chunk_owner_kernel");
  }
  batch_diff_rows_kernel<<<(unsigned)div_up64(p.diff_rows, 8), 256, 0, s>>>(diff, tab, p.n_images, p.diff_rows);
  BS_LAUNCHED("batch_diff_rows_kernel");
  batch_diff_cols_kernel<<<(unsigned)div_up64(p.diff_cols, 8), 256, 0, s>>>(diff, tab, p.n_images, p.diff_cols);
  BS_LAUNCHED("batch_diff_cols_kernel");
  batch_tile_reduce_kernel<<<(unsigned)p.tile_blocks, kTileThreads, 0, s>>>(diff, tab, p.n_images, p.n_tiles,
                                                                            p.passes, p.digit_bits, tsum, hist);
  BS_LAUNCHED("batch_tile_reduce_kernel");
  scan_partials_kernel<<<1, 1024, 0, s>>>(tsum, p.tile_blocks, &hdr->tile_total, nullptr, 0);
  BS_LAUNCHED("scan_partials_kernel");
  batch_digits_kernel<<<1, 32 * kMaxPasses, 0, s>>>(hdr, p.capacity, p.passes, hist);
  BS_LAUNCHED("batch_digits_kernel");
  batch_tile_ranges_kernel<<<(unsigned)p.tile_blocks, kTileThreads, 0, s>>>(diff, tab, p.n_images, p.n_tiles, tsum,
                                                                            hdr, ranges);
  BS_LAUNCHED("batch_tile_ranges_kernel");
  // emit and sort, sized by the capacity: kernels past the pair count return
  const int bits0 = std::min(p.digit_bits, p.tbits);
  BS_CUDA(cudaMemsetAsync(part_offs, 0, sizeof(uint32_t) * ((size_t)1 << bits0) * (size_t)p.parts, s));
  batch_emit_kernel<<<(unsigned)div_up64(p.capacity, kEmitTile), kEmitThreads, 0, s>>>(
      local, partial, p.count_blocks, rects, p.n_gauss, &hdr->n_sorted, owner, keys0, bits0, part_offs,
      (uint32_t)p.parts);
  BS_LAUNCHED("batch_emit_kernel");
  unsigned long long *src = keys0;
  for (int pass = 0; pass < p.passes; ++pass) {
    const int shift = 32 + pass * p.digit_bits;
    const int bits = std::min(p.digit_bits, p.tbits - pass * p.digit_bits);
    if (pass > 0) {
      upsweep_kernel<unsigned long long><<<(unsigned)p.parts, kSortThreads, 0, s>>>(src, &hdr->n_sorted, shift, bits,
                                                                                   part_offs, (uint32_t)p.parts);
      BS_LAUNCHED("upsweep_kernel");
    }
    scan_parts_kernel<<<1u << bits, kScanThreads, 0, s>>>(part_offs, (uint32_t)p.parts, hist + pass * 256);
    BS_LAUNCHED("scan_parts_kernel");
    if (pass + 1 < p.passes) {
      unsigned long long *dst = src == keys0 ? keys1 : keys0;
      downsweep_kernel<unsigned long long, unsigned long long><<<(unsigned)p.parts, kSortThreads, 0, s>>>(
          src, dst, &hdr->n_sorted, shift, bits, part_offs, (uint32_t)p.parts);
      src = dst;
    } else {
      downsweep_kernel<unsigned long long, uint32_t><<<(unsigned)p.parts, kSortThreads, 0, s>>>(
          src, tile_vals, &hdr->n_sorted, shift, bits, part_offs, (uint32_t)p.parts);
    }
    BS_LAUNCHED("downsweep_kernel");
  }
  return BS_OK;
}

bs_status read_batch_status(const BatchPlan &p, const void *ws, int32_t *status, int64_t *n_pairs, cudaStream_t s) {
  BatchHdr h;
  BS_CUDA(cudaMemcpyAsync(&h, static_cast<const char *>(ws) + p.off_hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  *status = (h.status & kDevErrCapacity) ? BS_ERR_CAPACITY : BS_OK;
  if (h.status & kDevErrCounts) {
    set_error("batch binning: %llu pairs from the Gaussians but %llu from the tiles; nothing was sorted",
              h.n_pairs, h.tile_total);
    *status = BS_ERR_UNSUPPORTED;
  }
  if (n_pairs) *n_pairs = (int64_t)h.n_pairs;
  return BS_OK;
}

// ---- binning without caller-provided scratch ----
// The scratch lives in one file-scope device array of kStaticScratchBytes,
// which every GPU that loads the library holds until the process exits.
// Host code may not pass the array's name to a kernel (on the host it only
// names a stand-in); its device address is looked up once per device, with
// that device current, under a per-device once flag (so concurrent first
// calls from several host threads are safe), and kept.  A device reset
// (cudaDeviceReset) unloads the module and makes that address stale.
namespace {
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void *g_static_scratch_ptr[kMaxDevices] = {};
cudaError_t g_static_scratch_err[kMaxDevices] = {};
std::once_flag g_static_scratch_once[kMaxDevices];
}  // namespace

bs_status static_scratch(void **ptr) {
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d: at most %d devices supported", dev, kMaxDevices);
    return BS_ERR_UNSUPPORTED;
  }
  std::call_once(g_static_scratch_once[dev], [dev] {
    void *p = nullptr;
    g_static_scratch_err[dev] = cudaGetSymbolAddress(&p, g_static_scratch);
    g_static_scratch_ptr[dev] = p;
  });
  BS_CUDA(g_static_scratch_err[dev]);
  *ptr = g_static_scratch_ptr[dev];
  return BS_OK;
}

bs_status read_device_status(const void *ws, size_t ws_bytes, int32_t *out, cudaStream_t s, int64_t *n_pairs) {
  if (ws_bytes < sizeof(Hdr)) {
    set_error("workspace too small");
    return BS_ERR_INVALID_ARG;
  }
  Hdr h;
  BS_CUDA(cudaMemcpyAsync(&h, ws, sizeof(Hdr), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  *out = (h.status & kDevErrTimeout) ? BS_ERR_TIMEOUT : (h.status ? BS_ERR_CAPACITY : BS_OK);
  if (n_pairs) *n_pairs = (int64_t)h.n_pairs;
  return BS_OK;
}

}  // namespace bs
