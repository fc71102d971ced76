// Tile binning (Section 3.4): per-Gaussian tile rectangles, (tile, depth)
// keys, a hand-written stable onesweep LSD radix sort of the tile bits, and
// per-tile ranges.
//
// The keys are emitted Gaussian by Gaussian, so the emitted array is already
// ordered by the Gaussian index (the depth, since the table is in draw
// order).  A stable sort on the tile bits alone therefore orders the keys by
// (tile, depth): ceil(tile_bits / 8) passes instead of one per key byte.
//
// Sort pass (one launch per digit): every CTA takes the next partition of
// 4096 keys from an atomic counter (so a partition's predecessors are always
// resident), ranks its keys stably with warp match_any, publishes its digit
// counts, and resolves its global offsets by decoupled look-back over the
// partitions before it.  Every look-back wait is bounded; when a bound runs
// out the CTA records kDevErrTimeout in the workspace status word and goes on.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kCountThreads = 256;   // Gaussians per count/emit CTA
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per partition
constexpr int kMaxPasses = 4;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int64_t kMaxPairs = (1ll << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

struct Hdr {
  uint32_t status;
  uint32_t pad;
  unsigned long long n_pairs;
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

// ---- count + block-local exclusive scan ----
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Per Gaussian: its pair count, its block-local exclusive offset, and its
// rectangle packed as {tx0 | ty0 << 16, width | height << 16}.
__global__ void __launch_bounds__(kCountThreads) count_kernel(const float *gauss, int64_t n_gauss, int W, int H,
                                                              int tile, uint32_t *local,
                                                              unsigned long long *partial, uint2 *rects) {
  __shared__ uint32_t s_warp[kCountThreads / 32];
  const int64_t g = (int64_t)blockIdx.x * kCountThreads + threadIdx.x;
  uint32_t cnt = 0;
  Rect r;
  if (g < n_gauss) {
    uint2 packed = make_uint2(0u, 0u);
    if (tile_rect(gauss, g, W, H, tile, &r)) {
      const uint32_t w = (uint32_t)(r.tx1 - r.tx0 + 1), h = (uint32_t)(r.ty1 - r.ty0 + 1);
      cnt = w * h;
      packed = make_uint2((uint32_t)r.tx0 | ((uint32_t)r.ty0 << 16), w | (h << 16));
    }
    rects[g] = packed;
  }
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

// Exclusive scan of the per-CTA totals (one CTA); writes the pair count.
__global__ void __launch_bounds__(1024) scan_partials_kernel(unsigned long long *partial, int64_t n, Hdr *hdr) {
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
    hdr->n_pairs = carry;
    partial[n] = carry;  // sentinel for the owner search
  }
}

// ---- zero the per-call sort state and the tile ranges ----
__global__ void zero_kernel(uint32_t *a, size_t na, uint32_t *b, size_t nb) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
    if (i < na) a[i] = 0u;
    else b[i - na] = 0u;
  }
}

// ---- emit keys, one per thread, + digit histograms ----
// The owner of pair i is found by two binary searches (CTA offsets, then
// offsets inside the CTA), so every thread writes one key whatever the size
// of the rectangles: a Gaussian covering thousands of tiles is spread over
// many warps instead of serialising one.
__device__ __forceinline__ uint32_t pair_owner(const unsigned long long *__restrict__ partial, int64_t nb,
                                               const uint32_t *__restrict__ local, int64_t n_gauss, uint32_t i,
                                               uint32_t *l_out) {
  int64_t lo = 0, hi = nb;  // first block whose offset exceeds i
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
  const int64_t g = lo - 1;
  *l_out = i2 - local[g];
  return (uint32_t)g;
}

__global__ void __launch_bounds__(kCountThreads) emit_kernel(const uint32_t *__restrict__ local,
                                                             const unsigned long long *__restrict__ partial,
                                                             int64_t nb, const uint2 *__restrict__ rects,
                                                             int64_t n_gauss, const Hdr *hdr, int tiles_x, int gbits,
                                                             uint32_t *__restrict__ keys, int passes,
                                                             int digit_bits, uint32_t *hist) {
  __shared__ uint32_t s_hist[kMaxPasses * 256];
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) s_hist[i] = 0u;
  __syncthreads();
  const uint32_t n = (uint32_t)hdr->n_pairs;
  const int lane = threadIdx.x & 31;
  const uint32_t dmask = (1u << digit_bits) - 1;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    const bool valid = i < n;
    uint32_t tid = 0;
    if (valid) {
      uint32_t l;
      const uint32_t g = pair_owner(partial, nb, local, n_gauss, i, &l);
      const uint2 rc = rects[g];
      const uint32_t w = rc.y & 0xffffu;
      const uint32_t ry = l / w, rx = l - ry * w;
      tid = ((rc.x >> 16) + ry) * (uint32_t)tiles_x + (rc.x & 0xffffu) + rx;
      keys[i] = (tid << gbits) | g;
    }
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    for (int p = 0; p < passes; ++p) {
      const uint32_t d = (tid >> (p * digit_bits)) & dmask;
      const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu) & active;
      if (valid && (peers & ((1u << lane) - 1)) == 0) atomicAdd(&s_hist[p * 256 + d], __popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

// ---- one onesweep pass ----
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(const uint32_t *__restrict__ in,
                                                                uint32_t *__restrict__ out, const Hdr *hdr_in,
                                                                Hdr *hdr, int shift, int bits,
                                                                const uint32_t *ghist, uint32_t *lookback,
                                                                uint32_t *counter, uint32_t spin_limit,
                                                                int never_publish_part) {
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_whist[kSortWarps][256];
  __shared__ uint32_t s_bexcl[256];
  __shared__ uint32_t s_gstart[256];
  __shared__ uint32_t s_scan[256];
  __shared__ uint32_t s_part;
  const uint32_t n = (uint32_t)hdr_in->n_pairs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nbins = 1u << bits, dmask = nbins - 1;
  if (tid == 0) s_part = atomicAdd(counter, 1u);
  for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
  // global exclusive prefix of this pass's digit histogram
  s_scan[tid] = tid < (int)nbins ? ghist[tid] : 0u;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const uint32_t t = tid >= o ? s_scan[tid - o] : 0u;
    __syncthreads();
    s_scan[tid] += t;
    __syncthreads();
  }
  const uint32_t gexcl = s_scan[tid] - (tid < (int)nbins ? ghist[tid] : 0u);
  const uint32_t part = s_part;
  const uint32_t base = part * (uint32_t)kSortTile + (uint32_t)warp * (32u * kSortItems);
  const unsigned lt_mask = (1u << lane) - 1;

  uint32_t keys[kSortItems], rank[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + (uint32_t)i * 32u + (uint32_t)lane;
    keys[i] = idx < n ? in[idx] : 0u;
  }
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + (uint32_t)i * 32u + (uint32_t)lane;
    const bool valid = idx < n;
    const uint32_t d = (keys[i] >> shift) & dmask;
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu);
    const uint32_t cnt = valid ? s_whist[warp][d] : 0u;
    rank[i] = cnt + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_whist[warp][d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // per digit: exclusive offsets across warps, publish, look back
  uint32_t bcount = 0;
  if (tid < (int)nbins) {
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = bcount;
      bcount += c;
    }
    uint32_t *mine = lookback + (size_t)part * 256 + tid;
    const bool publish = (int)part != never_publish_part;
    if (part == 0) {
      if (publish) st_relaxed(mine, kFlagIncl | bcount);
      s_gstart[tid] = gexcl;
    } else {
      if (publish) st_relaxed(mine, kFlagAgg | bcount);
      uint32_t excl = 0;
      int64_t j = (int64_t)part - 1;
      uint32_t spins = 0;
      while (j >= 0) {
        const uint32_t v = ld_relaxed(lookback + (size_t)j * 256 + tid);
        const uint32_t flag = v & ~kCountMask;
        if (flag == 0u) {
          if (++spins > spin_limit) {
            atomicOr(&hdr->status, kDevErrTimeout);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += v & kCountMask;
        if (flag == kFlagIncl) break;
        --j;
      }
      if (publish) st_relaxed(mine, kFlagIncl | ((excl + bcount) & kCountMask));
      s_gstart[tid] = gexcl + excl;
    }
  }
  // block exclusive prefix over digits
  s_scan[tid] = bcount;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const uint32_t t = tid >= o ? s_scan[tid - o] : 0u;
    __syncthreads();
    s_scan[tid] += t;
    __syncthreads();
  }
  s_bexcl[tid] = s_scan[tid] - bcount;
  __syncthreads();
  // scatter into shared memory in (digit, input order) order
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + (uint32_t)i * 32u + (uint32_t)lane;
    if (idx < n) {
      const uint32_t d = (keys[i] >> shift) & dmask;
      s_keys[s_bexcl[d] + s_whist[warp][d] + rank[i]] = keys[i];
    }
  }
  __syncthreads();
  const uint32_t pstart = part * (uint32_t)kSortTile;
  const uint32_t n_here = n > pstart ? min((uint32_t)kSortTile, n - pstart) : 0u;
  for (uint32_t j = tid; j < n_here; j += kSortThreads) {
    const uint32_t k = s_keys[j];
    const uint32_t d = (k >> shift) & dmask;
    out[s_gstart[d] + (j - s_bexcl[d])] = k;
  }
}

__global__ void ranges_kernel(const uint32_t *keys, const Hdr *hdr, int gbits, uint32_t n_tiles, uint2 *ranges) {
  const uint32_t n = (uint32_t)hdr->n_pairs;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t t = keys[i] >> gbits;
    if (t >= n_tiles) continue;  // only after a sort that gave up waiting
    if (i == 0 || (keys[i - 1] >> gbits) != t) ranges[t].x = i;
    if (i + 1 == n || (keys[i + 1] >> gbits) != t) ranges[t].y = i + 1;
  }
}

int g_debug_never_publish = -1;     // test hook: a partition that never publishes
uint32_t g_spin_limit = kSpinLimit;

}  // namespace

bs_status plan_binning(int64_t n_gauss, const bs_canvas &cv, int64_t capacity, BinPlan *p) {
  if (n_gauss < 0 || n_gauss > (1ll << 31) - 1) {
    set_error("n_gauss %lld out of range", (long long)n_gauss);
    return BS_ERR_INVALID_ARG;
  }
  if (cv.width < 1 || cv.height < 1 || cv.width > 32768 || cv.height > 32768) {
    set_error("canvas %dx%d out of range", cv.width, cv.height);
    return BS_ERR_INVALID_ARG;
  }
  if (cv.tile != 16) {
    set_error("tile side %d not supported (16)", cv.tile);
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
  if (p->gbits + p->tbits > 32) {
    set_error("keys need %d tile + %d Gaussian bits > 32", p->tbits, p->gbits);
    return BS_ERR_UNSUPPORTED;
  }
  p->passes = div_up(p->tbits, 8);
  p->digit_bits = div_up(p->tbits, p->passes);
  p->capacity = capacity;
  p->count_blocks = div_up64(n_gauss > 0 ? n_gauss : 1, kCountThreads);
  p->parts = div_up64(capacity > 0 ? capacity : 1, kSortTile);
  size_t o = 0;
  p->off_hdr = o;        o = align256(o + sizeof(Hdr));
  p->off_local = o;      o = align256(o + sizeof(uint32_t) * (size_t)(n_gauss > 0 ? n_gauss : 1));
  p->off_partial = o;    o = align256(o + sizeof(unsigned long long) * (size_t)(p->count_blocks + 1));
  p->off_rects = o;      o = align256(o + sizeof(uint2) * (size_t)(n_gauss > 0 ? n_gauss : 1));
  p->off_keys_tmp = o;   o = align256(o + sizeof(uint32_t) * (size_t)(capacity > 0 ? capacity : 1));
  p->off_hist = o;       o = align256(o + sizeof(uint32_t) * kMaxPasses * 256);
  p->off_counter = o;    o = align256(o + sizeof(uint32_t) * kMaxPasses);
  p->off_lookback = o;   o = align256(o + sizeof(uint32_t) * (size_t)p->passes * (size_t)p->parts * 256);
  p->bytes = o;
  return BS_OK;
}

bs_status run_binning(const BinPlan &p, const float *gauss, const bs_canvas &cv, void *ws, int64_t *n_pairs,
                      uint32_t *tile_keys, uint32_t *tile_ranges, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  Hdr *hdr = reinterpret_cast<Hdr *>(base + p.off_hdr);
  uint32_t *local = reinterpret_cast<uint32_t *>(base + p.off_local);
  auto *partial = reinterpret_cast<unsigned long long *>(base + p.off_partial);
  uint2 *rects = reinterpret_cast<uint2 *>(base + p.off_rects);
  uint32_t *keys_tmp = reinterpret_cast<uint32_t *>(base + p.off_keys_tmp);
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + p.off_hist);
  uint32_t *counter = reinterpret_cast<uint32_t *>(base + p.off_counter);
  uint32_t *lookback = reinterpret_cast<uint32_t *>(base + p.off_lookback);

  BS_CUDA(cudaMemsetAsync(hdr, 0, sizeof(Hdr), s));
  if (p.n_gauss > 0) {
    count_kernel<<<(unsigned)p.count_blocks, kCountThreads, 0, s>>>(gauss, p.n_gauss, cv.width, cv.height,
                                                                    cv.tile, local, partial, rects);
    BS_LAUNCHED("count_kernel");
    scan_partials_kernel<<<1, 1024, 0, s>>>(partial, p.count_blocks, hdr);
    BS_LAUNCHED("scan_partials_kernel");
  }
  Hdr h;
  BS_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  *n_pairs = (int64_t)h.n_pairs;
  if ((int64_t)h.n_pairs > p.capacity) {
    set_error("%lld pairs exceed pair_capacity %lld", (long long)h.n_pairs, (long long)p.capacity);
    return BS_ERR_CAPACITY;
  }
  const int64_t P = (int64_t)h.n_pairs;
  const int64_t parts = div_up64(P, kSortTile);
  // zero the sort state for the partitions in use, and the tile ranges
  {
    const size_t na = (size_t)(p.off_lookback - p.off_hist) / sizeof(uint32_t) +
                      (size_t)p.passes * (size_t)parts * 256;  // hist, counter, (pad), lookback
    const size_t nb = (size_t)p.n_tiles * 2;
    const int blocks = (int)std::min<size_t>(div_up64((int64_t)(na + nb), 256), 152 * 8);
    zero_kernel<<<blocks, 256, 0, s>>>(hist, na, tile_ranges, nb);
    BS_LAUNCHED("zero_kernel");
  }
  if (P == 0) return BS_OK;
  // emit into the buffer that makes the last pass land in tile_keys
  uint32_t *bufs[2] = {tile_keys, keys_tmp};
  uint32_t *src = (p.passes % 2 == 0) ? tile_keys : keys_tmp;
  {
    const int blocks = (int)std::min<int64_t>(div_up64(P, kCountThreads), 152 * 16);
    emit_kernel<<<blocks, kCountThreads, 0, s>>>(local, partial, p.count_blocks, rects, p.n_gauss, hdr, p.tiles_x,
                                                 p.gbits, src, p.passes, p.digit_bits, hist);
  }
  BS_LAUNCHED("emit_kernel");
  for (int pass = 0; pass < p.passes; ++pass) {
    uint32_t *dst = (src == bufs[0]) ? bufs[1] : bufs[0];
    const int shift = p.gbits + pass * p.digit_bits;
    const int bits = std::min(p.digit_bits, p.tbits - pass * p.digit_bits);
    onesweep_kernel<<<(unsigned)parts, kSortThreads, 0, s>>>(
        src, dst, hdr, hdr, shift, bits, hist + pass * 256, lookback + (size_t)pass * (size_t)parts * 256,
        counter + pass, g_spin_limit, g_debug_never_publish);
    BS_LAUNCHED("onesweep_kernel");
    src = dst;
  }
  {
    const int blocks = (int)std::min<int64_t>(div_up64(P, 256), 152 * 16);
    ranges_kernel<<<blocks, 256, 0, s>>>(tile_keys, hdr, p.gbits, (uint32_t)p.n_tiles,
                                         reinterpret_cast<uint2 *>(tile_ranges));
    BS_LAUNCHED("ranges_kernel");
  }
  return BS_OK;
}

bs_status read_device_status(const void *ws, size_t ws_bytes, int32_t *out, cudaStream_t s) {
  if (ws_bytes < sizeof(Hdr)) {
    set_error("workspace too small");
    return BS_ERR_INVALID_ARG;
  }
  Hdr h;
  BS_CUDA(cudaMemcpyAsync(&h, ws, sizeof(Hdr), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  *out = (h.status & kDevErrTimeout) ? BS_ERR_TIMEOUT : (h.status ? BS_ERR_CAPACITY : BS_OK);
  return BS_OK;
}

void debug_set_sort_fault(int never_publish_part, uint32_t spin_limit) {
  g_debug_never_publish = never_publish_part;
  g_spin_limit = spin_limit ? spin_limit : kSpinLimit;
}

}  // namespace bs
