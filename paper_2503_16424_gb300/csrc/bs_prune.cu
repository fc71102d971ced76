// Adaptive pruning and densification (Section 3.5, Algorithm 1; the split
// rule of Appendix B).
//
// Kernels, in launch order:
//   curve_kernel     per curve: area key, box, colour, low-opacity and
//                    small-area flags
//   overlap_kernel   pairs (i, j) in 256 x 256 blocks: redundant-overlap flag
//   plan_kernel      one CTA: split flags, ordinals of the freed slots, the
//                    target slot of every split and the region index of
//                    every other freed slot
//   runs_kernel      one warp per image row: error mask and, per pixel, the
//                    first pixel of its horizontal run (ballot bit tricks)
//   union_kernel     vertical links between runs: lock-free union-find
//                    whose roots are the smallest pixel index (atomicMin)
//   heads_kernel     run heads point to their root
//   flatten_kernel   every pixel to its root; pixel count per root (warp-
//                    aggregated atomics)
//   roots_kernel     one 64-bit key per region: (count descending, root)
//   select_*         radix select (8 x 8 bits) of the n-th smallest key
//   gather/rank      the selected keys, ranked by counting (keys are unique)
//   sums_kernel      centroid and target colour sums of selected regions
//   apply_kernel     per curve: split halves, circle curves, transparency
// Every retry loop is bounded and reports BS_ERR_TIMEOUT through the header's
// status word.
#include <algorithm>
#include <cstddef>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kThreads = 256;
constexpr int kSegPx = 16;                   // pixels per thread in the run-aggregated passes
constexpr uint32_t kUnionAttempts = 1u << 20;  // default bound of the union step's linking attempts
constexpr uint32_t kSelected = 0x80000000u;  // area[root] holds the region's rank when set
constexpr int kSelectBlocks = 608;           // 152 SMs x 4

constexpr uint32_t kLowOp = 1u, kSmall = 2u, kOverlap = 4u, kSplit = 8u;
constexpr uint32_t kPruned = kLowOp | kSmall | kOverlap;

enum Count {
  kCntPruned, kCntLow, kCntSmall, kCntOverlap, kCntSplit, kCntSplitPlaced,
  kCntFreeOpen, kCntFreeClosed, kNumCounts
};

struct PdHeader {
  uint32_t status;
  uint32_t n_roots;         // connected error regions
  uint32_t n_sel;           // regions placed: min(n_roots, n_slots)
  uint32_t n_gathered;
  unsigned long long kth;   // radix-select prefix; the n_sel-th smallest key when done
  uint32_t rank_left;
  uint32_t n_slots;         // freed slots left for regions after the splits
  uint32_t counts[kNumCounts];
  uint32_t hist[256];
};

struct RegionAcc {
  unsigned long long sx, sy;  // sums of the pixel indices x, y
  double r, g, b;             // sums of the target colour
};

struct Layout {
  size_t hdr, box, colkey, flags, info, free_open, sel, sorted, acc, label, area, roots, bytes;
};

__host__ __device__ inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

Layout layout(int n, int64_t P) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  L.hdr = take(sizeof(PdHeader));
  L.box = take(sizeof(float4) * (size_t)n);
  L.colkey = take(sizeof(float4) * (size_t)n);
  L.flags = take(sizeof(uint32_t) * (size_t)n);
  L.info = take(sizeof(int32_t) * (size_t)n);
  L.free_open = take(sizeof(int32_t) * (size_t)n);
  L.sel = take(sizeof(unsigned long long) * (size_t)n);
  L.sorted = take(sizeof(unsigned long long) * (size_t)n);
  L.acc = take(sizeof(RegionAcc) * (size_t)n);
  L.label = take(sizeof(int32_t) * (size_t)P);
  L.area = take(sizeof(uint32_t) * (size_t)P);
  L.roots = take(sizeof(unsigned long long) * (size_t)(P / 2 + 1));  // at most ceil(P/2) 4-connected regions
  L.bytes = o;
  return L;
}

struct Curves {
  int n_open, n_closed;
  float *open_ctrl, *open_width, *open_color, *open_opac;
  float *closed_ctrl, *closed_color, *closed_opac;
};

// ---- pruning criteria ----

// tau = op_start (1 - f) + op_end f: the opacity threshold at step fraction f.
__global__ void curve_kernel(Curves c, float op_start, float op_end, float frac, float area_min, float4 *box,
                             float4 *colkey, uint32_t *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = c.n_open + c.n_closed;
  if (i >= n) return;
  const float tau = __fadd_rn(__fmul_rn(op_start, __fsub_rn(1.0f, frac)), __fmul_rn(op_end, frac));
  const float key = curve_area_key(c.n_open, c.open_ctrl, c.open_width, c.closed_ctrl, i);
  const bool open = i < c.n_open;
  const float *P = open ? c.open_ctrl + (size_t)i * 20 : c.closed_ctrl + (size_t)(i - c.n_open) * 24;
  const int np = open ? 10 : 12;
  float x0 = P[0], x1 = P[0], y0 = P[1], y1 = P[1];
  for (int j = 1; j < np; ++j) {
    x0 = fminf(x0, P[2 * j]);
    x1 = fmaxf(x1, P[2 * j]);
    y0 = fminf(y0, P[2 * j + 1]);
    y1 = fmaxf(y1, P[2 * j + 1]);
  }
  float op;
  float3 col;
  if (open) {
    const float hw = __fmul_rn(c.open_width[i], 0.5f);
    x0 = __fsub_rn(x0, hw);
    y0 = __fsub_rn(y0, hw);
    x1 = __fadd_rn(x1, hw);
    y1 = __fadd_rn(y1, hw);
    const float *o = c.open_opac + (size_t)i * 3;
    op = __fdiv_rn(__fadd_rn(__fadd_rn(o[0], o[1]), o[2]), 3.0f);
    col = make_float3(c.open_color[3 * i], c.open_color[3 * i + 1], c.open_color[3 * i + 2]);
  } else {
    const int j = i - c.n_open;
    op = c.closed_opac[j];
    col = make_float3(c.closed_color[3 * j], c.closed_color[3 * j + 1], c.closed_color[3 * j + 2]);
  }
  box[i] = make_float4(x0, y0, x1, y1);
  colkey[i] = make_float4(col.x, col.y, col.z, key);
  flags[i] = (op < tau ? kLowOp : 0u) | (key < area_min ? kSmall : 0u);
}

// Curve i is redundant when a curve j drawn in front of it (smaller key,
// equal keys: lower index) has a colour within color_eps and box IoU above
// iou_min.  blockIdx.y picks the 256 candidates j this CTA tests.
__global__ void __launch_bounds__(kThreads) overlap_kernel(int n, float color_eps, float iou_min, const float4 *box,
                                                           const float4 *colkey, uint32_t *flags) {
  __shared__ float4 s_box[kThreads], s_ck[kThreads];
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const int j0 = blockIdx.y * kThreads;
  const int m = min(kThreads, n - j0);
  if (threadIdx.x < m) {
    s_box[threadIdx.x] = box[j0 + threadIdx.x];
    s_ck[threadIdx.x] = colkey[j0 + threadIdx.x];
  }
  __syncthreads();
  if (i >= n) return;
  const float4 a = box[i], ci = colkey[i];
  const uint32_t ki = key_order(ci.w);
  for (int q = 0; q < m; ++q) {
    const float4 cj = s_ck[q];
    const uint32_t kj = key_order(cj.w);
    if (!(kj < ki || (kj == ki && j0 + q < i))) continue;
    const float d0 = __fsub_rn(ci.x, cj.x), d1 = __fsub_rn(ci.y, cj.y), d2 = __fsub_rn(ci.z, cj.z);
    const float dist =
        __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2)));
    if (!(dist < color_eps)) continue;
    const float4 b = s_box[q];
    const float iw = fmaxf(0.f, __fsub_rn(fminf(a.z, b.z), fmaxf(a.x, b.x)));
    const float ih = fmaxf(0.f, __fsub_rn(fminf(a.w, b.w), fmaxf(a.y, b.y)));
    const float inter = __fmul_rn(iw, ih);
    const float area_a = __fmul_rn(__fsub_rn(a.z, a.x), __fsub_rn(a.w, a.y));
    const float area_b = __fmul_rn(__fsub_rn(b.z, b.x), __fsub_rn(b.w, b.y));
    const float uni = __fsub_rn(__fadd_rn(area_a, area_b), inter);
    if (uni > 0.f && __fdiv_rn(inter, uni) > iou_min) {
      atomicOr(&flags[i], kOverlap);
      return;
    }
  }
}

// ---- slot plan (one CTA of 1024 threads) ----

constexpr int kPlanThreads = 1024;

// Inclusive block scan of a packed triple of counts (21 bits each).
__device__ unsigned long long block_scan_packed(unsigned long long v, unsigned long long *warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = warp_tot[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += u;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += warp_tot[warp - 1];
  return v;
}

constexpr int kF0 = 0, kF1 = 21, kF2 = 42;  // fields: free open, split, free closed
constexpr unsigned long long kFieldMask = (1ull << 21) - 1;

__global__ void __launch_bounds__(kPlanThreads) plan_kernel(Curves c, float split_drop, uint32_t *flags,
                                                            int32_t *info, int32_t *free_open, PdHeader *hdr) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_cnt[4];
  const int n = c.n_open + c.n_closed;
  if (threadIdx.x == 0) s_base = 0;
  if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  // pass A: split flags and the ordinals of freed open slots, splits and
  // freed closed slots, all in index order
  for (int base = 0; base < n; base += kPlanThreads) {
    const int i = base + threadIdx.x;
    uint32_t f = 0;
    unsigned long long v = 0;
    if (i < n) {
      f = flags[i];
      const bool pruned = f & kPruned;
      if (i < c.n_open && !pruned) {
        const float *o = c.open_opac + (size_t)i * 3;
        if (o[1] < __fsub_rn(o[0], split_drop) && o[1] < __fsub_rn(o[2], split_drop)) {
          f |= kSplit;
          flags[i] = f;
        }
      }
      if (pruned) v = i < c.n_open ? (1ull << kF0) : (1ull << kF2);
      if (f & kSplit) v = 1ull << kF1;
      if (f & kLowOp) atomicAdd(&s_cnt[0], 1u);
      if (f & kSmall) atomicAdd(&s_cnt[1], 1u);
      if (f & kOverlap) atomicAdd(&s_cnt[2], 1u);
    }
    const unsigned long long incl = block_scan_packed(v, warp_tot);
    const unsigned long long excl = s_base + incl - v;
    if (i < n) {
      if (v == (1ull << kF0)) {
        const int q = (int)((excl >> kF0) & kFieldMask);
        free_open[q] = i;
        info[i] = q;
      } else if (v == (1ull << kF1)) {
        info[i] = (int)((excl >> kF1) & kFieldMask);
      } else if (v == (1ull << kF2)) {
        info[i] = (int)((excl >> kF2) & kFieldMask);
      } else {
        info[i] = -1;
      }
    }
    __syncthreads();
    if (threadIdx.x == kPlanThreads - 1) s_base += incl;
    __syncthreads();
  }
  const int n_fo = (int)((s_base >> kF0) & kFieldMask);
  const int n_sp = (int)((s_base >> kF1) & kFieldMask);
  const int n_fc = (int)((s_base >> kF2) & kFieldMask);
  const int n_used = min(n_sp, n_fo);
  // pass B: split -> target slot (-1: none); freed slot -> region index, or
  // -1 when a split half fills it
  for (int i = threadIdx.x; i < n; i += kPlanThreads) {
    const uint32_t f = flags[i];
    const int q = info[i];
    if (f & kSplit) {
      info[i] = q < n_fo ? free_open[q] : -1;
    } else if (f & kPruned) {
      if (i < c.n_open) info[i] = q < n_used ? -1 : q - n_used;
      else info[i] = (n_fo - n_used) + q;
    }
  }
  if (threadIdx.x == 0) {
    hdr->counts[kCntPruned] = (uint32_t)(n_fo + n_fc);
    hdr->counts[kCntLow] = s_cnt[0];
    hdr->counts[kCntSmall] = s_cnt[1];
    hdr->counts[kCntOverlap] = s_cnt[2];
    hdr->counts[kCntSplit] = (uint32_t)n_sp;
    hdr->counts[kCntSplitPlaced] = (uint32_t)n_used;
    hdr->counts[kCntFreeOpen] = (uint32_t)n_fo;
    hdr->counts[kCntFreeClosed] = (uint32_t)n_fc;
    hdr->n_slots = (uint32_t)((n_fo - n_used) + n_fc);
  }
}

// ---- connected error regions ----

__device__ __forceinline__ bool in_error(const float *img, const float *tgt, size_t P, size_t p, float thr) {
  const float d0 = fabsf(__fsub_rn(img[p], tgt[p]));
  const float d1 = fabsf(__fsub_rn(img[P + p], tgt[P + p]));
  const float d2 = fabsf(__fsub_rn(img[2 * P + p], tgt[2 * P + p]));
  return __fdiv_rn(__fadd_rn(__fadd_rn(d0, d1), d2), 3.0f) > thr;
}

// One warp per row: label[p] = index of the first pixel of p's horizontal
// run of error pixels, -1 outside the mask; area[] cleared.
__global__ void runs_kernel(const float *img, const float *tgt, int W, int H, float thr, int32_t *label,
                            uint32_t *area) {
  const int lane = threadIdx.x & 31;
  const int y = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (y >= H) return;
  const size_t P = (size_t)W * H;
  const int row = y * W;
  int carry = -1;  // run start of the pixel left of this chunk, -1 if not in the mask
#pragma unroll 4
  for (int x0 = 0; x0 < W; x0 += 32) {
    const int x = x0 + lane;
    const bool in = x < W && in_error(img, tgt, P, (size_t)row + x, thr);
    const uint32_t m = __ballot_sync(0xffffffffu, in);
    int start = -1;
    if (in) {
      const uint32_t below = ~m & ((1u << lane) - 1u);
      start = below ? x0 + (32 - __clz(below)) : (carry >= 0 ? carry : x0);
    }
    if (x < W) {
      label[row + x] = in ? row + start : -1;
      area[row + x] = 0u;
    }
    carry = __shfl_sync(0xffffffffu, start, 31);
  }
}

// Root of x: follow parents, which only ever decrease, to the entry that is
// its own parent.
__device__ __forceinline__ int find_root(const int32_t *L, int x) {
  for (;;) {
    const int p = __ldcg(L + x);
    if (p == x) return x;
    x = p;
  }
}

// Link the trees of a and b; the larger root is hooked under the smaller one,
// so every root stays the smallest pixel index of its component.  A new
// attempt follows a root that another thread moved meanwhile; after
// max_attempts the step gives up and records kDevErrTimeout.
__device__ void unite(int32_t *L, int a, int b, uint32_t *status, uint32_t max_attempts) {
  for (uint32_t it = 0;; ++it) {
    a = find_root(L, a);
    b = find_root(L, b);
    if (a == b) return;
    if (it >= max_attempts) {
      atomicOr(status, kDevErrTimeout);
      return;
    }
    if (a < b) {
      const int old = atomicMin(L + b, a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(L + a, b);
      if (old == a) return;
      a = old;
    }
  }
}

// Vertical neighbours in the mask: unite their runs, once per overlap of two
// runs (at its leftmost column).
__global__ void union_kernel(int W, int64_t P, int32_t *L, uint32_t *status, uint32_t max_attempts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P || p < W) return;
  const int x = (int)(p % W);
  const int a = __ldcg(L + p), b = __ldcg(L + p - W);
  if (a < 0 || b < 0) return;
  if (x > 0 && __ldcg(L + p - 1) >= 0 && __ldcg(L + p - W - 1) >= 0) return;
  unite(L, a, b, status, max_attempts);
}

// Run heads (first pixel of a run) point straight to their root.
__global__ void heads_kernel(int W, int64_t P, int32_t *L) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int x = (int)(p % W);
  if (L[p] < 0 || (x > 0 && L[p - 1] >= 0)) return;
  L[p] = find_root(L, (int)p);
}

// A warp covers kWarpPx consecutive pixels of one row, lane l the pixels
// x0 + l + 32 k (coalesced).  Each lane accumulates while its root stays the
// same; at the end the lanes holding the same root add up their partial
// sums and one lane issues the atomics, so a large region costs one atomic
// per warp instead of one per pixel run.
constexpr int kWarpPx = 32 * kSegPx;

__device__ __forceinline__ int64_t warp_chunk(int W, int H, int *y, int *x0) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int cpr = (W + kWarpPx - 1) / kWarpPx;
  if (w >= (int64_t)cpr * H) return -1;
  *y = (int)(w / cpr);
  *x0 = (int)(w % cpr) * kWarpPx;
  return w;
}

// Every pixel to its root (head -> root); pixel counts per root.
__global__ void flatten_kernel(int W, int H, int32_t *L, uint32_t *area) {
  int y, x0;
  if (warp_chunk(W, H, &y, &x0) < 0) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  int cur = -1;
  uint32_t cnt = 0;
  for (int k = 0; k < kSegPx; ++k) {
    const int x = x0 + lane + 32 * k;
    int root = -1;
    if (x < W) {
      const size_t p = (size_t)y * W + x;
      const int l = L[p];
      if (l >= 0) {
        root = L[l];
        L[p] = root;
      }
    }
    if (root != cur) {
      if (cur >= 0) atomicAdd(area + cur, cnt);
      cur = root;
      cnt = 0;
    }
    if (root >= 0) ++cnt;
  }
  for (uint32_t pending = __ballot_sync(0xffffffffu, cur >= 0); pending;) {
    const int leader = __ffs(pending) - 1;
    const int r = __shfl_sync(0xffffffffu, cur, leader);
    const bool mine = cur == r;
    const uint32_t sum = __reduce_add_sync(0xffffffffu, mine ? cnt : 0u);
    if (lane == leader) atomicAdd(area + r, sum);
    pending &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// key = (0xffffffff - count) << 32 | root: ascending keys = count
// descending, then root ascending.  Keys are unique.
__global__ void roots_kernel(int64_t P, const int32_t *L, const uint32_t *area, unsigned long long *roots,
                             PdHeader *hdr) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool is_root = p < P && L[p] == (int32_t)p;
  const uint32_t m = __ballot_sync(0xffffffffu, is_root);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&hdr->n_roots, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (is_root) {
    const unsigned long long key = ((unsigned long long)(0xffffffffu - area[p]) << 32) | (unsigned long long)p;
    roots[base + __popc(m & ((1u << lane) - 1u))] = key;
  }
}

// ---- selection of the n_sel smallest keys ----

__global__ void select_init_kernel(PdHeader *hdr) {
  const uint32_t n_sel = min(hdr->n_roots, hdr->n_slots);
  hdr->n_sel = n_sel;
  hdr->rank_left = n_sel;
  hdr->kth = 0ull;
}

__global__ void __launch_bounds__(kThreads) select_hist_kernel(const unsigned long long *roots, PdHeader *hdr,
                                                               int shift) {
  __shared__ uint32_t h[256];
  if (hdr->n_sel == 0) return;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t n = hdr->n_roots;
  const unsigned long long prefix = hdr->kth;
  const int hi = shift + 8;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long k = roots[i];
    if (hi >= 64 || (k >> hi) == (prefix >> hi)) atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hdr->hist[threadIdx.x], h[threadIdx.x]);
}

// The digit holding the rank_left-th smallest key among those matching the
// prefix; clears the histogram for the next digit.
__global__ void __launch_bounds__(256) select_pick_kernel(PdHeader *hdr, int shift) {
  __shared__ uint32_t warp_tot[8];
  if (hdr->n_sel == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v = hdr->hist[threadIdx.x];
  uint32_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  for (int w = 0; w < warp; ++w) incl += warp_tot[w];
  const uint32_t excl = incl - v;
  const uint32_t k = hdr->rank_left;
  __syncthreads();
  if (excl < k && k <= incl) {
    hdr->kth |= (unsigned long long)threadIdx.x << shift;
    hdr->rank_left = k - excl;
  }
  hdr->hist[threadIdx.x] = 0;
}

__global__ void gather_sel_kernel(const unsigned long long *roots, unsigned long long *sel, PdHeader *hdr) {
  if (hdr->n_sel == 0) return;
  const uint32_t n = hdr->n_roots;
  const unsigned long long kth = hdr->kth;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long k = roots[i];
    if (k <= kth) sel[atomicAdd(&hdr->n_gathered, 1u)] = k;
  }
}

// Rank of each selected key among the selected ones (unique keys), by
// counting; marks area[root] with the rank.
__global__ void __launch_bounds__(kThreads) rank_sel_kernel(const unsigned long long *sel,
                                                            unsigned long long *sorted, uint32_t *area,
                                                            const PdHeader *hdr) {
  __shared__ unsigned long long s[kThreads];
  const uint32_t n = hdr->n_sel;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x >= n) return;
  const unsigned long long mine = t < n ? sel[t] : 0ull;
  uint32_t rank = 0;
  for (uint32_t base = 0; base < n; base += kThreads) {
    __syncthreads();
    if (base + threadIdx.x < n) s[threadIdx.x] = sel[base + threadIdx.x];
    __syncthreads();
    const uint32_t m = min((uint32_t)kThreads, n - base);
    for (uint32_t q = 0; q < m; ++q) rank += s[q] < mine;
  }
  if (t < n) {
    sorted[rank] = mine;
    area[(uint32_t)(mine & 0xffffffffu)] = kSelected | rank;
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums over the pixels of each selected region (same warp layout and
// aggregation as flatten_kernel).
__global__ void sums_kernel(const float *tgt, int W, int H, const int32_t *L, const uint32_t *area,
                            RegionAcc *acc) {
  int y, x0;
  if (warp_chunk(W, H, &y, &x0) < 0) return;
  const int lane = threadIdx.x & 31;
  const size_t P = (size_t)W * H;
  int cur = -1;
  unsigned long long sx = 0, sy = 0;
  double r = 0, g = 0, b = 0;
  for (int k = 0; k < kSegPx; ++k) {
    const int x = x0 + lane + 32 * k;
    int sel = -1;
    size_t p = 0;
    if (x < W) {
      p = (size_t)y * W + x;
      const int l = L[p];
      if (l >= 0) {
        const uint32_t v = area[l];
        if (v & kSelected) sel = (int)(v & ~kSelected);
      }
    }
    if (sel != cur) {
      if (cur >= 0) {
        RegionAcc *a = acc + cur;
        atomicAdd(&a->sx, sx);
        atomicAdd(&a->sy, sy);
        atomicAdd(&a->r, r);
        atomicAdd(&a->g, g);
        atomicAdd(&a->b, b);
      }
      cur = sel;
      sx = sy = 0;
      r = g = b = 0;
    }
    if (sel >= 0) {
      sx += (unsigned long long)x;
      sy += (unsigned long long)y;
      r += (double)tgt[p];
      g += (double)tgt[P + p];
      b += (double)tgt[2 * P + p];
    }
  }
  for (uint32_t pending = __ballot_sync(0xffffffffu, cur >= 0); pending;) {
    const int leader = __ffs(pending) - 1;
    const int k = __shfl_sync(0xffffffffu, cur, leader);
    const bool mine = cur == k;
    const unsigned long long tx = warp_sum_u64(mine ? sx : 0ull), ty = warp_sum_u64(mine ? sy : 0ull);
    const double tr = warp_sum_d(mine ? r : 0.0), tg = warp_sum_d(mine ? g : 0.0), tb = warp_sum_d(mine ? b : 0.0);
    if (lane == leader) {
      RegionAcc *a = acc + k;
      atomicAdd(&a->sx, tx);
      atomicAdd(&a->sy, ty);
      atomicAdd(&a->r, tr);
      atomicAdd(&a->g, tg);
      atomicAdd(&a->b, tb);
    }
    pending &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// ---- edits ----

__device__ __forceinline__ double lerp_rn(double a, double b, double t) {
  return __dadd_rn(__dmul_rn(a, 1.0 - t), __dmul_rn(b, t));
}

// de Casteljau split of the cubic p at t: left (p0, a0, b0, c), right (c, b1, a2, p3).
__device__ void casteljau(const double2 p[4], double t, double2 left[4], double2 right[4]) {
  double2 a[3], b[2], c;
  for (int j = 0; j < 3; ++j) a[j] = make_double2(lerp_rn(p[j].x, p[j + 1].x, t), lerp_rn(p[j].y, p[j + 1].y, t));
  for (int j = 0; j < 2; ++j) b[j] = make_double2(lerp_rn(a[j].x, a[j + 1].x, t), lerp_rn(a[j].y, a[j + 1].y, t));
  c = make_double2(lerp_rn(b[0].x, b[1].x, t), lerp_rn(b[0].y, b[1].y, t));
  left[0] = p[0], left[1] = a[0], left[2] = b[0], left[3] = c;
  right[0] = c, right[1] = b[1], right[2] = a[2], right[3] = p[3];
}

// One cubic segment (4 points from src) as three chained segments covering
// t in [0,1/3], [1/3,2/3], [2/3,1]: 10 points written to dst.
__device__ void write_thirds(const float *src, float *dst) {
  double2 p[4], s0[4], rest[4], s1[4], s2[4];
  for (int j = 0; j < 4; ++j) p[j] = make_double2((double)src[2 * j], (double)src[2 * j + 1]);
  casteljau(p, 1.0 / 3.0, s0, rest);
  casteljau(rest, 0.5, s1, s2);
  double2 out[10] = {s0[0], s0[1], s0[2], s0[3], s1[1], s1[2], s1[3], s2[1], s2[2], s2[3]};
  for (int j = 0; j < 10; ++j) {
    dst[2 * j] = (float)out[j].x;
    dst[2 * j + 1] = (float)out[j].y;
  }
}

__global__ void apply_kernel(Curves c, float new_opacity, float new_width, const uint32_t *flags,
                             const int32_t *info, const unsigned long long *sorted, const RegionAcc *acc,
                             const PdHeader *hdr, uint8_t *changed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = c.n_open + c.n_closed;
  if (i >= n) return;
  const uint32_t f = flags[i];
  const int q = info[i];
  const bool open = i < c.n_open;
  if (changed) changed[i] = (f & (kPruned | kSplit)) ? 1 : 0;
  if (f & kSplit) {
    float P[20], o[3], col[3];
    const float w = c.open_width[i];
    for (int j = 0; j < 20; ++j) P[j] = c.open_ctrl[(size_t)i * 20 + j];
    for (int j = 0; j < 3; ++j) o[j] = c.open_opac[(size_t)i * 3 + j], col[j] = c.open_color[(size_t)i * 3 + j];
    write_thirds(P, c.open_ctrl + (size_t)i * 20);
    for (int j = 0; j < 3; ++j) c.open_opac[(size_t)i * 3 + j] = o[0];
    if (q >= 0) {
      write_thirds(P + 12, c.open_ctrl + (size_t)q * 20);
      for (int j = 0; j < 3; ++j) {
        c.open_opac[(size_t)q * 3 + j] = o[2];
        c.open_color[(size_t)q * 3 + j] = col[j];
      }
      c.open_width[q] = w;
    }
    return;
  }
  if (!(f & kPruned) || q < 0) return;
  if ((uint32_t)q >= hdr->n_sel) {  // no region left for this slot
    if (open) {
      for (int j = 0; j < 3; ++j) c.open_opac[(size_t)i * 3 + j] = 0.f;
    } else {
      c.closed_opac[i - c.n_open] = 0.f;
    }
    return;
  }
  const unsigned long long key = sorted[q];
  const uint32_t cnt = 0xffffffffu - (uint32_t)(key >> 32);
  const RegionAcc a = acc[q];
  const double A = (double)cnt;
  // centroid of the pixel centres: (sum x + A/2) / A, one rounding
  const double cx = __ddiv_rn((double)(2 * a.sx + cnt), 2.0 * A);
  const double cy = __ddiv_rn((double)(2 * a.sy + cnt), 2.0 * A);
  const double rad = __dsqrt_rn(__ddiv_rn(A, 3.141592653589793));
  const float col[3] = {(float)__ddiv_rn(a.r, A), (float)__ddiv_rn(a.g, A), (float)__ddiv_rn(a.b, A)};
  const int np = open ? 10 : 12;
  const double span = open ? 11.0 : 12.0;
  float *dst = open ? c.open_ctrl + (size_t)i * 20 : c.closed_ctrl + (size_t)(i - c.n_open) * 24;
  for (int j = 0; j < np; ++j) {
    const double ang = __ddiv_rn(__dmul_rn(2.0 * 3.141592653589793, (double)j), span);
    dst[2 * j] = (float)__dadd_rn(cx, __dmul_rn(rad, cos(ang)));
    dst[2 * j + 1] = (float)__dadd_rn(cy, __dmul_rn(rad, sin(ang)));
  }
  if (open) {
    for (int j = 0; j < 3; ++j) {
      c.open_opac[(size_t)i * 3 + j] = new_opacity;
      c.open_color[(size_t)i * 3 + j] = col[j];
    }
    c.open_width[i] = new_width;
  } else {
    const int j = i - c.n_open;
    c.closed_opac[j] = new_opacity;
    for (int k = 0; k < 3; ++k) c.closed_color[(size_t)j * 3 + k] = col[k];
  }
}

uint32_t g_union_attempts = kUnionAttempts;

}  // namespace

void debug_set_retry_limit(int64_t max_attempts) {
  g_union_attempts = max_attempts < 0 ? kUnionAttempts : (uint32_t)std::min<int64_t>(max_attempts, 0xffffffffll);
}

size_t prune_densify_bytes(int n_open, int n_closed, int width, int height) {
  return layout(n_open + n_closed, (int64_t)width * height).bytes;
}

bs_status run_prune_densify(const bs_curves_mut &cm, const bs_pd_cfg &cfg, int W, int H, const float *img,
                            const float *target, void *ws, uint8_t *changed, bs_pd_stats *stats,
                            cudaStream_t s) {
  const int n = cm.n_open + cm.n_closed;
  const int64_t P = (int64_t)W * H;
  const Layout L = layout(n, P);
  char *base = static_cast<char *>(ws);
  PdHeader *hdr = reinterpret_cast<PdHeader *>(base + L.hdr);
  float4 *box = reinterpret_cast<float4 *>(base + L.box);
  float4 *colkey = reinterpret_cast<float4 *>(base + L.colkey);
  uint32_t *flags = reinterpret_cast<uint32_t *>(base + L.flags);
  int32_t *info = reinterpret_cast<int32_t *>(base + L.info);
  int32_t *free_open = reinterpret_cast<int32_t *>(base + L.free_open);
  unsigned long long *sel = reinterpret_cast<unsigned long long *>(base + L.sel);
  unsigned long long *sorted = reinterpret_cast<unsigned long long *>(base + L.sorted);
  RegionAcc *acc = reinterpret_cast<RegionAcc *>(base + L.acc);
  int32_t *label = reinterpret_cast<int32_t *>(base + L.label);
  uint32_t *area = reinterpret_cast<uint32_t *>(base + L.area);
  unsigned long long *roots = reinterpret_cast<unsigned long long *>(base + L.roots);

  Curves c{cm.n_open, cm.n_closed, cm.open_ctrl, cm.open_width, cm.open_color, cm.open_opac,
           cm.closed_ctrl, cm.closed_color, cm.closed_opac};
  const float frac = (float)std::min(1.0, (double)cfg.step / (double)std::max(1, cfg.t_end));

  BS_CUDA(cudaMemsetAsync(hdr, 0, sizeof(PdHeader), s));
  if (n > 0) BS_CUDA(cudaMemsetAsync(acc, 0, sizeof(RegionAcc) * (size_t)n, s));
  if (n > 0) {
    const int nb = div_up(n, kThreads);
    curve_kernel<<<nb, kThreads, 0, s>>>(c, cfg.op_start, cfg.op_end, frac, cfg.area_min, box, colkey, flags);
    BS_LAUNCHED("prune curve_kernel");
    overlap_kernel<<<dim3(nb, nb), kThreads, 0, s>>>(n, cfg.color_eps, cfg.iou_min, box, colkey, flags);
    BS_LAUNCHED("prune overlap_kernel");
    plan_kernel<<<1, kPlanThreads, 0, s>>>(c, cfg.split_drop, flags, info, free_open, hdr);
    BS_LAUNCHED("prune plan_kernel");
  }
  const unsigned pb = (unsigned)div_up64(P, kThreads);
  runs_kernel<<<div_up(H, kThreads / 32), kThreads, 0, s>>>(img, target, W, H, cfg.err_thresh, label, area);
  BS_LAUNCHED("prune runs_kernel");
  union_kernel<<<pb, kThreads, 0, s>>>(W, P, label, &hdr->status, g_union_attempts);
  BS_LAUNCHED("prune union_kernel");
  heads_kernel<<<pb, kThreads, 0, s>>>(W, P, label);
  BS_LAUNCHED("prune heads_kernel");
  const int64_t seg_threads = (int64_t)div_up(W, kWarpPx) * H * 32;
  const unsigned sb = (unsigned)div_up64(seg_threads, kThreads);
  flatten_kernel<<<sb, kThreads, 0, s>>>(W, H, label, area);
  BS_LAUNCHED("prune flatten_kernel");
  roots_kernel<<<pb, kThreads, 0, s>>>(P, label, area, roots, hdr);
  BS_LAUNCHED("prune roots_kernel");
  if (n > 0) {
    select_init_kernel<<<1, 1, 0, s>>>(hdr);
    BS_LAUNCHED("prune select_init_kernel");
    for (int shift = 56; shift >= 0; shift -= 8) {
      select_hist_kernel<<<kSelectBlocks, kThreads, 0, s>>>(roots, hdr, shift);
      BS_LAUNCHED("prune select_hist_kernel");
      select_pick_kernel<<<1, 256, 0, s>>>(hdr, shift);
      BS_LAUNCHED("prune select_pick_kernel");
    }
    gather_sel_kernel<<<kSelectBlocks, kThreads, 0, s>>>(roots, sel, hdr);
    BS_LAUNCHED("prune gather_sel_kernel");
    rank_sel_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(sel, sorted, area, hdr);
    BS_LAUNCHED("prune rank_sel_kernel");
    sums_kernel<<<sb, kThreads, 0, s>>>(target, W, H, label, area, acc);
    BS_LAUNCHED("prune sums_kernel");
    apply_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(c, cfg.new_opacity, cfg.new_width, flags, info, sorted,
                                                          acc, hdr, changed);
    BS_LAUNCHED("prune apply_kernel");
  }
  PdHeader h;
  BS_CUDA(cudaMemcpyAsync(&h, hdr, offsetof(PdHeader, hist), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    stats->pruned = (int32_t)h.counts[kCntPruned];
    stats->low_opacity = (int32_t)h.counts[kCntLow];
    stats->small_area = (int32_t)h.counts[kCntSmall];
    stats->overlap = (int32_t)h.counts[kCntOverlap];
    stats->split = (int32_t)h.counts[kCntSplit];
    stats->split_placed = (int32_t)h.counts[kCntSplitPlaced];
    stats->regions = (int32_t)h.n_roots;
    stats->inserted = (int32_t)h.n_sel;
    stats->transparent = (int32_t)(h.n_slots - h.n_sel);
  }
  if (h.status & kDevErrTimeout) {
    set_error("bs_prune_densify: a union step of the region labelling gave up after its bounded attempts");
    return BS_ERR_TIMEOUT;
  }
  return BS_OK;
}

}  // namespace bs
