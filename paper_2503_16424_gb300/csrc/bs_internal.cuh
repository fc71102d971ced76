// Internal declarations shared by the translation units of libbs.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "bs.h"

namespace bs {

// ---- thresholds of the blend (Eq. 9-10 with the tile rasterizer's rules) ----
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip a Gaussian below this alpha
constexpr float kAlphaMax = 0.99f;          // alpha clamp
constexpr float kTMin = 1e-4f;              // stop a pixel before T drops below
constexpr float kExtPad = 0.01f;            // px added to support half extents

constexpr int kMaxSamplesPerCurve = 3072;  // a closed curve's rows x samples per row
// Curves of at least this many samples are sampled by CTAs of
// kCurveThreadsWide threads, the others by CTAs of kCurveThreads.
constexpr int kWideSamples = 512;
constexpr int kCurveThreads = 64;
constexpr int kCurveThreadsWide = 256;

// ---- status plumbing ----
void set_error(const char *fmt, ...);
bs_status cuda_status(cudaError_t e, const char *what);
bs_status check_device();

#define BS_TRY(expr)                      \
  do {                                    \
    bs_status _s = (expr);                \
    if (_s != BS_OK) return _s;           \
  } while (0)

#define BS_CUDA(expr) BS_TRY(::bs::cuda_status((expr), #expr))

#define BS_LAUNCHED(what) BS_TRY(::bs::cuda_status(cudaGetLastError(), what))

// ---- device status words ----
// Inside the binning and batch workspaces:
constexpr uint32_t kDevErrTimeout = 1u;
constexpr uint32_t kDevErrCapacity = 2u;
constexpr uint32_t kDevErrCounts = 4u;   // batch binning: pair totals disagree (never expected)
// The library's own word on each device (bs_sync_status): a sampling or
// backward kernel wrote a non-finite table record or gradient.
constexpr uint32_t kDevErrNotFinite = 8u;
// Device address of the current device's library status word, looked up
// once per device (thread-safe).
bs_status lib_status_word(uint32_t **ptr);

// ---- small math helpers usable on host and device ----
__host__ __device__ inline int div_up(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t div_up64(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int bit_length(uint64_t v) {
  int n = 0;
  while (v) { ++n; v >>= 1; }
  return n;
}
inline int gauss_bits(int64_t n_gauss) { return n_gauss > 1 ? bit_length((uint64_t)(n_gauss - 1)) : 1; }
// Tile-id bits of a canvas.
inline int tile_bits(const bs_canvas &cv) {
  const int64_t n = (int64_t)div_up(cv.width, cv.tile) * div_up(cv.height, cv.tile);
  return n > 1 ? bit_length((uint64_t)(n - 1)) : 1;
}
// Bits of the Gaussian index inside a sorted key of one canvas: gauss_bits
// for 32-bit keys (tile << gbits | g); 32 when tile bits + gbits exceed 32
// and the binning sorts 64-bit keys, whose sorted output is g alone.
inline int key_gbits(int64_t n_gauss, const bs_canvas &cv) {
  const int g = gauss_bits(n_gauss);
  return g + tile_bits(cv) > 32 ? 32 : g;
}

// ---- draw-order key (Section 3.3), shared by the draw order and pruning ----
#ifdef __CUDACC__
// Area key of curve i in float32, each operation rounded in order: a closed
// curve's key is half the absolute shoelace sum of its 12-point control
// polygon, an open curve's the length of its 10-point control polygon times
// its width.  Curves i < n_open are open.
__device__ __forceinline__ float curve_area_key(int n_open, const float *open_ctrl, const float *open_width,
                                                const float *closed_ctrl, int i) {
  if (i < n_open) {
    const float *P = open_ctrl + (size_t)i * 20;
    float acc = 0.f;
    for (int j = 0; j < 9; ++j) {
      const float dx = __fsub_rn(P[2 * j + 2], P[2 * j]);
      const float dy = __fsub_rn(P[2 * j + 3], P[2 * j + 1]);
      acc = __fadd_rn(acc, __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy))));
    }
    return __fmul_rn(acc, open_width[i]);
  }
  const float *P = closed_ctrl + (size_t)(i - n_open) * 24;
  float acc = 0.f;
  for (int j = 0; j < 12; ++j) {
    const int jn = j == 11 ? 0 : j + 1;
    const float cross = __fsub_rn(__fmul_rn(P[2 * j], P[2 * jn + 1]), __fmul_rn(P[2 * jn], P[2 * j + 1]));
    acc = __fadd_rn(acc, cross);
  }
  return __fmul_rn(fabsf(acc), 0.5f);
}

// Order-preserving integer image of a float key (NaN last, -0 == +0).
__device__ __forceinline__ uint32_t key_order(float k) {
  if (k != k) return 0xffffffffu;
  k = __fadd_rn(k, 0.0f);
  const uint32_t b = __float_as_uint(k);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
#endif

// ---- launchers (one per translation unit) ----
// curves (bs_curves.cu)
bs_status launch_curve_order(const bs_curves &c, const bs_sample_cfg &cfg, uint32_t *rank,
                             uint32_t *first, cudaStream_t s);
bs_status launch_sample_fwd(const bs_curves &c, const bs_sample_cfg &cfg, float *gauss,
                            cudaStream_t s);
bs_status launch_sample_bwd(const bs_curves &c, const bs_sample_cfg &cfg, const float *dgauss,
                            const bs_curves_grad &g, cudaStream_t s);
bs_status launch_xing(const bs_curves &c, float lambda, double *loss, float *grad_closed_ctrl, cudaStream_t s);

// binning (bs_bin.cu)
struct BinPlan {
  int64_t n_gauss;
  int tiles_x, tiles_y, n_tiles;
  int gbits, tbits;
  bool wide;               // tbits + gbits > 32: 64-bit keys (tile << 32 | g), g alone written out
  int passes, digit_bits;
  int64_t capacity;
  int64_t count_blocks;    // blocks of the count/emit kernels
  int64_t parts;           // sort partitions for `capacity` keys
  // byte offsets inside the workspace
  size_t off_hdr, off_hist, off_diff, zero_bytes, off_parts;
  size_t off_local, off_partial, off_rects, off_owner, off_keys_tmp;  // keys_tmp: u32 [capacity], or u64 [2][capacity] when wide
  // the two-level counting sort instead of the radix passes (rows): level-1
  // chunks of 256 Gaussians, the most level-2 chunks, and its tables
  bool rows;
  int n_g1;
  int64_t n_ch_max;
  size_t off_t1, off_rowcnt, off_rowstart, off_chstart, off_t2, off_chrow;
  size_t bytes;
};
// allow_rows = false keeps the radix passes (the fixed scratch of
// bs_bin_tiles_static is sized for them).
bs_status plan_binning(int64_t n_gauss, const bs_canvas &cv, int64_t capacity, BinPlan *p, bool allow_rows = true);
bs_status run_binning(const BinPlan &p, const float *gauss, const bs_canvas &cv, void *ws,
                      int64_t *n_pairs, uint32_t *tile_keys, uint32_t *tile_ranges,
                      cudaStream_t s, bool sync = true, int64_t *n_pairs_dev = nullptr);
bs_status read_device_status(const void *ws, size_t ws_bytes, int32_t *out, cudaStream_t s,
                             int64_t *n_pairs = nullptr);
// Fixed scratch of bs_bin_tiles_static: 32 MiB of device memory per GPU.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
bs_status static_scratch(void **ptr);

// render (bs_render.cu)
bs_status launch_render_fwd(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                            const uint32_t *keys, const uint32_t *ranges, float *img,
                            float *T_final, uint32_t *n_contrib, cudaStream_t s,
                            unsigned long long *stats = nullptr);
bs_status launch_render_fwd_l2(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                               const uint32_t *keys, const uint32_t *ranges, const float *target, float *img,
                               float *T_final, uint32_t *n_contrib, float *dimg, double *loss, cudaStream_t s);
bs_status launch_render_bwd(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                            const uint32_t *keys, const uint32_t *ranges, const float *T_final,
                            const uint32_t *n_contrib, const float *dL_dimg, float *dgauss,
                            cudaStream_t s);
bs_status launch_l2(const float *img, const float *target, int64_t n, float *dimg, double *loss,
                    cudaStream_t s);

// ---- batches of images (bs_batch.cu and the batched kernels) ----
// One entry of the device table of a batch: where image b's curves,
// Gaussians, pixels, tiles and difference array start in the batch's
// concatenated arrays, and its canvas and sampling.
struct BatchImage {
  int W, H, tiles_x, tiles_y;
  int n_open, n_closed;
  int g_open, rows, kc;
  float rho, eps;
  float bg[3];
  float l2_scale;       // 2 / (3 W H)
  int order_chunks;     // ceil((n_open + n_closed) / 256)
  int tmode;            // its sampling's tangent_mode
  int64_t open0, closed0;  // first open / closed curve
  int64_t gauss0, n_gauss; // first Gaussian and count
  int64_t pix0;            // first pixel
  int64_t tile0;           // first tile of the batch's tile numbering
  int64_t diff0;           // first word of its (tiles_y + 1) x (tiles_x + 1) difference array
  int64_t row0, col0;      // first row / column of the stacked difference arrays
  int64_t order0;          // first CTA of the draw-order grid
};

struct BatchPlan {
  int n_images, tile;
  int64_t n_open, n_closed, n_curves, n_gauss, n_pix, n_tiles;
  int64_t diff_words, diff_rows, diff_cols, order_ctas;
  int tbits, passes, digit_bits;
  int64_t capacity, parts, count_blocks, tile_blocks;
  int n_max, k_max, rows_max;  // sampling: largest samples per curve / per row, rows
  // The curves of fewer than kWideSamples samples (sampled by narrow CTAs)
  // and the others (wide CTAs): their count and largest sizes (0: none).
  struct SampleClass {
    int64_t n_curves;
    int open_g, closed_n, closed_k, closed_rows;
  } narrow, wide;
  // byte offsets inside the batch workspace
  size_t off_hdr, off_hist, off_diff, off_queue, zero_bytes;
  size_t off_images, off_curve_ids, off_parts, off_local, off_partial, off_rects, off_owner, off_tsum, off_keys0, off_keys1;
  size_t bytes;
};

// Header of the batch workspace.  status bits: kDevErrCapacity when the
// pairs exceed the capacity (the ranges are then empty and nothing is
// sorted).  n_pairs is the number of pairs the binning found (the sum of
// the Gaussians' counts), n_sorted the number it sorted (0 on overflow),
// tile_total the same pairs summed over the tiles.
struct BatchHdr {
  uint32_t status;
  uint32_t pad;
  unsigned long long n_pairs;
  unsigned long long n_sorted;
  unsigned long long tile_total;
};

#ifdef __CUDACC__
// The batch's tables: image b owns Gaussians [gauss0, gauss0 + n_gauss),
// tiles [tile0, tile0 + tiles_x tiles_y), difference-array rows [row0,
// row0 + tiles_y + 1), columns [col0, col0 + tiles_x + 1), open curves
// [open0, open0 + n_open) and so on.  An index belongs to the last image
// whose first index is <= it (an image owning none of a kind shares its first
// index with the next image and is passed over).
template <int64_t BatchImage::*F>
__device__ __forceinline__ int last_image_le(const BatchImage *__restrict__ tab, int n_images, int64_t v) {
  int lo = 0, hi = n_images;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (tab[mid].*F <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}
#endif

bs_status plan_batch(const bs_batch_image *images, int32_t n_images, int32_t tile, int64_t capacity,
                     BatchPlan *p);
void fill_batch_table(const bs_batch_image *images, const BatchPlan &p, BatchImage *out);
// The batch's curve indices, the narrow class first, then the wide one
// (curves of fewer / at least kWideSamples samples); out holds n_curves.
void fill_curve_classes(const bs_batch_image *images, const BatchPlan &p, int32_t *out);

// launchers of the batched kernels; `table` is the device table in the workspace
bs_status launch_batch_curve_order(const BatchPlan &p, const BatchImage *table, const bs_curves &c,
                                   uint32_t *rank, uint32_t *first, cudaStream_t s);
bs_status launch_batch_sample_fwd(const BatchPlan &p, const BatchImage *table, const int32_t *curve_ids,
                                  const bs_curves &c, float *gauss, cudaStream_t s);
bs_status launch_batch_sample_bwd(const BatchPlan &p, const BatchImage *table, const int32_t *curve_ids,
                                  const bs_curves &c, const float *dgauss, const bs_curves_grad &g, cudaStream_t s);
bs_status run_batch_binning(const BatchPlan &p, void *ws, const float *gauss, uint32_t *tile_vals,
                            uint32_t *tile_ranges, cudaStream_t s);
bs_status read_batch_status(const BatchPlan &p, const void *ws, int32_t *status, int64_t *n_pairs, cudaStream_t s);
bs_status launch_batch_render_fwd(const BatchPlan &p, void *ws, const float *gauss, const uint32_t *vals,
                                  const uint32_t *ranges, const float *target, float *img, float *T_final,
                                  uint32_t *n_contrib, float *dimg, double *loss, cudaStream_t s);
bs_status launch_batch_render_bwd(const BatchPlan &p, void *ws, const float *gauss, const uint32_t *vals,
                                  const uint32_t *ranges, const float *T_final, const uint32_t *n_contrib,
                                  const float *dimg, float *dgauss, cudaStream_t s);

// Adam (bs_adam.cu)
bs_status launch_adam(const bs_adam_group *groups, int n_groups, const bs_adam_cfg &cfg, int32_t *step,
                      cudaStream_t s);

// pruning and densification (bs_prune.cu)
constexpr int kMaxPdCurves = 65536;
size_t prune_densify_bytes(int n_open, int n_closed, int width, int height);
bs_status run_prune_densify(const bs_curves_mut &c, const bs_pd_cfg &cfg, int width, int height,
                            const float *img, const float *target, void *ws, uint8_t *changed,
                            bs_pd_stats *stats, cudaStream_t s);

}  // namespace bs
