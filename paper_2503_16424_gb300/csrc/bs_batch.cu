// Batches of images (many targets optimised together, each by the method of
// Section 3) and the Adam update of Section 4.1.
//
// A batch is laid out image after image: curves, Gaussians, pixels, tiles
// and tile difference arrays of image b start at the prefix sums of the
// earlier images' counts.  plan_batch does that host arithmetic and the
// workspace layout; fill_batch_table writes the per-image table the batched
// kernels read.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "bs_internal.cuh"

namespace bs {

namespace {

constexpr int64_t kMaxBatchPairs = (1ll << 30) - 1;
constexpr int kOrderChunkHost = 256;    // curves per draw-order chunk (bs_curves.cu)
constexpr int kTilesPerCtaHost = 2048;  // tiles per CTA of the batch tile scan (bs_bin.cu)
constexpr int kSortTileHost = 4096;     // keys per sort partition (bs_bin.cu)
constexpr int kEmitTileHost = 2048;     // keys per emit CTA (bs_bin.cu)
constexpr int kCountThreadsHost = 256;  // Gaussians per count CTA (bs_bin.cu)
constexpr int kMaxPassesHost = 4;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

bs_status plan_batch(const bs_batch_image *images, int32_t n_images, int32_t tile, int64_t capacity,
                     BatchPlan *p) {
  if (!images || n_images < 1) {
    set_error("a batch needs at least one image");
    return BS_ERR_INVALID_ARG;
  }
  if (tile != 8 && tile != 16 && tile != 32) {
    set_error("tile side %d not supported (8, 16, 32)", tile);
    return BS_ERR_UNSUPPORTED;
  }
  if (capacity < 1 || capacity > kMaxBatchPairs) {
    set_error("pair_capacity %lld out of range [1, 2^30)", (long long)capacity);
    return BS_ERR_INVALID_ARG;
  }
  *p = BatchPlan{};
  p->n_images = n_images;
  p->tile = tile;
  for (int b = 0; b < n_images; ++b) {
    const bs_batch_image &im = images[b];
    if (im.width < 1 || im.height < 1 || im.width > 32768 || im.height > 32768) {
      set_error("image %d: canvas %dx%d out of range", b, im.width, im.height);
      return BS_ERR_INVALID_ARG;
    }
    if (im.n_open < 0 || im.n_closed < 0) {
      set_error("image %d: negative curve count", b);
      return BS_ERR_INVALID_ARG;
    }
    const int64_t tx = div_up(im.width, tile), ty = div_up(im.height, tile);
    const int64_t nc = (int64_t)im.n_open + im.n_closed;
    const int64_t ng = (int64_t)im.n_open * im.sample.g_open +
                       (int64_t)im.n_closed * im.sample.rows_closed * im.sample.k_closed;
    const int64_t chunks = div_up64(nc, kOrderChunkHost);
    p->n_open += im.n_open;
    p->n_closed += im.n_closed;
    p->n_gauss += ng;
    p->n_pix += (int64_t)im.width * im.height;
    p->n_tiles += tx * ty;
    p->diff_words += (tx + 1) * (ty + 1);
    p->diff_rows += ty + 1;
    p->diff_cols += tx + 1;
    p->order_ctas += chunks * chunks;
    const auto cls = [p](int n) -> BatchPlan::SampleClass & { return n < kWideSamples ? p->narrow : p->wide; };
    if (im.n_open > 0) {
      const int n = im.sample.g_open;
      p->n_max = std::max(p->n_max, n);
      p->k_max = std::max(p->k_max, n);
      BatchPlan::SampleClass &c = cls(n);
      c.n_curves += im.n_open;
      c.open_g = std::max(c.open_g, n);
    }
    if (im.n_closed > 0) {
      const int n = im.sample.rows_closed * im.sample.k_closed;
      p->n_max = std::max(p->n_max, n);
      p->k_max = std::max(p->k_max, im.sample.k_closed);
      p->rows_max = std::max(p->rows_max, im.sample.rows_closed);
      BatchPlan::SampleClass &c = cls(n);
      c.n_curves += im.n_closed;
      c.closed_n = std::max(c.closed_n, n);
      c.closed_k = std::max(c.closed_k, im.sample.k_closed);
      c.closed_rows = std::max(c.closed_rows, im.sample.rows_closed);
    }
  }
  p->n_curves = p->n_open + p->n_closed;
  if (p->n_curves > (1ll << 30)) {
    set_error("%lld curves: at most 2^30 per batch", (long long)p->n_curves);
    return BS_ERR_INVALID_ARG;
  }
  if (p->n_gauss > (1ll << 31) - 1) {
    set_error("%lld Gaussians: at most 2^31 - 1 per batch", (long long)p->n_gauss);
    return BS_ERR_INVALID_ARG;
  }
  if (p->n_tiles > 0xffffffffll || p->order_ctas > 0x7fffffffll) {
    set_error("batch too large: %lld tiles", (long long)p->n_tiles);
    return BS_ERR_INVALID_ARG;
  }
  p->tbits = p->n_tiles > 1 ? bit_length((uint64_t)(p->n_tiles - 1)) : 1;
  p->passes = div_up(p->tbits, 8);
  if (p->passes > kMaxPassesHost) {
    set_error("%d tile bits need more than %d sort passes", p->tbits, kMaxPassesHost);
    return BS_ERR_UNSUPPORTED;
  }
  p->digit_bits = div_up(p->tbits, p->passes);
  p->capacity = capacity;
  p->parts = div_up64(capacity, kSortTileHost);
  p->count_blocks = div_up64(p->n_gauss > 0 ? p->n_gauss : 1, kCountThreadsHost);
  p->tile_blocks = div_up64(p->n_tiles, kTilesPerCtaHost);
  const size_t ng = (size_t)(p->n_gauss > 0 ? p->n_gauss : 1);
  size_t o = 0;
  p->off_hdr = o;     o = align256(o + sizeof(BatchHdr));
  p->off_hist = o;    o = align256(o + sizeof(uint32_t) * kMaxPassesHost * 256);
  p->off_diff = o;    o = align256(o + sizeof(int) * (size_t)p->diff_words);
  p->zero_bytes = o;
  p->off_queue = o;   o = align256(o + sizeof(uint32_t) * 2);
  p->off_images = o;  o = align256(o + sizeof(BatchImage) * (size_t)n_images);
  p->off_curve_ids = o;  o = align256(o + sizeof(int32_t) * (size_t)(p->n_curves > 0 ? p->n_curves : 1));
  p->off_parts = o;   o = align256(o + sizeof(uint32_t) * 256 * (size_t)p->parts);
  p->off_local = o;   o = align256(o + sizeof(uint32_t) * ng);
  p->off_partial = o; o = align256(o + sizeof(unsigned long long) * (size_t)(p->count_blocks + 1));
  p->off_rects = o;   o = align256(o + sizeof(uint4) * ng);
  p->off_owner = o;   o = align256(o + sizeof(uint32_t) * (size_t)(div_up64(capacity, kEmitTileHost) + 1));
  p->off_tsum = o;    o = align256(o + sizeof(unsigned long long) * (size_t)(p->tile_blocks + 1));
  p->off_keys0 = o;   o = align256(o + sizeof(unsigned long long) * (size_t)capacity);
  p->off_keys1 = o;   o = align256(o + sizeof(unsigned long long) * (size_t)capacity);
  p->bytes = o;
  return BS_OK;
}

void fill_batch_table(const bs_batch_image *images, const BatchPlan &p, BatchImage *out) {
  int64_t open0 = 0, closed0 = 0, gauss0 = 0, pix0 = 0, tile0 = 0, diff0 = 0, row0 = 0, col0 = 0, order0 = 0;
  for (int b = 0; b < p.n_images; ++b) {
    const bs_batch_image &im = images[b];
    BatchImage &e = out[b];
    e = BatchImage{};
    e.W = im.width;
    e.H = im.height;
    e.tiles_x = div_up(im.width, p.tile);
    e.tiles_y = div_up(im.height, p.tile);
    e.n_open = im.n_open;
    e.n_closed = im.n_closed;
    e.g_open = im.sample.g_open;
    e.rows = im.sample.rows_closed;
    e.kc = im.sample.k_closed;
    e.rho = im.sample.rho;
    e.eps = im.sample.cov_eps;
    e.tmode = im.sample.tangent_mode;
    for (int c = 0; c < 3; ++c) e.bg[c] = im.bg[c];
    e.l2_scale = (float)(2.0 / (3.0 * (double)im.width * (double)im.height));
    const int64_t nc = (int64_t)im.n_open + im.n_closed;
    e.order_chunks = (int)div_up64(nc, kOrderChunkHost);
    e.open0 = open0;
    e.closed0 = closed0;
    e.gauss0 = gauss0;
    e.n_gauss = (int64_t)im.n_open * im.sample.g_open + (int64_t)im.n_closed * im.sample.rows_closed * im.sample.k_closed;
    e.pix0 = pix0;
    e.tile0 = tile0;
    e.diff0 = diff0;
    e.row0 = row0;
    e.col0 = col0;
    e.order0 = order0;
    open0 += im.n_open;
    closed0 += im.n_closed;
    gauss0 += e.n_gauss;
    pix0 += (int64_t)im.width * im.height;
    tile0 += (int64_t)e.tiles_x * e.tiles_y;
    diff0 += (int64_t)(e.tiles_x + 1) * (e.tiles_y + 1);
    row0 += e.tiles_y + 1;
    col0 += e.tiles_x + 1;
    order0 += (int64_t)e.order_chunks * e.order_chunks;
  }
}

void fill_curve_classes(const bs_batch_image *images, const BatchPlan &p, int32_t *out) {
  // curve indices: the open curves of all images, then the closed ones
  int64_t narrow = 0, wide = p.narrow.n_curves, open0 = 0, closed0 = p.n_open;
  for (int b = 0; b < p.n_images; ++b) {
    const bs_batch_image &im = images[b];
    const bool ow = im.sample.g_open >= kWideSamples;
    const bool cw = im.sample.rows_closed * im.sample.k_closed >= kWideSamples;
    for (int i = 0; i < im.n_open; ++i) out[ow ? wide++ : narrow++] = (int32_t)(open0 + i);
    for (int i = 0; i < im.n_closed; ++i) out[cw ? wide++ : narrow++] = (int32_t)(closed0 + i);
    open0 += im.n_open;
    closed0 += im.n_closed;
  }
}

// ---- Adam (Kingma and Ba, Algorithm 1), projected onto a box ----
namespace {

struct AdamArgs {
  bs_adam_group g[BS_ADAM_MAX_GROUPS];
  int64_t start[BS_ADAM_MAX_GROUPS + 1];  // prefix sums of the group sizes
  int n_groups;
};

// One thread per parameter (grid-stride); t = *step + 1 is read once per
// CTA, and step_advance_kernel writes it back after this kernel.
__global__ void __launch_bounds__(256) adam_kernel(const AdamArgs a, const bs_adam_cfg cfg,
                                                   const int32_t *__restrict__ step) {
  // the bias corrections 1 - beta^t, once per CTA (FP64 is slow here)
  __shared__ float s_bc[2];
  if (threadIdx.x == 0) {
    const int t = *step + 1;
    s_bc[0] = (float)(1.0 - pow((double)cfg.beta1, (double)t));
    s_bc[1] = (float)(1.0 - pow((double)cfg.beta2, (double)t));
  }
  __syncthreads();
  const float bc1 = s_bc[0], bc2 = s_bc[1];
  const int64_t total = a.start[a.n_groups];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    int k = 0;
    while (idx >= a.start[k + 1]) ++k;
    const bs_adam_group &G = a.g[k];
    const int64_t i = idx - a.start[k];
    const float g = G.grad[i];
    const float m = cfg.beta1 * G.m[i] + (1.f - cfg.beta1) * g;
    const float v = cfg.beta2 * G.v[i] + (1.f - cfg.beta2) * (g * g);
    G.m[i] = m;
    G.v[i] = v;
    const float lr = G.row_scale ? G.lr * G.row_scale[i / G.row_len] : G.lr;
    const float mh = m / bc1, vh = v / bc2;
    const float p = G.param[i] - lr * mh / (sqrtf(vh) + cfg.eps);
    G.param[i] = fminf(fmaxf(p, G.lo), G.hi);
  }
}

__global__ void step_advance_kernel(int32_t *step) { *step += 1; }

}  // namespace

bs_status launch_adam(const bs_adam_group *groups, int n_groups, const bs_adam_cfg &cfg, int32_t *step,
                      cudaStream_t s) {
  AdamArgs a{};
  a.n_groups = n_groups;
  a.start[0] = 0;
  for (int k = 0; k < n_groups; ++k) {
    a.g[k] = groups[k];
    a.start[k + 1] = a.start[k] + groups[k].n;
  }
  for (int k = n_groups; k < BS_ADAM_MAX_GROUPS; ++k) a.start[k + 1] = a.start[n_groups];
  const int64_t total = a.start[n_groups];
  if (total > 0) {
    const int blocks = (int)std::min<int64_t>(div_up64(total, 256), 152 * 16);
    adam_kernel<<<blocks, 256, 0, s>>>(a, cfg, step);
    BS_LAUNCHED("adam_kernel");
  }
  step_advance_kernel<<<1, 1, 0, s>>>(step);
  BS_LAUNCHED("step_advance_kernel");
  return BS_OK;
}

}  // namespace bs
