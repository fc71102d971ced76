// The C ABI of libbs.so: argument validation on the host, then the launchers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <string.h>

#include <string>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

namespace {
thread_local std::string g_last_error;
}

const char *last_error_cstr() { return g_last_error.c_str(); }

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

bs_status cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return BS_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return BS_ERR_CUDA;
}

// sm_103 only; checked once per device.
bs_status check_device() {
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  static int checked[64] = {0};  // 0 unknown, 1 ok, 2 unsupported
  if (dev >= 0 && dev < 64 && checked[dev] == 1) return BS_OK;
  int major = 0, minor = 0;
  BS_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  BS_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  const bool ok = major == 10 && minor == 3;
  if (dev >= 0 && dev < 64) checked[dev] = ok ? 1 : 2;
  if (!ok) {
    set_error("device %d is sm_%d%d; this library is built for sm_103a only", dev, major, minor);
    return BS_ERR_UNSUPPORTED;
  }
  return BS_OK;
}

void debug_set_retry_limit(int64_t max_attempts);
const char *last_error_cstr();

// The library's own status word on each device (kDevErrNotFinite); its
// device address is looked up once per device with that device current.
namespace {
__device__ uint32_t g_lib_status;
constexpr int kMaxStatusDevices = 64;
uint32_t *g_lib_status_ptr[kMaxStatusDevices] = {};
cudaError_t g_lib_status_err[kMaxStatusDevices] = {};
std::once_flag g_lib_status_once[kMaxStatusDevices];
}  // namespace

bs_status lib_status_word(uint32_t **ptr) {
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxStatusDevices) {
    set_error("device %d: at most %d devices supported", dev, kMaxStatusDevices);
    return BS_ERR_UNSUPPORTED;
  }
  std::call_once(g_lib_status_once[dev], [dev] {
    void *p = nullptr;
    g_lib_status_err[dev] = cudaGetSymbolAddress(&p, g_lib_status);
    g_lib_status_ptr[dev] = static_cast<uint32_t *>(p);
  });
  BS_CUDA(g_lib_status_err[dev]);
  *ptr = g_lib_status_ptr[dev];
  return BS_OK;
}

}  // namespace bs

using namespace bs;

namespace {

bs_status invalid(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_error("%s", buf);
  return BS_ERR_INVALID_ARG;
}

bs_status check_cfg(const bs_sample_cfg *cfg) {
  if (!cfg) return invalid("cfg is NULL");
  if (cfg->g_open < 2 || cfg->g_open > 1024) return invalid("g_open %d not in [2, 1024]", cfg->g_open);
  if (cfg->rows_closed < 2 || cfg->k_closed < 2) return invalid("rows_closed and k_closed must be >= 2");
  if ((int64_t)cfg->rows_closed * cfg->k_closed > kMaxSamplesPerCurve)
    return invalid("rows_closed * k_closed > %d", kMaxSamplesPerCurve);
  if (cfg->tangent_mode != 0 && cfg->tangent_mode != 1) return invalid("tangent_mode %d not 0 or 1", cfg->tangent_mode);
  if (!(cfg->rho > 0.f)) return invalid("rho must be > 0");
  if (!(cfg->cov_eps >= 0.f)) return invalid("cov_eps must be >= 0");
  return BS_OK;
}

bs_status check_curves(const bs_curves *c, bool need_first) {
  if (!c) return invalid("curves is NULL");
  if (c->n_open < 0 || c->n_closed < 0) return invalid("negative curve count");
  if (c->n_open > 0 && (!c->open_ctrl || !c->open_width || !c->open_color || !c->open_opac))
    return invalid("open curve arrays must be non-NULL when n_open > 0");
  if (c->n_closed > 0 && (!c->closed_ctrl || !c->closed_color || !c->closed_opac))
    return invalid("closed curve arrays must be non-NULL when n_closed > 0");
  if (need_first && c->n_open + c->n_closed > 0 && !c->draw_first) return invalid("draw_first is NULL");
  if ((int64_t)c->n_open + c->n_closed > (1 << 30)) return invalid("too many curves");
  return BS_OK;
}

bs_status check_canvas(const bs_canvas *cv) {
  if (!cv) return invalid("canvas is NULL");
  if (cv->width < 1 || cv->height < 1 || cv->width > 32768 || cv->height > 32768)
    return invalid("canvas %dx%d out of range", cv->width, cv->height);
  if (cv->tile != 8 && cv->tile != 16 && cv->tile != 32) {
    set_error("tile side %d not supported (8, 16, 32)", cv->tile);
    return BS_ERR_UNSUPPORTED;
  }
  return BS_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ---- SVG export (Appendix C, Algorithm 2) ----
// Numbers with 9 significant digits (a float32 reads back exactly); colours
// rgb(round(255 c)) of the colour clamped to [0, 1].
void svg_num(std::string &s, float v) {
  char b[32];
  snprintf(b, sizeof(b), "%.9g", (double)v);
  s += b;
}

void svg_pt(std::string &s, const float *p) {
  svg_num(s, p[0]);
  s += ' ';
  svg_num(s, p[1]);
}

void svg_rgb(std::string &s, const float *c) {
  char b[48];
  int v[3];
  for (int i = 0; i < 3; ++i) {
    const float x = c[i] < 0.f ? 0.f : (c[i] > 1.f ? 1.f : c[i]);
    v[i] = (int)lrintf(255.f * x);
  }
  snprintf(b, sizeof(b), "rgb(%d,%d,%d)", v[0], v[1], v[2]);
  s += b;
}

// The document: curves back to front (descending draw rank when rank is
// given, else in index order, open curves first).  Closed curve: "M P0 C P1
// P2 P3 C P4 P5 P6 C P7 P8 P9 C P10 P11 P0 Z" filled with its colour, at
// opacity 1 as in Algorithm 2 (flag 1: its own opacity); with a gradient
// fill a linearGradient from P0 to P6 (user space) with the two colours and
// opacities as stops.  Open curve: "M P0 C P1 P2 P3 C P4 P5 P6 C P7 P8 P9",
// unfilled, stroked with its colour, width 2 w and the mean of its three
// segment opacities.
bs_status svg_document(const bs_curves &c, const uint32_t *rank, int width, int height, int flags,
                       std::string *out) {
  const int n = c.n_open + c.n_closed;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  if (rank) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rank[a] > rank[b]; });
  std::string &s = *out;
  char b[256];
  snprintf(b, sizeof(b),
           "<svg xmlns=\"http://www.w3.org/2000/svg\" width=\"%d\" height=\"%d\" viewBox=\"0 0 %d %d\">\n", width,
           height, width, height);
  s += b;
  const bool grad = c.closed_color2 || c.closed_opac2;
  if (grad && c.n_closed > 0) {
    s += "<defs>\n";
    for (int j = 0; j < c.n_closed; ++j) {
      const float *P = c.closed_ctrl + (size_t)j * 24;
      const float *c0 = c.closed_color + (size_t)j * 3;
      const float *c1 = c.closed_color2 ? c.closed_color2 + (size_t)j * 3 : c0;
      const float o0 = c.closed_opac[j], o1 = c.closed_opac2 ? c.closed_opac2[j] : o0;
      snprintf(b, sizeof(b), "<linearGradient id=\"f%d\" gradientUnits=\"userSpaceOnUse\" x1=\"", j);
      s += b;
      svg_num(s, P[0]);
      s += "\" y1=\"";
      svg_num(s, P[1]);
      s += "\" x2=\"";
      svg_num(s, P[12]);
      s += "\" y2=\"";
      svg_num(s, P[13]);
      s += "\"><stop offset=\"0\" stop-color=\"";
      svg_rgb(s, c0);
      s += "\" stop-opacity=\"";
      svg_num(s, (flags & 1) ? o0 : 1.f);
      s += "\"/><stop offset=\"1\" stop-color=\"";
      svg_rgb(s, c1);
      s += "\" stop-opacity=\"";
      svg_num(s, (flags & 1) ? o1 : 1.f);
      s += "\"/></linearGradient>\n";
    }
    s += "</defs>\n";
  }
  for (int idx : order) {
    if (idx < c.n_open) {
      const float *P = c.open_ctrl + (size_t)idx * 20;
      s += "<path d=\"M ";
      svg_pt(s, P);
      for (int seg = 0; seg < 3; ++seg) {
        s += " C ";
        svg_pt(s, P + 2 * (3 * seg + 1));
        s += ' ';
        svg_pt(s, P + 2 * (3 * seg + 2));
        s += ' ';
        svg_pt(s, P + 2 * (3 * seg + 3));
      }
      s += "\" fill=\"none\" stroke=\"";
      svg_rgb(s, c.open_color + (size_t)idx * 3);
      s += "\" stroke-width=\"";
      svg_num(s, 2.f * c.open_width[idx]);
      const float *o = c.open_opac + (size_t)idx * 3;
      s += "\" stroke-opacity=\"";
      svg_num(s, ((o[0] + o[1]) + o[2]) / 3.f);
      s += "\" stroke-linecap=\"round\"/>\n";
    } else {
      const int j = idx - c.n_open;
      const float *P = c.closed_ctrl + (size_t)j * 24;
      s += "<path d=\"M ";
      svg_pt(s, P);
      for (int seg = 0; seg < 4; ++seg) {
        s += " C ";
        svg_pt(s, P + 2 * (3 * seg + 1));
        s += ' ';
        svg_pt(s, P + 2 * (3 * seg + 2));
        s += ' ';
        svg_pt(s, P + 2 * ((3 * seg + 3) % 12));
      }
      s += " Z\" fill=\"";
      if (grad) {
        snprintf(b, sizeof(b), "url(#f%d)", j);
        s += b;
        s += "\"/>\n";
      } else {
        svg_rgb(s, c.closed_color + (size_t)j * 3);
        s += "\" fill-opacity=\"";
        svg_num(s, (flags & 1) ? c.closed_opac[j] : 1.f);
        s += "\"/>\n";
      }
    }
  }
  s += "</svg>\n";
  return BS_OK;
}

bs_status check_pd_counts(int32_t n_open, int32_t n_closed) {
  if (n_open < 0 || n_closed < 0) return invalid("negative curve count");
  if ((int64_t)n_open + n_closed > kMaxPdCurves) return invalid("more than %d curves", kMaxPdCurves);
  return BS_OK;
}

bs_status check_pd_cfg(const bs_pd_cfg *cfg) {
  if (!cfg) return invalid("cfg is NULL");
  if (cfg->step < 0 || cfg->t_end < 1) return invalid("step must be >= 0 and t_end >= 1");
  const float v[] = {cfg->op_start, cfg->op_end, cfg->area_min, cfg->color_eps, cfg->iou_min,
                     cfg->err_thresh, cfg->split_drop, cfg->new_opacity, cfg->new_width};
  for (float x : v)
    if (!isfinite(x)) return invalid("prune/densify thresholds must be finite");
  if (!(cfg->new_opacity >= 0.f && cfg->new_opacity <= 1.f)) return invalid("new_opacity not in [0, 1]");
  if (!(cfg->new_width > 0.f)) return invalid("new_width must be > 0");
  return BS_OK;
}

// The plan of a batch, with every image's sampling validated.
bs_status batch_plan(const bs_batch *b, BatchPlan *p) {
  if (!b) return invalid("batch is NULL");
  if (!b->images || b->n_images < 1) return invalid("a batch needs a host array of at least one image");
  for (int i = 0; i < b->n_images; ++i) {
    const bs_status st = check_cfg(&b->images[i].sample);
    if (st != BS_OK) {
      const std::string msg = last_error_cstr();
      return invalid("image %d: %s", i, msg.c_str());
    }
  }
  return plan_batch(b->images, b->n_images, b->tile, b->pair_capacity, p);
}

// The plan, and a workspace large enough for it.
bs_status batch_plan_ws(const bs_batch *b, BatchPlan *p) {
  BS_TRY(batch_plan(b, p));
  if (!b->ws || b->ws_bytes < p->bytes || ((uintptr_t)b->ws & 255u))
    return invalid("batch workspace needs %zu bytes (256-byte aligned), got %zu", p->bytes, b->ws_bytes);
  return BS_OK;
}

bs_status check_batch_curves(const bs_curves *c, const BatchPlan &p, bool need_first) {
  BS_TRY(check_curves(c, need_first));
  if (c->n_open != p.n_open || c->n_closed != p.n_closed)
    return invalid("curves hold %d open + %d closed curves, the batch %lld + %lld", c->n_open, c->n_closed,
                   (long long)p.n_open, (long long)p.n_closed);
  return BS_OK;
}

const BatchImage *batch_table_of(const bs_batch *b, const BatchPlan &p) {
  return reinterpret_cast<const BatchImage *>(static_cast<const char *>(b->ws) + p.off_images);
}

const int32_t *batch_curve_ids_of(const bs_batch *b, const BatchPlan &p) {
  return reinterpret_cast<const int32_t *>(static_cast<const char *>(b->ws) + p.off_curve_ids);
}

}  // namespace

extern "C" {

int64_t bs_num_gaussians(int32_t n_open, int32_t n_closed, const bs_sample_cfg *cfg) {
  if (n_open < 0 || n_closed < 0 || check_cfg(cfg) != BS_OK) return -1;
  return (int64_t)n_open * cfg->g_open + (int64_t)n_closed * cfg->rows_closed * cfg->k_closed;
}

bs_status bs_curve_order(const bs_curves *curves, const bs_sample_cfg *cfg, uint32_t *rank_out,
                         uint32_t *first_out, bs_stream stream) {
  BS_TRY(check_curves(curves, false));
  BS_TRY(check_cfg(cfg));
  const int64_t n = (int64_t)curves->n_open + curves->n_closed;
  if (n > 0 && (!rank_out || !first_out)) return invalid("rank_out/first_out is NULL");
  if (bs_num_gaussians(curves->n_open, curves->n_closed, cfg) > (1ll << 31) - 1)
    return invalid("too many Gaussians");
  BS_TRY(check_device());
  return launch_curve_order(*curves, *cfg, rank_out, first_out, (cudaStream_t)stream);
}

bs_status bs_sample_curves(const bs_curves *curves, const bs_sample_cfg *cfg, float *gauss, bs_stream stream) {
  BS_TRY(check_curves(curves, true));
  BS_TRY(check_cfg(cfg));
  const int64_t ng = bs_num_gaussians(curves->n_open, curves->n_closed, cfg);
  if (ng > (1ll << 31) - 1) return invalid("too many Gaussians");
  if (ng > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  BS_TRY(check_device());
  return launch_sample_fwd(*curves, *cfg, gauss, (cudaStream_t)stream);
}

bs_status bs_sample_curves_bwd(const bs_curves *curves, const bs_sample_cfg *cfg, const float *dgauss,
                               const bs_curves_grad *grad, bs_stream stream) {
  BS_TRY(check_curves(curves, true));
  BS_TRY(check_cfg(cfg));
  if (!grad) return invalid("grad is NULL");
  if (curves->n_open > 0 && (!grad->open_ctrl || !grad->open_width || !grad->open_color || !grad->open_opac))
    return invalid("open gradient arrays must be non-NULL");
  if (curves->n_closed > 0 && (!grad->closed_ctrl || !grad->closed_color || !grad->closed_opac))
    return invalid("closed gradient arrays must be non-NULL");
  const int64_t ng = bs_num_gaussians(curves->n_open, curves->n_closed, cfg);
  if (ng > 0 && (!dgauss || !aligned16(dgauss))) return invalid("dgauss must be a 16-byte aligned device pointer");
  BS_TRY(check_device());
  return launch_sample_bwd(*curves, *cfg, dgauss, *grad, (cudaStream_t)stream);
}

bs_status bs_bin_tiles_workspace(int64_t n_gauss, const bs_canvas *canvas, int64_t pair_capacity, size_t *bytes) {
  BS_TRY(check_canvas(canvas));
  if (!bytes) return invalid("bytes is NULL");
  BinPlan p;
  BS_TRY(plan_binning(n_gauss, *canvas, pair_capacity, &p));
  *bytes = p.bytes;
  return BS_OK;
}

bs_status bs_bin_tiles(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, void *ws, size_t ws_bytes,
                       int64_t pair_capacity, int64_t *n_pairs_out, uint32_t *tile_keys, uint32_t *tile_ranges,
                       bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (!n_pairs_out) return invalid("n_pairs_out is NULL");
  *n_pairs_out = 0;
  BinPlan p;
  BS_TRY(plan_binning(n_gauss, *canvas, pair_capacity, &p));
  if (!ws || ws_bytes < p.bytes || !aligned16(ws))
    return invalid("workspace needs %zu bytes (16-byte aligned), got %zu", p.bytes, ws_bytes);
  if (n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_ranges || !aligned16(tile_ranges)) return invalid("tile_ranges must be an 8-byte aligned device pointer");
  if (pair_capacity > 0 && !tile_keys) return invalid("tile_keys is NULL");
  BS_TRY(check_device());
  return run_binning(p, gauss, *canvas, ws, n_pairs_out, tile_keys, tile_ranges, (cudaStream_t)stream);
}

bs_status bs_bin_tiles_async(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, void *ws, size_t ws_bytes,
                             int64_t pair_capacity, int64_t *n_pairs_dev, uint32_t *tile_keys, uint32_t *tile_ranges,
                             bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (pair_capacity < 1) return invalid("pair_capacity must be >= 1");
  BinPlan p;
  BS_TRY(plan_binning(n_gauss, *canvas, pair_capacity, &p));
  if (!ws || ws_bytes < p.bytes || !aligned16(ws))
    return invalid("workspace needs %zu bytes (16-byte aligned), got %zu", p.bytes, ws_bytes);
  if (n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_ranges || !aligned16(tile_ranges)) return invalid("tile_ranges must be an 8-byte aligned device pointer");
  if (!tile_keys) return invalid("tile_keys is NULL");
  if (n_pairs_dev && (reinterpret_cast<uintptr_t>(n_pairs_dev) & 7u))
    return invalid("n_pairs_dev must be 8-byte aligned");
  BS_TRY(check_device());
  int64_t unused = 0;
  return run_binning(p, gauss, *canvas, ws, &unused, tile_keys, tile_ranges, (cudaStream_t)stream, false,
                     n_pairs_dev);
}

bs_status bs_bin_tiles_result(const void *ws, size_t ws_bytes, int32_t *status_out, int64_t *n_pairs_out,
                              bs_stream stream) {
  if (!ws || !status_out) return invalid("NULL pointer");
  return read_device_status(ws, ws_bytes, status_out, (cudaStream_t)stream, n_pairs_out);
}

bs_status bs_bin_tiles_static(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, int64_t pair_capacity,
                              int64_t *n_pairs_out, uint32_t *tile_keys, uint32_t *tile_ranges, bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (!n_pairs_out) return invalid("n_pairs_out is NULL");
  *n_pairs_out = 0;
  BinPlan p;
  BS_TRY(plan_binning(n_gauss, *canvas, pair_capacity, &p, false));
  if (p.bytes > kStaticScratchBytes)
    return invalid("this binning needs %zu bytes of scratch; the fixed scratch of bs_bin_tiles_static holds %zu "
                   "(lower pair_capacity or n_gauss, or use bs_bin_tiles with a workspace)",
                   p.bytes, kStaticScratchBytes);
  if (n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_ranges || !aligned16(tile_ranges)) return invalid("tile_ranges must be an 8-byte aligned device pointer");
  if (pair_capacity > 0 && !tile_keys) return invalid("tile_keys is NULL");
  BS_TRY(check_device());
  void *ws = nullptr;
  BS_TRY(static_scratch(&ws));
  return run_binning(p, gauss, *canvas, ws, n_pairs_out, tile_keys, tile_ranges, (cudaStream_t)stream);
}

bs_status bs_render_fwd(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, const uint32_t *tile_keys,
                        const uint32_t *tile_ranges, float *img, float *T_final, uint32_t *n_contrib,
                        bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (n_gauss < 0 || n_gauss > (1ll << 31) - 1) return invalid("n_gauss out of range");
  if (n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_ranges || !img || !T_final || !n_contrib) return invalid("NULL output or tile_ranges");
  BS_TRY(check_device());
  return launch_render_fwd(gauss, n_gauss, *canvas, key_gbits(n_gauss, *canvas), tile_keys, tile_ranges, img, T_final, n_contrib,
                           (cudaStream_t)stream);
}

bs_status bs_render_fwd_l2(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, const uint32_t *tile_keys,
                           const uint32_t *tile_ranges, const float *target, float *img, float *T_final,
                           uint32_t *n_contrib, float *dL_dimg, double *loss_out, bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (n_gauss < 0 || n_gauss > (1ll << 31) - 1) return invalid("n_gauss out of range");
  if (n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_ranges || !img || !T_final || !n_contrib) return invalid("NULL output or tile_ranges");
  if (!target || !dL_dimg || !loss_out) return invalid("target, dL_dimg and loss_out must be non-NULL");
  BS_TRY(check_device());
  return launch_render_fwd_l2(gauss, n_gauss, *canvas, key_gbits(n_gauss, *canvas), tile_keys, tile_ranges, target, img,
                              T_final, n_contrib, dL_dimg, loss_out, (cudaStream_t)stream);
}

bs_status bs_render_stats(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, const uint32_t *tile_keys,
                          const uint32_t *tile_ranges, float *img, float *T_final, uint32_t *n_contrib,
                          unsigned long long *stats_out, bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (n_gauss < 0 || n_gauss > (1ll << 31) - 1) return invalid("n_gauss out of range");
  if (n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_ranges || !img || !T_final || !n_contrib || !stats_out) return invalid("NULL output or tile_ranges");
  BS_TRY(check_device());
  return launch_render_fwd(gauss, n_gauss, *canvas, key_gbits(n_gauss, *canvas), tile_keys, tile_ranges, img, T_final,
                           n_contrib, (cudaStream_t)stream, stats_out);
}

bs_status bs_l2_loss_grad(const float *img, const float *target, int64_t n, float *dL_dimg, double *loss_out,
                          bs_stream stream) {
  if (n < 0) return invalid("n < 0");
  if (!loss_out || (n > 0 && (!img || !target || !dL_dimg))) return invalid("NULL pointer");
  BS_TRY(check_device());
  return launch_l2(img, target, n, dL_dimg, loss_out, (cudaStream_t)stream);
}

bs_status bs_render_bwd(const float *gauss, int64_t n_gauss, const bs_canvas *canvas, const uint32_t *tile_keys,
                        const uint32_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                        const float *dL_dimg, float *dgauss, const bs_curves *curves, const bs_sample_cfg *cfg,
                        const bs_curves_grad *grad, bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (n_gauss < 0 || n_gauss > (1ll << 31) - 1) return invalid("n_gauss out of range");
  if (n_gauss > 0 && (!gauss || !aligned16(gauss) || !dgauss || !aligned16(dgauss)))
    return invalid("gauss/dgauss must be 16-byte aligned device pointers");
  if (!tile_ranges || !T_final || !n_contrib || !dL_dimg) return invalid("NULL input");
  if (grad) {
    BS_TRY(check_curves(curves, true));
    BS_TRY(check_cfg(cfg));
    if (bs_num_gaussians(curves->n_open, curves->n_closed, cfg) != n_gauss)
      return invalid("n_gauss does not match the curves and cfg");
  }
  BS_TRY(check_device());
  const cudaStream_t s = (cudaStream_t)stream;
  if (n_gauss > 0)
    BS_TRY(launch_render_bwd(gauss, n_gauss, *canvas, key_gbits(n_gauss, *canvas), tile_keys, tile_ranges, T_final,
                             n_contrib, dL_dimg, dgauss, s));
  if (grad) return bs_sample_curves_bwd(curves, cfg, dgauss, grad, stream);
  return BS_OK;
}

bs_status bs_batch_plan(const bs_batch *batch, bs_batch_sizes *out) {
  if (!out) return invalid("out is NULL");
  BatchPlan p;
  BS_TRY(batch_plan(batch, &p));
  out->n_open = p.n_open;
  out->n_closed = p.n_closed;
  out->n_gauss = p.n_gauss;
  out->n_pixels = p.n_pix;
  out->n_tiles = p.n_tiles;
  out->ws_bytes = p.bytes;
  return BS_OK;
}

bs_status bs_batch_setup(const bs_batch *batch, bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  BS_TRY(check_device());
  std::vector<BatchImage> tab((size_t)p.n_images);
  fill_batch_table(batch->images, p, tab.data());
  std::vector<int32_t> ids((size_t)p.n_curves);
  fill_curve_classes(batch->images, p, ids.data());
  const cudaStream_t s = (cudaStream_t)stream;
  BS_CUDA(cudaMemcpyAsync(static_cast<char *>(batch->ws) + p.off_images, tab.data(), sizeof(BatchImage) * tab.size(),
                          cudaMemcpyHostToDevice, s));
  if (!ids.empty())
    BS_CUDA(cudaMemcpyAsync(static_cast<char *>(batch->ws) + p.off_curve_ids, ids.data(), sizeof(int32_t) * ids.size(),
                            cudaMemcpyHostToDevice, s));
  BS_CUDA(cudaStreamSynchronize(s));
  return BS_OK;
}

bs_status bs_batch_curve_order(const bs_batch *batch, const bs_curves *curves, uint32_t *rank_out,
                               uint32_t *first_out, bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  BS_TRY(check_batch_curves(curves, p, false));
  if (p.n_curves > 0 && (!rank_out || !first_out)) return invalid("rank_out/first_out is NULL");
  BS_TRY(check_device());
  return launch_batch_curve_order(p, batch_table_of(batch, p), *curves, rank_out, first_out, (cudaStream_t)stream);
}

bs_status bs_batch_sample_curves(const bs_batch *batch, const bs_curves *curves, float *gauss, bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  BS_TRY(check_batch_curves(curves, p, true));
  if (p.n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  BS_TRY(check_device());
  return launch_batch_sample_fwd(p, batch_table_of(batch, p), batch_curve_ids_of(batch, p), *curves, gauss,
                                 (cudaStream_t)stream);
}

bs_status bs_batch_bin_tiles(const bs_batch *batch, const float *gauss, uint32_t *tile_vals, uint32_t *tile_ranges,
                             bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  if (p.n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_vals || !tile_ranges || !aligned16(tile_ranges))
    return invalid("tile_vals and tile_ranges (8-byte aligned) must be device pointers");
  BS_TRY(check_device());
  return run_batch_binning(p, batch->ws, gauss, tile_vals, tile_ranges, (cudaStream_t)stream);
}

bs_status bs_batch_render_fwd(const bs_batch *batch, const float *gauss, const uint32_t *tile_vals,
                              const uint32_t *tile_ranges, const float *target, float *img, float *T_final,
                              uint32_t *n_contrib, float *dL_dimg, double *loss_out, bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  if (p.n_gauss > 0 && (!gauss || !aligned16(gauss))) return invalid("gauss must be a 16-byte aligned device pointer");
  if (!tile_vals || !tile_ranges || !img || !T_final || !n_contrib) return invalid("NULL input or output");
  if (target && (!dL_dimg || !loss_out)) return invalid("with a target, dL_dimg and loss_out must be non-NULL");
  BS_TRY(check_device());
  return launch_batch_render_fwd(p, batch->ws, gauss, tile_vals, tile_ranges, target, img, T_final, n_contrib,
                                 dL_dimg, loss_out, (cudaStream_t)stream);
}

bs_status bs_batch_render_bwd(const bs_batch *batch, const float *gauss, const uint32_t *tile_vals,
                              const uint32_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                              const float *dL_dimg, float *dgauss, const bs_curves *curves,
                              const bs_curves_grad *grad, bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  if (p.n_gauss > 0 && (!gauss || !aligned16(gauss) || !dgauss || !aligned16(dgauss)))
    return invalid("gauss/dgauss must be 16-byte aligned device pointers");
  if (!tile_vals || !tile_ranges || !T_final || !n_contrib || !dL_dimg) return invalid("NULL input");
  if (grad) {
    BS_TRY(check_batch_curves(curves, p, true));
    if (p.n_open > 0 && (!grad->open_ctrl || !grad->open_width || !grad->open_color || !grad->open_opac))
      return invalid("open gradient arrays must be non-NULL");
    if (p.n_closed > 0 && (!grad->closed_ctrl || !grad->closed_color || !grad->closed_opac))
      return invalid("closed gradient arrays must be non-NULL");
  }
  BS_TRY(check_device());
  const cudaStream_t s = (cudaStream_t)stream;
  BS_TRY(launch_batch_render_bwd(p, batch->ws, gauss, tile_vals, tile_ranges, T_final, n_contrib, dL_dimg, dgauss,
                                 s));
  if (grad) return launch_batch_sample_bwd(p, batch_table_of(batch, p), batch_curve_ids_of(batch, p), *curves, dgauss,
                                           *grad, s);
  return BS_OK;
}

bs_status bs_batch_status(const bs_batch *batch, int32_t *status_out, int64_t *n_pairs_out, bs_stream stream) {
  BatchPlan p;
  BS_TRY(batch_plan_ws(batch, &p));
  if (!status_out) return invalid("status_out is NULL");
  return read_batch_status(p, batch->ws, status_out, n_pairs_out, (cudaStream_t)stream);
}

bs_status bs_adam_step(const bs_adam_group *groups, int32_t n_groups, const bs_adam_cfg *cfg, int32_t *step,
                       bs_stream stream) {
  if (!groups || n_groups < 1 || n_groups > BS_ADAM_MAX_GROUPS)
    return invalid("1 <= n_groups <= %d host groups needed", BS_ADAM_MAX_GROUPS);
  if (!cfg || !step) return invalid("cfg and step must be non-NULL");
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
    return invalid("betas must be in [0, 1) and eps > 0");
  for (int k = 0; k < n_groups; ++k) {
    const bs_adam_group &g = groups[k];
    if (g.n < 0) return invalid("group %d: n < 0", k);
    if (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v)) return invalid("group %d: NULL array", k);
    if (!(g.lr >= 0.f) || !(g.lo <= g.hi)) return invalid("group %d: lr must be >= 0 and lo <= hi", k);
    if (g.row_scale && g.row_len < 1) return invalid("group %d: row_len must be >= 1", k);
  }
  BS_TRY(check_device());
  return launch_adam(groups, n_groups, *cfg, step, (cudaStream_t)stream);
}

bs_status bs_xing_loss(const bs_curves *curves, float lambda, double *loss_out, float *grad_closed_ctrl,
                       bs_stream stream) {
  BS_TRY(check_curves(curves, false));
  if (!loss_out) return invalid("loss_out is NULL");
  if (!(lambda >= 0.f) || !isfinite(lambda)) return invalid("lambda must be finite and >= 0");
  BS_TRY(check_device());
  return launch_xing(*curves, lambda, loss_out, grad_closed_ctrl, (cudaStream_t)stream);
}

bs_status bs_svg_export(const bs_curves *curves, const uint32_t *rank, int32_t width, int32_t height, int32_t flags,
                        char *buf, size_t buf_bytes, size_t *needed_out) {
  BS_TRY(check_curves(curves, false));
  if (width < 1 || height < 1) return invalid("canvas %dx%d out of range", width, height);
  if (!needed_out) return invalid("needed_out is NULL");
  std::string out;
  BS_TRY(svg_document(*curves, rank, width, height, flags, &out));
  *needed_out = out.size() + 1;
  if (buf) {
    if (buf_bytes < out.size() + 1) return invalid("buffer of %zu bytes, %zu needed", buf_bytes, out.size() + 1);
    memcpy(buf, out.c_str(), out.size() + 1);
  }
  return BS_OK;
}

bs_status bs_prune_densify_workspace(int32_t n_open, int32_t n_closed, const bs_canvas *canvas, size_t *bytes) {
  BS_TRY(check_canvas(canvas));
  BS_TRY(check_pd_counts(n_open, n_closed));
  if (!bytes) return invalid("bytes is NULL");
  *bytes = prune_densify_bytes(n_open, n_closed, canvas->width, canvas->height);
  return BS_OK;
}

bs_status bs_prune_densify(const bs_curves_mut *curves, const bs_pd_cfg *cfg, const bs_canvas *canvas,
                           const float *img, const float *target, void *ws, size_t ws_bytes, uint8_t *changed_out,
                           bs_pd_stats *stats_out, bs_stream stream) {
  BS_TRY(check_canvas(canvas));
  if (!curves) return invalid("curves is NULL");
  BS_TRY(check_pd_counts(curves->n_open, curves->n_closed));
  if (curves->n_open > 0 && (!curves->open_ctrl || !curves->open_width || !curves->open_color || !curves->open_opac))
    return invalid("open curve arrays must be non-NULL when n_open > 0");
  if (curves->n_closed > 0 && (!curves->closed_ctrl || !curves->closed_color || !curves->closed_opac))
    return invalid("closed curve arrays must be non-NULL when n_closed > 0");
  BS_TRY(check_pd_cfg(cfg));
  if (!img || !target) return invalid("img and target must be non-NULL");
  const size_t need = prune_densify_bytes(curves->n_open, curves->n_closed, canvas->width, canvas->height);
  if (!ws || ws_bytes < need || !aligned16(ws))
    return invalid("workspace of %zu bytes (16-byte aligned) needed, got %zu", need, ws_bytes);
  BS_TRY(check_device());
  return run_prune_densify(*curves, *cfg, canvas->width, canvas->height, img, target, ws, changed_out, stats_out,
                           (cudaStream_t)stream);
}

bs_status bs_device_status(const void *ws, size_t ws_bytes, int32_t *status_out, bs_stream stream) {
  if (!ws || !status_out) return invalid("NULL pointer");
  return read_device_status(ws, ws_bytes, status_out, (cudaStream_t)stream);
}

bs_status bs_sync_status(int32_t clear, int32_t *status_out, bs_stream stream) {
  if (!status_out) return invalid("status_out is NULL");
  BS_TRY(check_device());
  uint32_t *word = nullptr;
  BS_TRY(lib_status_word(&word));
  const cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  BS_CUDA(cudaMemcpyAsync(&h, word, sizeof(h), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  if (clear) BS_CUDA(cudaMemsetAsync(word, 0, sizeof(uint32_t), s));
  *status_out = (h & kDevErrNotFinite) ? BS_ERR_NOT_FINITE : BS_OK;
  return BS_OK;
}

bs_status bs_debug_retry_limit(int64_t max_attempts) {
  debug_set_retry_limit(max_attempts);
  return BS_OK;
}

const char *bs_last_error(void) { return last_error_cstr(); }

const char *bs_status_string(bs_status status) {
  switch (status) {
    case BS_OK: return "BS_OK";
    case BS_ERR_INVALID_ARG: return "BS_ERR_INVALID_ARG";
    case BS_ERR_CUDA: return "BS_ERR_CUDA";
    case BS_ERR_CAPACITY: return "BS_ERR_CAPACITY";
    case BS_ERR_TIMEOUT: return "BS_ERR_TIMEOUT";
    case BS_ERR_NOT_FINITE: return "BS_ERR_NOT_FINITE";
    case BS_ERR_UNSUPPORTED: return "BS_ERR_UNSUPPORTED";
  }
  return "BS_ERR_UNKNOWN";
}

}  // extern "C"
