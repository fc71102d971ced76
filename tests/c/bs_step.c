/*
 * One optimisation step of the rasterizer through the C ABI alone (bs.h and
 * the CUDA runtime; no Python): draw order, sampling, binning, blend with
 * the L2 loss, blend and sampling backward.  Test program of
 * tests/test_c_abi.py.
 *
 *   bs_step IN OUT
 * IN: int32 {W, H, tile, n_open, n_closed, g_open, rows_closed, k_closed,
 *     tangent_mode}, float {rho, cov_eps, bg[3]}, then float32 arrays
 *     open_ctrl [n_open][10][2], open_width [n_open], open_color [n_open][3],
 *     open_opac [n_open][3], closed_ctrl [n_closed][12][2],
 *     closed_color [n_closed][3], closed_opac [n_closed], target [3][H][W].
 * OUT: double loss, int64 n_pairs, float32 img [3][H][W], then the curve
 *     gradients in the order of the input arrays (without the target).
 * Exit status 0 on success; a failing call prints bs_last_error().
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "bs.h"

#define CHECK_BS(call)                                                              \
  do {                                                                              \
    bs_status st_ = (call);                                                         \
    if (st_ != BS_OK) {                                                             \
      fprintf(stderr, "%s failed (%d): %s\n", #call, (int)st_, bs_last_error());    \
      return 1;                                                                     \
    }                                                                               \
  } while (0)

#define CHECK_CUDA(call)                                                            \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));            \
      return 1;                                                                     \
    }                                                                               \
  } while (0)

static int read_exact(FILE *f, void *dst, size_t bytes) { return fread(dst, 1, bytes, f) == bytes ? 0 : 1; }

/* a device copy of n floats read from f */
static float *upload(FILE *f, size_t n, int *err) {
  float *host = (float *)malloc(n ? n * sizeof(float) : 1), *dev = NULL;
  if (!host || read_exact(f, host, n * sizeof(float)) ||
      cudaMalloc((void **)&dev, n ? n * sizeof(float) : 4) != cudaSuccess ||
      cudaMemcpy(dev, host, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    *err = 1;
  free(host);
  return dev;
}

static float *zeros(size_t n, int *err) {
  float *dev = NULL;
  if (cudaMalloc((void **)&dev, n ? n * sizeof(float) : 4) != cudaSuccess || cudaMemset(dev, 0, n * sizeof(float)))
    *err = 1;
  return dev;
}

static int download(FILE *f, const float *dev, size_t n) {
  float *host = (float *)malloc(n ? n * sizeof(float) : 1);
  int bad = !host || cudaMemcpy(host, dev, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
            fwrite(host, sizeof(float), n, f) != n;
  free(host);
  return bad;
}

int main(int argc, char **argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: bs_step IN OUT\n");
    return 2;
  }
  FILE *in = fopen(argv[1], "rb");
  if (!in) return 2;
  int32_t hdr[9];
  float fl[5];
  if (read_exact(in, hdr, sizeof(hdr)) || read_exact(in, fl, sizeof(fl))) return 2;
  const int W = hdr[0], H = hdr[1], no = hdr[3], nc = hdr[4];
  bs_sample_cfg cfg = {hdr[5], hdr[6], hdr[7], fl[0], fl[1], hdr[8]};
  bs_canvas canvas = {W, H, hdr[2], {fl[2], fl[3], fl[4]}};
  int err = 0;
  float *oc = upload(in, (size_t)no * 20, &err), *ow = upload(in, (size_t)no, &err);
  float *ocol = upload(in, (size_t)no * 3, &err), *oop = upload(in, (size_t)no * 3, &err);
  float *cc = upload(in, (size_t)nc * 24, &err), *ccol = upload(in, (size_t)nc * 3, &err);
  float *cop = upload(in, (size_t)nc, &err);
  const size_t npix = (size_t)W * H;
  float *target = upload(in, 3 * npix, &err);
  fclose(in);
  if (err) {
    fprintf(stderr, "reading or uploading the input failed\n");
    return 2;
  }

  const int64_t n_gauss = bs_num_gaussians(no, nc, &cfg);
  if (n_gauss < 0) return 2;
  uint32_t *rank = NULL, *first = NULL, *keys = NULL, *ranges = NULL, *nc_map = NULL;
  float *gauss = NULL, *dgauss = NULL, *img = NULL, *T = NULL, *dimg = NULL;
  double *loss_d = NULL;
  void *ws = NULL;
  const int tx = (W + canvas.tile - 1) / canvas.tile, ty = (H + canvas.tile - 1) / canvas.tile;
  CHECK_CUDA(cudaMalloc((void **)&rank, sizeof(uint32_t) * (no + nc + 1)));
  CHECK_CUDA(cudaMalloc((void **)&first, sizeof(uint32_t) * (no + nc + 1)));
  CHECK_CUDA(cudaMalloc((void **)&gauss, sizeof(float) * BS_GAUSS_FLOATS * (n_gauss + 1)));
  CHECK_CUDA(cudaMalloc((void **)&dgauss, sizeof(float) * BS_DGAUSS_FLOATS * (n_gauss + 1)));
  CHECK_CUDA(cudaMalloc((void **)&ranges, sizeof(uint32_t) * 2 * (size_t)tx * ty));
  CHECK_CUDA(cudaMalloc((void **)&img, sizeof(float) * 3 * npix));
  CHECK_CUDA(cudaMalloc((void **)&dimg, sizeof(float) * 3 * npix));
  CHECK_CUDA(cudaMalloc((void **)&T, sizeof(float) * npix));
  CHECK_CUDA(cudaMalloc((void **)&nc_map, sizeof(uint32_t) * npix));
  CHECK_CUDA(cudaMalloc((void **)&loss_d, sizeof(double)));

  bs_curves curves = {no, nc, oc, ow, ocol, oop, cc, ccol, cop, first, NULL, NULL};
  CHECK_BS(bs_curve_order(&curves, &cfg, rank, first, NULL));
  CHECK_BS(bs_sample_curves(&curves, &cfg, gauss, NULL));

  /* binning: a first capacity, grown once to the pairs reported */
  int64_t capacity = 4 * n_gauss + 1024, n_pairs = 0;
  bs_status st = BS_ERR_CAPACITY;
  for (int attempt = 0; attempt < 2 && st == BS_ERR_CAPACITY; ++attempt) {
    size_t ws_bytes = 0;
    CHECK_BS(bs_bin_tiles_workspace(n_gauss, &canvas, capacity, &ws_bytes));
    cudaFree(ws);
    cudaFree(keys);
    CHECK_CUDA(cudaMalloc(&ws, ws_bytes));
    CHECK_CUDA(cudaMalloc((void **)&keys, sizeof(uint32_t) * (size_t)capacity));
    st = bs_bin_tiles(gauss, n_gauss, &canvas, ws, ws_bytes, capacity, &n_pairs, keys, ranges, NULL);
    if (st == BS_ERR_CAPACITY) capacity = n_pairs + 1024;
  }
  CHECK_BS(st);

  CHECK_BS(bs_render_fwd_l2(gauss, n_gauss, &canvas, keys, ranges, target, img, T, nc_map, dimg, loss_d, NULL));
  bs_curves_grad grad = {zeros((size_t)no * 20, &err), zeros((size_t)no, &err),      zeros((size_t)no * 3, &err),
                         zeros((size_t)no * 3, &err),  zeros((size_t)nc * 24, &err), zeros((size_t)nc * 3, &err),
                         zeros((size_t)nc, &err),      NULL,                         NULL};
  if (err) return 1;
  CHECK_BS(bs_render_bwd(gauss, n_gauss, &canvas, keys, ranges, T, nc_map, dimg, dgauss, &curves, &cfg, &grad,
                         NULL));
  CHECK_CUDA(cudaDeviceSynchronize());
  int32_t status = 0;
  CHECK_BS(bs_sync_status(1, &status, NULL));
  if (status != BS_OK) {
    fprintf(stderr, "device status %d\n", (int)status);
    return 1;
  }

  FILE *out = fopen(argv[2], "wb");
  if (!out) return 2;
  double loss = 0.0;
  CHECK_CUDA(cudaMemcpy(&loss, loss_d, sizeof(double), cudaMemcpyDeviceToHost));
  if (fwrite(&loss, sizeof(double), 1, out) != 1 || fwrite(&n_pairs, sizeof(int64_t), 1, out) != 1 ||
      download(out, img, 3 * npix) || download(out, grad.open_ctrl, (size_t)no * 20) ||
      download(out, grad.open_width, (size_t)no) || download(out, grad.open_color, (size_t)no * 3) ||
      download(out, grad.open_opac, (size_t)no * 3) || download(out, grad.closed_ctrl, (size_t)nc * 24) ||
      download(out, grad.closed_color, (size_t)nc * 3) || download(out, grad.closed_opac, (size_t)nc))
    return 1;
  fclose(out);
  return 0;
}
