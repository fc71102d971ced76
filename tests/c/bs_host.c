/*
 * The host-only calls of bs.h from plain C (no GPU needed): sizes, the
 * batch plan, the network's parameter counts, argument validation and the
 * SVG export.  Test program of tests/test_c_abi.py; prints "name value"
 * lines and writes the SVG document to the file given as its argument.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "bs.h"

int main(int argc, char **argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: bs_host SVG_OUT\n");
    return 2;
  }
  const bs_sample_cfg cfg = {16, 4, 8, 1.0f, 0.3f, 0};
  printf("num_gaussians %lld\n", (long long)bs_num_gaussians(5, 3, &cfg));
  const bs_sample_cfg bad_cfg = {1, 4, 8, 1.0f, 0.3f, 0};   /* g_open < 2 */
  printf("num_gaussians_bad %lld\n", (long long)bs_num_gaussians(5, 3, &bad_cfg));

  const bs_canvas canvas = {2048, 2048, 16, {0.0f, 0.0f, 0.0f}};
  size_t bytes = 0;
  if (bs_bin_tiles_workspace(262144, &canvas, 11428828, &bytes) != BS_OK) return 1;
  printf("bin_workspace %llu\n", (unsigned long long)bytes);
  const bs_canvas bad_canvas = {2048, 2048, 12, {0.0f, 0.0f, 0.0f}};   /* tile side 12 */
  const bs_status st = bs_bin_tiles_workspace(262144, &bad_canvas, 1024, &bytes);
  printf("bin_workspace_bad_tile %d %d\n", (int)st, bs_last_error()[0] != '\0');

  bs_batch_image images[2] = {{100, 73, 12, 6, {12, 5, 7, 1.0f, 0.3f, 0}, {0.2f, 0.5f, 0.1f}},
                              {256, 200, 60, 30, {16, 4, 8, 1.0f, 0.3f, 1}, {0.0f, 0.1f, 0.2f}}};
  const bs_batch batch = {images, 2, 16, 1 << 20, NULL, 0};
  bs_batch_sizes sz;
  if (bs_batch_plan(&batch, &sz) != BS_OK) return 1;
  printf("batch %lld %lld %lld %lld %lld %llu\n", (long long)sz.n_open, (long long)sz.n_closed,
         (long long)sz.n_gauss, (long long)sz.n_pixels, (long long)sz.n_tiles, (unsigned long long)sz.ws_bytes);

  printf("net_params %lld %lld\n", (long long)bs_net_param_count(0), (long long)bs_net_param_count(5));

  /* one open and one closed curve, host arrays */
  float open_ctrl[20], closed_ctrl[24];
  for (int j = 0; j < 10; ++j) {
    open_ctrl[2 * j] = 3.0f + 2.5f * (float)j;
    open_ctrl[2 * j + 1] = 10.0f + (float)(j % 3);
  }
  for (int j = 0; j < 12; ++j) {
    closed_ctrl[2 * j] = 30.0f + 0.5f * (float)(j * j % 7);
    closed_ctrl[2 * j + 1] = 20.0f + 1.25f * (float)j;
  }
  const float open_width[1] = {1.5f}, open_color[3] = {0.1f, 0.2f, 0.3f}, open_opac[3] = {0.9f, 0.5f, 0.7f};
  const float closed_color[3] = {0.6f, 0.25f, 1.0f}, closed_opac[1] = {0.8f};
  const uint32_t rank[2] = {1, 0};
  const bs_curves curves = {1, 1, open_ctrl, open_width, open_color, open_opac, closed_ctrl,
                            closed_color, closed_opac, NULL, NULL, NULL};
  size_t need = 0;
  if (bs_svg_export(&curves, rank, 64, 48, 1, NULL, 0, &need) != BS_OK) return 1;
  char *doc = (char *)malloc(need);
  if (!doc || bs_svg_export(&curves, rank, 64, 48, 1, doc, need, &need) != BS_OK) return 1;
  FILE *f = fopen(argv[1], "wb");
  if (!f || fwrite(doc, 1, need - 1, f) != need - 1) return 1;
  fclose(f);
  printf("svg_bytes %llu\n", (unsigned long long)need);
  free(doc);
  return 0;
}
