// Per-tile alpha blending (Section 3.4, Eq. 9-10) and its reverse-order
// backward, plus the L2 term of Eq. 13.
//
// One CTA per 16x16 tile, one pixel per thread.  The tile's list is staged
// into shared memory 256 Gaussians at a time.  A Gaussian is stored by its
// eigen-frame (Eq. 11-12): Sigma^-1 = R diag(isx^2, isy^2) R^T with
// R = [[ux, -uy], [uy, ux]], and is staged as the two scaled axes
//     (A1, B1) = k isx (ux, uy),   (A2, B2) = k isy (-uy, ux),   k^2 = log2(e)/2,
// so that a pixel at offset (dx, dy) from the mean evaluates
//     t1 = A1 dx + B1 dy,  t2 = A2 dx + B2 dy,
//     p  = log2(o) - t1^2 - t2^2 = log2(o exp(-0.5 d^T Sigma^-1 d)),
//     alpha = min(0.99, 2^p).
// A sum of two squares has no cancellation, unlike the conic form
// a dx^2 + 2 b dx dy + c dy^2 of a thin, rotated Gaussian far along its
// axis.  The forward and the backward stage and evaluate alpha with the same
// code, so both take the same skip decisions bit for bit.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kTile = 16;
constexpr int kThreads = kTile * kTile;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kKappa = 0.84932180028801907f;  // sqrt(log2(e) / 2)

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Staged {
  float4 a;    // mx, my, A1, B1
  float4 b;    // A2, B2, log2(o), r
  float4 c;    // g, b, o, 0
  float4 raw;  // ux, uy, isx, isy
};

// Stage Gaussian g; an index past the table (only possible after a sort that
// gave up waiting) stages an invisible Gaussian.
__device__ __forceinline__ Staged stage(const float *__restrict__ gauss, uint32_t g, uint32_t n_gauss) {
  Staged s;
  if (g >= n_gauss) {
    s.a = make_float4(0.f, 0.f, 0.f, 0.f);
    s.b = make_float4(0.f, 0.f, -INFINITY, 0.f);
    s.c = make_float4(0.f, 0.f, 0.f, 0.f);
    s.raw = make_float4(1.f, 0.f, 0.f, 0.f);
    return s;
  }
  const float4 *rec = reinterpret_cast<const float4 *>(gauss + (size_t)g * BS_GAUSS_FLOATS);
  const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
  const float ux = r0.z, uy = r0.w, isx = r1.x, isy = r1.y, o = r1.z;
  const float kx = __fmul_rn(kKappa, isx), ky = __fmul_rn(kKappa, isy);
  s.a = make_float4(r0.x, r0.y, __fmul_rn(kx, ux), __fmul_rn(kx, uy));
  s.b = make_float4(__fmul_rn(ky, -uy), __fmul_rn(ky, ux), o > 0.f ? log2f(o) : -INFINITY, r1.w);
  s.c = make_float4(r2.x, r2.y, o, 0.f);
  s.raw = make_float4(ux, uy, isx, isy);
  return s;
}

// log2 of the unclamped alpha of a staged Gaussian at pixel centre (px, py),
// with the offsets and the two axis projections.
__device__ __forceinline__ float log2_alpha(const float4 &a, const float4 &b, float px, float py, float &dx,
                                            float &dy, float &t1, float &t2) {
  dx = __fsub_rn(px, a.x);
  dy = __fsub_rn(py, a.y);
  t1 = __fmaf_rn(a.z, dx, __fmul_rn(a.w, dy));
  t2 = __fmaf_rn(b.x, dx, __fmul_rn(b.y, dy));
  return __fmaf_rn(-t1, t1, __fmaf_rn(-t2, t2, b.z));
}

// kStats: also count, per pixel, the list entries evaluated (E), the entries
// blended, and the entries of the tile lists times the tile's pixels, into
// stats[0..2] (for measurement; same blend otherwise).
template <bool kStats>
__global__ void __launch_bounds__(kThreads) render_fwd_kernel(const float *__restrict__ gauss,
                                                              const uint32_t *__restrict__ keys,
                                                              const uint2 *__restrict__ ranges, int W, int H,
                                                              int tiles_x, uint32_t gmask, uint32_t n_gauss,
                                                              float3 bg, float *__restrict__ img,
                                                              float *__restrict__ T_out,
                                                              uint32_t *__restrict__ nc_out,
                                                              unsigned long long *__restrict__ stats) {
  __shared__ float4 s_a[kThreads];
  __shared__ float4 s_b[kThreads];
  __shared__ float2 s_c[kThreads];
  uint32_t n_eval = 0, n_blend = 0;
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int x = tx * kTile + (threadIdx.x & (kTile - 1));
  const int y = ty * kTile + threadIdx.x / kTile;
  const bool inside = x < W && y < H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint2 r = ranges[tile];
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  uint32_t last = 0;
  bool done = !inside;
  for (uint32_t base = r.x; base < r.y; base += kThreads) {
    if (__syncthreads_count(done) == kThreads) break;
    const uint32_t i = base + threadIdx.x;
    if (i < r.y) {
      const Staged s = stage(gauss, keys[i] & gmask, n_gauss);
      s_a[threadIdx.x] = s.a;
      s_b[threadIdx.x] = s.b;
      s_c[threadIdx.x] = make_float2(s.c.x, s.c.y);
    }
    __syncthreads();
    if (!done) {
      const int n = (int)min((uint32_t)kThreads, r.y - base);
      for (int j = 0; j < n; ++j) {
        const float4 a = s_a[j], b = s_b[j];
        float dx, dy, t1, t2;
        const float al = fminf(kAlphaMax, ex2_approx(log2_alpha(a, b, px, py, dx, dy, t1, t2)));
        if (kStats) ++n_eval;
        if (al < kAlphaMin) continue;
        const float Tn = T * (1.f - al);
        if (Tn < kTMin) {
          done = true;
          break;
        }
        const float w = al * T;
        const float2 gb = s_c[j];
        c0 = __fmaf_rn(w, b.w, c0);
        c1 = __fmaf_rn(w, gb.x, c1);
        c2 = __fmaf_rn(w, gb.y, c2);
        T = Tn;
        last = base - r.x + (uint32_t)j + 1;
        if (kStats) ++n_blend;
      }
    }
  }
  if (kStats) {
    __shared__ unsigned long long s_st[2];
    if (threadIdx.x == 0) s_st[0] = s_st[1] = 0ull;
    __syncthreads();
    atomicAdd(&s_st[0], (unsigned long long)n_eval);
    atomicAdd(&s_st[1], (unsigned long long)n_blend);
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(&stats[0], s_st[0]);
      atomicAdd(&stats[1], s_st[1]);
      atomicAdd(&stats[2], (unsigned long long)(r.y - r.x) * kThreads);
    }
  }
  if (inside) {
    const size_t p = (size_t)y * W + x, plane = (size_t)W * H;
    img[p] = __fmaf_rn(T, bg.x, c0);
    img[plane + p] = __fmaf_rn(T, bg.y, c1);
    img[2 * plane + p] = __fmaf_rn(T, bg.z, c2);
    T_out[p] = T;
    nc_out[p] = last;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reverse walk.  With S the colour behind Gaussian j as seen through it,
// S <- alpha_j c_j + (1 - alpha_j) S (starting from bg behind the last
// blended Gaussian), the colour derivative is
//     dC/dalpha_j = T_j (c_j - S),
// which keeps the (1 - alpha_j)^-1 of the recovered transmittance out of the
// gradient.  Per Gaussian and pixel the walk accumulates
//   q1 = dp t1, q2 = dp t2 (dp = dL/dlog2(alpha)), q1 dx, q1 dy, q2 dx,
//   q2 dy, dp and w g (w = alpha T),
// and the chain rule through the staging turns their tile sums into
// d/d(mx, my, ux, uy, isx, isy, o, r, g, b).
__global__ void __launch_bounds__(kThreads) render_bwd_kernel(const float *__restrict__ gauss,
                                                              const uint32_t *__restrict__ keys,
                                                              const uint2 *__restrict__ ranges, int W, int H,
                                                              int tiles_x, uint32_t gmask, uint32_t n_gauss,
                                                              float3 bg, const float *__restrict__ T_final,
                                                              const uint32_t *__restrict__ n_contrib,
                                                              const float *__restrict__ dimg,
                                                              float *__restrict__ dgauss) {
  __shared__ float4 s_a[kThreads];
  __shared__ float4 s_b[kThreads];
  __shared__ float4 s_c[kThreads];
  __shared__ float4 s_raw[kThreads];
  __shared__ uint32_t s_g[kThreads];
  __shared__ uint32_t s_max_last;
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int x = tx * kTile + (threadIdx.x & (kTile - 1));
  const int y = ty * kTile + threadIdx.x / kTile;
  const bool inside = x < W && y < H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint2 r = ranges[tile];
  const int lane = threadIdx.x & 31;
  float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  uint32_t last = 0;
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  if (inside) {
    const size_t p = (size_t)y * W + x, plane = (size_t)W * H;
    T = T_final[p];
    last = n_contrib[p];
    g0 = dimg[p];
    g1 = dimg[plane + p];
    g2 = dimg[2 * plane + p];
    atomicMax(&s_max_last, last);
  }
  float gS = g0 * bg.x + g1 * bg.y + g2 * bg.z;  // g . S, S = bg behind the last blended Gaussian
  __syncthreads();
  const uint32_t max_last = min(s_max_last, r.y - r.x);
  for (uint32_t end = max_last; end > 0;) {
    const uint32_t start = end > (uint32_t)kThreads ? end - kThreads : 0u;
    __syncthreads();
    const uint32_t i = start + threadIdx.x;
    if (i < end) {
      const uint32_t g = keys[r.x + i] & gmask;
      const Staged s = stage(gauss, g, n_gauss);
      s_a[threadIdx.x] = s.a;
      s_b[threadIdx.x] = s.b;
      s_c[threadIdx.x] = s.c;
      s_raw[threadIdx.x] = s.raw;
      s_g[threadIdx.x] = g;
    }
    __syncthreads();
    for (int j = (int)(end - start) - 1; j >= 0; --j) {
      const uint32_t pos = start + (uint32_t)j;
      float v[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) v[q] = 0.f;
      bool contrib = false;
      if (pos < last) {
        const float4 a = s_a[j], b = s_b[j];
        float dx, dy, t1, t2;
        const float raw = ex2_approx(log2_alpha(a, b, px, py, dx, dy, t1, t2));
        const float al = fminf(kAlphaMax, raw);
        if (al >= kAlphaMin) {
          contrib = true;
          const float4 c = s_c[j];
          const float one_m = 1.f - al;
          T = __fdividef(T, one_m);             // T before this Gaussian
          const float w = al * T;
          const float gc = g0 * b.w + g1 * c.x + g2 * c.y;
          const float dal = T * (gc - gS);      // dL/dalpha
          gS = __fmaf_rn(al, gc, one_m * gS);
          v[7] = w * g0;
          v[8] = w * g1;
          v[9] = w * g2;
          if (raw <= kAlphaMax) {
            const float dp = dal * al * kLn2;   // dL/dlog2(alpha)
            const float q1 = dp * t1, q2 = dp * t2;
            v[0] = q1;
            v[1] = q2;
            v[2] = q1 * dx;
            v[3] = q1 * dy;
            v[4] = q2 * dx;
            v[5] = q2 * dy;
            v[6] = dp;
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int q = 0; q < 10; ++q) v[q] = warp_sum(v[q]);
        if (lane < 10) {
          const float4 a = s_a[j], b = s_b[j], u = s_raw[j];
          const float o = s_c[j].z;
          // dL/dA1 = -2 sum q1 dx, dL/dB1 = -2 sum q1 dy, dL/dA2 = -2 sum q2 dx, dL/dB2 = -2 sum q2 dy
          const float dA1 = -2.f * v[2], dB1 = -2.f * v[3], dA2 = -2.f * v[4], dB2 = -2.f * v[5];
          float val;
          switch (lane) {
            case 0: val = 2.f * (a.z * v[0] + b.x * v[1]); break;                // mx
            case 1: val = 2.f * (a.w * v[0] + b.y * v[1]); break;                // my
            case 2: val = kKappa * (u.z * dA1 + u.w * dB2); break;               // ux
            case 3: val = kKappa * (u.z * dB1 - u.w * dA2); break;               // uy
            case 4: val = kKappa * (u.x * dA1 + u.y * dB1); break;               // isx
            case 5: val = kKappa * (u.x * dB2 - u.y * dA2); break;               // isy
            case 6: val = o > 0.f ? v[6] / (o * kLn2) : 0.f; break;              // o
            case 7: val = v[7]; break;
            case 8: val = v[8]; break;
            default: val = v[9]; break;
          }
          if (val != 0.f && s_g[j] < n_gauss) atomicAdd(dgauss + (size_t)s_g[j] * BS_DGAUSS_FLOATS + lane, val);
        }
      }
    }
    end = start;
  }
}

__global__ void l2_kernel(const float *__restrict__ img, const float *__restrict__ target, int64_t n,
                          float *__restrict__ dimg, double *loss) {
  __shared__ double s_sum[32];
  double acc = 0.0;
  const float scale = (float)(2.0 / (double)n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double d = (double)img[i] - (double)target[i];   // exact
    dimg[i] = scale * (float)d;
    acc += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_sum[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < (int)(blockDim.x / 32) ? s_sum[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(loss, acc / (double)n);
  }
}

}  // namespace

bs_status launch_render_fwd(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                            const uint32_t *keys,
                            const uint32_t *ranges, float *img, float *T_final, uint32_t *n_contrib,
                            cudaStream_t s, unsigned long long *stats) {
  const int tiles_x = div_up(cv.width, kTile), tiles_y = div_up(cv.height, kTile);
  const uint32_t gmask = gbits >= 32 ? 0xffffffffu : ((1u << gbits) - 1u);
  const auto bg = make_float3(cv.bg[0], cv.bg[1], cv.bg[2]);
  const auto *rg = reinterpret_cast<const uint2 *>(ranges);
  if (stats) {
    BS_CUDA(cudaMemsetAsync(stats, 0, 4 * sizeof(unsigned long long), s));
    render_fwd_kernel<true><<<tiles_x * tiles_y, kThreads, 0, s>>>(
        gauss, keys, rg, cv.width, cv.height, tiles_x, gmask, (uint32_t)n_gauss, bg, img, T_final, n_contrib, stats);
  } else {
    render_fwd_kernel<false><<<tiles_x * tiles_y, kThreads, 0, s>>>(
        gauss, keys, rg, cv.width, cv.height, tiles_x, gmask, (uint32_t)n_gauss, bg, img, T_final, n_contrib,
        nullptr);
  }
  BS_LAUNCHED("render_fwd_kernel");
  return BS_OK;
}

bs_status launch_render_bwd(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                            const uint32_t *keys, const uint32_t *ranges, const float *T_final,
                            const uint32_t *n_contrib, const float *dL_dimg, float *dgauss, cudaStream_t s) {
  const int tiles_x = div_up(cv.width, kTile), tiles_y = div_up(cv.height, kTile);
  const uint32_t gmask = gbits >= 32 ? 0xffffffffu : ((1u << gbits) - 1u);
  BS_CUDA(cudaMemsetAsync(dgauss, 0, sizeof(float) * BS_DGAUSS_FLOATS * (size_t)n_gauss, s));
  render_bwd_kernel<<<tiles_x * tiles_y, kThreads, 0, s>>>(
      gauss, keys, reinterpret_cast<const uint2 *>(ranges), cv.width, cv.height, tiles_x, gmask,
      (uint32_t)n_gauss, make_float3(cv.bg[0], cv.bg[1], cv.bg[2]), T_final, n_contrib, dL_dimg, dgauss);
  BS_LAUNCHED("render_bwd_kernel");
  return BS_OK;
}

bs_status launch_l2(const float *img, const float *target, int64_t n, float *dimg, double *loss, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
  if (n == 0) return BS_OK;
  const int blocks = (int)std::min<int64_t>(div_up64(n, 256 * 4), 152 * 8);
  l2_kernel<<<blocks, 256, 0, s>>>(img, target, n, dimg, loss);
  BS_LAUNCHED("l2_kernel");
  return BS_OK;
}

}  // namespace bs
