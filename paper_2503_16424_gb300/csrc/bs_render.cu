// Per-tile alpha blending (Section 3.4, Eq. 9-10) and its reverse-order
// backward, plus the L2 term of Eq. 13.
//
// One CTA per 16x16 tile, one pixel per thread.  The tile's list is staged
// into shared memory 256 Gaussians at a time; each Gaussian is staged as a
// log2-domain quadratic form so that a pixel evaluates
//     p = qa dx^2 + qb2 dx dy + qc dy^2 + log2(o),    alpha = min(0.99, 2^p)
// with qa = -a log2(e)/2, qb2 = -b log2(e), qc = -c log2(e)/2 for the conic
// [[a, b], [b, c]].  The forward and the backward stage and evaluate alpha
// with the same code, so both take the same skip decisions bit for bit.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kTile = 16;
constexpr int kThreads = kTile * kTile;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kQ = -0.5f * kLog2e;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Staged {
  float4 a;  // mx, my, qa, qb2
  float4 b;  // qc, lo, r, g
  float2 c;  // b, o
};

// Stage Gaussian g; an index past the table (only possible after a sort that
// gave up waiting) stages an invisible Gaussian.
__device__ __forceinline__ Staged stage(const float *__restrict__ gauss, uint32_t g, uint32_t n_gauss) {
  Staged s;
  if (g >= n_gauss) {
    s.a = make_float4(0.f, 0.f, 0.f, 0.f);
    s.b = make_float4(0.f, -INFINITY, 0.f, 0.f);
    s.c = make_float2(0.f, 0.f);
    return s;
  }
  const float4 *rec = reinterpret_cast<const float4 *>(gauss + (size_t)g * BS_GAUSS_FLOATS);
  const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
  const float blue = __ldg(gauss + (size_t)g * BS_GAUSS_FLOATS + 8);
  const float o = r1.y;
  s.a = make_float4(r0.x, r0.y, __fmul_rn(kQ, r0.z), __fmul_rn(2.0f * kQ, r0.w));
  s.b = make_float4(__fmul_rn(kQ, r1.x), o > 0.f ? log2f(o) : -INFINITY, r1.z, r1.w);
  s.c = make_float2(blue, o);
  return s;
}

// log2 of the unclamped alpha of a staged Gaussian at pixel centre (px, py).
__device__ __forceinline__ float log2_alpha(const float4 &a, const float4 &b, float px, float py, float &dx,
                                            float &dy) {
  dx = __fsub_rn(px, a.x);
  dy = __fsub_rn(py, a.y);
  const float u = __fmaf_rn(a.z, dx, __fmul_rn(a.w, dy));
  const float v = __fmul_rn(b.x, dy);
  return __fmaf_rn(dx, u, __fmaf_rn(dy, v, b.y));
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
  __shared__ float s_c[kThreads];
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
      s_c[threadIdx.x] = s.c.x;
    }
    __syncthreads();
    if (!done) {
      const int n = (int)min((uint32_t)kThreads, r.y - base);
      for (int j = 0; j < n; ++j) {
        const float4 a = s_a[j], b = s_b[j];
        float dx, dy;
        const float al = fminf(kAlphaMax, ex2_approx(log2_alpha(a, b, px, py, dx, dy)));
        if (kStats) ++n_eval;
        if (al < kAlphaMin) continue;
        const float Tn = T * (1.f - al);
        if (Tn < kTMin) {
          done = true;
          break;
        }
        const float w = al * T;
        c0 = __fmaf_rn(w, b.z, c0);
        c1 = __fmaf_rn(w, b.w, c1);
        c2 = __fmaf_rn(w, s_c[j], c2);
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
  __shared__ float2 s_c[kThreads];
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
  // g . A, A = colour accumulated behind the current Gaussian, starts at T_final bg
  float gA = T * (g0 * bg.x + g1 * bg.y + g2 * bg.z);
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
      s_g[threadIdx.x] = g;
    }
    __syncthreads();
    for (int j = (int)(end - start) - 1; j >= 0; --j) {
      const uint32_t pos = start + (uint32_t)j;
      float v[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = 0.f;
      bool contrib = false;
      if (pos < last) {
        const float4 a = s_a[j], b = s_b[j];
        float dx, dy;
        const float raw = ex2_approx(log2_alpha(a, b, px, py, dx, dy));
        const float al = fminf(kAlphaMax, raw);
        if (al >= kAlphaMin) {
          contrib = true;
          const float one_m = 1.f - al;
          const float inv = 1.f / one_m;
          T = T * inv;                         // T before this Gaussian
          const float w = al * T;
          const float cb = s_c[j].x;
          const float gc = g0 * b.z + g1 * b.w + g2 * cb;
          const float dal = T * gc - gA * inv;  // dL/dalpha
          gA = __fmaf_rn(gc, w, gA);
          v[6] = w * g0;
          v[7] = w * g1;
          v[8] = w * g2;
          if (raw <= kAlphaMax) {
            const float dp = dal * al * kLn2;   // dL/d(log2 alpha)
            const float t1 = dp * dx, t2 = dp * dy;
            v[0] = -(t1 * (2.f * a.z) + t2 * a.w);  // sum dp (2qa dx + qb2 dy), negated: d/dmx
            v[1] = -(t1 * a.w + t2 * (2.f * b.x));  // d/dmy
            v[2] = t1 * dx;                         // sum dp dx^2
            v[3] = t1 * dy;                         // sum dp dx dy
            v[4] = t2 * dy;                         // sum dp dy^2
            v[5] = dp;                              // sum dp
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = warp_sum(v[q]);
        if (lane < 9) {
          float val = v[0];
#pragma unroll
          for (int q = 1; q < 9; ++q)
            if (lane == q) val = v[q];
          const float o = s_c[j].y;
          // constant factors of the chain rule (see the staging above)
          if (lane == 2 || lane == 4) val *= kQ;
          else if (lane == 3) val *= 2.f * kQ;
          else if (lane == 5) val = o > 0.f ? val / (o * kLn2) : 0.f;
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
    const float d = img[i] - target[i];
    dimg[i] = scale * d;
    acc += (double)d * (double)d;
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
