// Curves -> Gaussians: draw order (Section 3.3 "depth from area"), sampling
// (Section 3.3, Eq. 3-8, Eq. 11-12) and its backward.
//
// One CTA per curve.  The CTA evaluates the curve's sample points X into
// shared memory, then each thread turns one sample and its neighbours into
// a Gaussian record (forward), or pushes one Gaussian's gradient back to the
// sample points and from there, with the Bernstein weights of Eq. 1-2, to the
// control points (backward).  A curve's Gaussians are contiguous in the
// draw-ordered table, so the backward needs no global atomics.
//
// Precision: the sample points and the differences of neighbouring samples
// (Eq. 7-8) are computed in double, relative to the curve's first control
// point.  Subtracting two float32 positions loses the digits that a short
// tangent or a thin row spacing needs; the difference vectors, once formed,
// are well conditioned and everything after them runs in float32.
#include <cuda_runtime.h>
#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kCurveThreads = 64;

struct Cfg {
  int g_open, rows, kc;
  float rho, eps;
};

__device__ __forceinline__ void bern3(double t, double w[4]) {
  const double u = 1.0 - t;
  w[0] = u * u * u;
  w[1] = 3.0 * u * u * t;
  w[2] = 3.0 * u * t * t;
  w[3] = t * t * t;
}

// Segment of sample k of K on a chain of S segments, u = k/(K-1):
// s = min(floor(S u), S-1), decided in integers.
__device__ __forceinline__ int chain_seg(int k, int K, int S) {
  const int s = (S * k) / (K - 1);
  return s > S - 1 ? S - 1 : s;
}
// Local parameter t = S u - s, u = k / (K - 1), with inv = 1 / (K - 1).
__device__ __forceinline__ double chain_t_inv(int k, int K, int S, int s, double inv) {
  return (double)(S * k - s * (K - 1)) * inv;
}

// Boundary groups of a closed curve: A = P0..P6, B = P0, P11, ..., P7, P6.
__device__ __forceinline__ int closed_b_index(int j) { return (j == 0 || j == 6) ? j : 12 - j; }

// tau_r = (1 - cos(pi r/(R+1)))/2 with rows = R + 2.
__device__ __forceinline__ double closed_tau(int r, int rows) {
  return 0.5 * (1.0 - cospi((double)r / (double)(rows - 1)));
}

__device__ __forceinline__ float2 ld2(const float *p, int i) { return make_float2(p[2 * i], p[2 * i + 1]); }

__device__ __forceinline__ const float *curve_ctrl(const bs_curves &c, int curve) {
  return curve < c.n_open ? c.open_ctrl + (size_t)curve * 20 : c.closed_ctrl + (size_t)(curve - c.n_open) * 24;
}

// Per-CTA tables shared by every sample of the curve: the Bernstein weights
// of each sample index k (double [K][4]) and, for closed curves, the row
// weights tau_r (double [rows]).  A closed curve's rows reuse the same K
// weights, and the divisions and cosines run once per index, not per sample.
__device__ void build_tables(const Cfg &cfg, bool closed, double *Wt, double *taut) {
  __shared__ double s_inv;
  const int K = closed ? cfg.kc : cfg.g_open, S = closed ? 2 : 3;
  if (threadIdx.x == 0) s_inv = 1.0 / (double)(K - 1);  // one double division per curve
  __syncthreads();
  const double inv = s_inv;
  for (int k = threadIdx.x; k < K; k += blockDim.x) bern3(chain_t_inv(k, K, S, chain_seg(k, K, S), inv), Wt + 4 * k);
  if (closed)
    for (int r = threadIdx.x; r < cfg.rows; r += blockDim.x) taut[r] = closed_tau(r, cfg.rows);
}

// Sample points X of a curve relative to its first control point, into
// shared memory (after build_tables and a barrier); returns the number of
// samples.
__device__ int eval_samples(const bs_curves &c, const Cfg &cfg, int curve, const double *Wt, const double *taut,
                            double2 *X) {
  const float *P = curve_ctrl(c, curve);
  const double ox = P[0], oy = P[1];
  if (curve < c.n_open) {
    const int K = cfg.g_open;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const int s = chain_seg(k, K, 3);
      const double *w = Wt + 4 * k;
      double ax = 0.0, ay = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 p = ld2(P, 3 * s + i);
        ax += w[i] * ((double)p.x - ox);
        ay += w[i] * ((double)p.y - oy);
      }
      X[k] = make_double2(ax, ay);
    }
    return K;
  }
  const int K = cfg.kc, R2 = cfg.rows, n = R2 * K;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int r = idx / K, k = idx - r * K;
    const double tau = taut[r];
    const int s = chain_seg(k, K, 2);
    const double *w = Wt + 4 * k;
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = 3 * s + i;
      const float2 a = ld2(P, j), b = ld2(P, closed_b_index(j));
      const double qx = (1.0 - tau) * ((double)a.x - ox) + tau * ((double)b.x - ox);  // Eq. 4
      const double qy = (1.0 - tau) * ((double)a.y - oy) + tau * ((double)b.y - oy);
      ax += w[i] * qx;
      ay += w[i] * qy;
    }
    X[idx] = make_double2(ax, ay);
  }
  return n;
}

__device__ __forceinline__ float2 diff(const double2 *X, int hi, int lo) {
  return make_float2((float)(X[hi].x - X[lo].x), (float)(X[hi].y - X[lo].y));
}

// Local geometry of one sample (Eq. 7-8): the along-row difference e (for
// sigma_x), the tangent difference t (for the rotation), the across-row
// difference f (closed curves, for sigma_y); the scales; the unit tangent u.
struct Local {
  float2 e, t, f;
  int e_hi, e_lo, t_hi, t_lo, f_hi, f_lo;  // sample indices the differences use
  float le, lt, lf;                         // their lengths
  float sx, sy, ux, uy;
};

__device__ __forceinline__ Local local_geometry(const double2 *X, int idx, int K, int R2, bool closed,
                                                float width, float rho) {
  Local L;
  const int r = closed ? idx / K : 0;
  const int k = idx - r * K;
  const int row = r * K;
  if (k + 1 < K) { L.e_hi = row + k + 1; L.e_lo = row + k; }
  else { L.e_hi = row + k; L.e_lo = row + k - 1; }
  if (k == 0) { L.t_hi = row + 1; L.t_lo = row; }
  else if (k == K - 1) { L.t_hi = row + k; L.t_lo = row + k - 1; }
  else { L.t_hi = row + k + 1; L.t_lo = row + k - 1; }
  L.e = diff(X, L.e_hi, L.e_lo);
  L.t = diff(X, L.t_hi, L.t_lo);
  L.le = sqrtf(L.e.x * L.e.x + L.e.y * L.e.y);
  L.lt = sqrtf(L.t.x * L.t.x + L.t.y * L.t.y);
  L.sx = L.le / rho;
  if (closed) {
    if (r + 1 < R2) { L.f_hi = idx + K; L.f_lo = idx; }
    else { L.f_hi = idx; L.f_lo = idx - K; }
    L.f = diff(X, L.f_hi, L.f_lo);
    L.lf = sqrtf(L.f.x * L.f.x + L.f.y * L.f.y);
    L.sy = L.lf / rho;
  } else {
    L.f = make_float2(0.f, 0.f);
    L.f_hi = L.f_lo = idx;
    L.lf = 0.f;
    L.sy = width;
  }
  if (L.lt > 0.f) { L.ux = L.t.x / L.lt; L.uy = L.t.y / L.lt; }
  else { L.ux = 1.f; L.uy = 0.f; }
  return L;
}

struct CurveAttr {
  float width;
  float opac;
  float3 col;
};

__device__ __forceinline__ CurveAttr curve_attr(const bs_curves &c, int curve, int seg) {
  CurveAttr a;
  if (curve < c.n_open) {
    a.width = c.open_width[curve];
    a.opac = c.open_opac[curve * 3 + seg];
    a.col = make_float3(c.open_color[curve * 3], c.open_color[curve * 3 + 1], c.open_color[curve * 3 + 2]);
  } else {
    const int j = curve - c.n_open;
    a.width = 0.f;
    a.opac = c.closed_opac[j];
    a.col = make_float3(c.closed_color[j * 3], c.closed_color[j * 3 + 1], c.closed_color[j * 3 + 2]);
  }
  return a;
}

// Dynamic shared memory of the sampling kernels: n_max double2 sample points,
// [bwd: n_max float2 gradients,] k_max x 4 double weights, rows double tau.
struct CurveSmem {
  double2 *X;
  float2 *dX;
  double *Wt, *taut;
};

__device__ __forceinline__ CurveSmem carve(void *base, int n_max, int k_max, bool with_grad) {
  CurveSmem m;
  char *p = static_cast<char *>(base);
  m.X = reinterpret_cast<double2 *>(p);
  p += sizeof(double2) * n_max;
  m.Wt = reinterpret_cast<double *>(p);
  p += sizeof(double) * 4 * k_max;
  m.taut = reinterpret_cast<double *>(p);
  p += sizeof(double) * 64 * ((n_max + 63) / 64);  // rows <= n_max
  m.dX = with_grad ? reinterpret_cast<float2 *>(p) : nullptr;
  return m;
}

__global__ void __launch_bounds__(kCurveThreads) sample_fwd_kernel(bs_curves c, Cfg cfg, float *gauss, int n_max,
                                                                   int k_max) {
  extern __shared__ double2 smem_fwd[];
  const CurveSmem m = carve(smem_fwd, n_max, k_max, false);
  double2 *X = m.X;
  const int curve = blockIdx.x;
  const bool closed = curve >= c.n_open;
  build_tables(cfg, closed, m.Wt, m.taut);
  __syncthreads();
  const int n = eval_samples(c, cfg, curve, m.Wt, m.taut, X);
  __syncthreads();
  const int K = closed ? cfg.kc : cfg.g_open;
  const uint32_t first = c.draw_first[curve];
  const float *P = curve_ctrl(c, curve);
  const double ox = P[0], oy = P[1];
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int seg = closed ? 0 : chain_seg(idx, K, 3);
    const CurveAttr at = curve_attr(c, curve, seg);
    const Local L = local_geometry(X, idx, K, cfg.rows, closed, at.width, cfg.rho);
    // Sigma = R diag(lx, ly) R^T (Eq. 11-12 with the eps floor)
    const float lx = L.sx * L.sx + cfg.eps, ly = L.sy * L.sy + cfg.eps;
    float ex = -1.f, ey = -1.f;
    if (at.opac >= kAlphaMin) {
      const float lth = logf(255.0f * at.opac);  // alpha >= 1/255 <=> 0.5 d^T Sigma^-1 d <= lth
      const float sxx = L.ux * L.ux * lx + L.uy * L.uy * ly;
      const float syy = L.uy * L.uy * lx + L.ux * L.ux * ly;
      ex = sqrtf(2.0f * lth * sxx) + kExtPad;
      ey = sqrtf(2.0f * lth * syy) + kExtPad;
    }
    float4 *rec = reinterpret_cast<float4 *>(gauss + (size_t)(first + idx) * BS_GAUSS_FLOATS);
    rec[0] = make_float4((float)(ox + X[idx].x), (float)(oy + X[idx].y), L.ux, L.uy);
    rec[1] = make_float4(rsqrtf(lx), rsqrtf(ly), at.opac, at.col.x);
    rec[2] = make_float4(at.col.y, at.col.z, ex, ey);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void sadd2(float2 *p, float x, float y) {
  atomicAdd(&p->x, x);
  atomicAdd(&p->y, y);
}

__global__ void __launch_bounds__(kCurveThreads) sample_bwd_kernel(bs_curves c, Cfg cfg, const float *dgauss,
                                                                   bs_curves_grad g, int n_max, int k_max) {
  extern __shared__ double2 smem_bwd[];
  const CurveSmem m = carve(smem_bwd, n_max, k_max, true);
  double2 *X = m.X;
  float2 *dX = m.dX;
  __shared__ float2 dP[12];
  __shared__ float sAttr[8];  // opac[3] (open) or opac (closed), colour[3], width
  const int curve = blockIdx.x;
  const bool closed = curve >= c.n_open;
  for (int i = threadIdx.x; i < 12; i += blockDim.x) dP[i] = make_float2(0.f, 0.f);
  if (threadIdx.x < 8) sAttr[threadIdx.x] = 0.f;
  build_tables(cfg, closed, m.Wt, m.taut);
  __syncthreads();
  const int n = eval_samples(c, cfg, curve, m.Wt, m.taut, X);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dX[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int K = closed ? cfg.kc : cfg.g_open;
  const uint32_t first = c.draw_first[curve];
  const int lane = threadIdx.x & 31;
  const int n_rounds = div_up(n, blockDim.x);
  for (int round = 0; round < n_rounds; ++round) {
    const int idx = round * blockDim.x + threadIdx.x;
    float d_op[3] = {0.f, 0.f, 0.f}, d_col[3] = {0.f, 0.f, 0.f}, d_w = 0.f;
    if (idx < n) {
      const int seg = closed ? 0 : chain_seg(idx, K, 3);
      const CurveAttr at = curve_attr(c, curve, seg);
      const Local L = local_geometry(X, idx, K, cfg.rows, closed, at.width, cfg.rho);
      const float *dg = dgauss + (size_t)(first + idx) * BS_DGAUSS_FLOATS;
      const float4 d0 = *reinterpret_cast<const float4 *>(dg);      // mx, my, ux, uy
      const float4 d1 = *reinterpret_cast<const float4 *>(dg + 4);  // isx, isy, o, r
      const float4 d2 = *reinterpret_cast<const float4 *>(dg + 8);  // g, b, -, -
      // isx = (sx^2 + eps)^-1/2  ->  d isx / d sx = -sx isx^3
      const float isx = rsqrtf(L.sx * L.sx + cfg.eps), isy = rsqrtf(L.sy * L.sy + cfg.eps);
      const float dsx = -d1.x * L.sx * isx * isx * isx;
      const float dsy = -d1.y * L.sy * isy * isy * isy;
      // mean
      sadd2(&dX[idx], d0.x, d0.y);
      // sigma_x = |e| / rho
      if (L.le > 0.f) {
        const float k = dsx / (L.le * cfg.rho);
        sadd2(&dX[L.e_hi], k * L.e.x, k * L.e.y);
        sadd2(&dX[L.e_lo], -k * L.e.x, -k * L.e.y);
      }
      // u = t / |t|  ->  dL/dt = (du - u (u . du)) / |t|
      if (L.lt > 0.f) {
        const float proj = L.ux * d0.z + L.uy * d0.w;
        const float gx = (d0.z - L.ux * proj) / L.lt, gy = (d0.w - L.uy * proj) / L.lt;
        sadd2(&dX[L.t_hi], gx, gy);
        sadd2(&dX[L.t_lo], -gx, -gy);
      }
      if (closed) {
        if (L.lf > 0.f) {
          const float k = dsy / (L.lf * cfg.rho);
          sadd2(&dX[L.f_hi], k * L.f.x, k * L.f.y);
          sadd2(&dX[L.f_lo], -k * L.f.x, -k * L.f.y);
        }
        d_op[0] = d1.z;
      } else {
        d_w = dsy;
        d_op[seg] = d1.z;
      }
      d_col[0] = d1.w;
      d_col[1] = d2.x;
      d_col[2] = d2.y;
    }
    // per-curve scalars: warp sums, then one shared atomic per warp
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float a = warp_sum(d_op[i]);
      const float b = warp_sum(d_col[i]);
      if (lane == 0) {
        atomicAdd(&sAttr[i], a);
        atomicAdd(&sAttr[3 + i], b);
      }
    }
    const float w = warp_sum(d_w);
    if (lane == 0) atomicAdd(&sAttr[6], w);
  }
  __syncthreads();
  // sample points -> control points (Eq. 1-2; closed rows also Eq. 4)
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const float2 d = dX[idx];
    if (!closed) {
      const int s = chain_seg(idx, K, 3);
      const double *wd = m.Wt + 4 * idx;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float w = (float)wd[i];
        sadd2(&dP[3 * s + i], w * d.x, w * d.y);
      }
    } else {
      const int r = idx / K, k = idx - r * K;
      const float tau = (float)m.taut[r];
      const int s = chain_seg(k, K, 2);
      float w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) w[i] = (float)m.Wt[4 * k + i];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = 3 * s + i;
        const float wa = w[i] * (1.0f - tau), wb = w[i] * tau;
        sadd2(&dP[j], wa * d.x, wa * d.y);
        sadd2(&dP[closed_b_index(j)], wb * d.x, wb * d.y);
      }
    }
  }
  __syncthreads();
  if (!closed) {
    float *gp = g.open_ctrl + (size_t)curve * 20;
    for (int i = threadIdx.x; i < 10; i += blockDim.x) {
      gp[2 * i] = dP[i].x;
      gp[2 * i + 1] = dP[i].y;
    }
    if (threadIdx.x < 3) {
      g.open_opac[curve * 3 + threadIdx.x] = sAttr[threadIdx.x];
      g.open_color[curve * 3 + threadIdx.x] = sAttr[3 + threadIdx.x];
    }
    if (threadIdx.x == 0) g.open_width[curve] = sAttr[6];
  } else {
    const int j = curve - c.n_open;
    float *gp = g.closed_ctrl + (size_t)j * 24;
    for (int i = threadIdx.x; i < 12; i += blockDim.x) {
      gp[2 * i] = dP[i].x;
      gp[2 * i + 1] = dP[i].y;
    }
    if (threadIdx.x < 3) g.closed_color[j * 3 + threadIdx.x] = sAttr[3 + threadIdx.x];
    if (threadIdx.x == 0) g.closed_opac[j] = sAttr[0];
  }
}

// ---- draw order ----
__device__ __forceinline__ float area_key(const bs_curves &c, int i) {
  if (i < c.n_open) {
    const float *P = c.open_ctrl + (size_t)i * 20;
    float acc = 0.f;
    for (int j = 0; j < 9; ++j) {
      const float dx = __fsub_rn(P[2 * j + 2], P[2 * j]);
      const float dy = __fsub_rn(P[2 * j + 3], P[2 * j + 1]);
      acc = __fadd_rn(acc, __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy))));
    }
    return __fmul_rn(acc, c.open_width[i]);
  }
  const float *P = c.closed_ctrl + (size_t)(i - c.n_open) * 24;
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

constexpr int kOrderThreads = 256;
constexpr int kOrderChunk = 1024;  // keys compared per CTA

// Rank by counting: rank_i = #{j : key_j < key_i or (key_j == key_i, j < i)}.
// CTA (x, y) compares its 256 curves against the keys of chunk y and adds its
// counts (rank, and how many of the preceding curves are open) atomically.
__global__ void __launch_bounds__(kOrderThreads) curve_order_count_kernel(bs_curves c, uint32_t *rank,
                                                                         uint32_t *open_before) {
  __shared__ uint32_t sk[kOrderChunk];
  const int n = c.n_open + c.n_closed;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int base = blockIdx.y * kOrderChunk;
  const int m = min(kOrderChunk, n - base);
  for (int q = threadIdx.x; q < m; q += blockDim.x) sk[q] = key_order(area_key(c, base + q));
  const uint32_t mine = i < n ? key_order(area_key(c, i)) : 0u;
  __syncthreads();
  if (i >= n) return;
  uint32_t before = 0, ob = 0;
  const int open_end = c.n_open - base;  // chunk entries q < open_end are open curves
  for (int q = 0; q < m; ++q) {
    const uint32_t kq = sk[q];
    const bool prec = kq < mine || (kq == mine && base + q < i);
    before += prec;
    ob += prec && q < open_end;
  }
  if (before) atomicAdd(&rank[i], before);
  if (ob) atomicAdd(&open_before[i], ob);
}

// first_i = g_open * (open curves before i) + g_closed * (closed curves before i)
__global__ void curve_order_first_kernel(int n, int g_open, int g_closed, const uint32_t *rank, uint32_t *first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t ob = first[i];
  first[i] = ob * (uint32_t)g_open + (rank[i] - ob) * (uint32_t)g_closed;
}

Cfg to_cfg(const bs_sample_cfg &s) { return Cfg{s.g_open, s.rows_closed, s.k_closed, s.rho, s.cov_eps}; }

int max_samples(const bs_curves &c, const bs_sample_cfg &cfg) {
  int m = 0;
  if (c.n_open > 0) m = cfg.g_open;
  if (c.n_closed > 0) m = max(m, cfg.rows_closed * cfg.k_closed);
  return m;
}

int max_k(const bs_curves &c, const bs_sample_cfg &cfg) {
  int m = 0;
  if (c.n_open > 0) m = cfg.g_open;
  if (c.n_closed > 0) m = max(m, cfg.k_closed);
  return m;
}

size_t curve_smem(int n_max, int k_max, bool with_grad) {
  return sizeof(double2) * n_max + sizeof(double) * 4 * k_max + sizeof(double) * 64 * ((n_max + 63) / 64) +
         (with_grad ? sizeof(float2) * n_max : 0);
}

}  // namespace

bs_status launch_curve_order(const bs_curves &c, const bs_sample_cfg &cfg, uint32_t *rank, uint32_t *first,
                             cudaStream_t s) {
  const int n = c.n_open + c.n_closed;
  if (n == 0) return BS_OK;
  BS_CUDA(cudaMemsetAsync(rank, 0, sizeof(uint32_t) * n, s));
  BS_CUDA(cudaMemsetAsync(first, 0, sizeof(uint32_t) * n, s));
  const dim3 grid(div_up(n, kOrderThreads), div_up(n, kOrderChunk));
  curve_order_count_kernel<<<grid, kOrderThreads, 0, s>>>(c, rank, first);
  BS_LAUNCHED("curve_order_count_kernel");
  curve_order_first_kernel<<<div_up(n, 256), 256, 0, s>>>(n, cfg.g_open, cfg.rows_closed * cfg.k_closed, rank, first);
  BS_LAUNCHED("curve_order_first_kernel");
  return BS_OK;
}

bs_status launch_sample_fwd(const bs_curves &c, const bs_sample_cfg &cfg, float *gauss, cudaStream_t s) {
  const int n = c.n_open + c.n_closed;
  if (n == 0) return BS_OK;
  const int n_max = max_samples(c, cfg), k_max = max_k(c, cfg);
  const size_t smem = curve_smem(n_max, k_max, false);
  BS_CUDA(cudaFuncSetAttribute(sample_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sample_fwd_kernel<<<n, kCurveThreads, smem, s>>>(c, to_cfg(cfg), gauss, n_max, k_max);
  BS_LAUNCHED("sample_fwd_kernel");
  return BS_OK;
}

bs_status launch_sample_bwd(const bs_curves &c, const bs_sample_cfg &cfg, const float *dgauss,
                            const bs_curves_grad &g, cudaStream_t s) {
  const int n = c.n_open + c.n_closed;
  if (n == 0) return BS_OK;
  const int n_max = max_samples(c, cfg), k_max = max_k(c, cfg);
  const size_t smem = curve_smem(n_max, k_max, true);
  BS_CUDA(cudaFuncSetAttribute(sample_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sample_bwd_kernel<<<n, kCurveThreads, smem, s>>>(c, to_cfg(cfg), dgauss, g, n_max, k_max);
  BS_LAUNCHED("sample_bwd_kernel");
  return BS_OK;
}

}  // namespace bs
