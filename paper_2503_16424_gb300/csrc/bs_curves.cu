// Curves -> Gaussians: draw order (Section 3.3 "depth from area"), sampling
// (Section 3.3, Eq. 3-8, Eq. 11-12) and its backward.
//
// One CTA per curve (64 threads, 256 for curves of 512 samples or more).
// The CTA evaluates the curve's sample points X into
// shared memory, then each thread turns one sample and its neighbours into
// a Gaussian record (forward), or pushes one Gaussian's gradient back to the
// sample points and from there, with the Bernstein weights of Eq. 1-2, to the
// control points (backward).  A curve's Gaussians are contiguous in the
// draw-ordered table, so the backward needs no global atomics.
//
// Precision: a short tangent or a thin row spacing is the difference of two
// nearby sample points far from the curve's first control point, and
// subtracting two float32 positions would lose the digits it needs.  The
// sample points are therefore formed in float-float arithmetic (a float pair
// hi + lo carrying about 48 bits, from the error-free two-sum of Knuth and
// the FMA two-product, the construction of double-double arithmetic carried
// over to floats; FP64 units are a small fraction of FP32 ones on this GPU),
// relative to the first control point, and the difference vectors are taken
// in that arithmetic before being rounded to float32.  A closed curve's row r
// is (1 - tau_r) A + tau_r B (Eq. 4), so its points are X_A + tau_r (X_B - X_A)
// and its differences are those of the two boundaries interpolated by tau_r;
// the across-row difference is (tau_{r+1} - tau_r)(X_B - X_A), with the tau
// step from a product of sines, accurate however thin the row.  Everything
// after the difference vectors runs in float32.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "bs_internal.cuh"

namespace bs {
namespace {

__host__ __device__ inline int curve_threads(int n_max) { return n_max >= kWideSamples ? kCurveThreadsWide : kCurveThreads; }

struct Cfg {
  int g_open, rows, kc;
  float rho, eps;
  int tmode;  // 0: rotation from the neighbour difference (Eq. 8); 1: from B'(t)
};

// ---- float-float arithmetic: x = hi + lo, |lo| <= ulp(hi) / 2 ----
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {  // a + b exactly (Knuth)
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

__device__ __forceinline__ ff quick_sum(float a, float b) {  // a + b exactly when |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff two_prod(float a, float b) {  // a b exactly (one FMA)
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return quick_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const ff p = two_prod(a.hi, b.hi);
  return quick_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ float ff_round(ff a) { return __fadd_rn(a.hi, a.lo); }

// b - a of two float-float points (x.hi, x.lo, y.hi, y.lo), rounded to float
__device__ __forceinline__ float2 ff2_diff(const float4 &b, const float4 &a) {
  return make_float2(ff_round(ff_add(ff{b.x, b.y}, ff_neg(ff{a.x, a.y}))),
                     ff_round(ff_add(ff{b.z, b.w}, ff_neg(ff{a.z, a.w}))));
}

// Segment of sample k of K on a chain of S segments, u = k/(K-1):
// s = min(floor(S u), S-1), decided in integers.
__device__ __forceinline__ int chain_seg(int k, int K, int S) {
  const int s = (S * k) / (K - 1);
  return s > S - 1 ? S - 1 : s;
}

// First sample of segment s (0 <= s <= S): the least k with
// chain_seg(k, K, S) >= s, i.e. ceil(s (K - 1) / S); K for s = S.
__device__ __forceinline__ int seg_first(int s, int K, int S) { return s >= S ? K : (s * (K - 1) + S - 1) / S; }

// Local parameter t = S u - s = (S k - s (K - 1)) / (K - 1) in float-float
// (the remainder of a correctly rounded quotient is exact under an FMA).
__device__ __forceinline__ ff chain_t(int k, int K, int S, int s) {
  const float num = (float)(S * k - s * (K - 1)), den = (float)(K - 1);
  const float q = __fdiv_rn(num, den);
  return ff{q, __fdiv_rn(__fmaf_rn(-q, den, num), den)};
}

// The cubic Bernstein weights of Eq. 1-2 at t, in float-float.
__device__ __forceinline__ void bern3_ff(ff t, ff w[4]) {
  const ff u = ff_add(ff{1.f, 0.f}, ff_neg(t));
  const ff uu = ff_mul(u, u), tt = ff_mul(t, t), three{3.f, 0.f};
  w[0] = ff_mul(uu, u);
  w[1] = ff_mul(three, ff_mul(uu, t));
  w[2] = ff_mul(three, ff_mul(u, tt));
  w[3] = ff_mul(tt, t);
}

// Boundary groups of a closed curve: A = P0..P6, B = P0, P11, ..., P7, P6.
__device__ __forceinline__ int closed_b_index(int j) { return (j == 0 || j == 6) ? j : 12 - j; }

__device__ __forceinline__ const float *curve_ctrl(const bs_curves &c, int curve) {
  return curve < c.n_open ? c.open_ctrl + (size_t)curve * 20 : c.closed_ctrl + (size_t)(curve - c.n_open) * 24;
}

// Shared memory of the sampling kernels, per CTA (one curve), by column k
// (open curves: one column per sample; closed curves: a column of R2 rows):
//   Q    [12]     float4  control points minus the first one, float-float (x.hi, x.lo, y.hi, y.lo)
//   W    [k_max]  float4  Bernstein weights of column k (float, for the backward's gather)
//   XA   [k_max]  float4  the point of boundary A (open: the curve) at k, float-float, relative to P0
//   EA   [k_max]  float4  along-row difference e and tangent difference t of boundary A
//   EB   [k_max]  float4  the same of boundary B (closed)
//   D    [k_max]  float2  X_B - X_A (closed)
//   tau  [rows]   float2  (tau_r, tau_{r+1} - tau_r) (closed)
//   backward only: G [4][n_max] float2  per-sample gradient pieces, whose
//   first plane is overwritten with dL/dX by the gather.
//   XB   [k_max]  float4  boundary B while the columns are built (in G's place when there is a G)
struct CurveSmem {
  float4 *Q, *W, *XA, *EA, *EB, *XB;
  float2 *D, *tau, *G;
};

// Bytes of one curve's tables in carve's layout: n samples, k columns,
// rows rows; an open curve has no EB, XB, D or tau.
__host__ __device__ inline size_t curve_smem_bytes(bool closed, int n, int k, int rows, bool with_grad) {
  size_t b = sizeof(float4) * (12 + (closed ? 4 : 3) * (size_t)k);
  if (with_grad) b += sizeof(float2) * 4 * (size_t)(n > k ? n : k);  // G (XB in its place)
  else if (closed) b += sizeof(float4) * (size_t)k;                     // XB
  if (closed) b += sizeof(float2) * ((size_t)k + (size_t)rows);         // D, tau
  return b;
}

// The tables of one curve from its own sizes: the float4 tables first, then
// G (or XB), then the float2 tables, so that every table starts on a
// multiple of its element size.
__device__ __forceinline__ CurveSmem carve(void *base, bool closed, int n, int k, int rows, bool with_grad) {
  CurveSmem m;
  char *p = static_cast<char *>(base);
  m.Q = reinterpret_cast<float4 *>(p);
  p += sizeof(float4) * 12;
  m.W = reinterpret_cast<float4 *>(p);
  p += sizeof(float4) * k;
  m.XA = reinterpret_cast<float4 *>(p);
  p += sizeof(float4) * k;
  m.EA = reinterpret_cast<float4 *>(p);
  p += sizeof(float4) * k;
  m.EB = nullptr;
  if (closed) {
    m.EB = reinterpret_cast<float4 *>(p);
    p += sizeof(float4) * k;
  }
  m.XB = reinterpret_cast<float4 *>(p);  // with a G: in G's place ([k] float4 fits in [4][n] float2)
  m.G = nullptr;
  if (with_grad) {
    m.G = reinterpret_cast<float2 *>(p);
    p += sizeof(float2) * 4 * (size_t)(n > k ? n : k);
  } else if (closed) {
    p += sizeof(float4) * k;
  }
  m.D = m.tau = nullptr;
  if (closed) {
    m.D = reinterpret_cast<float2 *>(p);
    p += sizeof(float2) * k;
    m.tau = reinterpret_cast<float2 *>(p);
  }
  return m;
}

// Point of a boundary at column k: sum_i w_i Q[j(3s + i)], float-float.
__device__ __forceinline__ float4 boundary_point(const float4 *Q, const ff w[4], int s, bool b_side) {
  ff x{0.f, 0.f}, y{0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = b_side ? closed_b_index(3 * s + i) : 3 * s + i;
    const float4 q = Q[j];
    x = ff_add(x, ff_mul(w[i], ff{q.x, q.y}));
    y = ff_add(y, ff_mul(w[i], ff{q.z, q.w}));
  }
  return make_float4(x.hi, x.lo, y.hi, y.lo);
}

// Derivative weights of the cubic Bernstein basis at t (d/dt of Eq. 2):
// dB/dt = sum_i dw_i Q_i.
__device__ __forceinline__ float4 bern3_dt(float t) {
  const float u = 1.f - t;
  return make_float4(-3.f * u * u, 3.f * u * u - 6.f * u * t, 6.f * u * t - 3.f * t * t, 3.f * t * t);
}

// tangent_mode 1: dX/dt of a boundary at column k, the hodograph of its
// segment, 3 (u^2 (Q1 - Q0) + 2 u t (Q2 - Q1) + t^2 (Q3 - Q2)), u = 1 - t, from
// control-point differences taken in float-float (the same vector as
// sum_i dw_i Q_i, since the dw_i sum to 0).
__device__ __forceinline__ float2 boundary_tangent(const float4 *Q, int k, int K, int S, bool b_side) {
  const int s = chain_seg(k, K, S);
  const float t = ff_round(chain_t(k, K, S, s)), u = 1.f - t;
  float2 d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j0 = b_side ? closed_b_index(3 * s + i) : 3 * s + i;
    const int j1 = b_side ? closed_b_index(3 * s + i + 1) : 3 * s + i + 1;
    d[i] = ff2_diff(Q[j1], Q[j0]);
  }
  const float a = 3.f * u * u, b = 6.f * u * t, c = 3.f * t * t;
  return make_float2(a * d[0].x + b * d[1].x + c * d[2].x, a * d[0].y + b * d[1].y + c * d[2].y);
}

// Along-row difference e_k and tangent difference t_k of a column table X
// (one-sided at both ends), each rounded to float from float-float.
__device__ __forceinline__ float4 column_diffs(const float4 *X, int k, int K) {
  const float2 e = k + 1 < K ? ff2_diff(X[k + 1], X[k]) : ff2_diff(X[k], X[k - 1]);
  const float2 t = k == 0 ? ff2_diff(X[1], X[0]) : (k == K - 1 ? ff2_diff(X[k], X[k - 1]) : ff2_diff(X[k + 1], X[k - 1]));
  return make_float4(e.x, e.y, t.x, t.y);
}

// Fill the per-CTA column tables of one curve (ends with a barrier);
// returns its sample count.
__device__ int eval_samples(const bs_curves &c, const Cfg &cfg, int curve, const CurveSmem &m) {
  const bool closed = curve >= c.n_open;
  const float *P = curve_ctrl(c, curve);
  const int K = closed ? cfg.kc : cfg.g_open, S = closed ? 2 : 3, R2 = closed ? cfg.rows : 1;
  const int npts = closed ? 12 : 10;
  for (int j = threadIdx.x; j < npts; j += blockDim.x) {
    const ff x = two_sum(P[2 * j], -P[0]), y = two_sum(P[2 * j + 1], -P[1]);  // exact
    m.Q[j] = make_float4(x.hi, x.lo, y.hi, y.lo);
  }
  if (closed) {
    // tau_r = (1 - cos(pi r / N)) / 2 = sin^2(pi r / 2N), N = R2 - 1, and
    // tau_{r+1} - tau_r = sin(pi (2r + 1) / 2N) sin(pi / 2N)
    const float inv2n = 1.f / (float)(2 * (R2 - 1)), s1 = sinpif(inv2n);
    for (int r = threadIdx.x; r < R2; r += blockDim.x) {
      const float sr = sinpif((float)r * inv2n);
      m.tau[r] = make_float2(sr * sr, r + 1 < R2 ? sinpif((float)(2 * r + 1) * inv2n) * s1 : 0.f);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int s = chain_seg(k, K, S);
    ff w[4];
    bern3_ff(chain_t(k, K, S, s), w);
    m.W[k] = make_float4(ff_round(w[0]), ff_round(w[1]), ff_round(w[2]), ff_round(w[3]));
    m.XA[k] = boundary_point(m.Q, w, s, false);
    if (closed) m.XB[k] = boundary_point(m.Q, w, s, true);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float4 ea = column_diffs(m.XA, k, K);
    if (cfg.tmode) {  // the tangent from B'(t) instead of the neighbour difference
      const float2 ta = boundary_tangent(m.Q, k, K, S, false);
      ea.z = ta.x;
      ea.w = ta.y;
    }
    m.EA[k] = ea;
    if (closed) {
      float4 eb = column_diffs(m.XB, k, K);
      if (cfg.tmode) {
        const float2 tb = boundary_tangent(m.Q, k, K, S, true);
        eb.z = tb.x;
        eb.w = tb.y;
      }
      m.EB[k] = eb;
      m.D[k] = ff2_diff(m.XB[k], m.XA[k]);
    }
  }
  __syncthreads();
  return R2 * K;
}

// Local geometry of one sample (Eq. 7-8): the along-row difference e (for
// sigma_x), the tangent difference t (for the rotation), the across-row
// difference f (closed curves, for sigma_y); the scales; the unit tangent u;
// the mean relative to the first control point.
struct Local {
  float2 e, t, f;
  float le, lt, lf;  // their lengths
  float sx, sy, ux, uy;
  float mx, my;
};

__device__ __forceinline__ Local local_geometry(const CurveSmem &m, int idx, int K, int R2, bool closed,
                                                float width, float rho) {
  Local L;
  const int r = closed ? idx / K : 0;
  const int k = idx - r * K;
  const float4 ea = m.EA[k], xa = m.XA[k];
  if (closed) {
    const float tau = m.tau[r].x, omt = 1.f - tau;
    const float4 eb = m.EB[k];
    const float2 d = m.D[k];
    L.e = make_float2(omt * ea.x + tau * eb.x, omt * ea.y + tau * eb.y);
    L.t = make_float2(omt * ea.z + tau * eb.z, omt * ea.w + tau * eb.w);
    const float dt = r + 1 < R2 ? m.tau[r].y : m.tau[r - 1].y;
    L.f = make_float2(dt * d.x, dt * d.y);
    L.mx = xa.x + (xa.y + tau * d.x);
    L.my = xa.z + (xa.w + tau * d.y);
  } else {
    L.e = make_float2(ea.x, ea.y);
    L.t = make_float2(ea.z, ea.w);
    L.f = make_float2(0.f, 0.f);
    L.mx = xa.x + xa.y;
    L.my = xa.z + xa.w;
  }
  L.le = sqrtf(L.e.x * L.e.x + L.e.y * L.e.y);
  L.lt = sqrtf(L.t.x * L.t.x + L.t.y * L.t.y);
  L.sx = L.le / rho;
  if (closed) {
    L.lf = sqrtf(L.f.x * L.f.x + L.f.y * L.f.y);
    L.sy = L.lf / rho;
  } else {
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

// Width, opacity and colour of a sample.  Closed curves with a
// linear-gradient fill (Appendix D; closed_color2 / closed_opac2 non-NULL)
// interpolate from the values at P0 to those at P6 by the sample's position
// u = k / (K - 1) along its row: x = x0 + u (x1 - x0).
__device__ __forceinline__ float lerp_f(float a, float b, float u) { return a + u * (b - a); }

__device__ __forceinline__ CurveAttr curve_attr(const bs_curves &c, int curve, int seg, float u) {
  CurveAttr a;
  if (curve < c.n_open) {
    a.width = c.open_width[curve];
    a.opac = c.open_opac[curve * 3 + seg];
    a.col = make_float3(c.open_color[curve * 3], c.open_color[curve * 3 + 1], c.open_color[curve * 3 + 2]);
  } else {
    const int j = curve - c.n_open;
    a.width = 0.f;
    a.opac = c.closed_opac2 ? lerp_f(c.closed_opac[j], c.closed_opac2[j], u) : c.closed_opac[j];
    a.col = make_float3(c.closed_color[j * 3], c.closed_color[j * 3 + 1], c.closed_color[j * 3 + 2]);
    if (c.closed_color2)
      a.col = make_float3(lerp_f(a.col.x, c.closed_color2[j * 3], u), lerp_f(a.col.y, c.closed_color2[j * 3 + 1], u),
                          lerp_f(a.col.z, c.closed_color2[j * 3 + 2], u));
  }
  return a;
}

// u of sample idx of a closed curve with K samples per row
__device__ __forceinline__ float row_u(int idx, int K) {
  const int k = idx % K;
  return (float)k / (float)(K - 1);
}

// The sampling of curve `curve` of a batch: its image's.
__device__ __forceinline__ Cfg batch_cfg(const BatchImage *__restrict__ tab, int n_images, const bs_curves &c,
                                         int curve) {
  const int b = curve < c.n_open ? last_image_le<&BatchImage::open0>(tab, n_images, curve)
                                 : last_image_le<&BatchImage::closed0>(tab, n_images, curve - c.n_open);
  const BatchImage &im = tab[b];
  return Cfg{im.g_open, im.rows, im.kc, im.rho, im.eps, im.tmode};
}

// tab == nullptr: one canvas, sampling cfg, CTA b samples curve b; else a
// batch, CTA b samples curve curve_ids[b] with its image's sampling
// (dynamic shared memory sized for the largest curve of the launch).
__global__ void __launch_bounds__(kCurveThreadsWide) sample_fwd_kernel(bs_curves c, Cfg cfg, float *gauss,
                                                                   uint32_t *status,
                                                                   const BatchImage *tab = nullptr,
                                                                   int n_images = 0,
                                                                   const int32_t *curve_ids = nullptr) {
  extern __shared__ float4 smem_fwd[];
  const int curve = curve_ids ? curve_ids[blockIdx.x] : (int)blockIdx.x;
  const bool closed = curve >= c.n_open;
  if (tab) cfg = batch_cfg(tab, n_images, c, curve);
  const CurveSmem m = carve(smem_fwd, closed, closed ? cfg.rows * cfg.kc : cfg.g_open, closed ? cfg.kc : cfg.g_open,
                            closed ? cfg.rows : 1, false);
  const int n = eval_samples(c, cfg, curve, m);
  const int K = closed ? cfg.kc : cfg.g_open;
  const uint32_t first = c.draw_first[curve];
  const float *P = curve_ctrl(c, curve);
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int seg = closed ? 0 : chain_seg(idx, K, 3);
    const CurveAttr at = curve_attr(c, curve, seg, closed ? row_u(idx, K) : 0.f);
    const Local L = local_geometry(m, idx, K, cfg.rows, closed, at.width, cfg.rho);
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
    const float4 r0 = make_float4(P[0] + L.mx, P[1] + L.my, L.ux, L.uy);
    const float4 r1 = make_float4(rsqrtf(lx), rsqrtf(ly), at.opac, at.col.x);
    rec[0] = r0;
    rec[1] = r1;
    rec[2] = make_float4(at.col.y, at.col.z, ex, ey);
    // a non-finite record (0 * x is NaN exactly when x is not finite)
    const float probe = 0.f * r0.x + 0.f * r0.y + 0.f * r0.z + 0.f * r0.w + 0.f * r1.x + 0.f * r1.y + 0.f * r1.z +
                        0.f * r1.w + 0.f * at.col.y + 0.f * at.col.z;
    if (probe != 0.f) atomicOr(status, kDevErrNotFinite);
  }
}

__device__ __forceinline__ float w_at(const float4 &w, int i) { return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Backward of the sampling, without atomics on the geometry.  Phase 1: each
// sample turns its Gaussian's gradient into the gradients of its mean and
// of its three difference vectors (e: sigma_x, t: the rotation, f: sigma_y of
// a closed row), kept per sample.  Phase 2: each sample point gathers the
// pieces of every difference that uses it.  Phase 3: each control point
// coordinate gathers the Bernstein-weighted (and, for closed rows,
// tau-weighted, Eq. 4) gradients of the sample points it moves.
__global__ void __launch_bounds__(kCurveThreadsWide) sample_bwd_kernel(bs_curves c, Cfg cfg, const float *dgauss,
                                                                   bs_curves_grad g, uint32_t *status,
                                                                   const BatchImage *tab = nullptr,
                                                                   int n_images = 0,
                                                                   const int32_t *curve_ids = nullptr) {
  extern __shared__ float4 smem_bwd[];
  const int curve = curve_ids ? curve_ids[blockIdx.x] : (int)blockIdx.x;
  if (tab) cfg = batch_cfg(tab, n_images, c, curve);
  const bool closed = curve >= c.n_open;
  const int n_here = closed ? cfg.rows * cfg.kc : cfg.g_open;
  const CurveSmem m = carve(smem_bwd, closed, n_here, closed ? cfg.kc : cfg.g_open, closed ? cfg.rows : 1, true);
  float2 *GM = m.G, *GE = m.G + n_here, *GT = m.G + 2 * n_here, *GF = m.G + 3 * n_here;
  // opac[3] (open) or opac (closed), colour[3], width, then (gradient
  // fills) the far-end opacity [7] and colour [8..10]
  __shared__ float sAttr[12];
  if (threadIdx.x < 12) sAttr[threadIdx.x] = 0.f;
  const int n = eval_samples(c, cfg, curve, m);
  const int K = closed ? cfg.kc : cfg.g_open, R2 = closed ? cfg.rows : 1;
  const uint32_t first = c.draw_first[curve];
  const int lane = threadIdx.x & 31;
  const int n_rounds = div_up(n, blockDim.x);
  for (int round = 0; round < n_rounds; ++round) {
    const int idx = round * blockDim.x + threadIdx.x;
    float d_op[3] = {0.f, 0.f, 0.f}, d_col[3] = {0.f, 0.f, 0.f}, d_w = 0.f;
    float d_op2 = 0.f, d_col2[3] = {0.f, 0.f, 0.f};
    if (idx < n) {
      const int seg = closed ? 0 : chain_seg(idx, K, 3);
      const float u = closed ? row_u(idx, K) : 0.f;
      const CurveAttr at = curve_attr(c, curve, seg, u);
      const Local L = local_geometry(m, idx, K, cfg.rows, closed, at.width, cfg.rho);
      const float *dg = dgauss + (size_t)(first + idx) * BS_DGAUSS_FLOATS;
      const float4 d0 = *reinterpret_cast<const float4 *>(dg);      // mx, my, ux, uy
      const float4 d1 = *reinterpret_cast<const float4 *>(dg + 4);  // isx, isy, o, r
      const float4 d2 = *reinterpret_cast<const float4 *>(dg + 8);  // g, b, -, -
      // isx = (sx^2 + eps)^-1/2  ->  d isx / d sx = -sx isx^3
      const float isx = rsqrtf(L.sx * L.sx + cfg.eps), isy = rsqrtf(L.sy * L.sy + cfg.eps);
      const float dsx = -d1.x * L.sx * isx * isx * isx;
      const float dsy = -d1.y * L.sy * isy * isy * isy;
      GM[idx] = make_float2(d0.x, d0.y);
      // sigma_x = |e| / rho
      const float ke = L.le > 0.f ? dsx / (L.le * cfg.rho) : 0.f;
      GE[idx] = make_float2(ke * L.e.x, ke * L.e.y);
      // u = t / |t|  ->  dL/dt = (du - u (u . du)) / |t|
      if (L.lt > 0.f) {
        const float proj = L.ux * d0.z + L.uy * d0.w;
        GT[idx] = make_float2((d0.z - L.ux * proj) / L.lt, (d0.w - L.uy * proj) / L.lt);
      } else {
        GT[idx] = make_float2(0.f, 0.f);
      }
      if (closed) {
        const float kf = L.lf > 0.f ? dsy / (L.lf * cfg.rho) : 0.f;
        GF[idx] = make_float2(kf * L.f.x, kf * L.f.y);
        if (c.closed_opac2) {
          d_op[0] = (1.f - u) * d1.z;
          d_op2 = u * d1.z;
        } else {
          d_op[0] = d1.z;
        }
      } else {
        GF[idx] = make_float2(0.f, 0.f);
        d_w = dsy;
        d_op[seg] = d1.z;
      }
      d_col[0] = d1.w;
      d_col[1] = d2.x;
      d_col[2] = d2.y;
      if (closed && c.closed_color2) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          d_col2[i] = u * d_col[i];
          d_col[i] -= d_col2[i];
        }
      }
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
    if (closed && (c.closed_opac2 || c.closed_color2)) {
      const float o2 = warp_sum(d_op2);
      if (lane == 0) atomicAdd(&sAttr[7], o2);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float b2 = warp_sum(d_col2[i]);
        if (lane == 0) atomicAdd(&sAttr[8 + i], b2);
      }
    }
  }
  __syncthreads();
  // phase 2: dL/dX_m from the differences that use sample m (see local_geometry)
  for (int mi = threadIdx.x; mi < n; mi += blockDim.x) {
    const int r = mi / K, k = mi - r * K;
    float2 d = GM[mi];
    // e_k = X_{k+1} - X_k (k < K-1), X_k - X_{k-1} (k = K-1)
    if (k >= 1) { d.x += GE[mi - 1].x; d.y += GE[mi - 1].y; }
    if (k == K - 1) { d.x += GE[mi].x; d.y += GE[mi].y; }
    if (k < K - 1) { d.x -= GE[mi].x; d.y -= GE[mi].y; }
    if (k == K - 2) { d.x -= GE[mi + 1].x; d.y -= GE[mi + 1].y; }
    // t_k = X_{k+1} - X_{k-1}, one-sided at both ends (tangent_mode 0; in
    // mode 1 t_k is B'(t), which phase 3 takes to the control points)
    if (!cfg.tmode) {
      if (k >= 1) { d.x += GT[mi - 1].x; d.y += GT[mi - 1].y; }
      if (k == K - 1) { d.x += GT[mi].x; d.y += GT[mi].y; }
      if (k <= K - 2) { d.x -= GT[mi + 1].x; d.y -= GT[mi + 1].y; }
      if (k == 0) { d.x -= GT[mi].x; d.y -= GT[mi].y; }
    }
    if (closed) {
      // f_k = X_{r+1,k} - X_{r,k} (r < R2-1), X_{r,k} - X_{r-1,k} (last row)
      if (r >= 1) { d.x += GF[mi - K].x; d.y += GF[mi - K].y; }
      if (r == R2 - 1) { d.x += GF[mi].x; d.y += GF[mi].y; }
      if (r < R2 - 1) { d.x -= GF[mi].x; d.y -= GF[mi].y; }
      if (r == R2 - 2) { d.x -= GF[mi + K].x; d.y -= GF[mi + K].y; }
    }
    GM[mi] = d;  // only this thread reads GM[mi]
  }
  __syncthreads();
  // phase 3: control points (Eq. 1-2; closed rows through Eq. 4)
  const float2 *dX = GM;
  const int npts = closed ? 12 : 10;
  const int S = closed ? 2 : 3;
  // Row r of a closed curve is (1 - tau_r) A + tau_r B (Eq. 4), so the
  // gradient of a boundary point through column k is the same Bernstein
  // weight times sum_r (1 - tau_r) dX_rk (boundary A) or sum_r tau_r dX_rk
  // (boundary B): those column sums first (one thread per column), kept in
  // the no longer needed GE / GT planes, then every control point runs over
  // the K columns only.
  // With tangent_mode 1 the row tangents t_rk = (1 - tau_r) tA_k + tau_r tB_k
  // (local_geometry) are summed the same way into tangent columns (the GF
  // plane, free after phase 2; GT is then still read, so the point columns
  // go to the GE plane alone: R2 >= 2, so it holds both).  Open curves use
  // dX and GT as their columns.
  float2 *colA = GE, *colB = cfg.tmode ? GE + K : GT;
  const float2 *colTA = GT, *colTB = GT;
  if (closed) {
    float2 *tA = GF, *tB = GF + K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
      float2 ta = make_float2(0.f, 0.f), tb = make_float2(0.f, 0.f);
      for (int r = 0; r < R2; ++r) {
        const float tau = m.tau[r].x;
        const float2 dx = dX[r * K + k];
        a.x += (1.f - tau) * dx.x;
        a.y += (1.f - tau) * dx.y;
        b.x += tau * dx.x;
        b.y += tau * dx.y;
        if (cfg.tmode) {
          const float2 gt = GT[r * K + k];
          ta.x += (1.f - tau) * gt.x;
          ta.y += (1.f - tau) * gt.y;
          tb.x += tau * gt.x;
          tb.y += tau * gt.y;
        }
      }
      if (cfg.tmode) {
        tA[k] = ta;
        tB[k] = tb;
      }
      colA[k] = a;
      colB[k] = b;
    }
    __syncthreads();
    colTA = tA;
    colTB = tB;
  }
  // Each (control point, segment it shapes, coordinate) item sums over that
  // segment's samples only (a contiguous k range, no division per sample);
  // then each control point coordinate adds its items in a fixed order.
  // Items q = 0..n_items/2-1 per coordinate: open, q < 10: P_q on segment
  // min(q/3, 2); q = 10, 11: P3 on segment 0, P6 on segment 1 (weight 3).
  // Closed, side A (q < 8) and B (q >= 8), boundary index j = q % 8 < 7 on
  // segment min(j/3, 1), and j = 3 on segment 0 for q % 8 = 7.
  __shared__ float s_item[64];
  const int n_items = closed ? 32 : 24;
  for (int it = threadIdx.x; it < n_items; it += blockDim.x) {
    const int comp = it & 1, q = it >> 1;
    int j, sg;
    const float2 *src = dX, *srcT = colTA;
    if (!closed) {
      j = q < 10 ? q : (q == 10 ? 3 : 6);
      sg = q < 10 ? min(q / 3, 2) : (q == 10 ? 0 : 1);
    } else {
      const int r = q & 7;
      j = r < 7 ? r : 3;
      sg = r < 7 ? min(r / 3, 1) : 0;
      src = q < 8 ? colA : colB;
      srcT = q < 8 ? colTA : colTB;
    }
    const int i = j - 3 * sg;
    const int k0 = seg_first(sg, K, S), k1 = seg_first(sg + 1, K, S);
    float acc = 0.f;
    for (int k = k0; k < k1; ++k) acc += w_at(m.W[k], i) * (comp ? src[k].y : src[k].x);
    if (cfg.tmode) {  // t_k = sum_i dw_i(t_k) Q_i (Eq. 1 differentiated)
      for (int k = k0; k < k1; ++k) {
        const float4 dw = bern3_dt(ff_round(chain_t(k, K, S, sg)));
        acc += w_at(dw, i) * (comp ? srcT[k].y : srcT[k].x);
      }
    }
    s_item[it] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * npts; t += blockDim.x) {
    const int p = t >> 1, comp = t & 1;
    float acc = 0.f;
    for (int q = 0; q < n_items / 2; ++q) {
      int pq;  // the control point item q shapes
      if (!closed) {
        pq = q < 10 ? q : (q == 10 ? 3 : 6);
      } else {
        const int r = q & 7, j = r < 7 ? r : 3;
        pq = q < 8 ? j : closed_b_index(j);
      }
      if (pq == p) acc += s_item[2 * q + comp];
    }
    if (!closed) g.open_ctrl[(size_t)curve * 20 + t] = acc;
    else g.closed_ctrl[(size_t)(curve - c.n_open) * 24 + t] = acc;
    if (0.f * acc != 0.f) atomicOr(status, kDevErrNotFinite);
  }
  if (threadIdx.x < 11 && 0.f * sAttr[threadIdx.x] != 0.f) atomicOr(status, kDevErrNotFinite);
  if (!closed) {
    if (threadIdx.x < 3) {
      g.open_opac[curve * 3 + threadIdx.x] = sAttr[threadIdx.x];
      g.open_color[curve * 3 + threadIdx.x] = sAttr[3 + threadIdx.x];
    }
    if (threadIdx.x == 0) g.open_width[curve] = sAttr[6];
  } else {
    const int j = curve - c.n_open;
    if (threadIdx.x < 3) g.closed_color[j * 3 + threadIdx.x] = sAttr[3 + threadIdx.x];
    if (threadIdx.x == 0) g.closed_opac[j] = sAttr[0];
    if (c.closed_color2 && g.closed_color2 && threadIdx.x < 3) g.closed_color2[j * 3 + threadIdx.x] = sAttr[8 + threadIdx.x];
    if (c.closed_opac2 && g.closed_opac2 && threadIdx.x == 0) g.closed_opac2[j] = sAttr[7];
  }
}

// ---- draw order ----
__device__ __forceinline__ float area_key(const bs_curves &c, int i) {
  return curve_area_key(c.n_open, c.open_ctrl, c.open_width, c.closed_ctrl, i);
}

constexpr int kOrderThreads = 256;
constexpr int kOrderChunk = 256;  // keys compared per CTA

// The keys among sk[q0, q1) below `mine` (kLe: or equal to it), four at a
// time from the first multiple of 4 (sk 16-byte aligned).
template <bool kLe>
__device__ __forceinline__ uint32_t count_keys(const uint32_t *sk, int q0, int q1, uint32_t mine) {
  uint32_t c = 0;
  int q = q0;
  for (; q < q1 && (q & 3); ++q) c += kLe ? sk[q] <= mine : sk[q] < mine;
  for (; q + 4 <= q1; q += 4) {
    const uint4 k = *reinterpret_cast<const uint4 *>(sk + q);
    c += kLe ? (uint32_t)(k.x <= mine) + (k.y <= mine) + (k.z <= mine) + (k.w <= mine)
             : (uint32_t)(k.x < mine) + (k.y < mine) + (k.z < mine) + (k.w < mine);
  }
  for (; q < q1; ++q) c += kLe ? sk[q] <= mine : sk[q] < mine;
  return c;
}

// Of the chunk entries q < m (curve base + q, key sk[q]), those preceding
// curve i (key mine): an entry before i precedes it when its key is <= mine,
// one at or after i when its key is < mine.  `before` counts them all, `ob`
// those with q < open_end (the open curves).
__device__ __forceinline__ void count_preceding(const uint32_t *sk, int m, int base, int i, uint32_t mine,
                                                int open_end, uint32_t &before, uint32_t &ob) {
  const int e = min(max(i - base, 0), m), oe = min(max(open_end, 0), m);
  const int lo = min(e, oe), hi = max(e, oe);
  const uint32_t a = count_keys<true>(sk, 0, lo, mine);     // before i, open
  const uint32_t b = count_keys<true>(sk, lo, e, mine);     // before i, closed (oe < e)
  const uint32_t d = count_keys<false>(sk, e, hi, mine);    // after i, open (oe > e)
  const uint32_t f = count_keys<false>(sk, hi, m, mine);    // after i, closed
  before = a + b + d + f;
  ob = a + d;
}

// Rank by counting: rank_i = #{j : key_j < key_i or (key_j == key_i, j < i)}.
// CTA (x, y) compares its 256 curves against the keys of chunk y and adds its
// counts (rank, and how many of the preceding curves are open) atomically.
__global__ void __launch_bounds__(kOrderThreads) curve_order_count_kernel(bs_curves c, uint32_t *rank,
                                                                         uint32_t *open_before) {
  __shared__ __align__(16) uint32_t sk[kOrderChunk];
  const int n = c.n_open + c.n_closed;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int base = blockIdx.y * kOrderChunk;
  const int m = min(kOrderChunk, n - base);
  for (int q = threadIdx.x; q < m; q += blockDim.x) sk[q] = key_order(area_key(c, base + q));
  const uint32_t mine = i < n ? key_order(area_key(c, i)) : 0u;
  __syncthreads();
  if (i >= n) return;
  uint32_t before, ob;
  count_preceding(sk, m, base, i, mine, c.n_open - base, before, ob);  // entries q < n_open - base are open
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

// Draw order of a batch: ranks within each image.  CTA k of the grid is
// (image b, chunk ci of its curves, chunk cj of the keys it compares with),
// k - order0_b = ci order_chunks_b + cj.  Image-local curve l is open curve
// open0_b + l for l < n_open_b, else closed curve closed0_b + l - n_open_b,
// and equal keys rank by l, as bs_curve_order does on the image alone.
__device__ __forceinline__ int batch_curve(const BatchImage &im, int total_open, int l) {
  return l < im.n_open ? (int)im.open0 + l : total_open + (int)im.closed0 + (l - im.n_open);
}

__global__ void __launch_bounds__(kOrderThreads) batch_curve_order_count_kernel(bs_curves c,
                                                                               const BatchImage *__restrict__ tab,
                                                                               int n_images, uint32_t *rank,
                                                                               uint32_t *open_before) {
  __shared__ __align__(16) uint32_t sk[kOrderChunk];
  const int b = last_image_le<&BatchImage::order0>(tab, n_images, blockIdx.x);
  const BatchImage &im = tab[b];
  const int local = blockIdx.x - (int)im.order0;
  const int ci = local / im.order_chunks, cj = local - ci * im.order_chunks;
  const int n = im.n_open + im.n_closed;
  const int i = ci * kOrderThreads + threadIdx.x;  // image-local
  const int base = cj * kOrderChunk;
  const int m = min(kOrderChunk, n - base);
  for (int q = threadIdx.x; q < m; q += blockDim.x) sk[q] = key_order(area_key(c, batch_curve(im, c.n_open, base + q)));
  const int gi = i < n ? batch_curve(im, c.n_open, i) : 0;
  const uint32_t mine = i < n ? key_order(area_key(c, gi)) : 0u;
  __syncthreads();
  if (i >= n) return;
  uint32_t before, ob;
  count_preceding(sk, m, base, i, mine, im.n_open - base, before, ob);  // entries q < n_open - base are open
  if (before) atomicAdd(&rank[gi], before);
  if (ob) atomicAdd(&open_before[gi], ob);
}

// first_i = gauss0_b + g_open_b (open curves before i) + G_closed_b (closed curves before i)
__global__ void batch_curve_order_first_kernel(bs_curves c, const BatchImage *__restrict__ tab, int n_images,
                                               const uint32_t *rank, uint32_t *first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.n_open + c.n_closed) return;
  const int b = i < c.n_open ? last_image_le<&BatchImage::open0>(tab, n_images, i)
                             : last_image_le<&BatchImage::closed0>(tab, n_images, i - c.n_open);
  const BatchImage &im = tab[b];
  const uint32_t ob = first[i];
  first[i] = (uint32_t)im.gauss0 + ob * (uint32_t)im.g_open + (rank[i] - ob) * (uint32_t)(im.rows * im.kc);
}

// ---- Xing loss (the convexity term of Eq. 13) ----
// Per cubic segment (A, B, C, D) of a closed curve, with u = B - A,
// v = C - B, w = D - C:
//   D1 = 1 if u x v >= 0 else 0,  D2 = (u x w) / (|u| |w|),
//   L  = D1 relu(-D2) + (1 - D1) relu(D2)
// (zero, with zero gradient, when |u| or |w| is 0).  One thread per closed
// curve walks its four segments (segment s: P_3s .. P_3s+3, P_12 = P_0), so
// its control-point gradient needs no atomics; the loss is lambda times the
// mean over all segments, added to *loss with one double atomic per CTA.
__global__ void xing_kernel(const float *__restrict__ ctrl, int n_closed, float lambda, double *__restrict__ loss,
                            float *__restrict__ grad) {
  __shared__ double s_sum[8];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (c < n_closed) {
    const float *P = ctrl + (size_t)c * 24;
    float g[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) g[i] = 0.f;
    const float scale = lambda / (4.f * (float)n_closed);
#pragma unroll
    for (int sgm = 0; sgm < 4; ++sgm) {
      const int ia = 3 * sgm, ib = ia + 1, ic = ia + 2, id = (ia + 3) % 12;
      const float ux = P[2 * ib] - P[2 * ia], uy = P[2 * ib + 1] - P[2 * ia + 1];
      const float vx = P[2 * ic] - P[2 * ib], vy = P[2 * ic + 1] - P[2 * ib + 1];
      const float wx = P[2 * id] - P[2 * ic], wy = P[2 * id + 1] - P[2 * ic + 1];
      const float nu = sqrtf(ux * ux + uy * uy), nw = sqrtf(wx * wx + wy * wy);
      if (!(nu > 0.f) || !(nw > 0.f)) continue;
      const float d1 = (ux * vy - uy * vx) >= 0.f ? 1.f : 0.f;
      const float cr = ux * wy - uy * wx, inv = 1.f / (nu * nw), d2 = cr * inv;
      l += d1 * fmaxf(-d2, 0.f) + (1.f - d1) * fmaxf(d2, 0.f);
      const float sgn = (d1 > 0.f && d2 < 0.f) ? -1.f : ((d1 == 0.f && d2 > 0.f) ? 1.f : 0.f);  // dL/dD2
      if (sgn == 0.f) continue;
      // dD2/du = (w_y, -w_x) inv - D2 u / |u|^2,  dD2/dw = (-u_y, u_x) inv - D2 w / |w|^2
      const float k = sgn * scale;
      const float dux = k * (wy * inv - d2 * ux / (nu * nu)), duy = k * (-wx * inv - d2 * uy / (nu * nu));
      const float dwx = k * (-uy * inv - d2 * wx / (nw * nw)), dwy = k * (ux * inv - d2 * wy / (nw * nw));
      g[2 * ia] -= dux;
      g[2 * ia + 1] -= duy;
      g[2 * ib] += dux;
      g[2 * ib + 1] += duy;
      g[2 * ic] -= dwx;
      g[2 * ic + 1] -= dwy;
      g[2 * id] += dwx;
      g[2 * id + 1] += dwy;
    }
    if (grad) {
      float *G = grad + (size_t)c * 24;
#pragma unroll
      for (int i = 0; i < 24; ++i) G[i] += g[i];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_sum[w];
    if (t != 0.0) atomicAdd(loss, t * (double)lambda / (4.0 * (double)n_closed));
  }
}

Cfg to_cfg(const bs_sample_cfg &s) {
  return Cfg{s.g_open, s.rows_closed, s.k_closed, s.rho, s.cov_eps, s.tangent_mode};
}

int max_samples(const bs_curves &c, const bs_sample_cfg &cfg) {
  int m = 0;
  if (c.n_open > 0) m = cfg.g_open;
  if (c.n_closed > 0) m = max(m, cfg.rows_closed * cfg.k_closed);
  return m;
}

// Shared memory for a launch whose largest open curve has open_g samples
// and whose largest closed curve closed_n samples in closed_rows rows of
// closed_k (0: no such curve).
size_t launch_smem(int open_g, int closed_n, int closed_k, int closed_rows, bool with_grad) {
  size_t b = 0;
  if (open_g > 0) b = curve_smem_bytes(false, open_g, open_g, 1, with_grad);
  if (closed_n > 0) b = std::max(b, curve_smem_bytes(true, closed_n, closed_k, closed_rows, with_grad));
  return b;
}

size_t launch_smem(const BatchPlan::SampleClass &k, bool with_grad) {
  return launch_smem(k.open_g, k.closed_n, k.closed_k, k.closed_rows, with_grad);
}

size_t launch_smem(const bs_curves &c, const bs_sample_cfg &cfg, bool with_grad) {
  return launch_smem(c.n_open > 0 ? cfg.g_open : 0, c.n_closed > 0 ? cfg.rows_closed * cfg.k_closed : 0,
                     cfg.k_closed, cfg.rows_closed, with_grad);
}

}  // namespace

// Dynamic shared memory of the sampling kernels: the attribute is raised
// per device and kernel to the largest size asked so far, never lowered (a
// batch sizes it for its largest image).
template <typename Kernel>
bs_status raise_smem(Kernel k, size_t smem, int slot) {
  constexpr int kMaxDev = 64;
  static size_t done[kMaxDev][2] = {};  // per device and slot, under mu
  static std::mutex mu;
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) {
    set_error("device %d: at most %d devices supported", dev, kMaxDev);
    return BS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (smem > done[dev][slot]) {
    BS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done[dev][slot] = smem;
  }
  return BS_OK;
}

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
  const size_t smem = launch_smem(c, cfg, false);
  BS_TRY(raise_smem(sample_fwd_kernel, smem, 0));
  uint32_t *status = nullptr;
  BS_TRY(lib_status_word(&status));
  sample_fwd_kernel<<<n, curve_threads(max_samples(c, cfg)), smem, s>>>(c, to_cfg(cfg), gauss, status);
  BS_LAUNCHED("sample_fwd_kernel");
  return BS_OK;
}

bs_status launch_sample_bwd(const bs_curves &c, const bs_sample_cfg &cfg, const float *dgauss,
                            const bs_curves_grad &g, cudaStream_t s) {
  const int n = c.n_open + c.n_closed;
  if (n == 0) return BS_OK;
  const size_t smem = launch_smem(c, cfg, true);
  BS_TRY(raise_smem(sample_bwd_kernel, smem, 1));
  uint32_t *status = nullptr;
  BS_TRY(lib_status_word(&status));
  sample_bwd_kernel<<<n, curve_threads(max_samples(c, cfg)), smem, s>>>(c, to_cfg(cfg), dgauss, g, status);
  BS_LAUNCHED("sample_bwd_kernel");
  return BS_OK;
}

bs_status launch_batch_curve_order(const BatchPlan &p, const BatchImage *table, const bs_curves &c,
                                   uint32_t *rank, uint32_t *first, cudaStream_t s) {
  const int n = c.n_open + c.n_closed;
  if (n == 0) return BS_OK;
  BS_CUDA(cudaMemsetAsync(rank, 0, sizeof(uint32_t) * n, s));
  BS_CUDA(cudaMemsetAsync(first, 0, sizeof(uint32_t) * n, s));
  batch_curve_order_count_kernel<<<(unsigned)p.order_ctas, kOrderThreads, 0, s>>>(c, table, p.n_images, rank, first);
  BS_LAUNCHED("batch_curve_order_count_kernel");
  batch_curve_order_first_kernel<<<div_up(n, 256), 256, 0, s>>>(c, table, p.n_images, rank, first);
  BS_LAUNCHED("batch_curve_order_first_kernel");
  return BS_OK;
}

bs_status launch_batch_sample_fwd(const BatchPlan &p, const BatchImage *table, const int32_t *curve_ids,
                                  const bs_curves &c, float *gauss, cudaStream_t s) {
  // curves below kWideSamples samples on narrow CTAs, the rest on wide ones
  // (curve_ids lists the narrow curves, then the wide ones), each launch
  // with the shared memory of its own largest curves
  uint32_t *status = nullptr;
  BS_TRY(lib_status_word(&status));
  if (p.narrow.n_curves > 0) {
    const size_t smem = launch_smem(p.narrow, false);
    BS_TRY(raise_smem(sample_fwd_kernel, smem, 0));
    sample_fwd_kernel<<<(unsigned)p.narrow.n_curves, kCurveThreads, smem, s>>>(c, Cfg{}, gauss, status, table,
                                                                               p.n_images, curve_ids);
    BS_LAUNCHED("sample_fwd_kernel");
  }
  if (p.wide.n_curves > 0) {
    const size_t smem = launch_smem(p.wide, false);
    BS_TRY(raise_smem(sample_fwd_kernel, smem, 0));
    sample_fwd_kernel<<<(unsigned)p.wide.n_curves, kCurveThreadsWide, smem, s>>>(c, Cfg{}, gauss, status, table,
                                                                                 p.n_images,
                                                                                 curve_ids + p.narrow.n_curves);
    BS_LAUNCHED("sample_fwd_kernel");
  }
  return BS_OK;
}

bs_status launch_batch_sample_bwd(const BatchPlan &p, const BatchImage *table, const int32_t *curve_ids,
                                  const bs_curves &c, const float *dgauss, const bs_curves_grad &g,
                                  cudaStream_t s) {
  uint32_t *status = nullptr;
  BS_TRY(lib_status_word(&status));
  if (p.narrow.n_curves > 0) {
    const size_t smem = launch_smem(p.narrow, true);
    BS_TRY(raise_smem(sample_bwd_kernel, smem, 1));
    sample_bwd_kernel<<<(unsigned)p.narrow.n_curves, kCurveThreads, smem, s>>>(c, Cfg{}, dgauss, g, status, table,
                                                                               p.n_images, curve_ids);
    BS_LAUNCHED("sample_bwd_kernel");
  }
  if (p.wide.n_curves > 0) {
    const size_t smem = launch_smem(p.wide, true);
    BS_TRY(raise_smem(sample_bwd_kernel, smem, 1));
    sample_bwd_kernel<<<(unsigned)p.wide.n_curves, kCurveThreadsWide, smem, s>>>(c, Cfg{}, dgauss, g, status,
                                                                                 table, p.n_images,
                                                                                 curve_ids + p.narrow.n_curves);
    BS_LAUNCHED("sample_bwd_kernel");
  }
  return BS_OK;
}

bs_status launch_xing(const bs_curves &c, float lambda, double *loss, float *grad_closed_ctrl, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
  if (c.n_closed == 0) return BS_OK;
  xing_kernel<<<div_up(c.n_closed, 256), 256, 0, s>>>(c.closed_ctrl, c.n_closed, lambda, loss, grad_closed_ctrl);
  BS_LAUNCHED("xing_kernel");
  return BS_OK;
}

}  // namespace bs
