// Per-tile alpha blending (Section 3.4, Eq. 9-10) and its reverse-order
// backward, plus the L2 term of Eq. 13.
//
// One CTA per T x T tile, T = 8, 16 or 32 (Geo<T>).  A warp covers a region
// of 8x4-pixel blocks: 8 x 8 pixels (two blocks) for T = 8, 16 x 8 pixels
// (four blocks) for T = 16 and 32, so a tile has 1, 2 or 8 warps.  Lane l
// owns pixel (l & 7, l >> 3) of each of its warp's blocks (its slots).  The
// tile's list is staged into shared memory one Gaussian per thread at a
// time (in the forward by cp.async, one batch ahead of the blend), each
// with one bit per block of the tile telling whether its
// alpha >= 1/255 region reaches the block, so a warp skips a block for a
// Gaussian without touching its pixels, and the work of a slot stays within
// one compact block.
//
// A Gaussian is stored by its eigen-frame (Eq. 11-12): Sigma^-1 =
// R diag(isx^2, isy^2) R^T with R = [[ux, -uy], [uy, ux]], and is staged as the
// two scaled axes
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

// Geometry of a T x T tile.
template <int kT>
struct Geo {
  static_assert(kT == 8 || kT == 16 || kT == 32, "tile side 8, 16 or 32");
  static constexpr int kBC = kT == 8 ? 1 : 2;        // 8x4 block columns per warp
  static constexpr int kWX = kT / (8 * kBC);         // warps across the tile
  static constexpr int kWY = kT / 8;                 // warps down the tile (two block rows each)
  static constexpr int kWarps = kWX * kWY;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kPix = 2 * kBC;               // pixels (slots) per thread
  static constexpr int kBatch = kThreads;            // Gaussians staged per round
  static constexpr int kBits = kWarps * kPix;        // block bits of a tile
  static constexpr uint32_t kSlotMask = (1u << kPix) - 1u;
  // bit of block (bc, br) of the tile: warp-major, then slot
  __host__ __device__ static constexpr int bit(int bc, int br) {
    return kPix * ((br >> 1) * kWX + bc / kBC) + (bc % kBC) + kBC * (br & 1);
  }
  __host__ __device__ static constexpr unsigned bcol(unsigned b) { return ((b / kPix) % kWX) * kBC + (b % kPix) % kBC; }
  __host__ __device__ static constexpr unsigned brow(unsigned b) { return 2 * ((b / kPix) / kWX) + (b % kPix) / kBC; }
  // the bits of block row br for the block columns in `cols`
  __host__ __device__ static constexpr uint32_t row_bits(uint32_t cols, int br) {
    return kT == 8 ? cols << br
         : kT == 16 ? cols << (2 * br)
                    : ((cols & 3u) | ((cols & 12u) << 2)) << (8 * (br >> 1) + 2 * (br & 1));
  }
};
static_assert(Geo<16>::bit(1, 3) == 7 && Geo<16>::bcol(7) == 1 && Geo<16>::brow(7) == 3, "T = 16 block bits");
static_assert(Geo<32>::row_bits(15u, 5) == ((1u << Geo<32>::bit(0, 5)) | (1u << Geo<32>::bit(1, 5)) |
                                            (1u << Geo<32>::bit(2, 5)) | (1u << Geo<32>::bit(3, 5))),
              "T = 32 row bits");
static_assert(Geo<32>::bcol(Geo<32>::bit(3, 6)) == 3 && Geo<32>::brow(Geo<32>::bit(3, 6)) == 6, "T = 32 block bits");
static_assert(Geo<8>::row_bits(1u, 1) == (1u << Geo<8>::bit(0, 1)), "T = 8 row bits");
static_assert(Geo<32>::kBits == 32 && Geo<8>::kBits == 2, "block bits fit a word");
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kKappa = 0.84932180028801907f;      // sqrt(log2(e) / 2)
constexpr float kLog2_255 = 7.99435343685885793f;   // alpha >= 1/255 <=> t1^2 + t2^2 <= log2(o) + log2(255)

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Staged {
  float4 a;  // mx, my, A1, B1
  float4 b;  // A2, B2, log2(o), r
  float2 c;  // g, b
  float2 ext;
};

__device__ __forceinline__ void scaled_axes(float ux, float uy, float isx, float isy, float &A1, float &B1,
                                            float &A2, float &B2) {
  const float kx = __fmul_rn(kKappa, isx), ky = __fmul_rn(kKappa, isy);
  A1 = __fmul_rn(kx, ux);
  B1 = __fmul_rn(kx, uy);
  A2 = __fmul_rn(ky, -uy);
  B2 = __fmul_rn(ky, ux);
}

// Stage one record (its three float4s); an index past the table (only
// possible after a sort that gave up waiting) stages an invisible Gaussian.
__device__ __forceinline__ Staged stage_none() {
  Staged s;
  s.a = make_float4(0.f, 0.f, 0.f, 0.f);
  s.b = make_float4(0.f, 0.f, -INFINITY, 0.f);
  s.c = make_float2(0.f, 0.f);
  s.ext = make_float2(-1.f, -1.f);
  return s;
}

__device__ __forceinline__ Staged stage_rec(const float4 r0, const float4 r1, const float4 r2) {
  Staged s;
  float A1, B1, A2, B2;
  scaled_axes(r0.z, r0.w, r1.x, r1.y, A1, B1, A2, B2);
  const float o = r1.z;
  s.a = make_float4(r0.x, r0.y, A1, B1);
  s.b = make_float4(A2, B2, o > 0.f ? lg2_approx(o) : -INFINITY, r1.w);
  s.c = make_float2(r2.x, r2.y);
  s.ext = make_float2(r2.z, r2.w);
  return s;
}

// Stage Gaussian g straight from global memory (the backward's path).
__device__ __forceinline__ Staged stage(const float *__restrict__ gauss, uint32_t g, uint32_t n_gauss) {
  if (g >= n_gauss) return stage_none();
  const float4 *rec = reinterpret_cast<const float4 *>(gauss + (size_t)g * BS_GAUSS_FLOATS);
  return stage_rec(__ldg(rec), __ldg(rec + 1), __ldg(rec + 2));
}

// Asynchronous staging of a tile's list (the forward's path).  While the
// CTA blends one batch of kBatch entries, thread t has in flight the
// cp.async copies of its entry of the next batch (the 48-byte record, three
// 16-byte copies into rec[.][t]) and of its key two batches ahead (into
// key[.][t]).  A thread reads only the slots it wrote, so
// cp.async.wait_group alone makes them visible; a slot is overwritten only
// after the thread has consumed what it held (the copy is issued after the
// instructions that use the loaded values).  The backward stages with plain
// loads: the same prefetch there measured 2 % slower (5 % more warp
// instructions at the same occupancy).
template <int kBatch>
struct StageBuf {
  float4 rec[3][kBatch];
  uint32_t key[2][kBatch];
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Copy Gaussian g's record into this thread's slot (nothing for g past the
// table; stage_slot stages it as invisible).
template <int kBatch>
__device__ __forceinline__ void issue_rec(StageBuf<kBatch> &buf, const float *__restrict__ gauss, uint32_t g,
                                          uint32_t n_gauss) {
  if (g >= n_gauss) return;
  const float4 *rec = reinterpret_cast<const float4 *>(gauss + (size_t)g * BS_GAUSS_FLOATS);
#pragma unroll
  for (int k = 0; k < 3; ++k) cp_async16(&buf.rec[k][threadIdx.x], rec + k);
}

template <int kBatch>
__device__ __forceinline__ Staged stage_slot(const StageBuf<kBatch> &buf, uint32_t g, uint32_t n_gauss) {
  if (g >= n_gauss) return stage_none();
  return stage_rec(buf.rec[0][threadIdx.x], buf.rec[1][threadIdx.x], buf.rec[2][threadIdx.x]);
}

// Bit Geo<T>::bit(block_col, block_row) set: the Gaussian can reach alpha
// >= 1/255 at some pixel centre of the 8x4 block (block_col, block_row) of
// the tile whose first pixel is (x0, y0), by an exact test per block row.
// With q = t1^2 + t2^2 = axx dx^2 + 2 axy dx dy + byy dy^2 and L the
// threshold, the chord of the ellipse q <= L at height dy is
//     dx in [r dy - h(dy), r dy + h(dy)],  r = -axy / axx,
//     h(dy) = sqrt((L - k dy^2) / axx),     k = det / axx,
// det = axx byy - axy^2 = (A1 B2 - A2 B1)^2.  Over a block row's band of
// pixel-centre heights the right end r dy + h(dy) is concave in dy, so its
// largest value is at the band point nearest the height of the ellipse's
// rightmost point, dy* = -(axy / byy) Xm with Xm = sqrt(L byy / det) (the
// left end likewise at -dy*): one chord per side and band gives the
// ellipse's x-extent in the band, tested against each block column.
// Conservative by a margin far above the float32 error of either side, so a
// cleared bit only skips pixels that the blend would skip anyway.
// The blocks whose pixel centres overlap the box mean +- ext (the fallback
// for a record without a proper frame).
template <int kT>
__device__ __forceinline__ uint32_t box_bits(const Staged &s, float ext_x, float ext_y, int x0, int y0) {
  using G = Geo<kT>;
  const float bx0 = s.a.x - ext_x - ((float)x0 + 0.5f), bx1 = s.a.x + ext_x - ((float)x0 + 0.5f);
  const float by0 = s.a.y - ext_y - ((float)y0 + 0.5f), by1 = s.a.y + ext_y - ((float)y0 + 0.5f);
  uint32_t cols = 0u, cand = 0u;
#pragma unroll
  for (int bc = 0; bc < kT / 8; ++bc)
    if (bx1 >= 8.f * bc - 0.5f && bx0 <= 8.f * bc + 7.5f) cols |= 1u << bc;
#pragma unroll
  for (int br = 0; br < kT / 4; ++br)
    if (by1 >= 4.f * br - 0.5f && by0 <= 4.f * br + 3.5f) cand |= G::row_bits(cols, br);
  return cand;
}

template <int kT>
__device__ __forceinline__ uint32_t block_bits(const Staged &s, float ext_x, float ext_y, int x0, int y0) {
  using G = Geo<kT>;
  const float thr = s.b.z + kLog2_255;
  if (!(thr >= 0.f)) return 0u;  // o < 1/255 (or not finite): never visible
  const float L = thr + (1e-2f + 1e-4f * thr);
  const float A1 = s.a.z, B1 = s.a.w, A2 = s.b.x, B2 = s.b.y;
  const float axx = A1 * A1 + A2 * A2, byy = B1 * B1 + B2 * B2, axy = A1 * B1 + A2 * B2;
  const float sq = A1 * B2 - A2 * B1, det = sq * sq;
  // a staged Gaussian has axx, byy, det > 0 (isx, isy > 0, (ux, uy) a unit
  // vector); anything else keeps the blocks of its box
  if (!(axx > 0.f && byy > 0.f && det > 0.f && det < INFINITY)) return box_bits<kT>(s, ext_x, ext_y, x0, y0);
  // approximate reciprocals and roots (relative error ~1e-7): the padding below covers them
  const float inv_axx = rcp_approx(axx), inv_det = rcp_approx(det);
  const float Xm = sqrt_approx(L * byy * inv_det), Ym = sqrt_approx(L * axx * inv_det);
  const float r = -axy * inv_axx, k = det * inv_axx, ys = -axy * rcp_approx(byy) * Xm;
  const float pad = 1e-3f + 1e-4f * (Xm + Ym);  // rounding of the chord ends, px
  const float ox = ((float)x0 + 0.5f) - s.a.x, oy = ((float)y0 + 0.5f) - s.a.y;
  uint32_t bits = 0u;
#pragma unroll
  for (int br = 0; br < kT / 4; ++br) {
    const float ya = fmaxf(oy + 4.f * br, -Ym), yb = fminf(oy + 4.f * br + 3.f, Ym);
    if (!(ya <= yb)) continue;
    const float yr = fminf(fmaxf(ys, ya), yb), yl = fminf(fmaxf(-ys, ya), yb);
    const float xr = fmaf(r, yr, sqrt_approx(fmaxf(0.f, fmaf(-k * yr, yr, L)) * inv_axx)) + pad;
    const float xl = fmaf(r, yl, -sqrt_approx(fmaxf(0.f, fmaf(-k * yl, yl, L)) * inv_axx)) - pad;
    uint32_t c = 0u;
#pragma unroll
    for (int bc = 0; bc < kT / 8; ++bc) {
      const float cx0 = ox + 8.f * bc;
      if (cx0 + 7.f >= xl && cx0 <= xr) c |= 1u << bc;
    }
    bits |= G::row_bits(c, br);
  }
  return bits;
}

// log2 of the unclamped alpha at a pixel: dx = px - mx, and the shared
// b1dy = B1 dy, b2dy = B2 dy of its row.
__device__ __forceinline__ float pixel_log2_alpha(const float4 &a, const float4 &b, float dx, float b1dy,
                                                  float b2dy, float &t1, float &t2) {
  t1 = __fmaf_rn(a.z, dx, b1dy);
  t2 = __fmaf_rn(b.x, dx, b2dy);
  return __fmaf_rn(-t1, t1, __fmaf_rn(-t2, t2, b.z));
}

// Per consumer warp, the staged entries whose block bits reach it, in order:
// each staging warp writes, for each of its qualifying lanes (ballot +
// prefix count), the entry's index with the consumer's block bits above it
// (index | slots << 8) into its own part of the consumer's list.  The caller
// synchronises before the lists are read.
template <int kT>
__device__ __forceinline__ void compact_lists(uint32_t bits, uint16_t (*list)[Geo<kT>::kWarps][32],
                                              uint32_t (*cnt)[Geo<kT>::kWarps]) {
  using G = Geo<kT>;
  const int sw = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int cw = 0; cw < G::kWarps; ++cw) {
    const uint32_t slots = (bits >> (G::kPix * cw)) & G::kSlotMask;
    const unsigned m = __ballot_sync(0xffffffffu, slots != 0u);
    if (slots) list[cw][sw][__popc(m & lt)] = (uint16_t)(threadIdx.x | (slots << 8));
    if (lane == 0) cnt[cw][sw] = (uint32_t)__popc(m);
  }
}

template <int kT>
struct ThreadPixels {
  int x[Geo<kT>::kBC], y[2];  // slot q is pixel (x[q % kBC], y[q / kBC])
  float px[Geo<kT>::kBC], py[2];
  unsigned inside;            // bit q: slot q lies on the canvas
  int tile_x0, tile_y0;
};

template <int kT>
__device__ __forceinline__ ThreadPixels<kT> thread_pixels(int tile_x0, int tile_y0, int W, int H) {
  using G = Geo<kT>;
  ThreadPixels<kT> t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wx = warp % G::kWX, wy = warp / G::kWX;
  t.tile_x0 = tile_x0;
  t.tile_y0 = tile_y0;
#pragma unroll
  for (int c = 0; c < G::kBC; ++c) {
    t.x[c] = tile_x0 + 8 * G::kBC * wx + 8 * c + (lane & 7);
    t.px[c] = (float)t.x[c] + 0.5f;
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    t.y[r] = tile_y0 + 8 * wy + 4 * r + (lane >> 3);
    t.py[r] = (float)t.y[r] + 0.5f;
  }
  t.inside = 0;
#pragma unroll
  for (int q = 0; q < G::kPix; ++q)
    if (t.x[q % G::kBC] < W && t.y[q / G::kBC] < H) t.inside |= 1u << q;
  return t;
}

// One tile of one image as the blend kernels see it: its first pixel, the
// canvas, its list range, and the image's planes (plane = W H floats).
struct TileView {
  int x0, y0, W, H;
  uint2 r;
  float3 bg;
};

struct FwdOut {
  float *img, *T_out;
  uint32_t *nc_out;
  const float *target;  // kL2 only
  float *dimg;          // kL2 only
  float scale;          // kL2 only: 2 / (3 W H)
};

// The forward blend of one tile.  kStats: also count the (pixel, list
// entry) evaluations performed, the entries blended, the entries of the tile
// list times the tile's pixels, and the entries each pixel visits up to its
// stop point (the entry that would bring T below 1e-4, or the list's end),
// into stats[0..3] (for measurement; same blend otherwise).  kL2: also the L2 term of Eq. 13 on the finished
// pixels: dL/dimg = scale (img - target); returns this thread's sum of
// (img - target)^2 (0 without kL2).  Starts and ends with every thread of
// the CTA past a barrier.
template <int kT, bool kStats, bool kL2>
__device__ __forceinline__ float fwd_tile(const TileView &v, const FwdOut &o, const float *__restrict__ gauss,
                                          const uint32_t *__restrict__ keys, uint32_t gmask, uint32_t n_gauss,
                                          unsigned long long *__restrict__ stats) {
  using G = Geo<kT>;
  constexpr int kPix = G::kPix, kBatch = G::kBatch, kW = G::kWarps, kBC = G::kBC;
  __shared__ float4 s_a[kBatch];
  __shared__ float4 s_b[kBatch];
  __shared__ float2 s_c[kBatch];
  __shared__ uint16_t s_list[kW][kW][32];  // [consumer warp][staging warp][k]: entries reaching the warp
  __shared__ uint32_t s_cnt[kW][kW];
  uint32_t n_eval = 0, n_blend = 0;
  const ThreadPixels<kT> tp = thread_pixels<kT>(v.x0, v.y0, v.W, v.H);
  const uint2 r = v.r;
  float T[kPix], c0[kPix], c1[kPix], c2[kPix];
  uint32_t last[kPix], stop[kStats ? kPix : 1];
#pragma unroll
  for (int i = 0; i < kPix; ++i) {
    T[i] = 1.f;
    c0[i] = c1[i] = c2[i] = 0.f;
    last[i] = 0;
    if (kStats) stop[i] = (tp.inside >> i) & 1u ? r.y - r.x : 0u;
  }
  __shared__ uint32_t s_alive[kW];  // per warp: slots (8x4 blocks) with a pixel still blending
  __shared__ __align__(16) StageBuf<kBatch> s_buf;
  // batch 0's key and record, batch 1's key
  if (r.x + threadIdx.x < r.y) {
    const uint32_t key = keys[r.x + threadIdx.x];
    s_buf.key[0][threadIdx.x] = key;
    issue_rec(s_buf, gauss, key & gmask, n_gauss);
  }
  if (r.x + kBatch + threadIdx.x < r.y) cp_async4(&s_buf.key[1][threadIdx.x], keys + r.x + kBatch + threadIdx.x);
  cp_async_commit();
  unsigned alive = tp.inside;
  uint32_t kb = 0;  // key slot of this batch
  for (uint32_t base = r.x; base < r.y; base += kBatch, kb ^= 1u) {
    const uint32_t walive = __reduce_or_sync(0xffffffffu, alive);
    if ((threadIdx.x & 31) == 0) s_alive[threadIdx.x >> 5] = walive;
    if (__syncthreads_count(alive != 0) == 0) break;
    cp_async_wait_all();
    const uint32_t i = base + threadIdx.x;
    uint32_t my_bits = 0u;
    if (i < r.y) {
      const Staged s = stage_slot(s_buf, s_buf.key[kb][threadIdx.x] & gmask, n_gauss);
      s_a[threadIdx.x] = s.a;
      s_b[threadIdx.x] = s.b;
      s_c[threadIdx.x] = s.c;
      uint32_t alive_all = 0u;
#pragma unroll
      for (int w = 0; w < kW; ++w) alive_all |= s_alive[w] << (kPix * w);
      my_bits = block_bits<kT>(s, s.ext.x, s.ext.y, tp.tile_x0, tp.tile_y0) & alive_all;
    }
    // in flight while this batch blends: the next batch's record, the key after it
    if (i + kBatch < r.y) issue_rec(s_buf, gauss, s_buf.key[kb ^ 1u][threadIdx.x] & gmask, n_gauss);
    if (i + 2 * kBatch < r.y) cp_async4(&s_buf.key[kb][threadIdx.x], keys + i + 2 * kBatch);
    cp_async_commit();
    compact_lists<kT>(my_bits, s_list, s_cnt);
    __syncthreads();
    const int cw = threadIdx.x >> 5;
    for (int sw = 0; sw < kW && alive; ++sw) {
    const int cnt = (int)s_cnt[cw][sw];
    for (int k = 0; k < cnt && alive; ++k) {
      const uint32_t ent = s_list[cw][sw][k];
      const int j = (int)(ent & 0xffu);
      const uint32_t bits = ent >> 8;  // this warp's block bits: warp-uniform, not 0
      const float4 a = s_a[j], b = s_b[j];
      const float2 gb = s_c[j];
      float dx[kBC], b1dy[2], b2dy[2];
#pragma unroll
      for (int k = 0; k < kBC; ++k) dx[k] = __fsub_rn(tp.px[k], a.x);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float dy = __fsub_rn(tp.py[k], a.y);
        b1dy[k] = __fmul_rn(a.w, dy);
        b2dy[k] = __fmul_rn(b.y, dy);
      }
      const auto blend = [&](const int q, const float al) {
        if (kStats) ++n_eval;
        if (al < kAlphaMin) return;
        const float Tn = __fmaf_rn(-T[q], al, T[q]);
        if (Tn < kTMin) {
          alive &= ~(1u << q);
          if (kStats) stop[q] = base - r.x + (uint32_t)j + 1;
          return;
        }
        const float w = al * T[q];
        c0[q] = __fmaf_rn(w, b.w, c0[q]);
        c1[q] = __fmaf_rn(w, gb.x, c1[q]);
        c2[q] = __fmaf_rn(w, gb.y, c2[q]);
        T[q] = Tn;
        last[q] = base - r.x + (uint32_t)j + 1;
        if (kStats) ++n_blend;
      };
      const auto alpha = [&](const int q) {
        float t1, t2;
        return fminf(kAlphaMax,
                     ex2_approx(pixel_log2_alpha(a, b, dx[q % kBC], b1dy[q / kBC], b2dy[q / kBC], t1, t2)));
      };
      // T (1 - alpha) as one FMA; when the entry reaches every block of the
      // warp, the four alphas in one straight run whose chains interleave,
      // otherwise only the reached blocks' alphas, each behind its
      // warp-uniform bit (0.541 -> 0.515 ms at 2048^2)
      if (bits == G::kSlotMask) {  // every block reached: the alphas in one straight run
        float al[kPix];
#pragma unroll
        for (int q = 0; q < kPix; ++q) al[q] = alpha(q);
#pragma unroll
        for (int q = 0; q < kPix; ++q)
          if (alive & (1u << q)) blend(q, al[q]);
      } else {  // each reached block behind its warp-uniform bit
#pragma unroll
        for (int q = 0; q < kPix; ++q)
          if (bits & (1u << q)) {
            const float al = alpha(q);
            if (alive & (1u << q)) blend(q, al);
          }
      }
    }
    }
  }
  cp_async_wait_all();  // nothing in flight into s_buf past the tile
  if (kStats) {
    __shared__ unsigned long long s_st[3];
    if (threadIdx.x == 0) s_st[0] = s_st[1] = s_st[2] = 0ull;
    __syncthreads();
    unsigned long long visits = 0;
#pragma unroll
    for (int q = 0; q < kPix; ++q) visits += kStats ? stop[q] : 0u;
    atomicAdd(&s_st[0], (unsigned long long)n_eval);
    atomicAdd(&s_st[1], (unsigned long long)n_blend);
    atomicAdd(&s_st[2], visits);
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(&stats[0], s_st[0]);
      atomicAdd(&stats[1], s_st[1]);
      atomicAdd(&stats[2], (unsigned long long)(r.y - r.x) * (kT * kT));
      atomicAdd(&stats[3], s_st[2]);
    }
  }
  const size_t plane = (size_t)v.W * v.H;
  float l2 = 0.f;
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    if (!(tp.inside & (1u << q))) continue;
    const size_t p = (size_t)tp.y[q / kBC] * v.W + tp.x[q % kBC];
    const float v0 = __fmaf_rn(T[q], v.bg.x, c0[q]);
    const float v1 = __fmaf_rn(T[q], v.bg.y, c1[q]);
    const float v2 = __fmaf_rn(T[q], v.bg.z, c2[q]);
    o.img[p] = v0;
    o.img[plane + p] = v1;
    o.img[2 * plane + p] = v2;
    o.T_out[p] = T[q];
    o.nc_out[p] = last[q];
    if (kL2) {
      const float d0 = v0 - o.target[p], d1 = v1 - o.target[plane + p], d2 = v2 - o.target[2 * plane + p];
      o.dimg[p] = o.scale * d0;
      o.dimg[plane + p] = o.scale * d1;
      o.dimg[2 * plane + p] = o.scale * d2;
      l2 += d0 * d0 + d1 * d1 + d2 * d2;
    }
  }
  return l2;
}

// CTA sum of one float per thread, in double (valid in thread 0).
template <int kT>
__device__ __forceinline__ double cta_sum(float x) {
  constexpr int kThreads = Geo<kT>::kThreads;
  __shared__ double s_l2[kThreads / 32];
  double v = x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_l2[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += s_l2[w];
  }
  return t;
}

// Resident CTAs per SM the blend kernels are compiled for: the forward
// fits 64 registers a thread, the backward 80.
template <int kT> constexpr int fwd_min_blocks() { return kT == 8 ? 32 : (kT == 16 ? 16 : 4); }
template <int kT> constexpr int bwd_min_blocks() { return kT == 8 ? 24 : (kT == 16 ? 12 : 3); }

// One CTA per tile of one canvas.  kL2: mean((img - target)^2) added to
// *loss (one double atomic per CTA; *loss zeroed by the launcher).
template <int kT, bool kStats, bool kL2 = false>
__global__ void __launch_bounds__(Geo<kT>::kThreads, fwd_min_blocks<kT>()) render_fwd_kernel(const float *__restrict__ gauss,
                                                                  const uint32_t *__restrict__ keys,
                                                                  const uint2 *__restrict__ ranges, int W, int H,
                                                                  int tiles_x, uint32_t gmask, uint32_t n_gauss,
                                                                  float3 bg, float *__restrict__ img,
                                                                  float *__restrict__ T_out,
                                                                  uint32_t *__restrict__ nc_out,
                                                                  unsigned long long *__restrict__ stats,
                                                                  const float *__restrict__ target = nullptr,
                                                                  float *__restrict__ dimg = nullptr,
                                                                  double *__restrict__ loss = nullptr) {
  const int tile = blockIdx.x;
  const TileView v{(tile % tiles_x) * kT, (tile / tiles_x) * kT, W, H, ranges[tile], bg};
  const size_t plane = (size_t)W * H;
  const FwdOut o{img, T_out, nc_out, target, dimg, kL2 ? (float)(2.0 / (double)(3 * plane)) : 0.f};
  const float l2 = fwd_tile<kT, kStats, kL2>(v, o, gauss, keys, gmask, n_gauss, stats);
  if (kL2) {
    const double t = cta_sum<kT>(l2);
    if (threadIdx.x == 0) atomicAdd(loss, t / (double)(3 * plane));
  }
}

// Image of global tile t.
__device__ __forceinline__ int batch_image_of_tile(const BatchImage *__restrict__ tab, int n_images, uint32_t t) {
  return last_image_le<&BatchImage::tile0>(tab, n_images, (int64_t)t);
}

// The tile view of global tile t of a batch (image b).
template <int kT>
__device__ __forceinline__ TileView batch_view(const BatchImage &im, uint32_t t, const uint2 *__restrict__ ranges) {
  const int local = (int)((int64_t)t - im.tile0);
  const int ty = local / im.tiles_x, tx = local - ty * im.tiles_x;
  return TileView{tx * kT, ty * kT, im.W, im.H, ranges[t], make_float3(im.bg[0], im.bg[1], im.bg[2])};
}

// Persistent forward over a batch: each CTA takes tiles from the atomic
// queue *queue (zeroed by the launcher) until all n_tiles are done.  kL2:
// loss[b] += mean over image b of (img - target)^2; a CTA keeps a running
// sum while its tiles stay in one image and adds it once per change.
template <int kT, bool kL2>
__global__ void __launch_bounds__(Geo<kT>::kThreads, fwd_min_blocks<kT>()) batch_render_fwd_kernel(
    const float *__restrict__ gauss, const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges,
    const BatchImage *__restrict__ tab, int n_images, uint32_t n_tiles, uint32_t n_gauss,
    unsigned int *__restrict__ queue, const float *__restrict__ target, float *__restrict__ img,
    float *__restrict__ T_out, uint32_t *__restrict__ nc_out, float *__restrict__ dimg,
    double *__restrict__ loss) {
  __shared__ uint32_t s_t;
  __shared__ int s_b;
  double acc = 0.0;  // thread 0: pending sum of image acc_b
  int acc_b = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(queue, 1u);
      s_t = t;
      s_b = t < n_tiles ? batch_image_of_tile(tab, n_images, t) : -1;
    }
    __syncthreads();
    const uint32_t t = s_t;
    const int b = s_b;
    if (t >= n_tiles) break;
    const BatchImage &im = tab[b];
    const TileView v = batch_view<kT>(im, t, ranges);
    const FwdOut o{img + 3 * im.pix0, T_out + im.pix0, nc_out + im.pix0, kL2 ? target + 3 * im.pix0 : nullptr,
                   kL2 ? dimg + 3 * im.pix0 : nullptr, im.l2_scale};
    const float l2 = fwd_tile<kT, false, kL2>(v, o, gauss, vals, 0xffffffffu, n_gauss, nullptr);
    if (kL2) {
      const double s = cta_sum<kT>(l2);
      if (threadIdx.x == 0) {
        if (b != acc_b) {
          if (acc_b >= 0) atomicAdd(loss + acc_b, acc / (3.0 * (double)tab[acc_b].W * (double)tab[acc_b].H));
          acc = 0.0;
          acc_b = b;
        }
        acc += s;
      }
    }
    __syncthreads();
  }
  if (kL2 && threadIdx.x == 0 && acc_b >= 0)
    atomicAdd(loss + acc_b, acc / (3.0 * (double)tab[acc_b].W * (double)tab[acc_b].H));
}


// Number of per-Gaussian sums the backward accumulates (see render_bwd_kernel).
constexpr int kSums = 9;
// The backward parks the per-lane partial sums of up to kPend entries of a
// warp in shared memory (4; 2 for 32 x 32 tiles, whose eight warps would
// otherwise need more shared memory than a CTA's static 48 KB), then reduces
// them transposed: lane l adds up row l (entry l / 8, sum l % 8) and eight
// lanes per entry finish sum 8.  A row holds the 32 lanes' partials padded
// to 36 floats, so the 128-bit reads of a quarter-warp hit distinct banks.
template <int kT> constexpr int pend_of() { return kT == 32 ? 2 : 4; }
constexpr int kRow = 36;

// Reduce the parked partials of n_pend (<= kPend) entries of this warp and
// add the totals to the per-Gaussian sums.  part is the warp's
// [kPend * kSums][kRow] block, pend_g the entries' Gaussian indices.
template <int kPend>
__device__ __forceinline__ void flush_pending(const float *part, const uint32_t *pend_g, int n_pend, int lane,
                                              float *__restrict__ sums, uint32_t n_gauss) {
  __syncwarp();
  const int e = lane >> 3;                   // this lane's entry
  const bool mine = kPend == 4 || e < kPend;  // lanes past the parked entries add nothing
  {  // sums 0..7 of each entry: one row per lane
    const int k = lane & 7;
    float tot = 0.f;
    if (mine) {
      const float4 *row = reinterpret_cast<const float4 *>(part + (e * kSums + k) * kRow);
      float4 acc = row[0];
#pragma unroll
      for (int c = 1; c < 8; ++c) {
        const float4 x = row[c];
        acc.x += x.x;
        acc.y += x.y;
        acc.z += x.z;
        acc.w += x.w;
      }
      tot = (acc.x + acc.y) + (acc.z + acc.w);
    }
    const uint32_t g = mine ? pend_g[e] : 0xffffffffu;
    if (e < n_pend && tot != 0.f && g < n_gauss) atomicAdd(sums + (size_t)g * BS_DGAUSS_FLOATS + k, tot);
  }
  {  // sum 8 of each entry: eight lanes, four partials each
    const int c = lane & 7;
    float tot = 0.f;
    if (mine) {
      const float4 x = reinterpret_cast<const float4 *>(part + (e * kSums + 8) * kRow)[c];
      tot = (x.x + x.y) + (x.z + x.w);
    }
    tot += __shfl_xor_sync(0xffffffffu, tot, 4);
    tot += __shfl_xor_sync(0xffffffffu, tot, 2);
    tot += __shfl_xor_sync(0xffffffffu, tot, 1);
    const uint32_t g = mine ? pend_g[e] : 0xffffffffu;
    if (c == 0 && e < n_pend && tot != 0.f && g < n_gauss) atomicAdd(sums + (size_t)g * BS_DGAUSS_FLOATS + 8, tot);
  }
  __syncwarp();
}

// Reverse walk.  With S the colour behind Gaussian j as seen through it,
// S <- alpha_j c_j + (1 - alpha_j) S (starting from bg behind the last
// blended Gaussian), the colour derivative is
//     dC/dalpha_j = T_j (c_j - S),
// which keeps the (1 - alpha_j)^-1 of the recovered transmittance out of the
// gradient.  With dq = alpha dL/dalpha (= dL/dp / ln 2 below the clamp) and
// (t1, t2) the pixel's offset in the Gaussian's scaled frame, each Gaussian
// accumulates over its tile's pixels
//   [0] sum dq t1  [1] sum dq t2  [2] sum dq t1^2  [3] sum dq t1 t2
//   [4] sum dq t2^2  [5] sum dq  [6..8] sum alpha T dL/dC.
// The frame keeps every term O(1) inside the Gaussian's support (the same
// sums in pixel offsets cancel badly for a thin Gaussian far along its
// axis); grads_from_sums turns the totals into d/d(record).
struct BwdIn {
  const float *T_final;
  const uint32_t *n_contrib;
  const float *dimg;
};

// The reverse walk of one tile (see above).  Starts and ends with every
// thread of the CTA past a barrier.
template <int kT>
__device__ __forceinline__ void bwd_tile(const TileView &v, const BwdIn &in, const float *__restrict__ gauss,
                                         const uint32_t *__restrict__ keys, uint32_t gmask, uint32_t n_gauss,
                                         float *__restrict__ sums) {
  using G = Geo<kT>;
  constexpr int kPix = G::kPix, kBatch = G::kBatch, kW = G::kWarps, kBC = G::kBC, kPend = pend_of<kT>();
  __shared__ float4 s_a[kBatch];
  __shared__ float4 s_b[kBatch];
  __shared__ float2 s_c[kBatch];
  __shared__ uint32_t s_g[kBatch];
  __shared__ uint16_t s_list[kW][kW][32];  // [consumer warp][staging warp][k]: entries reaching the warp
  __shared__ uint32_t s_cnt[kW][kW];
  __shared__ uint32_t s_max_last;
  __shared__ __align__(16) uint32_t s_wlast[kW][kPix];
  __shared__ __align__(16) float s_part[kW][kPend * kSums * kRow];
  __shared__ uint32_t s_pend_g[kW][kPend];
  const ThreadPixels<kT> tp = thread_pixels<kT>(v.x0, v.y0, v.W, v.H);
  const uint2 r = v.r;
  const float3 bg = v.bg;
  const int lane = threadIdx.x & 31;
  float T[kPix], g0[kPix], g1[kPix], g2[kPix], gS[kPix];
  uint32_t last[kPix];
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  uint32_t my_max = 0;
  const size_t plane = (size_t)v.W * v.H;
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    T[q] = 1.f;
    g0[q] = g1[q] = g2[q] = 0.f;
    last[q] = 0;
    if (tp.inside & (1u << q)) {
      const size_t p = (size_t)tp.y[q / kBC] * v.W + tp.x[q % kBC];
      T[q] = in.T_final[p];
      last[q] = in.n_contrib[p];
      g0[q] = in.dimg[p];
      g1[q] = in.dimg[plane + p];
      g2[q] = in.dimg[2 * plane + p];
      my_max = max(my_max, last[q]);
    }
    gS[q] = g0[q] * bg.x + g1[q] * bg.y + g2[q] * bg.z;  // g . S, S = bg behind the last blended Gaussian
  }
  atomicMax(&s_max_last, my_max);
  // per warp and slot (8x4 block), the deepest last entry of its pixels: an
  // entry at or past it is left out of that block when it is staged
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    const uint32_t wl = __reduce_max_sync(0xffffffffu, last[q]);
    if (lane == 0) s_wlast[threadIdx.x >> 5][q] = wl;
  }
  float *const part = s_part[threadIdx.x >> 5];
  uint32_t *const pend_g = s_pend_g[threadIdx.x >> 5];
  int n_pend = 0;  // warp-uniform
  __syncthreads();
  const uint32_t max_last = min(s_max_last, r.y - r.x);
  for (uint32_t end = max_last; end > 0;) {
    const uint32_t start = end > (uint32_t)kBatch ? end - kBatch : 0u;
    __syncthreads();
    const uint32_t i = start + threadIdx.x;
    uint32_t my_bits = 0u;
    if (i < end) {
      const uint32_t g = keys[r.x + i] & gmask;
      const Staged s = stage(gauss, g, n_gauss);
      s_a[threadIdx.x] = s.a;
      s_b[threadIdx.x] = s.b;
      s_c[threadIdx.x] = s.c;
      s_g[threadIdx.x] = g;
      my_bits = block_bits<kT>(s, s.ext.x, s.ext.y, tp.tile_x0, tp.tile_y0);
#pragma unroll
      for (int b = 0; b < G::kBits; ++b)
        if (i >= s_wlast[b / kPix][b % kPix]) my_bits &= ~(1u << b);
    }
    compact_lists<kT>(my_bits, s_list, s_cnt);
    __syncthreads();
    const int cw = threadIdx.x >> 5;
    for (int sw = kW - 1; sw >= 0; --sw)
    for (int k = (int)s_cnt[cw][sw] - 1; k >= 0; --k) {
      const uint32_t ent = s_list[cw][sw][k];
      const int j = (int)(ent & 0xffu);
      const uint32_t pos = start + (uint32_t)j;
      const uint32_t bits = ent >> 8;  // this warp's block bits: warp-uniform, not 0
      const float4 a = s_a[j], b = s_b[j];
      const float2 gb = s_c[j];
      float dx[kBC], b1dy[2], b2dy[2];
#pragma unroll
      for (int k = 0; k < kBC; ++k) dx[k] = __fsub_rn(tp.px[k], a.x);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float dy = __fsub_rn(tp.py[k], a.y);
        b1dy[k] = __fmul_rn(a.w, dy);
        b2dy[k] = __fmul_rn(b.y, dy);
      }
      float v[kSums];
#pragma unroll
      for (int q = 0; q < kSums; ++q) v[q] = 0.f;
      // One slot (8x4 block) of this thread.  Branch-free per pixel: a pixel
      // past its last blended Gaussian, or below the alpha threshold, gets
      // alpha = 0, an exact no-op below (rcp.approx(1) is exactly 1, so T
      // stays as it is).
      const auto slot = [&](const int q) {
        float t1, t2;
        const float raw = ex2_approx(pixel_log2_alpha(a, b, dx[q % kBC], b1dy[q / kBC], b2dy[q / kBC], t1, t2));
        const float al0 = fminf(kAlphaMax, raw);
        const bool on = pos < last[q] && al0 >= kAlphaMin;
        const float al = on ? al0 : 0.f;
        T[q] = T[q] * rcp_approx(1.f - al);  // T before this Gaussian
        const float w = al * T[q];
        const float gc = __fmaf_rn(g2[q], gb.y, __fmaf_rn(g1[q], gb.x, g0[q] * b.w));
        const float diff = gc - gS[q];
        gS[q] = __fmaf_rn(al, diff, gS[q]);
        v[6] = __fmaf_rn(w, g0[q], v[6]);
        v[7] = __fmaf_rn(w, g1[q], v[7]);
        v[8] = __fmaf_rn(w, g2[q], v[8]);
        const float dq = raw <= kAlphaMax ? w * diff : 0.f;  // alpha dL/dalpha; 0 past the clamp
        const float e1 = dq * t1, e2 = dq * t2;
        v[0] += e1;
        v[1] += e2;
        v[2] = __fmaf_rn(e1, t1, v[2]);
        v[3] = __fmaf_rn(e1, t2, v[3]);
        v[4] = __fmaf_rn(e2, t2, v[4]);
        v[5] += dq;
      };
      if (bits == G::kSlotMask) {  // every block reached: one straight run, the slots' chains interleave
#pragma unroll
        for (int q = 0; q < kPix; ++q) slot(q);
      } else {  // each block behind its warp-uniform bit
#pragma unroll
        for (int q = 0; q < kPix; ++q)
          if (bits & (1u << q)) slot(q);
      }
      // every walked entry is parked: 98 % of them reach a pixel, and an
      // entry that reaches none parks zeros, which the flush does not add
      // (a vote to skip those cost more than it saved: 0.941 -> 0.938 ms)
      float *dst = part + n_pend * kSums * kRow + lane;
#pragma unroll
      for (int q = 0; q < kSums; ++q) dst[q * kRow] = v[q];
      if (lane == 0) pend_g[n_pend] = s_g[j];
      if (++n_pend == kPend) {
        flush_pending<kPend>(part, pend_g, n_pend, lane, sums, n_gauss);
        n_pend = 0;
      }
    }
    end = start;
  }
  if (n_pend) flush_pending<kPend>(part, pend_g, n_pend, lane, sums, n_gauss);
  __syncthreads();
}

// One CTA per tile of one canvas.
template <int kT>
__global__ void __launch_bounds__(Geo<kT>::kThreads, bwd_min_blocks<kT>()) render_bwd_kernel(const float *__restrict__ gauss,
                                                                  const uint32_t *__restrict__ keys,
                                                                  const uint2 *__restrict__ ranges, int W, int H,
                                                                  int tiles_x, uint32_t gmask, uint32_t n_gauss,
                                                                  float3 bg, const float *__restrict__ T_final,
                                                                  const uint32_t *__restrict__ n_contrib,
                                                                  const float *__restrict__ dimg,
                                                                  float *__restrict__ sums) {
  // the tiles in reverse order: the forward's last-written blend state
  // (T_final, n_contrib, dL/dimg) is the likeliest still in L2
  // (0.937 -> 0.930 ms at 2048^2)
  const int tile = gridDim.x - 1 - blockIdx.x;
  const TileView v{(tile % tiles_x) * kT, (tile / tiles_x) * kT, W, H, ranges[tile], bg};
  bwd_tile<kT>(v, BwdIn{T_final, n_contrib, dimg}, gauss, keys, gmask, n_gauss, sums);
}

// Persistent backward over a batch (the queue of batch_render_fwd_kernel).
template <int kT>
__global__ void __launch_bounds__(Geo<kT>::kThreads, bwd_min_blocks<kT>()) batch_render_bwd_kernel(
    const float *__restrict__ gauss, const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges,
    const BatchImage *__restrict__ tab, int n_images, uint32_t n_tiles, uint32_t n_gauss,
    unsigned int *__restrict__ queue, const float *__restrict__ T_final, const uint32_t *__restrict__ n_contrib,
    const float *__restrict__ dimg, float *__restrict__ sums) {
  __shared__ uint32_t s_t;
  __shared__ int s_b;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(queue, 1u);
      s_t = t;
      s_b = t < n_tiles ? batch_image_of_tile(tab, n_images, t) : -1;
    }
    __syncthreads();
    const uint32_t t = s_t;
    const int b = s_b;
    if (t >= n_tiles) break;
    const BatchImage &im = tab[b];
    const TileView v = batch_view<kT>(im, t, ranges);
    bwd_tile<kT>(v, BwdIn{T_final + im.pix0, n_contrib + im.pix0, dimg + 3 * im.pix0}, gauss, vals, 0xffffffffu,
                 n_gauss, sums);
  }
}

// The chain rule from the tile sums of render_bwd_kernel to the record.
// With p = log2(o) - |t|^2, t = M d, M = [[A1, B1], [A2, B2]] = k D R^T,
// D = diag(isx, isy), dL/dp = ln2 dq and Tm = [[s2, s3], [s3, s4]]:
//   d/d(mx, my) = 2 ln2 M^T (s0, s1),
//   d/dM = -2 ln2 sum dq t d^T = -2 ln2 Tm M^-T = -(2 ln2 / k) Tm D^-1 R^T,
//   A1 = k isx ux, B1 = k isx uy, A2 = -k isy uy, B2 = k isy ux,
//   d/do = s5 / o,   d/dcolour = s6..s8.   In place, one thread per Gaussian.
// A non-finite gradient sets kDevErrNotFinite in the library status word.
__global__ void grads_from_sums_kernel(const float *__restrict__ gauss, float *__restrict__ dgauss, int64_t n,
                                       uint32_t *status) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const float4 *rec = reinterpret_cast<const float4 *>(gauss + g * BS_GAUSS_FLOATS);
  const float4 r0 = rec[0], r1 = rec[1];
  float4 *d = reinterpret_cast<float4 *>(dgauss + g * BS_DGAUSS_FLOATS);
  const float4 s0 = d[0], s1 = d[1], s2 = d[2];
  const float T1 = s0.x, T2 = s0.y, T11 = s0.z, T12 = s0.w, T22 = s1.x, S = s1.y;
  const float ux = r0.z, uy = r0.w, isx = r1.x, isy = r1.y, o = r1.z;
  float A1, B1, A2, B2;
  scaled_axes(ux, uy, isx, isy, A1, B1, A2, B2);
  const float c = 2.f * kLn2;
  // X = Tm D^-1 R^T, R^T = [[ux, uy], [-uy, ux]]
  const float sx = isx > 0.f ? 1.f / isx : 0.f, sy = isy > 0.f ? 1.f / isy : 0.f;
  const float p00 = T11 * sx, p01 = T12 * sy, p10 = T12 * sx, p11 = T22 * sy;
  const float X00 = p00 * ux - p01 * uy, X01 = p00 * uy + p01 * ux;
  const float X10 = p10 * ux - p11 * uy, X11 = p10 * uy + p11 * ux;
  const float f = -c / kKappa;
  const float dA1 = f * X00, dB1 = f * X01, dA2 = f * X10, dB2 = f * X11;
  const float4 o0 = make_float4(c * (A1 * T1 + A2 * T2), c * (B1 * T1 + B2 * T2),
                                kKappa * (isx * dA1 + isy * dB2), kKappa * (isx * dB1 - isy * dA2));
  const float4 o1 = make_float4(kKappa * (ux * dA1 + uy * dB1), kKappa * (ux * dB2 - uy * dA2), o > 0.f ? S / o : 0.f,
                                s1.z);
  const float4 o2 = make_float4(s1.w, s2.x, 0.f, 0.f);
  d[0] = o0;
  d[1] = o1;
  d[2] = o2;
  // 0 * x is 0 for a finite x and NaN otherwise
  const float probe = 0.f * o0.x + 0.f * o0.y + 0.f * o0.z + 0.f * o0.w + 0.f * o1.x + 0.f * o1.y + 0.f * o1.z +
                      0.f * o1.w + 0.f * o2.x + 0.f * o2.y;
  if (probe != 0.f) atomicOr(status, kDevErrNotFinite);
}

// L2 loss and its gradient, float4 at a time; per-thread float partial sums
// (a few dozen terms each), combined in double.
__global__ void l2_kernel(const float *__restrict__ img, const float *__restrict__ target, int64_t n,
                          float *__restrict__ dimg, double *loss) {
  __shared__ double s_sum[32];
  float acc = 0.f;
  const float scale = (float)(2.0 / (double)n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = n / 4;
  const float4 *a4 = reinterpret_cast<const float4 *>(img);
  const float4 *t4 = reinterpret_cast<const float4 *>(target);
  float4 *d4 = reinterpret_cast<float4 *>(dimg);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 a = a4[i], t = t4[i];
    const float4 d = make_float4(a.x - t.x, a.y - t.y, a.z - t.z, a.w - t.w);
    d4[i] = make_float4(scale * d.x, scale * d.y, scale * d.z, scale * d.w);
    acc += d.x * d.x + d.y * d.y + d.z * d.z + d.w * d.w;
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float d = img[i] - target[i];
    dimg[i] = scale * d;
    acc += d * d;
  }
  double dacc = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_sum[warp] = dacc;
  __syncthreads();
  if (warp == 0) {
    dacc = lane < (int)(blockDim.x / 32) ? s_sum[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    if (lane == 0) atomicAdd(loss, dacc / (double)n);
  }
}

}  // namespace

// Tile side -> one instantiation of a launcher template.
#define BS_BY_TILE(tile, call)                                                  \
  switch (tile) {                                                              \
    case 8: { constexpr int kT = 8; call; } break;                             \
    case 16: { constexpr int kT = 16; call; } break;                           \
    case 32: { constexpr int kT = 32; call; } break;                           \
    default: set_error("tile side %d not supported (8, 16, 32)", (int)(tile)); \
      return BS_ERR_UNSUPPORTED;                                               \
  }

template <int kT>
void fwd_plain(const float *gauss, int64_t n_gauss, const bs_canvas &cv, uint32_t gmask, const uint32_t *keys,
               const uint2 *rg, float *img, float *T_final, uint32_t *n_contrib, cudaStream_t s,
               unsigned long long *stats, const float *target, float *dimg, double *loss) {
  const int tiles_x = div_up(cv.width, kT), tiles_y = div_up(cv.height, kT);
  const auto bg = make_float3(cv.bg[0], cv.bg[1], cv.bg[2]);
  constexpr int kThreads = Geo<kT>::kThreads;
  if (stats)
    render_fwd_kernel<kT, true><<<tiles_x * tiles_y, kThreads, 0, s>>>(
        gauss, keys, rg, cv.width, cv.height, tiles_x, gmask, (uint32_t)n_gauss, bg, img, T_final, n_contrib, stats);
  else if (target)
    render_fwd_kernel<kT, false, true><<<tiles_x * tiles_y, kThreads, 0, s>>>(
        gauss, keys, rg, cv.width, cv.height, tiles_x, gmask, (uint32_t)n_gauss, bg, img, T_final, n_contrib,
        nullptr, target, dimg, loss);
  else
    render_fwd_kernel<kT, false><<<tiles_x * tiles_y, kThreads, 0, s>>>(
        gauss, keys, rg, cv.width, cv.height, tiles_x, gmask, (uint32_t)n_gauss, bg, img, T_final, n_contrib,
        nullptr);
}

template <int kT>
void bwd_plain(const float *gauss, int64_t n_gauss, const bs_canvas &cv, uint32_t gmask, const uint32_t *keys,
               const uint2 *rg, const float *T_final, const uint32_t *n_contrib, const float *dL_dimg, float *dgauss,
               cudaStream_t s) {
  const int tiles_x = div_up(cv.width, kT), tiles_y = div_up(cv.height, kT);
  render_bwd_kernel<kT><<<tiles_x * tiles_y, Geo<kT>::kThreads, 0, s>>>(
      gauss, keys, rg, cv.width, cv.height, tiles_x, gmask, (uint32_t)n_gauss,
      make_float3(cv.bg[0], cv.bg[1], cv.bg[2]), T_final, n_contrib, dL_dimg, dgauss);
}

uint32_t gauss_mask(int gbits) { return gbits >= 32 ? 0xffffffffu : ((1u << gbits) - 1u); }

bs_status launch_render_fwd(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                            const uint32_t *keys,
                            const uint32_t *ranges, float *img, float *T_final, uint32_t *n_contrib,
                            cudaStream_t s, unsigned long long *stats) {
  const auto *rg = reinterpret_cast<const uint2 *>(ranges);
  if (stats) BS_CUDA(cudaMemsetAsync(stats, 0, 4 * sizeof(unsigned long long), s));
  BS_BY_TILE(cv.tile, (fwd_plain<kT>(gauss, n_gauss, cv, gauss_mask(gbits), keys, rg, img, T_final, n_contrib, s,
                                     stats, nullptr, nullptr, nullptr)));
  BS_LAUNCHED("render_fwd_kernel");
  return BS_OK;
}

bs_status launch_render_fwd_l2(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                               const uint32_t *keys, const uint32_t *ranges, const float *target, float *img,
                               float *T_final, uint32_t *n_contrib, float *dimg, double *loss, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
  const auto *rg = reinterpret_cast<const uint2 *>(ranges);
  BS_BY_TILE(cv.tile, (fwd_plain<kT>(gauss, n_gauss, cv, gauss_mask(gbits), keys, rg, img, T_final, n_contrib, s,
                                     nullptr, target, dimg, loss)));
  BS_LAUNCHED("render_fwd_kernel");
  return BS_OK;
}

bs_status launch_render_bwd(const float *gauss, int64_t n_gauss, const bs_canvas &cv, int gbits,
                            const uint32_t *keys, const uint32_t *ranges, const float *T_final,
                            const uint32_t *n_contrib, const float *dL_dimg, float *dgauss, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(dgauss, 0, sizeof(float) * BS_DGAUSS_FLOATS * (size_t)n_gauss, s));
  const auto *rg = reinterpret_cast<const uint2 *>(ranges);
  BS_BY_TILE(cv.tile, (bwd_plain<kT>(gauss, n_gauss, cv, gauss_mask(gbits), keys, rg, T_final, n_contrib, dL_dimg,
                                     dgauss, s)));
  BS_LAUNCHED("render_bwd_kernel");
  uint32_t *status = nullptr;
  BS_TRY(lib_status_word(&status));
  grads_from_sums_kernel<<<(unsigned)div_up64(n_gauss, 256), 256, 0, s>>>(gauss, dgauss, n_gauss, status);
  BS_LAUNCHED("grads_from_sums_kernel");
  return BS_OK;
}

bs_status launch_l2(const float *img, const float *target, int64_t n, float *dimg, double *loss, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
  if (n == 0) return BS_OK;
  if (((uintptr_t)img | (uintptr_t)target | (uintptr_t)dimg) & 15) {
    set_error("img, target and dL_dimg must be 16-byte aligned");
    return BS_ERR_INVALID_ARG;
  }
  const int blocks = (int)std::min<int64_t>(div_up64(n, 256 * 4 * 4), 152 * 8);
  l2_kernel<<<blocks, 256, 0, s>>>(img, target, n, dimg, loss);
  BS_LAUNCHED("l2_kernel");
  return BS_OK;
}

// Persistent grids: as many CTAs as fit on the device at once (queried once
// per device and kernel; slot names the kernel).
template <typename Kernel>
bs_status persistent_grid(Kernel k, int threads, int slot, int *grid) {
  constexpr int kMaxDev = 64, kSlots = 16;
  static int cache[kMaxDev][kSlots] = {};
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev || slot < 0 || slot >= kSlots) {
    set_error("device %d: at most %d devices supported", dev, kMaxDev);
    return BS_ERR_UNSUPPORTED;
  }
  if (!cache[dev][slot]) {
    int per_sm = 0, sms = 0;
    BS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0));
    BS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cache[dev][slot] = std::max(1, per_sm) * std::max(1, sms);
  }
  *grid = cache[dev][slot];
  return BS_OK;
}

template <int kT> constexpr int tile_slot() { return kT == 8 ? 0 : (kT == 16 ? 1 : 2); }

// The workspace's two queue counters: [0] forward, [1] backward.
unsigned int *batch_queue(const BatchPlan &p, void *ws) {
  return reinterpret_cast<unsigned int *>(static_cast<char *>(ws) + p.off_queue);
}

const BatchImage *batch_table(const BatchPlan &p, const void *ws) {
  return reinterpret_cast<const BatchImage *>(static_cast<const char *>(ws) + p.off_images);
}

template <int kT>
bs_status fwd_batch(const BatchPlan &p, void *ws, const float *gauss, const uint32_t *vals, const uint2 *rg,
                    const float *target, float *img, float *T_final, uint32_t *n_contrib, float *dimg, double *loss,
                    cudaStream_t s) {
  constexpr int kThreads = Geo<kT>::kThreads;
  unsigned int *queue = batch_queue(p, ws);
  int grid = 0;
  if (target) {
    BS_TRY(persistent_grid(batch_render_fwd_kernel<kT, true>, kThreads, tile_slot<kT>(), &grid));
    grid = (int)std::min<int64_t>(grid, p.n_tiles);
    batch_render_fwd_kernel<kT, true><<<grid, kThreads, 0, s>>>(gauss, vals, rg, batch_table(p, ws), p.n_images,
                                                               (uint32_t)p.n_tiles, (uint32_t)p.n_gauss, queue,
                                                               target, img, T_final, n_contrib, dimg, loss);
  } else {
    BS_TRY(persistent_grid(batch_render_fwd_kernel<kT, false>, kThreads, 3 + tile_slot<kT>(), &grid));
    grid = (int)std::min<int64_t>(grid, p.n_tiles);
    batch_render_fwd_kernel<kT, false><<<grid, kThreads, 0, s>>>(gauss, vals, rg, batch_table(p, ws), p.n_images,
                                                                (uint32_t)p.n_tiles, (uint32_t)p.n_gauss, queue,
                                                                nullptr, img, T_final, n_contrib, nullptr, nullptr);
  }
  return BS_OK;
}

template <int kT>
bs_status bwd_batch(const BatchPlan &p, void *ws, const float *gauss, const uint32_t *vals, const uint2 *rg,
                    const float *T_final, const uint32_t *n_contrib, const float *dimg, float *dgauss,
                    cudaStream_t s) {
  constexpr int kThreads = Geo<kT>::kThreads;
  int grid = 0;
  BS_TRY(persistent_grid(batch_render_bwd_kernel<kT>, kThreads, 6 + tile_slot<kT>(), &grid));
  grid = (int)std::min<int64_t>(grid, p.n_tiles);
  batch_render_bwd_kernel<kT><<<grid, kThreads, 0, s>>>(gauss, vals, rg, batch_table(p, ws), p.n_images,
                                                        (uint32_t)p.n_tiles, (uint32_t)p.n_gauss,
                                                        batch_queue(p, ws) + 1, T_final, n_contrib, dimg, dgauss);
  return BS_OK;
}

bs_status launch_batch_render_fwd(const BatchPlan &p, void *ws, const float *gauss, const uint32_t *vals,
                                  const uint32_t *ranges, const float *target, float *img, float *T_final,
                                  uint32_t *n_contrib, float *dimg, double *loss, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(batch_queue(p, ws), 0, sizeof(unsigned int), s));
  if (target) BS_CUDA(cudaMemsetAsync(loss, 0, sizeof(double) * (size_t)p.n_images, s));
  const auto *rg = reinterpret_cast<const uint2 *>(ranges);
  BS_BY_TILE(p.tile, BS_TRY((fwd_batch<kT>(p, ws, gauss, vals, rg, target, img, T_final, n_contrib, dimg, loss, s))));
  BS_LAUNCHED("batch_render_fwd_kernel");
  return BS_OK;
}

bs_status launch_batch_render_bwd(const BatchPlan &p, void *ws, const float *gauss, const uint32_t *vals,
                                  const uint32_t *ranges, const float *T_final, const uint32_t *n_contrib,
                                  const float *dimg, float *dgauss, cudaStream_t s) {
  BS_CUDA(cudaMemsetAsync(batch_queue(p, ws) + 1, 0, sizeof(unsigned int), s));
  BS_CUDA(cudaMemsetAsync(dgauss, 0, sizeof(float) * BS_DGAUSS_FLOATS * (size_t)p.n_gauss, s));
  const auto *rg = reinterpret_cast<const uint2 *>(ranges);
  BS_BY_TILE(p.tile, BS_TRY((bwd_batch<kT>(p, ws, gauss, vals, rg, T_final, n_contrib, dimg, dgauss, s))));
  BS_LAUNCHED("batch_render_bwd_kernel");
  if (p.n_gauss > 0) {
    uint32_t *status = nullptr;
    BS_TRY(lib_status_word(&status));
    grads_from_sums_kernel<<<(unsigned)div_up64(p.n_gauss, 256), 256, 0, s>>>(gauss, dgauss, p.n_gauss, status);
    BS_LAUNCHED("grads_from_sums_kernel");
  }
  return BS_OK;
}

}  // namespace bs
