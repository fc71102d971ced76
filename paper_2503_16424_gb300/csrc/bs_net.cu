// The learned initialiser: a 5-layer convolutional encoder that maps a
// 256 x 256 RGB patch to curve proposals, one closed curve and one open
// stroke per cell of an 8 x 8 grid, trained on curve sets the method itself
// optimised.
//
// Layers: five 4 x 4 convolutions of stride 2 and padding 1 (channels 8 -> 32
// -> 64 -> 128 -> 256 -> 256; the RGB input is padded to 8 channels), each
// followed by ReLU, then a 1 x 1 head (256 -> 64, the first 55 used).
// Activations are NHWC bfloat16, weights bfloat16 copies of float32 master
// weights, accumulation float32.
//
// Every convolution and its two backward products is one implicit GEMM on
// the tensor cores (mma.sync m16n8k16, bf16 inputs, f32 accumulators):
//   forward   out[m][co] = sum_k patch[m][k] w[co][k]        (k = tap, ci)
//   input     din[m][ci] = sum_k dout[m'][co] w[co][tap][ci] (one GEMM per
//             parity class of the input pixel: a stride-2 4 x 4 kernel reaches
//             each input pixel through 2 x 2 taps of fixed parity)
//   weights   dw[co][k]  = sum_m dout[m][co] patch[m][k]      (split over m,
//             float32 atomics)
// Operands are gathered into shared memory 8 bf16 (16 bytes) at a time by
// the op's load functions; a 64 x 64 tile per CTA, four warps of 32 x 32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 32, kSK = kBK + 8;  // smem row stride (bf16): conflict-free fragments
constexpr int kGemmThreads = 128;

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

// A decoded operand row (its meaning is the op's; a < 0: a row past the matrix).
struct Row {
  int a, b, c, d;
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] = sum_k A[m][k] B[n][k] over k in the op's range for blockIdx.z.
// Op: k_begin(z), k_end(z) (multiples of 8); row_a(m) / row_b(n): what a row
// needs to be read, decoded once per thread before the K loop (a row with
// a < 0 reads as zeros); load_a(row, k) / load_b(row, k): the 8 bf16 at
// k..k+7 of the row; store(m, n, v0, v1): the results at (m, n) and
// (m, n + 1) (n even).
template <class Op>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(const Op op) {
  __shared__ __align__(16) __nv_bfloat16 sA[kBM][kSK];
  __shared__ __align__(16) __nv_bfloat16 sB[kBN][kSK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int kb = op.k_begin(blockIdx.z), ke = op.k_end(blockIdx.z);
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
  // each thread stages two 16-byte vectors of A and two of B per chunk:
  // vector v = tid + 128 i covers row v / 4, columns 8 (v % 4) .. + 7
  uint4 ra[2], rb[2];
  Row rowa[2], rowb[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int row = (tid + kGemmThreads * i) >> 2;
    rowa[i] = op.row_a(m0 + row);
    rowb[i] = op.row_b(n0 + row);
  }
  auto fetch = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int v = tid + kGemmThreads * i, kk = k0 + 8 * (v & 3);
      ra[i] = kk < ke ? op.load_a(rowa[i], kk) : zero4();
      rb[i] = kk < ke ? op.load_b(rowb[i], kk) : zero4();
    }
  };
  if (kb < ke) fetch(kb);
  for (int k0 = kb; k0 < ke; k0 += kBK) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int v = tid + kGemmThreads * i, row = v >> 2, col = 8 * (v & 3);
      *reinterpret_cast<uint4 *>(&sA[row][col]) = ra[i];
      *reinterpret_cast<uint4 *>(&sB[row][col]) = rb[i];
    }
    __syncthreads();
    if (k0 + kBK < ke) fetch(k0 + kBK);  // the next chunk's loads overlap these MMAs
#pragma unroll
    for (int ks = 0; ks < kBK; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        a[i][0] = *reinterpret_cast<const uint32_t *>(&sA[r][ks + 2 * t]);
        a[i][1] = *reinterpret_cast<const uint32_t *>(&sA[r + 8][ks + 2 * t]);
        a[i][2] = *reinterpret_cast<const uint32_t *>(&sA[r][ks + 2 * t + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t *>(&sA[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = wn + 8 * j + g;
        b[j][0] = *reinterpret_cast<const uint32_t *>(&sB[n][ks + 2 * t]);
        b[j][1] = *reinterpret_cast<const uint32_t *>(&sB[n][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + wm + 16 * i + g, n = n0 + wn + 8 * j + 2 * t;
      op.store(m, n, acc[i][j][0], acc[i][j][1]);
      op.store(m + 8, n, acc[i][j][2], acc[i][j][3]);
    }
}

// ---- the same GEMM on the 5th-generation tensor cores (tcgen05) ----
// A CTA of eight warps computes a 128 x 64 tile.  Per 32-wide K chunk every
// thread gathers its share of A (128 x 32) and B (64 x 32) with the op's
// load functions into shared memory in the canonical K-major layout without
// swizzle: 8 x 16-byte core matrices, the core matrix of rows 8i..8i+7 and
// columns 8j..8j+7 at byte (i * 512 + j * 128), one row per 16 bytes inside.
// One thread then issues two tcgen05.mma (M 128, N 64, K 16, bf16 inputs,
// float32 accumulator in tensor memory) per chunk and commits them to the
// chunk's mbarrier; two stages, so the gather of a chunk overlaps the MMAs
// of the previous one.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w reads tensor-memory lanes 32 (w % 4).., the tile's
// rows, and columns 32 (w / 4)..+31) and hands it to the op's store.  Every wait on an mbarrier is bounded; a
// wait that gives up counts in *err and the tile is not stored.
constexpr int kUM = 128, kUN = 64, kUK = 32;
constexpr int kUThreads = 256;  // eight warps gather; warps w and w + 4 share tensor-memory lanes 32 (w % 4)..
constexpr uint32_t kUmmaLbo = 128, kUmmaSbo = 512;          // bytes: next 8 K columns / next 8 rows
constexpr uint32_t kUmmaCols = 64;                          // tensor-memory columns (float32 accumulators)
constexpr uint32_t kWaitLimit = 1u << 24;
// instruction descriptor, kind::f16: D float32 (bit 4), A and B bf16 (bits
// 7 and 10), both K-major, N / 8 at bit 17, M / 16 at bit 24
constexpr uint32_t kUmmaIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kUN >> 3) << 17) |
                                ((uint32_t)(kUM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(const void *p, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait until the phase of `parity` of the barrier completed, trying at most
// `limit` times; false when the bounded wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kUmmaIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// byte offset of the 16-byte vector (row r, columns 8j..8j+7) in a stage
__device__ __forceinline__ uint32_t core_off(int r, int j) { return (uint32_t)((r >> 3) * kUmmaSbo + j * kUmmaLbo + (r & 7) * 16); }

// err[0]: tiles whose wait gave up, cumulative; err[1]: the same, for the
// current library call (zeroed at its start).  first_wait: the tries of the
// wait for the last commit before the read-back (kWaitLimit; lowered only by
// the test hook bs_debug_umma_wait); every other wait, and the draining wait
// before the tensor memory is released, keep kWaitLimit.
template <class Op>
__global__ void __launch_bounds__(kUThreads) umma_gemm_kernel(const Op op, unsigned int *err, uint32_t first_wait) {
  __shared__ __align__(128) uint8_t sA[2][kUM * kUK * 2];
  __shared__ __align__(128) uint8_t sB[2][kUN * kUK * 2];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kUM, n0 = blockIdx.y * kUN;
  const int kb = op.k_begin(blockIdx.z), ke = op.k_end(blockIdx.z);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kUmmaCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  // A: 512 vectors (row v / 4, columns 8 (v % 4)..), two per thread; B: 256, one
  uint4 ra[2], rb;
  Row rowa[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) rowa[i] = op.row_a(m0 + ((tid + kUThreads * i) >> 2));
  const Row rowb = op.row_b(n0 + (tid >> 2));
  auto fetch = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int v = tid + kUThreads * i, kk = k0 + 8 * (v & 3);
      ra[i] = kk < ke ? op.load_a(rowa[i], kk) : zero4();
    }
    const int kk = k0 + 8 * (tid & 3);
    rb = kk < ke ? op.load_b(rowb, kk) : zero4();
  };
  const int n_chunks = ke > kb ? (ke - kb + kUK - 1) / kUK : 0;
  bool ok = true;
  int last = n_chunks - 1;  // the last chunk whose MMAs were committed
  if (n_chunks > 0) fetch(kb);
  for (int c = 0; c < n_chunks; ++c) {
    const int st = c & 1;
    if (c >= 2) {  // the MMAs that read this stage: thread 0 waits, the CTA follows its outcome
      const bool w = tid == 0 ? mbar_wait(&bar[st], (uint32_t)(((c - 2) >> 1) & 1)) : true;
      if (!__syncthreads_and(w)) {
        ok = false;
        last = c - 1;
        break;
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int v = tid + kUThreads * i;
      *reinterpret_cast<uint4 *>(sA[st] + core_off(v >> 2, v & 3)) = ra[i];
    }
    *reinterpret_cast<uint4 *>(sB[st] + core_off(tid >> 2, tid & 3)) = rb;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stores, visible to the tensor cores
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kUK / 16; ++ks) {
        const uint64_t da = umma_desc(sA[st] + ks * 2 * kUmmaLbo, kUmmaLbo, kUmmaSbo);
        const uint64_t db = umma_desc(sB[st] + ks * 2 * kUmmaLbo, kUmmaLbo, kUmmaSbo);
        umma_bf16(tmem, da, db, (c > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&bar[st]);
    }
    if (c + 1 < n_chunks) fetch(kb + (c + 1) * kUK);
  }
  if (n_chunks > 0) {
    // thread 0 waits for the last commit, which covers every MMA it issued;
    // after a wait that gave up, a second bounded wait (full limit) before
    // the tensor memory is released, and the tile is not stored
    bool w = true;
    if (tid == 0) {
      w = ok && mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), first_wait);
      if (!w) {
        mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1));
        atomicAdd(err, 1u);
        atomicAdd(err + 1, 1u);
      }
    }
    ok = __syncthreads_and(w) && ok;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool store = __syncthreads_and(ok);
  if (store) {
    const int q = warp & 3, half = warp >> 2;
    const int m = m0 + q * 32 + lane;
#pragma unroll
    for (int col = 32 * half; col < 32 * half + 32; col += 8) {
      uint32_t v[8];
      if (n_chunks > 0) {
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
            "tcgen05.wait::ld.sync.aligned;\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
            : "r"(ta)
            : "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0u;
      }
#pragma unroll
      for (int j = 0; j < 8; j += 2) op.store(m, n0 + col + j, __uint_as_float(v[j]), __uint_as_float(v[j + 1]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUmmaCols) : "memory");
}

// ---- forward convolutions fed by the tensor memory accelerator ----
// For the 4 x 4, stride-2 convolutions whose input has 64 or more channels
// (and output channels a multiple of 128): a CTA computes a 128 x 128 tile
// (output pixels x output channels) over K = 16 taps x Cin, in chunks of 64
// input channels of one tap.  (A 32-channel input, output channels a
// multiple of 64, runs the same way with 32-channel chunks in 64-byte
// swizzled rows and 128 x 64 tiles.)  Per chunk one thread issues two TMA
// loads into a ring of kTStages shared-memory stages:
//   A: an im2col load of the NHWC input: 128 output pixels (the tile's
//      rows, traversed W, H, N with stride 2 inside the box [-1, dim - 3],
//      the padding zero-filled) x 64 channels of the tap (ky, kx), given as
//      im2col offsets; 128-byte rows, 128-byte swizzle;
//   B: a tiled load of the weights [Cout][K] (K-major): 128 rows x 64.
// Both land in the canonical K-major layout with 128-byte swizzle (8-row
// groups of 1024 bytes), which the tcgen05 descriptors read directly.
// Another thread waits for each stage, issues four tcgen05.mma (M 128, N
// 128, K 16; the descriptor's start advances 32 bytes per K step inside the
// swizzled row) and commits them to the stage's "empty" barrier, which frees
// it for the next load.  The accumulator (128 x 128 float32) lives in tensor
// memory; the epilogue reads it back (warp w: lanes 32 w ..), adds the bias,
// applies ReLU and stores bf16 NHWC rows.  Every mbarrier wait is bounded: a
// wait that gives up counts in err[0] and err[1] and the tile is not stored.
constexpr int kTM = 128, kTK = 64, kTStages = 3, kTThreads = 128;
constexpr uint32_t kTStageA = kTM * kTK * 2;   // bytes of an A stage of 64 channels

// K-major operand descriptor with 128-byte swizzle: start address, stride
// between 8-row groups 1024 bytes, version 1, layout type 2 (128B swizzle).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// K-major operand descriptor for rows of kRow bytes (128: 128-byte
// swizzle, layout type 2; 64: 64-byte swizzle, layout type 4): 8-row
// groups 8 kRow bytes apart.
template <int kRow>
__device__ __forceinline__ uint64_t umma_desc_kmajor(uint32_t addr) {
  static_assert(kRow == 128 || kRow == 64, "128- or 64-byte rows");
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((8 * kRow) >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)(kRow == 128 ? 2 : 4) << 61);
}

// Operand descriptor without swizzle (8-row x 16-byte core matrices): start,
// leading and stride byte offsets given (layout type 0).
__device__ __forceinline__ uint64_t umma_desc_plain(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

template <int kN>
__device__ __forceinline__ void umma_bf16_m128(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_im2col_4d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int c, int w, int h,
                                              int n, uint16_t off_w, uint16_t off_h) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.im2col.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6], {%7, %8};" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(w), "r"(h), "r"(n), "r"(smem_u32(bar)), "h"(off_w), "h"(off_h)
      : "memory");
}

__device__ __forceinline__ void tma_tile_2d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}


// ---- input gradients fed by the tensor memory accelerator ----
// For the 4 x 4 stride-2 convolutions with Cout a multiple of 64 and Cin 32,
// 64 or a multiple of 128.  An input pixel (2a + qy, 2c + qx) of parity
// class q = (qy, qx) is reached by the 2 x 2 taps of that parity, so per
// class the input gradient is a stride-1 2 x 2 correlation over dout:
//   din[n, 2a + qy, 2c + qx, ci] = relu'(act_in) sum over taps (ta, tb) and co
//       of dout[n, a + qy - ta, c + qx - tb, co] wq[q][ci][(2 ta + tb) Cout + co]
// (wq as DgradOp reads it).  A CTA computes a 128 x kN tile (class pixels x
// ci) over K = 4 Cout in chunks of 64 output channels of one tap:
//   A: an im2col load of dout with the class's own map (the 2 x 2 window's
//      corner runs over [q - 1, dim + q - 2] per axis at stride 1; taps as
//      im2col offsets (1 - tb, 1 - ta); outside dout reads zeros);
//   B: a tiled load of the rows q Cin + n0 .. of wq (K-major).
// Stages, descriptors, waits and commits as in conv_tma_kernel (N = kN);
// the epilogue applies the ReLU mask of act_in and stores bf16 NHWC rows at
// the class's pixels.  One launch covers the four classes (grid z).
struct DgradMaps {
  CUtensorMap a[4];
  CUtensorMap b;
};


template <int kN> constexpr uint32_t dgrad_smem() { return kTStages * (kTStageA + kN * kTK * 2) + 1024; }

// grid (ceil(M / 128), Cin / kN, 4); M = N Ho Wo pixels per class.
template <int kN>
__global__ void __launch_bounds__(kTThreads) dgrad_tma_kernel(const __grid_constant__ DgradMaps maps, int M, int Ho,
                                                              int Wo, int Cin, int Cout,
                                                              const __nv_bfloat16 *__restrict__ act_in,
                                                              __nv_bfloat16 *__restrict__ din, unsigned int *err,
                                                              uint32_t first_wait) {
  constexpr uint32_t kStageB = kN * kTK * 2;
  extern __shared__ uint8_t d_smem[];
  __shared__ __align__(8) uint64_t full[kTStages], empty[kTStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (smem_u32(d_smem) + 1023u) & ~1023u;
  const uint32_t sA = base, sB = base + kTStages * kTStageA;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kN, q = blockIdx.z, qy = q >> 1, qx = q & 1;
  const int per_tap = Cout / kTK, n_chunks = 4 * per_tap;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"((uint32_t)kN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kTStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const int hw = Ho * Wo;
  if (tid == 0) {
    // producer: the window's corner for the tile's first class pixel
    const int img = m0 / hw, r0 = m0 - img * hw, a0 = r0 / Wo, c0 = r0 - a0 * Wo;
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % kTStages;
      if (c >= kTStages && !mbar_wait(&empty[st], (uint32_t)((c / kTStages - 1) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      const int tap = c / per_tap, cb = (c - tap * per_tap) * kTK, ta = tap >> 1, tb = tap & 1;
      mbar_expect_tx(&full[st], kTStageA + kStageB);
      tma_im2col_4d(sA + st * kTStageA, &maps.a[q], &full[st], cb, c0 + qx - 1, a0 + qy - 1, img, (uint16_t)(1 - tb),
                    (uint16_t)(1 - ta));
      tma_tile_2d(sB + st * kStageB, &maps.b, &full[st], tap * Cout + cb, q * Cin + n0);
    }
  } else if (tid == 32) {
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % kTStages;
      if (!mbar_wait(&full[st], (uint32_t)((c / kTStages) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kTK / 16; ++ks) {
        const uint64_t da = umma_desc_sw128(sA + st * kTStageA + 32u * ks);
        const uint64_t db = umma_desc_sw128(sB + st * kStageB + 32u * ks);
        umma_bf16_m128<kN>(tmem, da, db, (c > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&empty[st]);
    }
    umma_commit(&done);
  }
  bool w = mbar_wait(&done, 0u, first_wait);
  if (!w) {
    mbar_wait(&done, 0u);
    if (tid == 0) {
      atomicAdd(err, 1u);
      atomicAdd(err + 1, 1u);
    }
  }
  const bool store = __syncthreads_and(w) && s_fail == 0;
  if (!store && tid == 0 && w) {
    atomicAdd(err, 1u);
    atomicAdd(err + 1, 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (store) {
    const int m = m0 + 32 * warp + lane;
    size_t o = 0;
    if (m < M) {
      const int img = m / hw, r = m - img * hw, a = r / Wo, cc = r - a * Wo;
      o = (((size_t)img * 2 * Ho + 2 * a + qy) * 2 * Wo + 2 * cc + qx) * Cin + n0;
    }
#pragma unroll
    for (int col = 0; col < kN; col += 8) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(ta)
          : "memory");
      if (m < M) {
        const uint4 x = *reinterpret_cast<const uint4 *>(act_in + o + col);
        const __nv_bfloat162 *xh = reinterpret_cast<const __nv_bfloat162 *>(&x);
        __align__(16) __nv_bfloat162 res[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 xf = __bfloat1622float2(xh[j]);
          res[j] = __floats2bfloat162_rn(xf.x > 0.f ? __uint_as_float(v[2 * j]) : 0.f,
                                         xf.y > 0.f ? __uint_as_float(v[2 * j + 1]) : 0.f);
        }
        *reinterpret_cast<uint4 *>(din + o + col) = *reinterpret_cast<const uint4 *>(res);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kN) : "memory");
}

// ---- weight gradients fed by the tensor memory accelerator ----
// For the convolutions conv_tma_kernel runs whose Ho Wo is a multiple of 64:
// dW^T[kk][co] = sum over output pixels m of patch[m][kk] dout[m][co],
// kk = (tap, ci).  A CTA computes a 128 x kN tile (kk x co) over one split
// of the pixels, in chunks of 64 pixels, and adds it to dw with float
// atomics.  Per chunk one thread issues its TMA loads into a ring of
// kWStages stages:
//   A: 128 / kACh im2col loads of the NHWC input (64 output pixels x kACh
//      channels of one tap each: the tile's kk in kACh-wide pieces);
//   B: kN / 64 tiled loads of dout [M][Cout] (64 pixels x 64 output
//      channels).
// Every box lands as 64 pixel rows of 2 kACh (A) or up to 128 (B) bytes,
// swizzled at the row width (16-byte rows: unswizzled core matrices): the
// pixels are the GEMM's reduction axis, so both operands are MN-major (the
// instruction descriptor's transpose bits).  The descriptors advance 16
// rows per K step; with swizzle the pieces of M (N) lie one box apart
// (leading byte offset) and the 8-row groups eight rows apart (stride byte
// offset); without, the two offsets trade places.  Waits, commits and the
// error count work as in conv_tma_kernel.
constexpr int kWStages = 3, kWThreads = 128;
constexpr uint32_t kWBoxB = 64 * 64 * 2;   // bytes of one dout box
template <int kACh, int kN> constexpr uint32_t wgrad_stage() {
  return 128 * 64 * 2 + (kN >= 64 ? (kN / 64) * kWBoxB : 64 * kN * 2);
}
template <int kACh, int kN> constexpr uint32_t wgrad_smem() { return kWStages * wgrad_stage<kACh, kN>() + 1024; }

// MN-major operand descriptor for rows of kRow bytes (128: 128-byte
// swizzle, layout type 2; 64: 64-byte swizzle, layout type 4); the 8-row
// groups eight rows apart.
template <int kRow>
__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t addr, uint32_t lbo) {
  static_assert(kRow == 128 || kRow == 64, "128- or 64-byte rows");
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((8 * kRow) >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)(kRow == 128 ? 2 : 4) << 61);
}

template <int kN>
__device__ __forceinline__ void umma_bf16_mn(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// grid (K / 128, Cout / kN, splits); split z takes chunks
// [z per, min(n_chunks, (z + 1) per)) of 64 pixels.
template <int kACh, int kN>
__global__ void __launch_bounds__(kWThreads) wgrad_tma_kernel(const __grid_constant__ CUtensorMap map_in,
                                                              const __grid_constant__ CUtensorMap map_dout, int Ho,
                                                              int Wo, int Cin, int K, int n_chunks, int per,
                                                              float *__restrict__ dw, unsigned int *err,
                                                              uint32_t first_wait) {
  constexpr int kRowA = 2 * kACh, kNA = 128 / kACh, kNB = kN >= 64 ? kN / 64 : 1;
  constexpr uint32_t kBoxA = 64 * kRowA, kStage = wgrad_stage<kACh, kN>();
  constexpr uint32_t kBoxB = kN >= 64 ? kWBoxB : 64 * kN * 2;  // B: 64-channel boxes, or one of kN < 64
  extern __shared__ uint8_t w_smem[];
  __shared__ __align__(8) uint64_t full[kWStages], empty[kWStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int c0 = blockIdx.z * per, n = min(n_chunks, c0 + per) - c0;
  if (n <= 0) return;  // uniform over the CTA, before any allocation
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (smem_u32(w_smem) + 1023u) & ~1023u;
  const int kk0 = blockIdx.x * 128, co0 = blockIdx.y * kN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"((uint32_t)kN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kWStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    // producer
    const int hw = Ho * Wo;
    for (int c = 0; c < n; ++c) {
      const int st = c % kWStages;
      if (c >= kWStages && !mbar_wait(&empty[st], (uint32_t)((c / kWStages - 1) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      const int m = (c0 + c) * 64, img = m / hw, r = m - img * hw, oy = r / Wo, ox = r - oy * Wo;
      const uint32_t sa = base + st * kStage, sb = sa + kNA * kBoxA;
      mbar_expect_tx(&full[st], kStage);
#pragma unroll 4
      for (int j = 0; j < kNA; ++j) {
        const int kk = kk0 + j * kACh, tap = kk / Cin, ci = kk - tap * Cin;
        tma_im2col_4d(sa + j * kBoxA, &map_in, &full[st], ci, 2 * ox - 1, 2 * oy - 1, img, (uint16_t)(tap & 3),
                      (uint16_t)(tap >> 2));
      }
#pragma unroll
      for (int j = 0; j < kNB; ++j) tma_tile_2d(sb + j * kBoxB, &map_dout, &full[st], co0 + 64 * j, m);
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int c = 0; c < n; ++c) {
      const int st = c % kWStages;
      if (!mbar_wait(&full[st], (uint32_t)((c / kWStages) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + st * kStage, sb = sa + kNA * kBoxA;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        // A: 16-byte rows (8 channels) use core matrices without swizzle;
        // for this MN-major form the leading byte offset steps along the
        // pixels (eight rows, 128 bytes) and the stride byte offset along
        // kk (one tap's box), the reverse of the swizzled forms
        const uint64_t da = kRowA == 16 ? umma_desc_plain(sa + 256u * ks, 128, kBoxA)
                                        : umma_desc_mn<kRowA == 16 ? 64 : kRowA>(sa + 16u * kRowA * ks, kBoxA);
        constexpr int kRowB = kN >= 64 ? 128 : 2 * kN;
        const uint64_t db = umma_desc_mn<kRowB>(sb + 16u * kRowB * ks, kBoxB);
        umma_bf16_mn<kN>(tmem, da, db, (c > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&empty[st]);
    }
    umma_commit(&done);
  }
  bool w = mbar_wait(&done, 0u, first_wait);
  if (!w) {
    mbar_wait(&done, 0u);
    if (tid == 0) {
      atomicAdd(err, 1u);
      atomicAdd(err + 1, 1u);
    }
  }
  const bool store = __syncthreads_and(w) && s_fail == 0;
  if (!store && tid == 0 && w) {
    atomicAdd(err, 1u);
    atomicAdd(err + 1, 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (store) {
    const int kk = kk0 + 32 * warp + lane;
#pragma unroll 4
    for (int col = 0; col < kN; col += 8) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(ta)
          : "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) atomicAdd(dw + (size_t)(co0 + col + j) * K + kk, __uint_as_float(v[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kN) : "memory");
}

// kCh input channels per chunk (64: 128-byte rows and swizzle; 32: 64-byte
// rows and swizzle, for a 32-channel input), kN output channels per tile.
// M = N Ho Wo output pixels, Cout a multiple of kN, Cin a multiple of kCh;
// grid (ceil(M / kTM), Cout / kN).
template <int kCh, int kN> constexpr uint32_t conv_smem() { return kTStages * (kTM + kN) * kCh * 2 + 1024; }

template <int kCh, int kN>
__global__ void __launch_bounds__(kTThreads) conv_tma_kernel(const __grid_constant__ CUtensorMap map_in,
                                                             const __grid_constant__ CUtensorMap map_w, int M, int Ho,
                                                             int Wo, int Cin, int Cout, const float *__restrict__ bias,
                                                             __nv_bfloat16 *__restrict__ out, unsigned int *err,
                                                             uint32_t first_wait) {
  constexpr uint32_t kStageA = kTM * kCh * 2, kStageB = kN * kCh * 2;
  extern __shared__ uint8_t t_smem[];
  __shared__ __align__(8) uint64_t full[kTStages], empty[kTStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base = (smem_u32(t_smem) + 1023u) & ~1023u;   // 1024-byte aligned stages
  const uint32_t sA = base, sB = base + kTStages * kStageA;
  const int m0 = blockIdx.x * kTM, co0 = blockIdx.y * kN;
  const int per_tap = Cin / kCh, n_chunks = 16 * per_tap;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"((uint32_t)kN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kTStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    // producer: the receptive field's corner of the tile's first output pixel
    const int hw = Ho * Wo, n0 = m0 / hw, r0 = m0 - n0 * hw, oy = r0 / Wo, ox = r0 - oy * Wo;
    const int w0 = 2 * ox - 1, h0 = 2 * oy - 1;
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % kTStages;
      if (c >= kTStages && !mbar_wait(&empty[st], (uint32_t)((c / kTStages - 1) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      const int tap = c / per_tap, cb = (c - tap * per_tap) * kCh;
      mbar_expect_tx(&full[st], kStageA + kStageB);
      tma_im2col_4d(sA + st * kStageA, &map_in, &full[st], cb, w0, h0, n0, (uint16_t)(tap & 3), (uint16_t)(tap >> 2));
      tma_tile_2d(sB + st * kStageB, &map_w, &full[st], tap * Cin + cb, co0);
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % kTStages;
      if (!mbar_wait(&full[st], (uint32_t)((c / kTStages) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kCh / 16; ++ks) {
        const uint64_t da = umma_desc_kmajor<kCh * 2>(sA + st * kStageA + 32u * ks);
        const uint64_t db = umma_desc_kmajor<kCh * 2>(sB + st * kStageB + 32u * ks);
        umma_bf16_m128<kN>(tmem, da, db, (c > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&empty[st]);
    }
    umma_commit(&done);  // arrives once every MMA issued before it has completed
  }
  // epilogue: every thread waits for the last commit (bounded; after a wait
  // that gave up, a second wait with the full bound before the tensor memory
  // is released), then reads its row of the accumulator
  bool w = mbar_wait(&done, 0u, first_wait);
  if (!w) {
    mbar_wait(&done, 0u);
    if (tid == 0) {
      atomicAdd(err, 1u);
      atomicAdd(err + 1, 1u);
    }
  }
  const bool store = __syncthreads_and(w) && s_fail == 0;
  if (!store && tid == 0 && w) {
    atomicAdd(err, 1u);
    atomicAdd(err + 1, 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (store) {
    const int m = m0 + 32 * warp + lane;
#pragma unroll 4
    for (int col = 0; col < kN; col += 8) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(ta)
          : "memory");
      if (m < M) {
        __align__(16) __nv_bfloat162 o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          o[j] = __floats2bfloat162_rn(fmaxf(__uint_as_float(v[2 * j]) + bias[co0 + col + 2 * j], 0.f),
                                       fmaxf(__uint_as_float(v[2 * j + 1]) + bias[co0 + col + 2 * j + 1], 0.f));
        *reinterpret_cast<uint4 *>(out + (size_t)m * Cout + co0 + col) = *reinterpret_cast<const uint4 *>(o);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kN) : "memory");
}

// ---- the operations ----
// lcin, lcout, lks: log2 of Cin, Cout, KS (all powers of two here)
struct Geom {
  int N, Hi, Wi, Cin, Ho, Wo, Cout, KS, S, P;
  int lcin, lcout, lks;
  __host__ __device__ int M() const { return N * Ho * Wo; }
  __host__ __device__ int K() const { return KS * KS * Cin; }
};

// Forward: out = act(patch . w^T + b).  Relu: bf16 NHWC output with ReLU;
// else float32 [M][Cout] (the head).  A row is an output pixel: (image,
// first input row, first input column); k = tap * Cin + ci reads the 8
// channels ci..ci+7 of tap (ky, kx) (zero in the padding).
template <bool kRelu>
struct FwdOp {
  Geom g;
  const __nv_bfloat16 *in, *w;
  const float *bias;
  __nv_bfloat16 *out_bf;
  float *out_f;
  __device__ int k_begin(int) const { return 0; }
  __device__ int k_end(int) const { return g.K(); }
  __device__ Row row_a(int m) const {
    if (m >= g.M()) return Row{-1, 0, 0, 0};
    const int hw = g.Ho * g.Wo, n = m / hw, r = m - n * hw, oy = r / g.Wo, ox = r - oy * g.Wo;
    return Row{n, g.S * oy - g.P, g.S * ox - g.P, 0};
  }
  __device__ uint4 load_a(const Row &r, int k) const {
    if (r.a < 0) return zero4();
    const int tap = k >> g.lcin, ci = k & (g.Cin - 1);
    const int iy = r.b + (tap >> g.lks), ix = r.c + (tap & (g.KS - 1));
    if (iy < 0 || iy >= g.Hi || ix < 0 || ix >= g.Wi) return zero4();
    return *reinterpret_cast<const uint4 *>(in + (((size_t)r.a * g.Hi + iy) * g.Wi + ix) * g.Cin + ci);
  }
  __device__ Row row_b(int n) const { return Row{n < g.Cout ? n : -1, 0, 0, 0}; }
  __device__ uint4 load_b(const Row &r, int k) const {
    return r.a >= 0 ? *reinterpret_cast<const uint4 *>(w + (size_t)r.a * g.K() + k) : zero4();
  }
  __device__ void store(int m, int n, float v0, float v1) const {
    if (m >= g.M() || n >= g.Cout) return;
    v0 += bias[n];
    v1 += bias[n + 1];
    if (kRelu) {
      *reinterpret_cast<__nv_bfloat162 *>(out_bf + (size_t)m * g.Cout + n) =
          __floats2bfloat162_rn(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
    } else {
      out_f[(size_t)m * g.Cout + n] = v0;
      out_f[(size_t)m * g.Cout + n + 1] = v1;
    }
  }
};

// Input gradient of a 4 x 4, stride-2, padding-1 convolution for the input
// pixels of parity (qy, qx): iy = 2 hy + qy.  Such a pixel is reached by the
// taps ky = (1 - qy) + 2a, a = 0, 1, from output row oy = hy + qy - a (and
// likewise in x), so din = sum over k = (a, b, co) of dout[oy, ox, co] wq[ci][k]
// with wq the class's weights gathered by net_dgrad_weights_kernel.  The
// result is multiplied by the ReLU mask of the input activation (the gradient
// of the previous layer's pre-activation).  A row is an input pixel of the
// class: (image, hy + qy, hx + qx).
struct DgradOp {
  Geom g;
  int qy, qx;
  const __nv_bfloat16 *dout, *wq, *act_in;
  __nv_bfloat16 *din;
  __device__ int Mh() const { return g.N * (g.Hi / 2) * (g.Wi / 2); }
  __device__ int k_begin(int) const { return 0; }
  __device__ int k_end(int) const { return 4 * g.Cout; }
  __device__ void pixel(int m, int &n, int &iy, int &ix) const {
    const int hh = g.Hi / 2, wh = g.Wi / 2, hw = hh * wh;
    n = m / hw;
    const int r = m - n * hw, hy = r / wh, hx = r - hy * wh;
    iy = 2 * hy + qy;
    ix = 2 * hx + qx;
  }
  __device__ Row row_a(int m) const {
    if (m >= Mh()) return Row{-1, 0, 0, 0};
    int n, iy, ix;
    pixel(m, n, iy, ix);
    return Row{n, (iy >> 1) + qy, (ix >> 1) + qx, 0};
  }
  __device__ uint4 load_a(const Row &r, int k) const {
    if (r.a < 0) return zero4();
    const int tp = k >> g.lcout, co = k & (g.Cout - 1);
    const int oy = r.b - (tp >> 1), ox = r.c - (tp & 1);
    if (oy < 0 || oy >= g.Ho || ox < 0 || ox >= g.Wo) return zero4();
    return *reinterpret_cast<const uint4 *>(dout + (((size_t)r.a * g.Ho + oy) * g.Wo + ox) * g.Cout + co);
  }
  __device__ Row row_b(int n) const { return Row{n < g.Cin ? n : -1, 0, 0, 0}; }
  __device__ uint4 load_b(const Row &r, int k) const {
    return r.a >= 0 ? *reinterpret_cast<const uint4 *>(wq + (size_t)r.a * 4 * g.Cout + k) : zero4();
  }
  __device__ void store(int m, int ci, float v0, float v1) const {
    if (m >= Mh() || ci >= g.Cin) return;
    int n, iy, ix;
    pixel(m, n, iy, ix);
    const size_t o = (((size_t)n * g.Hi + iy) * g.Wi + ix) * g.Cin + ci;
    const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162 *>(act_in + o);
    const float m0 = __bfloat162float(x.x) > 0.f ? 1.f : 0.f, m1 = __bfloat162float(x.y) > 0.f ? 1.f : 0.f;
    *reinterpret_cast<__nv_bfloat162 *>(din + o) = __floats2bfloat162_rn(v0 * m0, v1 * m1);
  }
};

// Input gradient of the 1 x 1 head: din[m][ci] = sum_co dout[m][co] w[co][ci],
// times the ReLU mask of the head's input.  wt = w transposed, [Cin][Cout].
struct HeadDgradOp {
  int M, Cin, Cout;
  const __nv_bfloat16 *dout, *wt, *act_in;
  __nv_bfloat16 *din;
  __device__ int k_begin(int) const { return 0; }
  __device__ int k_end(int) const { return Cout; }
  __device__ Row row_a(int m) const { return Row{m < M ? m : -1, 0, 0, 0}; }
  __device__ uint4 load_a(const Row &r, int k) const {
    return r.a >= 0 ? *reinterpret_cast<const uint4 *>(dout + (size_t)r.a * Cout + k) : zero4();
  }
  __device__ Row row_b(int n) const { return Row{n < Cin ? n : -1, 0, 0, 0}; }
  __device__ uint4 load_b(const Row &r, int k) const {
    return r.a >= 0 ? *reinterpret_cast<const uint4 *>(wt + (size_t)r.a * Cout + k) : zero4();
  }
  __device__ void store(int m, int ci, float v0, float v1) const {
    if (m >= M || ci >= Cin) return;
    const size_t o = (size_t)m * Cin + ci;
    const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162 *>(act_in + o);
    const float m0 = __bfloat162float(x.x) > 0.f ? 1.f : 0.f, m1 = __bfloat162float(x.y) > 0.f ? 1.f : 0.f;
    *reinterpret_cast<__nv_bfloat162 *>(din + o) = __floats2bfloat162_rn(v0 * m0, v1 * m1);
  }
};

// Weight gradient: dw[co][k] += sum over output pixels m of this split of
// dout[m][co] patch[m][k]; K of the GEMM = the pixels, 8 at a time.
struct WgradOp {
  Geom g;
  int chunk;  // pixels per split, a multiple of kBK
  const __nv_bfloat16 *dout, *in;
  float *dw;
  __device__ int k_begin(int z) const { return z * chunk; }
  __device__ int k_end(int z) const { return min(g.M(), (z + 1) * chunk); }
  __device__ Row row_a(int co) const { return Row{co < g.Cout ? co : -1, 0, 0, 0}; }
  __device__ uint4 load_a(const Row &r, int m) const {  // dout[m..m+7][co]
    if (r.a < 0) return zero4();
    const int co = r.a;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      v[i] = m + i < g.M() ? dout[(size_t)(m + i) * g.Cout + co] : __float2bfloat16(0.f);
    return *reinterpret_cast<const uint4 *>(v);
  }
  __device__ Row row_b(int kk) const {  // (ci, ky, kx) of weight column kk
    if (kk >= g.K()) return Row{-1, 0, 0, 0};
    const int tap = kk >> g.lcin;
    return Row{kk & (g.Cin - 1), tap >> g.lks, tap & (g.KS - 1), 0};
  }
  __device__ uint4 load_b(const Row &rw, int m) const {  // patch[m..m+7][kk]
    if (rw.a < 0) return zero4();
    const int ci = rw.a, ky = rw.b, kx = rw.c;
    const int hw = g.Ho * g.Wo;
    __align__(16) __nv_bfloat16 v[8];
    {  // the 8 pixels in one output row: one input row, x in steps of S
      const int n = m / hw, r = m - n * hw, oy = r / g.Wo, ox = r - oy * g.Wo;
      if (m + 7 < g.M() && ox + 7 < g.Wo) {
        const int iy = g.S * oy + ky - g.P;
        if (iy < 0 || iy >= g.Hi) return zero4();
        const __nv_bfloat16 *row = in + (((size_t)n * g.Hi + iy) * g.Wi) * g.Cin + ci;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int ix = g.S * (ox + i) + kx - g.P;
          v[i] = (ix >= 0 && ix < g.Wi) ? row[(size_t)ix * g.Cin] : __float2bfloat16(0.f);
        }
        return *reinterpret_cast<const uint4 *>(v);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      v[i] = __float2bfloat16(0.f);
      const int mm = m + i;
      if (mm < g.M()) {
        const int n = mm / hw, r = mm - n * hw, oy = r / g.Wo, ox = r - oy * g.Wo;
        const int iy = g.S * oy + ky - g.P, ix = g.S * ox + kx - g.P;
        if (iy >= 0 && iy < g.Hi && ix >= 0 && ix < g.Wi)
          v[i] = in[(((size_t)n * g.Hi + iy) * g.Wi + ix) * g.Cin + ci];
      }
    }
    return *reinterpret_cast<const uint4 *>(v);
  }
  __device__ void store(int co, int kk, float v0, float v1) const {
    if (co >= g.Cout || kk >= g.K()) return;
    if (v0 != 0.f) atomicAdd(dw + (size_t)co * g.K() + kk, v0);
    if (v1 != 0.f) atomicAdd(dw + (size_t)co * g.K() + kk + 1, v1);
  }
};

// The GEMM engine: 1 (default) = tcgen05 for a reduction of at least
// kUmmaMinK per CTA, mma.sync below (a tcgen05 CTA pays a fixed cost for its
// tensor memory, barriers and read-back, which a few K chunks do not
// amortise); 2 = tcgen05 always, 0 = mma.sync always (the test hook
// bs_debug_gemm_engine selects them).
int g_gemm_engine = 1;   // 3: tcgen05 with thread-gathered operands for every GEMM
constexpr int kUmmaMinK = 1024;
// [0] tiles whose wait gave up since the process started, [1] in the
// current library call
__device__ unsigned int g_umma_timeouts[2];
uint32_t g_first_wait = kWaitLimit;

// The device address of g_umma_timeouts, looked up once per device.
bs_status umma_err_ptr(unsigned int **out) {
  constexpr int kMaxDev = 64;
  static unsigned int *cache[kMaxDev] = {};
  static std::once_flag once[kMaxDev];
  static cudaError_t err[kMaxDev] = {};
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) {
    set_error("device %d: at most %d devices supported", dev, kMaxDev);
    return BS_ERR_UNSUPPORTED;
  }
  std::call_once(once[dev], [dev] { err[dev] = cudaGetSymbolAddress((void **)&cache[dev], g_umma_timeouts); });
  BS_CUDA(err[dev]);
  *out = cache[dev];
  return BS_OK;
}

// Start of a network call: zero its count of tensor-core waits that gave up.
bs_status call_timeouts_reset(cudaStream_t s) {
  unsigned int *err = nullptr;
  BS_TRY(umma_err_ptr(&err));
  BS_CUDA(cudaMemsetAsync(err + 1, 0, sizeof(unsigned int), s));
  return BS_OK;
}

// End of a network call: read that count (one synchronisation); a wait that
// gave up left its tile's outputs unwritten, so the call fails.
bs_status call_timeouts_check(cudaStream_t s, const char *what) {
  unsigned int *err = nullptr;
  BS_TRY(umma_err_ptr(&err));
  unsigned int n = 0;
  BS_CUDA(cudaMemcpyAsync(&n, err + 1, sizeof(n), cudaMemcpyDeviceToHost, s));
  BS_CUDA(cudaStreamSynchronize(s));
  if (n) {
    set_error("%s: %u tensor-core tile(s) gave up a bounded wait on their MMAs; their outputs were not written",
              what, n);
    return BS_ERR_TIMEOUT;
  }
  return BS_OK;
}

template <class Op>
bs_status run_gemm(const Op &op, int M, int N, int K, int splits, cudaStream_t s) {
  if (g_gemm_engine >= 2 || (g_gemm_engine == 1 && K >= kUmmaMinK)) {
    unsigned int *err = nullptr;
    BS_TRY(umma_err_ptr(&err));
    const dim3 grid((unsigned)div_up(M, kUM), (unsigned)div_up(N, kUN), (unsigned)splits);
    umma_gemm_kernel<Op><<<grid, kUThreads, 0, s>>>(op, err, g_first_wait);
    BS_LAUNCHED("umma_gemm_kernel");
    return BS_OK;
  }
  const dim3 grid((unsigned)div_up(M, kBM), (unsigned)div_up(N, kBN), (unsigned)splits);
  gemm_kernel<Op><<<grid, kGemmThreads, 0, s>>>(op);
  BS_LAUNCHED("gemm_kernel");
  return BS_OK;
}

// ---- tensor maps for conv_tma_kernel ----
// The driver's encoders, taken through the runtime's entry-point lookup (the
// library links no driver library).
using EncodeIm2col = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const int *, const int *, cuuint32_t, cuuint32_t,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bs_status tma_encoders(EncodeIm2col *im2col, EncodeTiled *tiled) {
  static std::once_flag once;
  static void *f_im2col = nullptr, *f_tiled = nullptr;
  static bool ok = false;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeIm2col", &f_im2col, 12000,
                                                            cudaEnableDefault, &q1);
    const cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f_tiled, 12000,
                                                            cudaEnableDefault, &q2);
    ok = e1 == cudaSuccess && e2 == cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
         q2 == cudaDriverEntryPointSuccess && f_im2col && f_tiled;
  });
  if (!ok) {
    set_error("the driver's tensor-map encoders are not available");
    return BS_ERR_UNSUPPORTED;
  }
  *im2col = reinterpret_cast<EncodeIm2col>(f_im2col);
  *tiled = reinterpret_cast<EncodeTiled>(f_tiled);
  return BS_OK;
}

template <int kCh, int kN>
bs_status launch_conv_tma(const CUtensorMap &map_in, const CUtensorMap &map_w, const Geom &g, const float *bias,
                          __nv_bfloat16 *out, unsigned int *err, cudaStream_t s) {
  constexpr int kMaxDev = 64;
  static bool attr[kMaxDev] = {};
  static std::mutex mu;
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDev || !attr[dev]) {
      BS_CUDA(cudaFuncSetAttribute(conv_tma_kernel<kCh, kN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)conv_smem<kCh, kN>()));
      if (dev >= 0 && dev < kMaxDev) attr[dev] = true;
    }
  }
  const dim3 grid((unsigned)div_up(g.M(), kTM), (unsigned)(g.Cout / kN));
  conv_tma_kernel<kCh, kN><<<grid, kTThreads, conv_smem<kCh, kN>(), s>>>(map_in, map_w, g.M(), g.Ho, g.Wo, g.Cin,
                                                                         g.Cout, bias, out, err, g_first_wait);
  BS_LAUNCHED("conv_tma_kernel");
  return BS_OK;
}

// The TMA box width for layer g: 64 channels (Cin a multiple of 64, Cout of
// 128), 32 (a 32-channel input, Cout a multiple of 64) or 8 (an 8-channel
// input, Cout a multiple of 32; the weight gradient only: as a forward its
// tiles are too small to pay for sixteen loads each); 0: the gathered
// engines.
int conv_tma_channels(const Geom &g) {
  if (!(g_gemm_engine == 1 || g_gemm_engine == 2) || g.KS != 4 || g.S != 2 || g.P != 1) return 0;
  if (g.Cin % 64 == 0 && g.Cout % 128 == 0) return 64;
  if (g.Cin == 32 && g.Cout % 64 == 0) return 32;
  if (g.Cin == 8 && g.Cout % 32 == 0) return 8;
  return 0;
}

// The forward convolution of layer g (4 x 4, stride 2, padding 1) by
// conv_tma_kernel, with the chunk width of conv_tma_channels.
bs_status run_conv_tma(const Geom &g, const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias,
                       __nv_bfloat16 *out, cudaStream_t s) {
  const int ch = conv_tma_channels(g);
  const int nt = ch == 64 ? 128 : 64;
  const CUtensorMapSwizzle swz = ch == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  EncodeIm2col enc_im2col;
  EncodeTiled enc_tiled;
  BS_TRY(tma_encoders(&enc_im2col, &enc_tiled));
  CUtensorMap map_in, map_w;
  const cuuint64_t dims[4] = {(cuuint64_t)g.Cin, (cuuint64_t)g.Wi, (cuuint64_t)g.Hi, (cuuint64_t)g.N};
  const cuuint64_t strides[3] = {(cuuint64_t)g.Cin * 2, (cuuint64_t)g.Wi * g.Cin * 2,
                                 (cuuint64_t)g.Hi * g.Wi * g.Cin * 2};
  // the receptive field's corner runs over [-P, dim - 1 + P - (KS - 1)]
  const int lower[2] = {-g.P, -g.P}, upper[2] = {g.P - (g.KS - 1), g.P - (g.KS - 1)};
  const cuuint32_t estr[4] = {1, (cuuint32_t)g.S, (cuuint32_t)g.S, 1};
  CUresult r = enc_im2col(&map_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(in), dims, strides,
                          lower, upper, (cuuint32_t)ch, kTM, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeIm2col failed (%d) for a %dx%dx%d input", (int)r, g.Hi, g.Wi, g.Cin);
    return BS_ERR_CUDA;
  }
  const cuuint64_t wdims[2] = {(cuuint64_t)g.K(), (cuuint64_t)g.Cout};
  const cuuint64_t wstrides[1] = {(cuuint64_t)g.K() * 2};
  const cuuint32_t box[2] = {(cuuint32_t)ch, (cuuint32_t)nt}, wes[2] = {1, 1};
  r = enc_tiled(&map_w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(w), wdims, wstrides, box,
                wes, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for the %dx%d weights", (int)r, g.Cout, g.K());
    return BS_ERR_CUDA;
  }
  unsigned int *err = nullptr;
  BS_TRY(umma_err_ptr(&err));
  if (ch == 64) return launch_conv_tma<64, 128>(map_in, map_w, g, bias, out, err, s);
  return launch_conv_tma<32, 64>(map_in, map_w, g, bias, out, err, s);
}

// The layers whose forward runs on conv_tma_kernel.
bool uses_tma(const Geom &g) { return conv_tma_channels(g) >= 32; }

template <int kACh, int kN>
bs_status launch_wgrad_tma(const CUtensorMap &map_in, const CUtensorMap &map_dout, const Geom &g, float *dw,
                           unsigned int *err, cudaStream_t s) {
  constexpr int kMaxDev = 64;
  static bool attr[kMaxDev] = {};
  static std::mutex mu;
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDev || !attr[dev]) {
      BS_CUDA(cudaFuncSetAttribute(wgrad_tma_kernel<kACh, kN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)wgrad_smem<kACh, kN>()));
      if (dev >= 0 && dev < kMaxDev) attr[dev] = true;
    }
  }
  // splits of the pixels so that about two CTAs per SM run
  const int tiles = (g.K() / 128) * (g.Cout / kN), n_chunks = g.M() / 64;
  int splits = std::max(1, std::min(n_chunks, div_up(2 * 152, tiles)));
  const int per = div_up(n_chunks, splits);
  splits = div_up(n_chunks, per);
  const dim3 grid((unsigned)(g.K() / 128), (unsigned)(g.Cout / kN), (unsigned)splits);
  wgrad_tma_kernel<kACh, kN><<<grid, kWThreads, wgrad_smem<kACh, kN>(), s>>>(map_in, map_dout, g.Ho, g.Wo, g.Cin,
                                                                             g.K(), n_chunks, per, dw, err,
                                                                             g_first_wait);
  BS_LAUNCHED("wgrad_tma_kernel");
  return BS_OK;
}

// The weight gradient of layer g by wgrad_tma_kernel (the layers
// conv_tma_kernel runs, with Ho Wo a multiple of 64): A pieces of the
// forward's box width, co tiles of 128 (64 for a 32-channel input, 32 for
// an 8-channel one).
bs_status run_wgrad_tma(const Geom &g, const __nv_bfloat16 *in, const __nv_bfloat16 *dout, float *dw, cudaStream_t s) {
  const int ch = conv_tma_channels(g);
  EncodeIm2col enc_im2col;
  EncodeTiled enc_tiled;
  BS_TRY(tma_encoders(&enc_im2col, &enc_tiled));
  CUtensorMap map_in, map_dout;
  const cuuint64_t dims[4] = {(cuuint64_t)g.Cin, (cuuint64_t)g.Wi, (cuuint64_t)g.Hi, (cuuint64_t)g.N};
  const cuuint64_t strides[3] = {(cuuint64_t)g.Cin * 2, (cuuint64_t)g.Wi * g.Cin * 2,
                                 (cuuint64_t)g.Hi * g.Wi * g.Cin * 2};
  const int lower[2] = {-g.P, -g.P}, upper[2] = {g.P - (g.KS - 1), g.P - (g.KS - 1)};
  const cuuint32_t estr[4] = {1, (cuuint32_t)g.S, (cuuint32_t)g.S, 1};
  CUresult r = enc_im2col(&map_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(in), dims, strides,
                          lower, upper, (cuuint32_t)ch, 64, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          ch == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : (ch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE),
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeIm2col failed (%d) for a %dx%dx%d input", (int)r, g.Hi, g.Wi, g.Cin);
    return BS_ERR_CUDA;
  }
  const cuuint64_t ddims[2] = {(cuuint64_t)g.Cout, (cuuint64_t)g.M()};
  const cuuint64_t dstrides[1] = {(cuuint64_t)g.Cout * 2};
  const int nb = g.Cout >= 64 ? 64 : g.Cout;   // dout box width: 64 channels, or all of fewer
  const cuuint32_t box[2] = {(cuuint32_t)nb, 64}, es[2] = {1, 1};
  r = enc_tiled(&map_dout, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(dout), ddims, dstrides, box,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE, nb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for the %dx%d output gradient", (int)r, g.M(), g.Cout);
    return BS_ERR_CUDA;
  }
  unsigned int *err = nullptr;
  BS_TRY(umma_err_ptr(&err));
  if (ch == 64) return launch_wgrad_tma<64, 128>(map_in, map_dout, g, dw, err, s);
  if (ch == 32) return launch_wgrad_tma<32, 64>(map_in, map_dout, g, dw, err, s);
  return launch_wgrad_tma<8, 32>(map_in, map_dout, g, dw, err, s);
}

bool uses_tma_wgrad(const Geom &g) { return conv_tma_channels(g) != 0 && (g.Ho * g.Wo) % 64 == 0; }
// The input gradient of layer g by dgrad_tma_kernel: dout [N][Ho][Wo][Cout],
// wq the four classes' weights [4][Cin][4 Cout] (bf16), act_in / din
// [N][Hi][Wi][Cin].
template <int kN>
bs_status launch_dgrad_tma(const DgradMaps &maps, const Geom &g, const __nv_bfloat16 *act_in, __nv_bfloat16 *din,
                           unsigned int *err, cudaStream_t s) {
  constexpr int kMaxDev = 64;
  static bool attr[kMaxDev] = {};
  static std::mutex mu;
  int dev = 0;
  BS_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDev || !attr[dev]) {
      BS_CUDA(cudaFuncSetAttribute(dgrad_tma_kernel<kN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)dgrad_smem<kN>()));
      if (dev >= 0 && dev < kMaxDev) attr[dev] = true;
    }
  }
  const int M = g.N * g.Ho * g.Wo;
  const dim3 grid((unsigned)div_up(M, kTM), (unsigned)(g.Cin / kN), 4u);
  dgrad_tma_kernel<kN><<<grid, kTThreads, dgrad_smem<kN>(), s>>>(maps, M, g.Ho, g.Wo, g.Cin, g.Cout, act_in, din, err,
                                                                 g_first_wait);
  BS_LAUNCHED("dgrad_tma_kernel");
  return BS_OK;
}

bs_status run_dgrad_tma(const Geom &g, const __nv_bfloat16 *dout, const __nv_bfloat16 *wq, const __nv_bfloat16 *act_in,
                        __nv_bfloat16 *din, cudaStream_t s) {
  EncodeIm2col enc_im2col;
  EncodeTiled enc_tiled;
  BS_TRY(tma_encoders(&enc_im2col, &enc_tiled));
  const int kN = g.Cin >= 128 ? 128 : g.Cin;
  DgradMaps maps;
  const cuuint64_t dims[4] = {(cuuint64_t)g.Cout, (cuuint64_t)g.Wo, (cuuint64_t)g.Ho, (cuuint64_t)g.N};
  const cuuint64_t strides[3] = {(cuuint64_t)g.Cout * 2, (cuuint64_t)g.Wo * g.Cout * 2,
                                 (cuuint64_t)g.Ho * g.Wo * g.Cout * 2};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int q = 0; q < 4; ++q) {
    // the 2 x 2 window's corner runs over [q - 1, dim + q - 2] on each axis
    const int lower[2] = {(q & 1) - 1, (q >> 1) - 1}, upper[2] = {(q & 1) - 1, (q >> 1) - 1};
    const CUresult r = enc_im2col(&maps.a[q], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(dout),
                                  dims, strides, lower, upper, kTK, kTM, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeIm2col failed (%d) for a %dx%dx%d output gradient", (int)r, g.Ho, g.Wo, g.Cout);
      return BS_ERR_CUDA;
    }
  }
  const cuuint64_t wdims[2] = {(cuuint64_t)4 * g.Cout, (cuuint64_t)4 * g.Cin};
  const cuuint64_t wstrides[1] = {(cuuint64_t)4 * g.Cout * 2};
  const cuuint32_t box[2] = {kTK, (cuuint32_t)kN}, wes[2] = {1, 1};
  const CUresult r = enc_tiled(&maps.b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(wq), wdims,
                               wstrides, box, wes, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for the %dx%d class weights", (int)r, 4 * g.Cin, 4 * g.Cout);
    return BS_ERR_CUDA;
  }
  unsigned int *err = nullptr;
  BS_TRY(umma_err_ptr(&err));
  switch (kN) {
    case 32: return launch_dgrad_tma<32>(maps, g, act_in, din, err, s);
    case 64: return launch_dgrad_tma<64>(maps, g, act_in, din, err, s);
    default: return launch_dgrad_tma<128>(maps, g, act_in, din, err, s);
  }
}

// The layers whose input gradient runs on dgrad_tma_kernel.
bool uses_tma_dgrad(const Geom &g) {
  return (g_gemm_engine == 1 || g_gemm_engine == 2) && g.KS == 4 && g.S == 2 && g.P == 1 && g.Cout % kTK == 0 &&
         (g.Cin == 32 || g.Cin == 64 || g.Cin % 128 == 0);
}

// ---- element-wise pieces ----
// Planar float32 patches [N][3][H][W] -> NHWC bf16 [N][H][W][8] (channels
// 3..7 zero).
__global__ void net_input_kernel(const float *__restrict__ x, int N, int H, int W, __nv_bfloat16 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)H * W;
  if (i >= N * plane) return;
  const int64_t n = i / plane, p = i - n * plane;
  const float *src = x + n * 3 * plane + p;
  __align__(16) __nv_bfloat16 v[8];
  v[0] = __float2bfloat16(src[0]);
  v[1] = __float2bfloat16(src[plane]);
  v[2] = __float2bfloat16(src[2 * plane]);
#pragma unroll
  for (int c = 3; c < 8; ++c) v[c] = __float2bfloat16(0.f);
  *reinterpret_cast<uint4 *>(out + i * 8) = *reinterpret_cast<const uint4 *>(v);
}

__global__ void to_bf16_kernel(const float *__restrict__ x, int64_t n, __nv_bfloat16 *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// wq[q][ci][(a, b, co)] = w[co][ky][kx][ci], ky = (1 - qy) + 2a, kx = (1 - qx) + 2b
// for the four parity classes q = 2 qy + qx of a 4 x 4 kernel.
__global__ void net_dgrad_weights_kernel(const float *__restrict__ w, int Cin, int Cout,
                                         __nv_bfloat16 *__restrict__ wq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)Cin * 4 * Cout;
  if (i >= 4 * per) return;
  const int q = (int)(i / per);
  const int64_t r = i - q * per;
  const int ci = (int)(r / (4 * Cout)), k = (int)(r - (int64_t)ci * 4 * Cout);
  const int tp = k / Cout, co = k - tp * Cout, a = tp >> 1, b = tp & 1;
  const int qy = q >> 1, qx = q & 1;
  const int ky = (1 - qy) + 2 * a, kx = (1 - qx) + 2 * b;
  wq[i] = __float2bfloat16(w[((size_t)co * 16 + ky * 4 + kx) * Cin + ci]);
}

// wt[ci][co] = w[co][ci] (the head), bf16.
__global__ void net_transpose_kernel(const float *__restrict__ w, int Cin, int Cout, __nv_bfloat16 *__restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Cin * Cout) return;
  const int ci = i / Cout, co = i - ci * Cout;
  wt[i] = __float2bfloat16(w[(size_t)co * Cin + ci]);
}

// db[co] += sum over m of dout[m][co] (bf16 dout [M][C], C a multiple of 8,
// at most 256).  Each CTA takes a contiguous chunk of rows; a thread reads
// 8 channels (16 bytes) of a row at a time, so consecutive threads read
// consecutive bytes, and accumulates them in float; the CTA then sums its
// threads' partials per channel in shared memory and adds one atomic per
// channel.
constexpr int kBiasThreads = 256;
__global__ void __launch_bounds__(kBiasThreads) net_bias_grad_kernel(const __nv_bfloat16 *__restrict__ dout, int M,
                                                                     int C, float *__restrict__ db) {
  __shared__ float s_acc[kBiasThreads][9];
  const int groups = C >> 3, grp = threadIdx.x % groups, rstep = kBiasThreads / groups;
  const int64_t chunk = div_up64(M, gridDim.x);
  const int64_t m0 = (int64_t)blockIdx.x * chunk, m1 = min((int64_t)M, m0 + chunk);
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;
#pragma unroll 4
  for (int64_t m = m0 + threadIdx.x / groups; m < m1; m += rstep) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(dout + m * C) + grp);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(h[k]);
      acc[2 * k] += f.x;
      acc[2 * k + 1] += f.y;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) s_acc[threadIdx.x][k] = acc[k];
  __syncthreads();
  if ((int)threadIdx.x < C) {
    const int g = threadIdx.x >> 3, k = threadIdx.x & 7;
    float t = 0.f;
    for (int r = 0; r < rstep; ++r) t += s_acc[r * groups + g][k];
    if (t != 0.f) atomicAdd(db + threadIdx.x, t);
  }
}

// The grid of net_bias_grad_kernel for M rows: about 8 rows per thread,
// at most four CTAs per SM.
unsigned bias_grid(int M, int C) {
  const int64_t rows_per_cta = (int64_t)(kBiasThreads / (C >> 3)) * 8;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, div_up64(M, rows_per_cta)));
}

// The head's 64 outputs per cell o -> one closed curve and one open stroke
// (the two kinds of Section 3.2) in the patch's pixel coordinates, around the
// cell centre C (cells row-major on the grid x grid lattice of side `cell`):
//   closed  P_j = C + reach tanh(o_{2j}, o_{2j+1}) (j < 12), colour
//           sigmoid(o_24..26), opacity sigmoid(o_27);
//   open    Q_j = C + reach tanh(o_{28+2j}, o_{29+2j}) (j < 10), width
//           wmax sigmoid(o_48), colour sigmoid(o_49..51), segment opacities
//           sigmoid(o_52..54); outputs 55..63 are unused.
// With targets (tgt.ctrl non-NULL): the loss, the mean over cells of
//   sum_j |P_j - P*_j|^2 / reach^2 + |c - c*|^2 + (a - a*)^2
//   + sum_j |Q_j - Q*_j|^2 / reach^2 + (w - w*)^2 / wmax^2 + |c' - c'*|^2 + sum_s (a'_s - a'*_s)^2,
// added to *loss (one double atomic per cell), and dL/do as bf16 [cells][64]
// (zero at the unused outputs) for the head's backward.
constexpr int kHeadOut = 64;

__device__ __forceinline__ float head_sigmoid(float x) { return 1.f / (1.f + __expf(-x)); }

__global__ void net_head_kernel(const float *__restrict__ o, int n_cells, int grid, float cell, float reach, float wmax,
                                bs_net_curves out, bs_net_curves tgt, double *__restrict__ loss,
                                __nv_bfloat16 *__restrict__ dout) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const float *oc = o + (size_t)c * kHeadOut;
  const bool train = tgt.ctrl != nullptr;
  __nv_bfloat16 *dc = train ? dout + (size_t)c * kHeadOut : nullptr;
  const int cc = c % (grid * grid), gy = cc / grid, gx = cc - gy * grid;
  const float cx = (gx + 0.5f) * cell, cy = (gy + 0.5f) * cell;
  double l = 0.0;
  const float inv = 1.f / (reach * reach), scale = 1.f / (float)n_cells;
  // control points: the closed curve's 12 at outputs 0..23, the stroke's 10 at 28..47
  for (int kind = 0; kind < 2; ++kind) {
    const int np = kind ? 10 : 12, o0 = kind ? 28 : 0;
    float *dst = kind ? out.open_ctrl : out.ctrl;
    const float *t = kind ? tgt.open_ctrl : tgt.ctrl;
    for (int j = 0; j < np; ++j) {
      const float tx = tanhf(oc[o0 + 2 * j]), ty = tanhf(oc[o0 + 2 * j + 1]);
      const float px = cx + reach * tx, py = cy + reach * ty;
      const size_t e0 = ((size_t)c * np + j) * 2;
      if (dst) {
        dst[e0] = px;
        dst[e0 + 1] = py;
      }
      if (train) {
        const float ex = px - t[e0], ey = py - t[e0 + 1];
        l += (double)(ex * ex + ey * ey) * inv;
        dc[o0 + 2 * j] = __float2bfloat16(scale * 2.f * ex * inv * reach * (1.f - tx * tx));
        dc[o0 + 2 * j + 1] = __float2bfloat16(scale * 2.f * ey * inv * reach * (1.f - ty * ty));
      }
    }
  }
  // the sigmoid outputs: value s, written to dst[i] and compared with t[i]
  auto unit = [&](int k, float *dst, const float *t, size_t i) {
    const float s = head_sigmoid(oc[k]);
    if (dst) dst[i] = s;
    if (train) {
      const float e = s - t[i];
      l += (double)(e * e);
      dc[k] = __float2bfloat16(scale * 2.f * e * s * (1.f - s));
    }
  };
  for (int k = 0; k < 3; ++k) {
    unit(24 + k, out.color, tgt.color, (size_t)c * 3 + k);
    unit(49 + k, out.open_color, tgt.open_color, (size_t)c * 3 + k);
    unit(52 + k, out.open_opac, tgt.open_opac, (size_t)c * 3 + k);
  }
  unit(27, out.opac, tgt.opac, c);
  {  // width: (w - w*) / wmax = s - w* / wmax, so the term is a unit one in s
    const float s = head_sigmoid(oc[48]);
    if (out.open_width) out.open_width[c] = wmax * s;
    if (train) {
      const float e = s - tgt.open_width[c] / wmax;
      l += (double)(e * e);
      dc[48] = __float2bfloat16(scale * 2.f * e * s * (1.f - s));
    }
  }
  if (train) {
    for (int k = 55; k < kHeadOut; ++k) dc[k] = __float2bfloat16(0.f);
    atomicAdd(loss, l / (double)n_cells);
  }
}

}  // namespace

// ---- host side ----
// The layer geometry of a batch of n patches of side `side` (a multiple of
// 32): layer l in 0..4 the 4 x 4 stride-2 convolutions, 5 the head.
static const int kNetCh[6] = {8, 32, 64, 128, 256, 256};

Geom net_layer(int l, int n, int side) {
  Geom g{};
  g.N = n;
  if (l < 5) {
    g.Hi = g.Wi = side >> l;
    g.Ho = g.Wo = side >> (l + 1);
    g.Cin = kNetCh[l];
    g.Cout = kNetCh[l + 1];
    g.KS = 4;
    g.S = 2;
    g.P = 1;
  } else {
    g.Hi = g.Wi = g.Ho = g.Wo = side >> 5;
    g.Cin = 256;
    g.Cout = kHeadOut;
    g.KS = 1;
    g.S = 1;
    g.P = 0;
  }
  g.lcin = bit_length((uint64_t)g.Cin) - 1;
  g.lcout = bit_length((uint64_t)g.Cout) - 1;
  g.lks = bit_length((uint64_t)g.KS) - 1;
  return g;
}

size_t net_param_count(int l) {
  const Geom g = net_layer(l, 1, 256);
  return (size_t)g.Cout * g.K() + g.Cout;  // weights then bias
}

}  // namespace bs

using namespace bs;

namespace {

bs_status net_invalid(const char *msg) {
  set_error("%s", msg);
  return BS_ERR_INVALID_ARG;
}

bs_status check_net(const bs_net *net, int32_t n, int32_t side) {
  if (!net) return net_invalid("net is NULL");
  if (n < 1 || side < 32 || side % 32 || side > 1024) return net_invalid("n >= 1 patches of side 32..1024, a multiple of 32");
  for (int l = 0; l < BS_NET_LAYERS; ++l)
    if (!net->w[l] || !net->w_bf16[l]) return net_invalid("net weights must be non-NULL");
  return BS_OK;
}

// Activation buffers inside the workspace: x0 (input, 8 channels) and the
// outputs of layers 0..4, NHWC bf16; the head output (float [cells][64]).
struct NetWs {
  __nv_bfloat16 *act[6];
  float *head;
  __nv_bfloat16 *dact[6];  // gradients of the activations (same shapes)
  __nv_bfloat16 *dhead;
  __nv_bfloat16 *wq;       // dgrad weights of the largest layer (4 classes)
  size_t bytes;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

NetWs carve_net(void *base, int n, int side) {
  NetWs w{};
  char *p = static_cast<char *>(base);
  size_t o = 0;
  for (int l = 0; l <= 5; ++l) {
    const int s = side >> l;
    const size_t e = (size_t)n * s * s * kNetCh[l];
    w.act[l] = base ? reinterpret_cast<__nv_bfloat16 *>(p + o) : nullptr;
    o = align256(o + 2 * e);
    w.dact[l] = base ? reinterpret_cast<__nv_bfloat16 *>(p + o) : nullptr;
    o = align256(o + 2 * e);
  }
  const size_t cells = (size_t)n * (side >> 5) * (side >> 5);
  w.head = base ? reinterpret_cast<float *>(p + o) : nullptr;
  o = align256(o + 4 * cells * kHeadOut);
  w.dhead = base ? reinterpret_cast<__nv_bfloat16 *>(p + o) : nullptr;
  o = align256(o + 2 * cells * kHeadOut);
  w.wq = base ? reinterpret_cast<__nv_bfloat16 *>(p + o) : nullptr;
  o = align256(o + 2 * (size_t)4 * 256 * 4 * 256);
  w.bytes = o;
  return w;
}

const __nv_bfloat16 *wbf(const bs_net *net, int l) { return reinterpret_cast<const __nv_bfloat16 *>(net->w_bf16[l]); }

bs_status net_forward(const bs_net *net, const float *patches, int n, int side, const NetWs &ws, cudaStream_t s) {
  const int64_t px = (int64_t)n * side * side;
  net_input_kernel<<<(unsigned)div_up64(px, 256), 256, 0, s>>>(patches, n, side, side, ws.act[0]);
  BS_LAUNCHED("net_input_kernel");
  for (int l = 0; l < 5; ++l) {
    const Geom g = net_layer(l, n, side);
    const float *bias = net->w[l] + (size_t)g.Cout * g.K();
    if (uses_tma(g)) {
      BS_TRY(run_conv_tma(g, ws.act[l], wbf(net, l), bias, ws.act[l + 1], s));
      continue;
    }
    const FwdOp<true> op{g, ws.act[l], wbf(net, l), bias, ws.act[l + 1], nullptr};
    BS_TRY(run_gemm(op, g.M(), g.Cout, g.K(), 1, s));
  }
  const Geom g = net_layer(5, n, side);
  const FwdOp<false> op{g, ws.act[5], wbf(net, 5), net->w[5] + (size_t)g.Cout * g.K(), nullptr, ws.head};
  return run_gemm(op, g.M(), g.Cout, g.K(), 1, s);
}

}  // namespace

extern "C" {

bs_status bs_debug_gemm_engine(int32_t engine, int64_t *timeouts_out) {
  if (engine < 0 || engine > 3)
    return net_invalid("engine must be 0 (mma.sync), 1 (by reduction length), 2 (tcgen05) or 3 (tcgen05, gathered)");
  g_gemm_engine = engine;
  if (timeouts_out) {
    unsigned int t[2] = {0, 0};
    BS_CUDA(cudaMemcpyFromSymbol(t, g_umma_timeouts, sizeof(t)));
    *timeouts_out = t[0];
  }
  return BS_OK;
}

bs_status bs_debug_umma_wait(int64_t first_wait) {
  g_first_wait = first_wait < 0 ? kWaitLimit : (uint32_t)std::min<int64_t>(first_wait, kWaitLimit);
  return BS_OK;
}

bs_status bs_net_workspace(int32_t n, int32_t side, size_t *bytes) {
  if (!bytes) return net_invalid("bytes is NULL");
  if (n < 1 || side < 32 || side % 32 || side > 1024) return net_invalid("n >= 1 patches of side 32..1024, a multiple of 32");
  *bytes = carve_net(nullptr, n, side).bytes;
  return BS_OK;
}

int64_t bs_net_param_count(int32_t layer) {
  if (layer < 0 || layer >= BS_NET_LAYERS) return -1;
  return (int64_t)net_param_count(layer);
}

bs_status bs_net_sync_weights(const bs_net *net, bs_stream stream) {
  if (!net) return net_invalid("net is NULL");
  for (int l = 0; l < BS_NET_LAYERS; ++l)
    if (!net->w[l] || !net->w_bf16[l]) return net_invalid("net weights must be non-NULL");
  BS_TRY(check_device());
  const cudaStream_t s = (cudaStream_t)stream;
  for (int l = 0; l < BS_NET_LAYERS; ++l) {
    const Geom g = net_layer(l, 1, 256);
    const int64_t nw = (int64_t)g.Cout * g.K();
    to_bf16_kernel<<<(unsigned)div_up64(nw, 256), 256, 0, s>>>(net->w[l], nw,
                                                              reinterpret_cast<__nv_bfloat16 *>(net->w_bf16[l]));
    BS_LAUNCHED("to_bf16_kernel");
  }
  return BS_OK;
}

bs_status bs_net_forward(const bs_net *net, const float *patches, int32_t n, int32_t side, void *ws, size_t ws_bytes,
                         float *head_out, const bs_net_curves *curves, bs_stream stream) {
  BS_TRY(check_net(net, n, side));
  const NetWs w = carve_net(ws, n, side);
  if (!ws || ws_bytes < w.bytes || ((uintptr_t)ws & 255u)) return net_invalid("workspace too small or not 256-byte aligned");
  if (!patches) return net_invalid("patches is NULL");
  BS_TRY(check_device());
  const cudaStream_t s = (cudaStream_t)stream;
  BS_TRY(call_timeouts_reset(s));
  BS_TRY(net_forward(net, patches, n, side, w, s));
  const int grid = side >> 5, cells = n * grid * grid;
  const bs_net_curves out = curves ? *curves : bs_net_curves{};
  net_head_kernel<<<div_up(cells, 128), 128, 0, s>>>(w.head, cells, grid, 32.f, BS_NET_REACH, BS_NET_WIDTH_MAX, out,
                                                     bs_net_curves{}, nullptr, nullptr);
  BS_LAUNCHED("net_head_kernel");
  if (head_out) BS_CUDA(cudaMemcpyAsync(head_out, w.head, sizeof(float) * cells * kHeadOut, cudaMemcpyDeviceToDevice, s));
  return call_timeouts_check(s, "bs_net_forward");
}

bs_status bs_net_train_step(const bs_net *net, const float *patches, int32_t n, int32_t side,
                            const bs_net_curves *target, void *ws, size_t ws_bytes, const bs_net_grad *grad,
                            double *loss_out, bs_stream stream) {
  BS_TRY(check_net(net, n, side));
  if (!grad || !target || !loss_out) return net_invalid("NULL target, gradient or loss");
  if (!target->ctrl || !target->color || !target->opac || !target->open_ctrl || !target->open_width ||
      !target->open_color || !target->open_opac)
    return net_invalid("every target array must be non-NULL");
  for (int l = 0; l < BS_NET_LAYERS; ++l)
    if (!grad->g[l]) return net_invalid("gradient buffers must be non-NULL");
  const NetWs w = carve_net(ws, n, side);
  if (!ws || ws_bytes < w.bytes || ((uintptr_t)ws & 255u)) return net_invalid("workspace too small or not 256-byte aligned");
  if (!patches) return net_invalid("patches is NULL");
  BS_TRY(check_device());
  const cudaStream_t s = (cudaStream_t)stream;
  BS_TRY(call_timeouts_reset(s));
  BS_TRY(net_forward(net, patches, n, side, w, s));
  const int grid = side >> 5, cells = n * grid * grid;
  BS_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(double), s));
  net_head_kernel<<<div_up(cells, 128), 128, 0, s>>>(w.head, cells, grid, 32.f, BS_NET_REACH, BS_NET_WIDTH_MAX,
                                                     bs_net_curves{}, *target, loss_out, w.dhead);
  BS_LAUNCHED("net_head_kernel");
  for (int l = 0; l < BS_NET_LAYERS; ++l)
    BS_CUDA(cudaMemsetAsync(grad->g[l], 0, sizeof(float) * net_param_count(l), s));
  // head: weights, bias, input gradient
  {
    const Geom g = net_layer(5, n, side);
    const int chunk = std::max(kBK, (int)div_up64(div_up64(g.M(), 152), kBK) * kBK);
    const WgradOp op{g, chunk, w.dhead, w.act[5], grad->g[5]};
    BS_TRY(run_gemm(op, g.Cout, g.K(), chunk, div_up(g.M(), chunk), s));
    net_bias_grad_kernel<<<bias_grid(g.M(), g.Cout), kBiasThreads, 0, s>>>(w.dhead, g.M(), g.Cout,
                                                                           grad->g[5] + (size_t)g.Cout * g.K());
    BS_LAUNCHED("net_bias_grad_kernel");
    net_transpose_kernel<<<div_up(g.Cin * g.Cout, 256), 256, 0, s>>>(net->w[5], g.Cin, g.Cout, w.wq);
    BS_LAUNCHED("net_transpose_kernel");
    const HeadDgradOp dop{g.M(), g.Cin, g.Cout, w.dhead, w.wq, w.act[5], w.dact[5]};
    BS_TRY(run_gemm(dop, g.M(), g.Cin, g.Cout, 1, s));
  }
  for (int l = 4; l >= 0; --l) {
    const Geom g = net_layer(l, n, side);
    const __nv_bfloat16 *dout = w.dact[l + 1];
    if (uses_tma_wgrad(g)) {
      BS_TRY(run_wgrad_tma(g, w.act[l], dout, grad->g[l], s));
    } else {
      const int chunk = std::max(kBK, (int)div_up64(div_up64(g.M(), 304), kBK) * kBK);
      const WgradOp op{g, chunk, dout, w.act[l], grad->g[l]};
      BS_TRY(run_gemm(op, g.Cout, g.K(), chunk, div_up(g.M(), chunk), s));
    }
    net_bias_grad_kernel<<<bias_grid(g.M(), g.Cout), kBiasThreads, 0, s>>>(dout, g.M(), g.Cout,
                                                                           grad->g[l] + (size_t)g.Cout * g.K());
    BS_LAUNCHED("net_bias_grad_kernel");
    if (l == 0) break;  // the input image needs no gradient
    const int64_t nq = 4ll * g.Cin * 4 * g.Cout;
    net_dgrad_weights_kernel<<<(unsigned)div_up64(nq, 256), 256, 0, s>>>(net->w[l], g.Cin, g.Cout, w.wq);
    BS_LAUNCHED("net_dgrad_weights_kernel");
    if (uses_tma_dgrad(g)) {
      BS_TRY(run_dgrad_tma(g, dout, w.wq, w.act[l], w.dact[l], s));
      continue;
    }
    for (int q = 0; q < 4; ++q) {
      const DgradOp dop{g, q >> 1, q & 1, dout, w.wq + (size_t)q * g.Cin * 4 * g.Cout, w.act[l], w.dact[l]};
      BS_TRY(run_gemm(dop, g.N * (g.Hi / 2) * (g.Wi / 2), g.Cin, 4 * g.Cout, 1, s));
    }
  }
  return call_timeouts_check(s, "bs_net_train_step");
}

}  // extern "C"
