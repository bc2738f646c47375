// Tensor-core Gram for the mixed-precision path: S = Z^T Z / n from FP32
// operands split into hi + lo parts and three products hi*hi + hi*lo + lo*hi
// (FP32 accumulation in tensor memory), on 5th-generation tensor cores
// (tcgen05), in two operand formats:
//   3xTF32   tf32 parts (11 significant bits each), tcgen05.mma kind::tf32;
//   3xBF16   bf16 parts (8 significant bits each), tcgen05.mma kind::f16 --
//            half the operand bytes and twice the MMA rate of tf32, at an
//            error of about 2^-16 instead of 2^-22 per product.
// A 128-byte swizzled row holds 32 tf32 or 64 bf16 values and one MMA covers
// 32 bytes of K in both formats, so tiles, stages and the MMA loop are shared.
//
// Layout: the split kernel writes Zt_hi / Zt_lo as p_pad x n_pad row-major
// FP32 (K-major operands: the reduction index k is contiguous), zero padded.
// Each CTA computes one 128 x 128 tile (bi, bj), bi <= bj, of the upper
// triangle and writes it and its mirror, so S is exactly symmetric.
//   * thread 0 streams K blocks (one 128-byte row) of A_hi, A_lo (rows of tile bi) and
//     B_hi, B_lo (rows of tile bj) with TMA (128-byte swizzle) into a
//     3-stage shared-memory ring guarded by mbarriers;
//   * thread 32 issues, per K block, 4 x 3 tcgen05.mma (32 bytes of K each) into one
//     of two 128-column FP32 accumulators in tensor memory (a new one every
//     4 K blocks) and commits each stage back to its producer barrier;
//   * eight epilogue warps drain each finished accumulator (tcgen05.ld, each
//     warp its own 32 lanes and 64 columns) into compensated FP32 running
//     sums (TwoSum: the high parts in registers, the low parts in the upper
//     half of tensor memory), then scale by 1/n and store S[i][j] and
//     S[j][i] for i <= j through a shared-memory transpose.
// Every wait is bounded (%globaltimer); a wait that runs out sets bit 4 of
// the caller's status word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kernels.h"
#include "fp_bits.cuh"

namespace concord {

__device__ __forceinline__ float to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Standardize, split and transpose: zt_hi[i * n_pad + k] = tf32(z_ki),
// zt_lo[i * n_pad + k] = tf32(z_ki - hi) with z = (x - mean_i) * inv_scale_i
// rounded to FP32; when zt is given, also zt[i * ldz + k] = z (k < ldz).
// hi / lo may be NULL (zt only).  32 x 32 tiles through shared memory;
// padding is zero.
template <typename TX>
__global__ void __launch_bounds__(256) k_split_tf32(const TX* __restrict__ X, int n, int p, int ldx,
                                                    const double* __restrict__ mean,
                                                    const double* __restrict__ inv_scale,
                                                    float* __restrict__ hi, float* __restrict__ lo,
                                                    int n_pad, int p_pad, float* __restrict__ zt,
                                                    int ldz) {
  __shared__ float th[32][33];
  __shared__ float tl[32][33];
  __shared__ float tz[32][33];
  const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, i = i0 + tx;
    float z = 0.f;
    if (k < n && i < p) z = narrow_f64((to_f64(X[(size_t)k * ldx + i]) - mean[i]) * inv_scale[i]);
    const float h = to_tf32(z);
    th[r][tx] = h;
    tl[r][tx] = to_tf32(z - h);
    tz[r][tx] = z;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    if (i < p_pad && k < n_pad && hi) {
      hi[(size_t)i * n_pad + k] = th[tx][r];
      lo[(size_t)i * n_pad + k] = tl[tx][r];
    }
    if (zt && i < p_pad && k < ldz) zt[(size_t)i * ldz + k] = tz[tx][r];
  }
}

cudaError_t launch_split_tf32(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, float* zt_hi, float* zt_lo, int n_pad,
                              int p_pad, cudaStream_t st, float* zt, int ldz) {
  dim3 grid((n_pad + 31) / 32, (p_pad + 31) / 32);
  if (x_f32)
    k_split_tf32<float><<<grid, 256, 0, st>>>((const float*)X, n, p, ldx, mean, inv_scale, zt_hi,
                                              zt_lo, n_pad, p_pad, zt, ldz);
  else
    k_split_tf32<double><<<grid, 256, 0, st>>>((const double*)X, n, p, ldx, mean, inv_scale, zt_hi,
                                               zt_lo, n_pad, p_pad, zt, ldz);
  note_launches(1);
  return cudaGetLastError();
}

// The same for the bf16 split: hi = bf16(z), lo = bf16(z - hi), both as raw
// 16-bit patterns; zt as in k_split_tf32.
template <typename TX>
__global__ void __launch_bounds__(256) k_split_bf16(const TX* __restrict__ X, int n, int p, int ldx,
                                                    const double* __restrict__ mean,
                                                    const double* __restrict__ inv_scale,
                                                    uint16_t* __restrict__ hi,
                                                    uint16_t* __restrict__ lo, int n_pad,
                                                    int p_pad, float* __restrict__ zt, int ldz) {
  __shared__ uint16_t th[32][34];
  __shared__ uint16_t tl[32][34];
  __shared__ float tz[32][33];
  const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, i = i0 + tx;
    float z = 0.f;
    if (k < n && i < p) z = narrow_f64((to_f64(X[(size_t)k * ldx + i]) - mean[i]) * inv_scale[i]);
    const __nv_bfloat16 h = __float2bfloat16_rn(z);
    th[r][tx] = __bfloat16_as_ushort(h);
    tl[r][tx] = __bfloat16_as_ushort(__float2bfloat16_rn(z - __bfloat162float(h)));
    tz[r][tx] = z;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    if (i < p_pad && k < n_pad) {
      hi[(size_t)i * n_pad + k] = th[tx][r];
      lo[(size_t)i * n_pad + k] = tl[tx][r];
    }
    if (zt && i < p_pad && k < ldz) zt[(size_t)i * ldz + k] = tz[tx][r];
  }
}

cudaError_t launch_split_bf16(const void* X, int x_f32, int n, int p, int ldx, const double* mean,
                              const double* inv_scale, uint16_t* zt_hi, uint16_t* zt_lo, int n_pad,
                              int p_pad, cudaStream_t st, float* zt, int ldz) {
  dim3 grid((n_pad + 31) / 32, (p_pad + 31) / 32);
  if (x_f32)
    k_split_bf16<float><<<grid, 256, 0, st>>>((const float*)X, n, p, ldx, mean, inv_scale, zt_hi,
                                              zt_lo, n_pad, p_pad, zt, ldz);
  else
    k_split_bf16<double><<<grid, 256, 0, st>>>((const double*)X, n, p, ldx, mean, inv_scale, zt_hi,
                                               zt_lo, n_pad, p_pad, zt, ldz);
  note_launches(1);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- tcgen05
constexpr int kTM = 128;                          // tile rows (M) and columns (N)
constexpr int kRowBytes = 128;                    // K block: one 128-byte swizzled row per tile row
constexpr int kStages = 3;
constexpr int kOpBytes = kTM * kRowBytes;         // one operand tile: 16 KB
constexpr int kStageBytes = 4 * kOpBytes;         // A_hi, A_lo, B_hi, B_lo
constexpr int kChunkKb = 4;                       // K blocks summed per FP32 accumulator chunk
constexpr int kEpiWarps = 8;                      // epilogue warps (2 per TMEM lane quadrant)
constexpr int kGramThreads = 32 * (2 + kEpiWarps);  // producer, MMA issuer, epilogue
constexpr int kTmemCols = 512;                    // two 128-column FP32 accumulators + low parts
constexpr int kSumLo = 2 * kTM;                   // tensor-memory columns of the sums' low parts
constexpr size_t kGramSmem = (size_t)kStages * kStageBytes + 1024;  // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false (and status bit 4)
// if it has not completed within 2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++it & 255u) == 0 && globaltimer_ns() - t0 > 2000000000ull) {
      atomicOr(status, 4);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored in the
// 128-byte swizzled layout TMA writes (rows of 128 bytes, 8-row groups 1024
// bytes apart): start address >> 4, leading offset (unused for swizzled
// K-major) 16 B, stride offset 1024 B, descriptor version 1, layout
// SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptors: D FP32 (bits 4-5 = 1), A and B format (bits 7-9,
// 10-12: 2 = TF32 for kind::tf32, 1 = BF16 for kind::f16), both K-major,
// N = 128 (bits 17-22, N >> 3), M = 128 (bits 24-28, M >> 4).
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTM >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTM >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);

// Operand formats: elements per 128-byte row (the K block).
struct Tf32Fmt {
  static constexpr int kTK = 32;
};
struct Bf16Fmt {
  static constexpr int kTK = 64;
};

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.b32 q, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %4, q;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(accumulate), "r"(kIdescTf32)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.b32 q, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, q;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(accumulate), "r"(kIdescBf16)
      : "memory");
}

template <typename F>
__device__ __forceinline__ void mma_fmt(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (F::kTK == Bf16Fmt::kTK) mma_bf16(d, a, b, acc);
  else mma_tf32(d, a, b, acc);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st_32x32b_x32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
      "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
      "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// hi + lo += x with the rounding error of hi + x kept exactly (Knuth's
// TwoSum: six FP32 additions, no ordering assumption on |hi| and |x|).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// Order of the upper-triangle tiles over the grid: bands of kGroupRows tile
// rows; within a band the tile columns in increasing order and, per column,
// the band's rows bi <= bj.  The CTAs resident at one time then read a few
// dozen operand row blocks (the band's own and a run of columns), each from
// several CTAs at nearly the same K, so L2 serves the repeats; in row-major
// order every resident CTA streams its own column block from HBM.
constexpr int kGroupRows = 8;

__host__ __device__ inline void gram_tile(int t, int nbt, int group, int& bi, int& bj) {
  int r0 = 0;
  for (;;) {
    const int g = nbt - r0 < group ? nbt - r0 : group;
    const int tri = g * (g + 1) / 2;  // columns r0 .. r0 + g - 1: rows r0 .. bj
    const int cnt = tri + (nbt - r0 - g) * g;
    if (t < cnt) {
      if (t < tri) {
        int c = 0;
        while (t > c) {
          t -= c + 1;
          ++c;
        }
        bj = r0 + c;
        bi = r0 + t;
      } else {
        t -= tri;
        bj = r0 + g + t / g;
        bi = r0 + t % g;
      }
      return;
    }
    t -= cnt;
    r0 += g;
  }
}

// Packed FP32 pair arithmetic (add / sub .f32x2, round to nearest on each
// element: the same results as two scalar operations, one instruction).
__device__ __forceinline__ void add_f32x2(float& d0, float& d1, float a0, float a1, float b0,
                                          float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

__device__ __forceinline__ void sub_f32x2(float& d0, float& d1, float a0, float a1, float b0,
                                          float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// two_sum_acc on two running sums at once: the same operations in the same
// order on each element, as packed pairs.
__device__ __forceinline__ void two_sum_acc2(float& h0, float& h1, float& l0, float& l1, float x0,
                                             float x1) {
  float s0, s1, b0, b1, t0, t1, u0, u1, v0, v1, e0, e1;
  add_f32x2(s0, s1, h0, h1, x0, x1);  // s = hi + x
  sub_f32x2(b0, b1, s0, s1, h0, h1);  // bp = s - hi
  sub_f32x2(t0, t1, s0, s1, b0, b1);  // s - bp
  sub_f32x2(u0, u1, h0, h1, t0, t1);  // hi - (s - bp)
  sub_f32x2(v0, v1, x0, x1, b0, b1);  // x - bp
  add_f32x2(e0, e1, u0, u1, v0, v1);  // err
  h0 = s0;
  h1 = s1;
  add_f32x2(l0, l1, l0, l1, e0, e1);  // lo += err
}

// One CTA per 128 x 128 tile of the upper triangle.  The K reduction is cut
// into chunks of kChunkKb blocks (128 elements): each chunk accumulates in
// FP32 in one of two tensor-memory buffers while the epilogue warps add the
// previous chunk into the compensated running sums, so FP32 rounding only
// ever covers one chunk's products and the tensor pipe does not wait for the
// drain.  (FP64 additions in the drain would stall it: this part's FP64 rate
// is a small fraction of its FP32 rate.)
template <typename F>
__global__ void __launch_bounds__(kGramThreads, 1)
    k_gram_3x(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
              int nkb, int p, float* __restrict__ S, int lds, float scale, int nbt, int group,
              int* status) {
  constexpr int kTK = F::kTK;
  extern __shared__ unsigned char gsm_raw[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ uint32_t tmem_base;
  // 1024-byte aligned operand ring (the 128-byte swizzle repeats every 1024)
  unsigned char* ring = (unsigned char*)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);

  int bi, bj;
  gram_tile(blockIdx.x, nbt, group, bi, bj);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (nkb + kChunkKb - 1) / kChunkKb;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps * 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ---- producer: TMA loads of the four operand tiles per K block
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kStages;
        if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1, status)) break;
        unsigned char* st = ring + (size_t)s * kStageBytes;
        mbar_expect_tx(&full[s], kStageBytes);
        tma_load_2d(st, &tm_hi, &full[s], kb * kTK, bi * kTM);
        tma_load_2d(st + kOpBytes, &tm_lo, &full[s], kb * kTK, bi * kTM);
        tma_load_2d(st + 2 * kOpBytes, &tm_hi, &full[s], kb * kTK, bj * kTM);
        tma_load_2d(st + 3 * kOpBytes, &tm_lo, &full[s], kb * kTK, bj * kTM);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: per K block hi*hi + hi*lo + lo*hi on four K = 8 slices
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2) {
          ok = mbar_wait(&acc_empty[b], ((c >> 1) - 1) & 1, status);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const uint32_t d = tbase + (uint32_t)(b * kTM);
        const int kb_end = min(nkb, (c + 1) * kChunkKb);
        for (int kb = c * kChunkKb; kb < kb_end; ++kb) {
          const int s = kb % kStages;
          ok = mbar_wait(&full[s], (kb / kStages) & 1, status);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(ring + (size_t)s * kStageBytes);
          const uint64_t ah = sw128_kmajor_desc(st), al = sw128_kmajor_desc(st + kOpBytes);
          const uint64_t bh = sw128_kmajor_desc(st + 2 * kOpBytes);
          const uint64_t bl = sw128_kmajor_desc(st + 3 * kOpBytes);
#pragma unroll
          for (int kk = 0; kk < kRowBytes / 32; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32 >> 4);  // one MMA: 32 bytes along K
            const uint32_t first = (kb == c * kChunkKb && kk == 0) ? 0u : 1u;
            mma_fmt<F>(d, ah + adv, bh + adv, first);
            mma_fmt<F>(d, ah + adv, bl + adv, 1u);
            mma_fmt<F>(d, al + adv, bh + adv, 1u);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&acc_full[b]);
      }
    }
  } else {
    // ---- epilogue: warp e owns TMEM lanes 32 (warp % 4) .. +31 (tile rows)
    //      and tile columns 64 * (e / 4) .. +63.  The compensated sums across
    //      chunks keep their high parts in registers (fully unrolled) and
    //      their low parts in tensor memory: with both parts in registers the
    //      drain spilled to local memory, whose traffic shares the SRAM the
    //      MMAs read their operands from
    const int e = warp - 2;
    const int quad = warp & 3;
    const int col0 = 64 * (e >> 2);
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    float sh[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) sh[q] = 0.f;
    const uint32_t lo_t = tbase + lanes + (uint32_t)(kSumLo + col0);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      ok = __all_sync(0xffffffffu, ok && mbar_wait(&acc_full[b], (c >> 1) & 1, status));
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tbase + lanes + (uint32_t)(b * kTM + col0);
      if (ok) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t v[32], l[32];
          tmem_ld_32x32b_x32(acc + 32 * h, v);
          if (c == 0) {
#pragma unroll
            for (int q = 0; q < 32; ++q) l[q] = 0u;
          } else {
            tmem_ld_32x32b_x32(lo_t + 32 * h, l);
          }
#pragma unroll
          for (int q = 0; q < 32; q += 2) {
            float l0 = __uint_as_float(l[q]), l1 = __uint_as_float(l[q + 1]);
            two_sum_acc2(sh[32 * h + q], sh[32 * h + q + 1], l0, l1, __uint_as_float(v[q]),
                         __uint_as_float(v[q + 1]));
            l[q] = __float_as_uint(l0);
            l[q + 1] = __float_as_uint(l1);
          }
          tmem_st_32x32b_x32(lo_t + 32 * h, l);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      // the accumulator is free once its loads have completed
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acc_empty[b]);
      if (!ok) break;
    }
    float sl[64];
    if (ok) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t l[32];
        tmem_ld_32x32b_x32(lo_t + 32 * h, l);
#pragma unroll
        for (int q = 0; q < 32; ++q) sl[32 * h + q] = __uint_as_float(l[q]);
      }
    }
    if (ok) {
      // (hi + lo) * scale -- one rounding of hi * scale plus the (tiny)
      // lo * scale: within an FP32 ulp of the exact product -- staged in
      // shared memory (the operand ring is idle here: every load was consumed
      // and the last MMA has completed), then written as S[j][i] (lanes over
      // i) and S[i][j] (lanes over j): one coalesced row segment per store
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      float* T = reinterpret_cast<float*>(ring) + e * (32 * 65);
#pragma unroll
      for (int q = 0; q < 64; ++q) T[lane * 65 + q] = fmaf(sh[q], scale, sl[q] * scale);
      __syncwarp();
      const int i0 = bi * kTM + quad * 32;
      const int j0 = bj * kTM + col0;
      const int i = i0 + lane;
      if (i < p)
        for (int q = 0; q < 64; ++q) {
          const int j = j0 + q;
          if (j < p && i <= j) S[(size_t)j * lds + i] = T[lane * 65 + q];
        }
      for (int r = 0; r < 32 && i0 + r < p; ++r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + 32 * h + lane;
          if (j < p && i0 + r <= j) S[(size_t)(i0 + r) * lds + j] = T[r * 65 + 32 * h + lane];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(kTmemCols)
                 : "memory");
}

namespace {

std::mutex g_tma_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t encode_fn(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lock(g_tma_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  *out = g_encode;
  return cudaSuccess;
}

// 2-D tensor map over a p_pad x n_pad array of FP32 (bf16 = false) or bf16,
// box one 128-byte row (K) x 128 rows, 128-byte swizzle.
cudaError_t make_map(CUtensorMap* map, const void* base, int n_pad, int p_pad, bool bf16) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  cudaError_t e = encode_fn(&enc);
  if (e != cudaSuccess) return e;
  cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)p_pad};
  const size_t esz = bf16 ? 2 : 4;
  cuuint64_t strides[1] = {(cuuint64_t)n_pad * esz};
  cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)kTM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

namespace {

template <typename F>
cudaError_t launch_gram_3x(const void* zt_hi, const void* zt_lo, int n_pad, int p_pad, int p, float* S,
                           int lds, float scale, int* status, cudaStream_t st,
                           int group = kGroupRows) {
  constexpr bool bf16 = F::kTK == Bf16Fmt::kTK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return cudaErrorNotSupported;
  if (n_pad % F::kTK != 0 || p_pad % kTM != 0 || n_pad <= 0 || p_pad <= 0)
    return cudaErrorInvalidValue;
  if (((uintptr_t)zt_hi & 15) || ((uintptr_t)zt_lo & 15)) return cudaErrorInvalidValue;
  CUtensorMap m_hi, m_lo;
  if ((e = make_map(&m_hi, zt_hi, n_pad, p_pad, bf16)) != cudaSuccess) return e;
  if ((e = make_map(&m_lo, zt_lo, n_pad, p_pad, bf16)) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gram_3x<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGramSmem);
  if (e != cudaSuccess) return e;
  const int nbt = p_pad / kTM;
  const int tiles = nbt * (nbt + 1) / 2;
  if (group < 1) return cudaErrorInvalidValue;
  k_gram_3x<F><<<tiles, kGramThreads, kGramSmem, st>>>(m_hi, m_lo, n_pad / F::kTK, p, S, lds, scale,
                                                      nbt, group, status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_tf32x3(const float* zt_hi, const float* zt_lo, int n_pad, int p_pad, int p,
                               float* S, int lds, float scale, int* status, cudaStream_t st) {
  return launch_gram_3x<Tf32Fmt>(zt_hi, zt_lo, n_pad, p_pad, p, S, lds, scale, status, st);
}

cudaError_t launch_gram_bf16x3(const uint16_t* zt_hi, const uint16_t* zt_lo, int n_pad, int p_pad,
                               int p, float* S, int lds, float scale, int* status, cudaStream_t st) {
  return launch_gram_3x<Bf16Fmt>(zt_hi, zt_lo, n_pad, p_pad, p, S, lds, scale, status, st);
}

}  // namespace concord
