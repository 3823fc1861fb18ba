// Trailing update of the Hermitian sweep on the tensor cores with FP64-level
// accuracy (error-free splitting of the operands, the Ozaki scheme).
//
// Each sweep step subtracts the rank-kb product P C^H from the lower triangle
// (kb <= 32).  With u_i = [Re P_i, Im P_i] and v_j = [Re C_j, Im C_j] (64 real
// values each), Re(P_i C_j^H) = u_i . v_j and
// Im(P_i C_j^H) = u_i[32:64] . v_j[0:32] - u_i[0:32] . v_j[32:64].
// Every row is scaled by a power of two sigma_i (>= its largest entry) and cut
// into S slices of 8 bits: u_i = sigma_i sum_a 2^{-8(a+1)} h_a, with integer
// h_a (|h_0| <= 256, |h_a| <= 128 for a >= 1) held exactly in FP16.  The
// slice products h_a . g_b are integers whose sums over 64 terms and over
// the pairs of one level L = a + b stay below 2^24, so the tensor cores'
// FP32 accumulation is exact: one FP32 accumulator per level (Re and Im) in
// tensor memory.  The levels a + b < S are kept; they are combined in
// double-FP32 (two-sum); the pair, scaled by the power of two
// sigma_i tau_j 2^-16, is subtracted from A in FP64.  The dropped levels and the double-FP32 sum
// bound the error near 2^-48 of |u_i| |v_j| 64.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "runtime.h"
#include "sweep_common.cuh"

namespace bgw {

namespace oz {

constexpr int S = 7;             // slices per value
constexpr int BETA = 8;          // bits per slice
constexpr int KR = 64;           // real inner length (32 complex)
constexpr int BM = 128;          // tile rows (i)
constexpr int BN = 32;           // tile cols (j)
constexpr int NB = 32;           // sweep block width
constexpr int kThreads = 512;          // 16 warps: four per tensor-memory lane quadrant in the epilogue
constexpr int kChunk = 4;              // epilogue columns per tensor-memory load round
constexpr int kUTile = BM * KR * 2;    // 16 KiB
constexpr int kVTile = BN * KR * 2;    // 4 KiB
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > kWaitNs) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// K-major operand, 128-byte swizzle: rows of 128 bytes, 8-row groups 1024
// bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;  // SWIZZLE_128B
  return d;
}
__host__ __device__ constexpr uint32_t idesc(bool neg_a) {
  return (1u << 4) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Per-matrix description of one batched sweep (device pointers).
struct OzMat {
  double2* A;
  const double2* C;   // [ng][NB]
  const double2* P;   // [ng][NB]
  double2* Dinv;      // [NB][NB] D^-1 of the next diagonal block (written by mode 1)
  int ng;
  int row_off;        // first slice row of this matrix (multiple of BM)
};
constexpr int kBatch = 96;
struct OzBatch {
  int n;
  OzMat m[kBatch];
};

// Balanced base-256 digits of a 56-bit fixed-point value: x = sum_a h_a
// 2^{-8(a+1)} for |x| < 1, |h_0| <= 256 and |h_a| <= 128 (a >= 1).  X is
// rint(x 2^56); integer arithmetic only.
__device__ __forceinline__ void digits7(long long X, __half* out, size_t stride) {
  int d[S];
#pragma unroll
  for (int p = 0; p < S - 1; ++p) {
    const long long dp = ((X + 128) & 255) - 128;
    d[S - 1 - p] = (int)dp;
    X = (X - dp) >> 8;
  }
  d[0] = (int)X;
#pragma unroll
  for (int a = 0; a < S; ++a) out[a * stride] = __int2half_rn(d[a]);
}

// Slices and exponent of one 64-value row held by a warp (lane: value k and
// k + 32); all lanes call it.
__device__ __forceinline__ void slice_row(double re, double im, int lane, __half* base, size_t stride, int* exp_out) {
  double m = fmax(fabs(re), fabs(im));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  if (m > 0.0) frexp(m, &e);  // |value| 2^-e < 1
  const long long Xr = llrint(ldexp(re, 56 - e)), Xi = llrint(ldexp(im, 56 - e));
  digits7(Xr, base + lane, stride);
  digits7(Xi, base + lane + 32, stride);
  if (lane == 0) *exp_out = e;
}

// Slices of P (z = 0) and C (z = 1): one warp per row, lane k holds the real
// parts of column k and the imaginary parts (k + 32).  Rows inside the swept
// block and padding rows get zero slices.
__global__ void __launch_bounds__(256) slice_kernel(const __grid_constant__ OzBatch b, int k0, int rows_total,
                                                    int buf, __half* __restrict__ U, __half* __restrict__ V,
                                                    int* __restrict__ sig, int* __restrict__ tau) {
  const OzMat& M = b.m[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  const int ngpad = (M.ng + BM - 1) / BM * BM;
  if (i >= ngpad) return;
  const int kb = min(NB, M.ng - k0);
  const bool live = k0 < M.ng && i < M.ng && (i < k0 || i >= k0 + kb);
  const double2* src = blockIdx.z == 0 ? M.P : M.C;
  double re = 0.0, im = 0.0;
  if (live && lane < kb) {
    const double2 v = src[(size_t)i * NB + lane];
    re = v.x;
    im = v.y;
  }
  const size_t row = (size_t)M.row_off + i;
  __half* out = (blockIdx.z == 0 ? U : V) + (size_t)buf * S * rows_total * KR + row * KR;
  slice_row(re, im, lane, out, (size_t)rows_total * KR,
            (blockIdx.z == 0 ? sig : tau) + (size_t)buf * rows_total + row);
}

// Slices for the general (Gauss-Jordan) update A -= Cp R of the pivoted
// inverse: z = 0 slices the column panel Cp [ng][NB] (rows of the block K
// zero: they are overwritten with R afterwards), z = 1 slices R^H, read
// transposed from R [NB][ng] (every row live: the block's columns receive
// -Cp D^-1).  M.P holds Cp, M.C holds R.
__global__ void __launch_bounds__(256) slice_general_kernel(const __grid_constant__ OzBatch b, int k0,
                                                            int rows_total, int buf, __half* __restrict__ U,
                                                            __half* __restrict__ V, int* __restrict__ sig,
                                                            int* __restrict__ tau) {
  const OzMat& M = b.m[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  const int ngpad = (M.ng + BM - 1) / BM * BM;
  if (i >= ngpad) return;
  const int kb = min(NB, M.ng - k0);
  double re = 0.0, im = 0.0;
  if (blockIdx.z == 0) {
    if (i < M.ng && (i < k0 || i >= k0 + kb) && lane < kb) {
      const double2 v = M.P[(size_t)i * NB + lane];
      re = v.x;
      im = v.y;
    }
  } else if (i < M.ng && lane < kb) {
    const double2 v = M.C[(size_t)lane * M.ng + i];
    re = v.x;
    im = -v.y;
  }
  const size_t row = (size_t)M.row_off + i;
  __half* out = (blockIdx.z == 0 ? U : V) + (size_t)buf * S * rows_total * KR + row * KR;
  slice_row(re, im, lane, out, (size_t)rows_total * KR,
            (blockIdx.z == 0 ? sig : tau) + (size_t)buf * rows_total + row);
}

// Rows of the block K after the general update: A[k0 + r][j] = R[r][j].
__global__ void rows_from_r_kernel(const __grid_constant__ OzBatch b, int k0) {
  const OzMat& M = b.m[blockIdx.y];
  const int kb = min(NB, M.ng - k0);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= M.ng || e >= (long long)kb * M.ng) return;
  const int r = (int)(e / M.ng), j = (int)(e - (long long)r * M.ng);
  M.A[(size_t)(k0 + r) * M.ng + j] = M.C[(size_t)r * M.ng + j];
}

// (double)f for a finite float, built from its bits with integer operations
// (the FP64 pipe, which a conversion would occupy, is the scarce one here).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u && m == 0u) return __longlong_as_double((long long)sign);  // +-0
  if (e == 0u || e == 0xFFu) return (double)f;                          // denormal, inf, nan
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)m << 29)));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// One CTA: the 128 x 32 tile (I, J) of the lower triangle of one matrix.
// mode 0: every lower tile; 1: only the tiles touching the next block
// (rows or columns k0 + NB .. k0 + 2 NB), which the next sweep step reads
// first; 2: every other tile.  Modes 1 and 2 split one step's update so the
// next step's diagonal block, panel and slices can proceed after mode 1.
// mode 3: the general Gauss-Jordan update of the pivoted inverse, every
// tile of the matrix: A_ij = (j in K ? 0 : A_ij) - (Cp R)_ij for rows
// outside K (slices from slice_general_kernel).
template <bool realv>
__global__ void __launch_bounds__(kThreads, 1)
    update_kernel(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap vmap,
                  const __grid_constant__ OzBatch b, int k0, int rows_total, int buf, int mode,
                  const int* __restrict__ sig, const int* __restrict__ tau, int* __restrict__ status) {
  const OzMat& M = b.m[blockIdx.y];
  const int ng = M.ng;
  if (k0 >= ng) return;
  const int kb = min(NB, ng - k0);
  const int nI = (ng + BM - 1) / BM, nJ = (ng + BN - 1) / BN;
  const int k1 = k0 + NB;                      // next block
  const bool has_next = k1 < ng;
  const int In = k1 / BM, Jn = k1 / BN;
  int I = 0, J = 0;
  if (mode == 1) {
    if (!has_next) return;
    const int crow = min(4 * In + 4, nJ);
    const int t = blockIdx.x;
    if (t < crow) {
      I = In;
      J = t;
    } else {
      I = In + 1 + (t - crow);
      J = Jn;
      if (I >= nI) return;
    }
  } else if (mode == 3) {
    I = blockIdx.x / nJ;
    J = blockIdx.x - I * nJ;
    if (I >= nI) return;
  } else {
    // tile decode: row tile I holds column tiles J = 0 .. min(4I+3, nJ-1)
    int t = blockIdx.x;
    for (; I < nI; ++I) {
      const int cI = min(4 * I + 4, nJ);
      if (t < cI) break;
      t -= cI;
    }
    if (I >= nI) return;
    J = t;
    if (mode == 2 && has_next && (I == In || J == Jn)) return;
  }
  const int i0 = I * BM, j0 = J * BN;
  const int slice_base = buf * S * rows_total;  // first slice row of this step's buffer
  if (i0 >= k0 && min(i0 + BM, ng) <= k0 + kb) return;
  if (mode != 3 && j0 >= k0 && min(j0 + BN, ng) <= k0 + kb) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* us = smem;                  // S x 16 KiB
  unsigned char* vs = smem + S * kUTile;     // S x 4 KiB
  uint64_t* full = reinterpret_cast<uint64_t*>(vs + S * kVTile);
  uint64_t* done = full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(full)),
                 "r"((uint32_t)(S * (kUTile + kVTile)))
                 : "memory");
    for (int a = 0; a < S; ++a) {
      tma_load_2d(us + a * kUTile, &umap, full, 0, slice_base + a * rows_total + M.row_off + i0);
      tma_load_2d(vs + a * kVTile, &vmap, full, 0, slice_base + a * rows_total + M.row_off + j0);
    }
    // the copies must land before this CTA may exit, whatever happens next
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(full, 0) && globaltimer() - t0 < kWaitNs) {
    }
  } else if (warp == 1 && lane == 0) {
    if (!mbar_wait(full, 0)) {
      ok = false;
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ub = smem_u32(us), vb = smem_u32(vs);
      const uint32_t id = idesc(false), idn = idesc(true);
      bool first[S];
#pragma unroll
      for (int L = 0; L < S; ++L) first[L] = true;
#pragma unroll 1
      for (int a = 0; a < S; ++a) {
#pragma unroll 1
        for (int bb = 0; bb + a < S; ++bb) {
          const int L = a + bb;
          const uint32_t dre = tmem + L * 2 * BN, dim = dre + BN;
          const uint32_t ua = ub + a * kUTile, vb2 = vb + bb * kVTile;
          if constexpr (realv) {
            // real values (imaginary slices zero): Re = u[0:32] . v[0:32], no Im
#pragma unroll
            for (int k = 0; k < 2; ++k)
              mma(dre, sdesc(ua + 32 * k), sdesc(vb2 + 32 * k), id, (first[L] && k == 0) ? 0u : 1u);
            first[L] = false;
            continue;
          }
          // Re: u . v over the 64 real components (4 steps of 16)
#pragma unroll
          for (int k = 0; k < 4; ++k) mma(dre, sdesc(ua + 32 * k), sdesc(vb2 + 32 * k), id, (first[L] && k == 0) ? 0u : 1u);
          // Im: u[32:64] . v[0:32] - u[0:32] . v[32:64]
          mma(dim, sdesc(ua + 64), sdesc(vb2 + 0), id, first[L] ? 0u : 1u);
          mma(dim, sdesc(ua + 96), sdesc(vb2 + 32), id, 1u);
          mma(dim, sdesc(ua + 0), sdesc(vb2 + 64), idn, 1u);
          mma(dim, sdesc(ua + 32), sdesc(vb2 + 96), idn, 1u);
          first[L] = false;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(done))
                   : "memory");
    }
  }
  __syncwarp();
  bool have = mbar_wait(done, 0);
  have = __all_sync(0xffffffffu, have) != 0;
  if (!have && threadIdx.x == 0) atomicExch(status, (int)kDevTimeout);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  if (have && ok) {
    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows of the tile)
    // and the columns BN/4 (w / 4) .. + BN/4 - 1, in chunks of kChunk: the
    // A values of a chunk are loaded first, then all 14 level loads (7
    // levels, Re and Im) are issued before a single wait.
    const int quad = warp & 3, part = warp >> 2;
    constexpr int kCols = BN / (kThreads / 128);
    const int r = quad * 32 + lane;
    const int i = i0 + r;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const bool row_ok = i < ng && !(i >= k0 && i < k0 + kb);
    const int ei = row_ok ? sig[buf * rows_total + M.row_off + i] : 0;
#pragma unroll 1
    for (int c0 = part * kCols; c0 < (part + 1) * kCols; c0 += kChunk) {
      double2 av[kChunk];
      int ex[kChunk];
#pragma unroll
      for (int q = 0; q < kChunk; ++q) {
        const int j = j0 + c0 + q;
        const bool jblock = j >= k0 && j < k0 + kb;
        const bool live = row_ok && j < ng && (mode == 3 ? true : (j <= i && !jblock));
        av[q] = (live && !jblock) ? M.A[(size_t)i * ng + j] : make_double2(0.0, 0.0);
        ex[q] = live ? ei + tau[buf * rows_total + M.row_off + j] - 2 * BETA : 1 << 20;
      }
      uint32_t x[S][kChunk], y[S][kChunk];
#pragma unroll
      for (int L = 0; L < S; ++L) {
        tmem_ld4(tmem + lane_off + L * 2 * BN + c0, x[L]);
        if constexpr (!realv) tmem_ld4(tmem + lane_off + L * 2 * BN + BN + c0, y[L]);
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if constexpr (realv) {
#pragma unroll
        for (int L = 0; L < S; ++L)
#pragma unroll
          for (int q = 0; q < kChunk; ++q) y[L][q] = 0u;
      }
#pragma unroll
      for (int q = 0; q < kChunk; ++q) {
        float hr = __uint_as_float(x[0][q]), lr = 0.f, hm = __uint_as_float(y[0][q]), lm = 0.f;
#pragma unroll
        for (int L = 1; L < S; ++L) {
          const float w = ldexpf(1.f, -BETA * L);
          const float vr = __fmul_rn(__uint_as_float(x[L][q]), w), vi = __fmul_rn(__uint_as_float(y[L][q]), w);
          float sm, e;
          two_sum(hr, vr, sm, e);
          hr = sm;
          lr = __fadd_rn(lr, e);
          two_sum(hm, vi, sm, e);
          hm = sm;
          lm = __fadd_rn(lm, e);
        }
        if (ex[q] == (1 << 20)) continue;
        const int j = j0 + c0 + q;
        // scale by sigma_i tau_j 2^-16 = 2^ex: exact power of two, applied to
        // the FP32 pair when it stays a normal number, else in FP64; four
        // FP64 adds per element, scaling and conversion off the FP64 pipe
        const double2 v = av[q];
        double2 o;
        const int e2 = ex[q];
        if (realv && e2 > -100 && e2 < 100) {
          o.x = (v.x - f2d(ldexpf(hr, e2))) - f2d(ldexpf(lr, e2));
          o.y = v.y;   // real values: the imaginary part stays zero
        } else if (!realv && e2 > -100 && e2 < 100) {
          o.x = (v.x - f2d(ldexpf(hr, e2))) - f2d(ldexpf(lr, e2));
          o.y = (v.y - f2d(ldexpf(hm, e2))) - f2d(ldexpf(lm, e2));
        } else {
          o.x = v.x - ldexp((double)hr + (double)lr, e2);
          o.y = v.y - ldexp((double)hm + (double)lm, e2);
        }
        M.A[(size_t)i * ng + j] = o;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
  // The tile holding the next diagonal block (rows and columns k1 .. k1+31)
  // now has that block's final values: sweep it here, which leaves the next
  // step's D^-1 in Dinv and -D^-1 in A_K1K1 without a separate launch.
  // (I, J, mode) are the same for every thread of the CTA; the success
  // flags are combined by the barrier so that all threads agree.
  if (mode == 1 && I == In && J == Jn && __syncthreads_and(have && ok)) {
    __shared__ DiagSmem dsm;
    const int kb1 = min(NB, ng - k1);
    for (int e = threadIdx.x; e < NB * NB; e += kThreads) {
      const int r = e / NB, c2 = e % NB;
      if (r < kb1 && c2 <= r) dsm.L[r][c2] = M.A[(size_t)(k1 + r) * ng + k1 + c2];
    }
    diag_sweep_smem_n<kThreads>(dsm, kb1, threadIdx.x, status);
    for (int e = threadIdx.x; e < NB * NB; e += kThreads) {
      const int r = e / NB, c2 = e % NB;
      if (r >= kb1 || c2 >= kb1) continue;
      const double2 v = (r >= c2) ? dsm.L[r][c2] : make_double2(dsm.L[c2][r].x, -dsm.L[c2][r].y);
      M.Dinv[r * NB + c2] = make_double2(-v.x, -v.y);
      if (r >= c2) M.A[(size_t)(k1 + r) * ng + k1 + c2] = v;
    }
  }
}

}  // namespace oz

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode_oz = nullptr;
}  // namespace

// State of one batched sweep that uses the tensor-core update.
struct OzPlan {
  bool general = false;   // Gauss-Jordan update (mode 3) of the pivoted inverse
  bool real_values = false;  // every matrix real (real flavor): only the real-part MMAs
  int nmat = 0;
  int rows_total = 0;
  int max_tiles = 0;
  oz::OzBatch batch;
  CUtensorMap umap, vmap;
  Scratch U, V, sig, tau;
};

int oz_prepare(Ctx* c, int nmat, const int* ng, double2* const* A, const double2* const* C, const double2* const* P,
               double2* const* D, OzPlan* plan, bool general, bool real_values) {
  using namespace oz;
  if (nmat > kBatch) return fail(c, BGW_EUNSUPPORTED, "tensor-core inverse: at most %d matrices per batch", kBatch);
  if (!g_encode_oz) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail(c, BGW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    g_encode_oz = reinterpret_cast<EncodeTiledFn>(fn);
  }
  plan->nmat = nmat;
  plan->general = general;
  plan->real_values = real_values;
  plan->batch.n = nmat;
  int rows = 0, tiles = 0;
  for (int m = 0; m < nmat; ++m) {
    plan->batch.m[m].A = A[m];
    plan->batch.m[m].C = C[m];
    plan->batch.m[m].P = P[m];
    plan->batch.m[m].Dinv = D ? D[m] : nullptr;
    plan->batch.m[m].ng = ng[m];
    plan->batch.m[m].row_off = rows;
    rows += (ng[m] + BM - 1) / BM * BM;
    const int nI = (ng[m] + BM - 1) / BM, nJ = (ng[m] + BN - 1) / BN;
    int t = 0;
    if (general)
      t = nI * nJ;
    else
      for (int I = 0; I < nI; ++I) t += std::min(4 * I + 4, nJ);
    tiles = std::max(tiles, t);
  }
  plan->rows_total = rows;
  plan->max_tiles = tiles;
  plan->U.pool = plan->V.pool = plan->sig.pool = plan->tau.pool = &c->pool;
  int rc;
  // two slice buffers: a step may slice while the previous step's update
  // still reads its own
  const size_t sb = (size_t)2 * S * rows * KR * sizeof(__half);
  if ((rc = c->pool.alloc(sb, &plan->U.ptr)) != BGW_OK || (rc = c->pool.alloc(sb, &plan->V.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * rows * sizeof(int), &plan->sig.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * rows * sizeof(int), &plan->tau.ptr)) != BGW_OK)
    return fail(c, rc, "tensor-core inverse: slice buffers (%zu B each) could not be allocated", sb);
  cuuint64_t gdim[2] = {(cuuint64_t)KR, (cuuint64_t)2 * S * rows};
  cuuint64_t gstride[1] = {(cuuint64_t)KR * sizeof(__half)};
  cuuint32_t estr[2] = {1, 1};
  cuuint32_t ubox[2] = {(cuuint32_t)KR, (cuuint32_t)BM};
  cuuint32_t vbox[2] = {(cuuint32_t)KR, (cuuint32_t)BN};
  if (g_encode_oz(&plan->umap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, plan->U.ptr, gdim, gstride, ubox, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      g_encode_oz(&plan->vmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, plan->V.ptr, gdim, gstride, vbox, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return fail(c, BGW_ECUDA, "tensor-core inverse: tensor map encoding failed");
  // about 142 KiB: leaves room on each SM for the look-ahead chain's kernels
  const size_t smem = (size_t)S * (kUTile + kVTile) + 1024 + 64;
  BGW_CUDA(c, cudaFuncSetAttribute(update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BGW_CUDA(c, cudaFuncSetAttribute(update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return BGW_OK;
}

// Slices of one sweep step (P and C of every matrix) into buffer buf.
int oz_slice(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, cudaStream_t st) {
  using namespace oz;
  const int rpad = (ngmax + BM - 1) / BM * BM;
  if (plan->general)
    slice_general_kernel<<<dim3(rpad / 8, plan->nmat, 2), 256, 0, st>>>(plan->batch, k0, plan->rows_total, buf,
                                                                        plan->U.as<__half>(), plan->V.as<__half>(),
                                                                        plan->sig.as<int>(), plan->tau.as<int>());
  else
    slice_kernel<<<dim3(rpad / 8, plan->nmat, 2), 256, 0, st>>>(plan->batch, k0, plan->rows_total, buf,
                                                                plan->U.as<__half>(), plan->V.as<__half>(),
                                                                plan->sig.as<int>(), plan->tau.as<int>());
  BGW_CUDA(c, cudaGetLastError());
  return BGW_OK;
}

// The trailing update of one sweep step from slice buffer buf: mode 0 all
// tiles, 1 the tiles touching the next block, 2 the others; a general plan
// runs mode 3 (every tile) and then writes R into the block's rows.
int oz_update(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, int mode, cudaStream_t st) {
  using namespace oz;
  int grid = plan->max_tiles;
  if (mode == 1) {
    const int k1 = k0 + NB;
    if (k1 >= ngmax) return BGW_OK;
    const int nI = (ngmax + BM - 1) / BM, nJ = (ngmax + BN - 1) / BN, In = k1 / BM;
    grid = std::min(4 * In + 4, nJ) + std::max(0, nI - In - 1);
  }
  if (plan->general) mode = 3;
  const size_t smem = (size_t)S * (kUTile + kVTile) + 1024 + 64;
  if (plan->real_values)
    update_kernel<true><<<dim3(grid, plan->nmat), kThreads, smem, st>>>(plan->umap, plan->vmap, plan->batch, k0,
                                                                      plan->rows_total, buf, mode, plan->sig.as<int>(),
                                                                      plan->tau.as<int>(), c->d_status);
  else
    update_kernel<false><<<dim3(grid, plan->nmat), kThreads, smem, st>>>(plan->umap, plan->vmap, plan->batch, k0,
                                                                       plan->rows_total, buf, mode, plan->sig.as<int>(),
                                                                       plan->tau.as<int>(), c->d_status);
  if (plan->general) {
    const long long ne = (long long)NB * ngmax;
    rows_from_r_kernel<<<dim3((unsigned)((ne + 255) / 256), plan->nmat), 256, 0, st>>>(plan->batch, k0);
  }
  BGW_CUDA(c, cudaGetLastError());
  return BGW_OK;
}

OzPlan* oz_plan_new() { return new OzPlan(); }
void oz_plan_delete(OzPlan* p) { delete p; }

}  // namespace bgw
