// Trailing update of the Hermitian sweep on the tensor cores with FP64-level
// accuracy (error-free splitting of the operands, the Ozaki scheme).  The
// sweep inverts eps~ = I - v^1/2 chi v^1/2 (Eq. epsilon in its symmetric
// form; the paper inverts eps with LAPACK's ZGESV, Section "RPA Dielectric
// Matrix: epsilon").
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
#include "sweep_items.cuh"

namespace bgw {

namespace oz {

constexpr int S = 7;             // slices per value
constexpr int BETA = 8;          // bits per slice
constexpr int KR = 64;           // real inner length (32 complex)
constexpr int NB = 32;           // sweep block width
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
__host__ __device__ constexpr uint32_t idesc(bool neg_a, int n = BN) {
  return (1u << 4) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
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
// 16 lanes x 256 bits: register pair (0, 1) holds lane base + l / 4, columns
// 2 (l % 4) and 2 (l % 4) + 1; pair (2, 3) the same columns of lane base + 8 + l / 4.
__device__ __forceinline__ void tmem_ld16x256(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
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
  float4* Dff;        // [NB][NB] the same as double-FP32 pairs (re hi, re lo, im hi, im lo)
  int ng;
  int row_off;        // first slice row of this matrix (multiple of BM)
};
constexpr int kBatch = 96;
struct OzBatch {
  int n;
  OzMat m[kBatch];
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Two consecutive complex values in one 256-bit access (p 32-byte aligned).
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  asm("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(a.x), "=d"(a.y), "=d"(b.x), "=d"(b.y) : "l"(p));
}
__device__ __forceinline__ void st_pair(double2* p, double2 a, double2 b) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(a.x), "d"(a.y), "d"(b.x), "d"(b.y) : "memory");
}

// two_sum(a, x w) for a power of two w (x w exact): the products enter fused
// multiply-adds, the results are those of two_sum(a, x w) bit for bit.
__device__ __forceinline__ void two_sum_scaled(float a, float x, float w, float& s, float& e) {
  s = __fmaf_rn(x, w, a);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fmaf_rn(x, w, -bb));
}

__device__ __forceinline__ double ff2d_scaled(float h, float l, int ex) {
  float s, t;
  two_sum(h, l, s, t);
  return ff2d_pair(s, t, ex);
}


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
  // |d| <= 256: FP16 bits 0x6600 + d are 1536 + d exactly (unit spacing in
  // [1024, 2048)); one FP16 subtraction leaves d, with no conversion
  // instruction
#pragma unroll
  for (int a = 0; a < S; ++a)
    out[a * stride] = __hsub(__ushort_as_half((unsigned short)(0x6600 + d[a])), __ushort_as_half(0x6600));
}

// rint(v 2^(56 - e)) for |v| < 2^e, rounded half to even, from v's own
// fields in the integer pipe (the FP64 scaling and conversion it replaces run
// on the SM's slow FP64 pipe): v = m 2^(E - 1075) with the 53-bit mantissa m
// (no implicit bit below the normal range), so the result is m shifted by
// E - 1019 - e (at most 3 to the left).
__device__ __forceinline__ long long fixed56(double v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FFull);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
  const int sh = (E ? E : 1) - 1019 - e;
  unsigned long long X;
  if (sh >= 0) {
    X = m << sh;
  } else if (sh > -64) {
    const int k = -sh;
    const unsigned long long q = m >> k, r = m & ((1ull << k) - 1ull), half = 1ull << (k - 1);
    X = q + ((r > half || (r == half && (q & 1ull))) ? 1ull : 0ull);
  } else {
    X = 0ull;
  }
  return (b >> 63) ? -(long long)X : (long long)X;
}

// Slices and exponent of one 64-value row held by a warp (lane: value k and
// k + 32); all lanes call it.
__device__ __forceinline__ void slice_row(double re, double im, int lane, __half* base, size_t stride, int* exp_out) {
  // e = frexp exponent of the row's largest magnitude, from the biased
  // exponent fields (integer max over the warp; 0 for a zero row, and rows
  // of subnormals alone are cut to zero)
  const unsigned er = ((unsigned)__double2hiint(re) >> 20) & 0x7FFu, ei = ((unsigned)__double2hiint(im) >> 20) & 0x7FFu;
  const unsigned emax = __reduce_max_sync(0xffffffffu, er > ei ? er : ei);
  const int e = emax ? (int)emax - 1022 : 0;   // |value| 2^-e < 1
  const long long Xr = fixed56(re, e), Xi = fixed56(im, e);
  digits7(Xr, base + lane, stride);
  digits7(Xi, base + lane + 32, stride);
  if (lane == 0) *exp_out = e;
}

// The Hermitian sweep's panel and its slices in one launch (the look-ahead
// chain's critical path): for every row i outside the block K (warp per
// row, lane k = column k), C_i = A_iK (read from the stored lower triangle),
// P_i = C_i D^-1, the panel buffers and A_iK <- P_i written as the panel
// kernel of the FP64 sweep does, then P_i and C_i cut into their slices.
// Rows of K and padding rows get zero slices.  grid (ngpad/8, nmat).
// FF: P_i = C_i D^-1 in double FP32 (the five-slice update, whose target
// precision, near 2^-34, is far above the pair arithmetic's 2^-43): the
// products as exact pairs, their high words two-summed and the errors
// gathered in the low word; the FP64 pipe keeps only the conversions.
template <bool FF, bool FFD>
__global__ void __launch_bounds__(256) panel_slice_kernel(const __grid_constant__ OzBatch b, int k0, int rows_total,
                                                          int buf, __half* __restrict__ U, __half* __restrict__ V,
                                                          int* __restrict__ sig, int* __restrict__ tau) {
  __shared__ double2 Ds[NB][NB];   // FF: float4 (re hi, re lo, im hi, im lo)
  __shared__ double2 Cs[8][NB];
  const OzMat& M = b.m[blockIdx.y];
  const int ng = M.ng;
  const int ngpad = (ng + BM - 1) / BM * BM;
  if (blockIdx.x * 8 >= ngpad) return;
  const int kb = min(NB, ng - k0);
  double2* A = M.A;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // FFD: the look-ahead CTA that swept the block (every step after the
  // first) left D^-1 as double-FP32 pairs; the first step's block comes in
  // FP64 (a template flag: a runtime test would leave the conversions
  // predicated in every launch)
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    if constexpr (FF) {
      if constexpr (FFD) {
        reinterpret_cast<float4*>(&Ds[0][0])[e] = M.Dff[e];
      } else {
        const double2 d = M.Dinv[e];
        const float2 r = ff_from(d.x), m = ff_from(d.y);
        reinterpret_cast<float4*>(&Ds[0][0])[e] = make_float4(r.x, r.y, m.x, m.y);
      }
    } else {
      Ds[e / NB][e % NB] = M.Dinv[e];
    }
  }
  const int i = blockIdx.x * 8 + warp;
  const bool row_ok = k0 < ng && i < ng && (i < k0 || i >= k0 + kb);
  double2 cv = make_double2(0.0, 0.0);
  if (row_ok && lane < kb) {
    if (i >= k0 + kb) {
      cv = A[(size_t)i * ng + k0 + lane];
    } else {
      const double2 t = A[(size_t)(k0 + lane) * ng + i];
      cv = make_double2(t.x, neg_bits(t.y));
    }
  }
  // FF: the conversions in the integer pipe (the FP64 pipe bounds this kernel)
  if constexpr (FF) {
    const float2 r = ff_from_int(cv.x), m = ff_from_int(cv.y);
    reinterpret_cast<float4*>(&Cs[0][0])[warp * NB + lane] = make_float4(r.x, r.y, m.x, m.y);
  } else {
    Cs[warp][lane] = cv;
  }
  __syncthreads();
  double2 pv = make_double2(0.0, 0.0);
  if (row_ok) {
    if constexpr (FF) {
      const float4* Cf = reinterpret_cast<const float4*>(&Cs[0][0]) + warp * NB;
      const float4* Df = reinterpret_cast<const float4*>(&Ds[0][0]);
      float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;   // high word, gathered low terms
      auto acc = [](float& S, float& c, float ah, float al, float bh, float bl) {
        const float p = __fmul_rn(ah, bh);
        float e = __fmaf_rn(ah, bh, -p);
        e = __fmaf_rn(ah, bl, e);
        e = __fmaf_rn(al, bh, e);
        const float2 t = ff_two_sum(S, p);
        S = t.x;
        c = __fadd_rn(c, __fadd_rn(t.y, e));
      };
      for (int t = 0; t < kb; ++t) {
        const float4 a = Cf[t], d = Df[t * NB + lane];
        acc(sr, cr, a.x, a.y, d.x, d.y);     // + a_r d_r
        acc(sr, cr, -a.z, -a.w, d.z, d.w);   // - a_i d_i
        acc(si, ci, a.x, a.y, d.z, d.w);     // + a_r d_i
        acc(si, ci, a.z, a.w, d.x, d.y);     // + a_i d_r
      }
      pv = make_double2(ff_to_any(sr, cr), ff_to_any(si, ci));
    } else {
      for (int t = 0; t < kb; ++t) {
        const double2 a = Cs[warp][t], d = Ds[t][lane];
        pv.x = fma(a.x, d.x, fma(-a.y, d.y, pv.x));
        pv.y = fma(a.x, d.y, fma(a.y, d.x, pv.y));
      }
    }
    if (lane < kb) {
      const_cast<double2*>(M.C)[(size_t)i * NB + lane] = cv;
      const_cast<double2*>(M.P)[(size_t)i * NB + lane] = pv;
      if (i >= k0 + kb)
        A[(size_t)i * ng + k0 + lane] = pv;
      else
        A[(size_t)(k0 + lane) * ng + i] = make_double2(pv.x, neg_bits(pv.y));
    }
  }
  if (lane >= kb) pv = cv = make_double2(0.0, 0.0);
  const size_t row = (size_t)M.row_off + i;
  const size_t base = (size_t)buf * S * rows_total * KR + row * KR;
  slice_row(pv.x, pv.y, lane, U + base, (size_t)rows_total * KR, sig + (size_t)buf * rows_total + row);
  slice_row(cv.x, cv.y, lane, V + base, (size_t)rows_total * KR, tau + (size_t)buf * rows_total + row);
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


// ---------------------------------------------------------------------------
// Persistent, pipelined form of the update.  A CTA takes work items of up to
// kJPI column tiles of one row tile I: the row's U slices are loaded once per item, the V slices of
// consecutive tiles are double-buffered, and one control thread (warp 16)
// issues the TMA copies and the MMAs.  The 16 epilogue warps first read the
// tile's 14 accumulators out of tensor memory and combine the levels in
// double FP32 (registers), then release tensor memory -- the next tile's
// MMAs start -- and apply the FP64 subtraction while they run.
constexpr int kPipeEpiWarps = 16;
constexpr int kPipeThreads = (kPipeEpiWarps + 1) * 32;


// Bounded wait that also gives up when the CTA aborts.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitNs) return false;
  }
  return true;
}

// SL: slices used per value (the most significant SL of the S stored): 7
// gives an update error near 2^-48 of its scale, 5 near 2^-34.  FFC: the
// look-ahead CTA sweeps the next diagonal block in double FP32 (about 2^-46
// per operation, on the FP32 pipe) instead of FP64.
template <bool realv, int SL, bool FFC, bool NARROW>
__global__ void __launch_bounds__(kPipeThreads, 1)   // 17 warps: at most 5 per sub-partition, 96 registers
    update_pipe_kernel(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap vmap,
                       const __grid_constant__ OzBatch b, int k0, int rows_total, int buf, int mode,
                       const int* __restrict__ sig, const int* __restrict__ tau, int* __restrict__ status) {
  // column tiles per bulk work item, a compile-time constant (a runtime
  // width costs 2% in the item decode)
  constexpr int wide = NARROW ? 2 : (SL < 7 ? 3 : kJPI);
  // Levels 1 .. kTwoSumLevels are summed exactly (two-sum) into the high
  // word: with 7 slices the target is near 2^-48, so levels 1 and 2 (2^-8,
  // 2^-16 of the sum) need it; with 5 slices (near 2^-34) only level 1.
  constexpr int kTwoSumLevels = SL >= 7 ? 2 : 1;
  const OzMat& M = b.m[blockIdx.y];
  const int ng = M.ng;
  if (k0 >= ng) return;
  const int kb = min(NB, ng - k0);
  const int nI = (ng + BM - 1) / BM, nJ = (ng + BN - 1) / BN;
  const int k1 = k0 + NB;
  const bool has_next = k1 < ng;
  const int In = k1 / BM, Jn = k1 / BN;
  if (mode == 1 && !has_next) return;
  const int nitems = pipe_items(mode, wide, nI, nJ, In, has_next);
  const int slice_base = buf * S * rows_total;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* us = smem;                          // SL x 16 KiB
  unsigned char* vs = smem + SL * kUTile;            // 2 x SL x 4 KiB
  uint64_t* u_full = reinterpret_cast<uint64_t*>(vs + 2 * SL * kVTile);
  uint64_t* v_full = u_full + 1;                     // [2]
  uint64_t* v_empty = v_full + 2;                    // [2]
  uint64_t* t_full = v_empty + 2;
  uint64_t* t_empty = t_full + 1;
  uint64_t* u_empty = t_empty + 1;                   // an item's MMAs are complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(u_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ DiagSmem dsm;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool control = warp == kPipeEpiWarps;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(u_full)) : "memory");
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(v_full + q)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(v_empty + q)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(t_full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(t_empty)), "r"(kPipeEpiWarps) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(u_empty)) : "memory");
    *abort_flag = 0;
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

  int t = 0;           // tiles processed by this CTA (buffer and phase bookkeeping)
  int items_done = 0;  // items processed
  int u_loads = 0;     // U loads issued (control; phase of u_full)
  int vissued = 0;     // V loads issued (control)
  PipeCursor cursor;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++items_done) {
    int I, J0, J1;
    pipe_decode_next(cursor, mode, wide, item, nI, nJ, In, Jn, has_next, I, J0, J1);
    const int i0 = I * BM;
    // tiles of the item that are not skipped, in order
    int Js[kJPI], nt = 0;
    for (int J = J0; J < J1; ++J)
      if (!pipe_skip(mode, item, I, J, ng, k0, kb, In, Jn, has_next)) Js[nt++] = J;
    if (control) {
      if (lane == 0 && nt > 0 && !*abort_flag) {
        // U slices of the row tile, once the previous item's MMAs have read
        // the last ones (its epilogue may still run: items are independent)
        bool ok = u_loads == 0 || mbar_wait_ab(u_empty, (u_loads - 1) & 1, abort_flag);
        const int u_phase = u_loads & 1;
        if (ok) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(u_full)),
                       "r"((uint32_t)(SL * kUTile))
                       : "memory");
          for (int a = 0; a < SL; ++a)
            tma_load_2d(us + a * kUTile, &umap, u_full, 0, slice_base + a * rows_total + M.row_off + i0);
          ++u_loads;
        }
        auto issue_v = [&](int tt, int J) {
          const int bq = tt & 1;
          if (tt >= 2 && !mbar_wait_ab(&v_empty[bq], ((tt - 2) >> 1) & 1, abort_flag)) return false;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(v_full + bq)),
                       "r"((uint32_t)(SL * kVTile))
                       : "memory");
          for (int a = 0; a < SL; ++a)
            tma_load_2d(vs + (bq * SL + a) * kVTile, &vmap, v_full + bq, 0,
                        slice_base + a * rows_total + M.row_off + J * BN);
          return true;
        };
        ok = ok && issue_v(t, Js[0]);
        if (ok) vissued = t + 1;
        for (int k = 0; k < nt && ok; ++k) {
          const int tt = t + k;
          if (k + 1 < nt) {
            ok = issue_v(tt + 1, Js[k + 1]);
            vissued = tt + 2;
            if (!ok) break;
          }
          if ((k == 0 && !mbar_wait_ab(u_full, u_phase, abort_flag)) ||
              !mbar_wait_ab(&v_full[tt & 1], (tt >> 1) & 1, abort_flag) ||
              (tt > 0 && !mbar_wait_ab(t_empty, (tt - 1) & 1, abort_flag))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // Tensor memory holds the real parts of the SL level sums in columns
          // 32 L and their imaginary parts in 32 (SL + L).  The V slices lie
          // one after the other in shared memory, so for one U slice a the
          // products with V slices 0 .. SL-1-a are one MMA of N = 32 (SL - a)
          // columns into levels a .. SL-1: each U chunk is read once per
          // slice instead of once per slice pair (shared-memory traffic per
          // tile 2.5x lower at seven slices).  A descriptor's start address
          // is its low 14 bits (address / 16, no carry below 256 KiB), so
          // every operand descriptor is the base's plus a constant; level L
          // is first written by slice a = 0.
          const uint64_t du = sdesc(smem_u32(us)), dv = sdesc(smem_u32(vs + (tt & 1) * SL * kVTile));
#pragma unroll
          for (int a = 0; a < SL; ++a) {
            const uint32_t dre = tmem + 32 * a, dim = tmem + 32 * (SL + a);
            const uint64_t ua = du + (uint64_t)((a * kUTile) >> 4);
            const uint32_t ida = idesc(false, 32 * (SL - a)), idna = idesc(true, 32 * (SL - a));
            const uint32_t acc0 = a == 0 ? 0u : 1u;
            if constexpr (realv) {
              mma(dre, ua, dv, ida, acc0);
              mma(dre, ua + 2, dv + 2, ida, 1u);
            } else {
              mma(dre, ua, dv, ida, acc0);            // byte offsets 32 q along K: +2 q in the descriptor
              mma(dre, ua + 2, dv + 2, ida, 1u);
              mma(dre, ua + 4, dv + 4, ida, 1u);
              mma(dre, ua + 6, dv + 6, ida, 1u);
              mma(dim, ua + 4, dv + 0, ida, acc0);
              mma(dim, ua + 6, dv + 2, ida, 1u);
              mma(dim, ua + 0, dv + 4, idna, 1u);
              mma(dim, ua + 2, dv + 6, idna, 1u);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(v_empty + (tt & 1)))
                       : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(t_full))
                       : "memory");
        }
        if (ok)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(u_empty))
                       : "memory");
        if (!ok) {
          *abort_flag = 1;
          atomicExch(status, (int)kDevTimeout);
        }
      }
      __syncwarp();
    } else {
      // ---------------- epilogue warps: rows 32 (warp % 4) .. + 31, columns 8 (warp / 4) .. + 7.
      // The accumulators are read in the 16x256b shape: lane l holds rows
      // g, g + 8, g + 16, g + 24 (g = l / 4) and columns 2 (l % 4), + 1, so one
      // warp-wide access of A touches 8 rows of 128 contiguous bytes instead
      // of 32 rows of 16 (four times fewer cache lines per instruction).
      const int quad = warp & 3, part = warp >> 2;
      const int g = lane >> 2, cl = 2 * (lane & 3);
      const int c0 = part * 8;
      // rows r0 + 8 m (m = 0 .. 3) and their exponents sigma
      const int r0 = i0 + quad * 32 + g;
      auto row_ok = [&](int i) { return i < ng && !(i >= k0 && i < k0 + kb); };
      int ei[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) ei[m] = row_ok(r0 + 8 * m) ? sig[buf * rows_total + M.row_off + r0 + 8 * m] : 0;
      // 128 bytes of A for tile kk (row g + 8 (lane % 4), the warp's eight
      // columns) into L2, one tile ahead
      const int prow = i0 + quad * 32 + g + 8 * (lane & 3);
      const bool prow_ok = prow < ng;
      auto prefetch_a = [&](int kk) {
        if (!prow_ok || kk >= nt) return;
        const int j = Js[kk] * BN + c0;
        if (j >= ng) return;
        const double2* row = M.A + (size_t)prow * ng;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(row + j));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(row + min(j + 7, ng - 1)));
      };
      // the column exponents of tile kk (read one tile ahead)
      auto load_tau = [&](int kk, int (&tv)[2]) {
#pragma unroll
        for (int n = 0; n < 2; ++n) {
          const int j = kk < nt ? Js[kk] * BN + c0 + cl + n : ng;
          tv[n] = j < ng ? tau[buf * rows_total + M.row_off + j] : 0;
        }
      };
      // element e = 2 m + n of tile kk: row r0 + 8 m, column Js[kk] BN + c0 + cl + n,
      // scale exponent ei[m] + tv[n] - 16.  Bit e of the mask: the element is
      // updated; bit 8 + e: its old value is read (columns of the block K
      // start from zero in the Gauss-Jordan form).
      int tv[2];
      unsigned mask = 0;
      auto tile_mask = [&](int kk) {
        const int j0 = Js[kk] * BN;
        unsigned mk = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int i = r0 + 8 * (e >> 1), j = j0 + c0 + cl + (e & 1);
          const bool jblock = j >= k0 && j < k0 + kb;
          const bool live = row_ok(i) && j < ng && (mode == 3 ? true : (j <= i && !jblock));
          mk |= (live ? 1u : 0u) << e;
          mk |= (live && !jblock ? 1u : 0u) << (8 + e);
        }
        return mk;
      };
      if (nt > 0) {
        load_tau(0, tv);
        mask = tile_mask(0);
      }
      prefetch_a(0);
      for (int k = 0; k < nt; ++k) {
        const int tt = t + k;
        const int j0 = Js[k] * BN;
        prefetch_a(k + 1);
        // the next tile's column exponents, used after this tile's FP64 part
        int tnext[2];
        load_tau(k + 1, tnext);
        bool have = mbar_wait_ab(t_full, tt & 1, abort_flag);
        have = __all_sync(0xffffffffu, have) != 0;
        float hr[8], lr[8], hm[8], lm[8];
        if (have) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // Four rounds (two 16-row halves, real then imaginary parts):
          // each issues the loads of all SL levels before one wait.
          // level L enters scaled by w = 2^-8L (exact), folded into fused
          // multiply-adds: the same roundings as scaling first
          auto combine = [&](const uint32_t (&x)[SL][4], int hb, float (&h)[8], float (&l)[8]) {
#pragma unroll
            for (int L = 0; L < SL; ++L) {
              const float w = ldexpf(1.f, -BETA * L);
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const int q = 4 * hb + qq;
                const float v = __uint_as_float(x[L][qq]);
                if (L == 0) {
                  h[q] = v;
                  l[q] = 0.f;
                } else if (L <= kTwoSumLevels) {
                  // levels that can reach the running sum's last bits: exact two-sum
                  float sm, e;
                  two_sum_scaled(h[q], v, w, sm, e);
                  h[q] = sm;
                  l[q] = __fadd_rn(l[q], e);
                } else {
                  // deeper levels lie below the sum's last bit at the target
                  // precision: they go to the low word
                  l[q] = __fmaf_rn(v, w, l[q]);
                }
              }
            }
          };
#pragma unroll
          for (int hb = 0; hb < 2; ++hb) {
            const uint32_t tl = tmem + ((uint32_t)(quad * 32 + 16 * hb) << 16) + c0;
#pragma unroll
            for (int part = 0; part < (realv ? 1 : 2); ++part) {
              uint32_t x[SL][4];
#pragma unroll
              for (int L = 0; L < SL; ++L) tmem_ld16x256(tl + 32 * (part * SL + L), x[L]);
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
              if (part == 0)
                combine(x, hb, hr, lr);
              else
                combine(x, hb, hm, lm);
            }
            if constexpr (realv) {
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) hm[4 * hb + qq] = lm[4 * hb + qq] = 0.f;
            }
          }
        } else if (lane == 0) {
          *abort_flag = 1;
          atomicExch(status, (int)kDevTimeout);
        }
        // tensor memory is free for the next tile's MMAs
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(t_empty)) : "memory");
        if (!have) continue;
        // the tile's FP64 values, read while the next tile's MMAs run
        // a lane's two columns are adjacent: one 256-bit access per row
        // where both are read (written) and the pair is 32-byte aligned
        // (every row for an even N_G and an aligned matrix), else one
        // 128-bit access per element
        double2 av[8];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const size_t off = (size_t)(r0 + 8 * m) * ng + j0 + c0 + cl;
          const unsigned rd = (mask >> (8 + 2 * m)) & 3u;
          av[2 * m] = av[2 * m + 1] = make_double2(0.0, 0.0);
          if (rd == 3u && !(reinterpret_cast<uintptr_t>(M.A + off) & 31u)) {
            ld_pair(M.A + off, av[2 * m], av[2 * m + 1]);
          } else {
            if (rd & 1u) av[2 * m] = M.A[off];
            if (rd & 2u) av[2 * m + 1] = M.A[off + 1];
          }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const size_t off = (size_t)(r0 + 8 * m) * ng + j0 + c0 + cl;
          double2 o[2];
#pragma unroll
          for (int n = 0; n < 2; ++n) {
            const int e = 2 * m + n;
            const double2 v = av[e];
            const int e2 = ei[m] + tv[n] - 2 * BETA;
            // scale 2^e2 (sigma_i tau_j 2^-16) applied in the conversion; one
            // FP64 add per word
            o[n].x = v.x - ff2d_scaled(hr[e], lr[e], e2);
            o[n].y = realv ? v.y : v.y - ff2d_scaled(hm[e], lm[e], e2);
          }
          const unsigned wr = (mask >> (2 * m)) & 3u;
          if (wr == 3u && !(reinterpret_cast<uintptr_t>(M.A + off) & 31u)) {
            st_pair(M.A + off, o[0], o[1]);
          } else {
            if (wr & 1u) M.A[off] = o[0];
            if (wr & 2u) M.A[off + 1] = o[1];
          }
        }
        if (k + 1 < nt) {
          tv[0] = tnext[0];
          tv[1] = tnext[1];
          mask = tile_mask(k + 1);
        }
      }
    }
    t += nt;
    // Items of the bulk launches are independent and the barriers order the
    // buffers' reuse, so the next item's copies and MMAs overlap this item's
    // last epilogue.  The look-ahead launch's first item is followed by the
    // next diagonal block's sweep (all threads, U as scratch).
    if (mode == 1) __syncthreads();
    // The tile holding the next diagonal block (rows and columns k1 .. k1+31)
    // has its final values: sweep it here (next step's D^-1 into Dinv, -D^-1
    // into A_K1K1) without a separate launch.
    if (mode == 1 && item == 0 && !*abort_flag) {
      const int kb1 = min(NB, ng - k1);
      for (int e = threadIdx.x; e < NB * NB; e += kPipeThreads) {
        const int rr = e / NB, c2 = e % NB;
        if (rr < kb1 && c2 <= rr) dsm.L[rr][c2] = M.A[(size_t)(k1 + rr) * ng + k1 + c2];
      }
      // double-FP32 chain: the block's sweep in double FP32 (about 2^-46),
      // off the SM's slow FP64 pipe; else FP64
      if constexpr (FFC)
        diag_sweep_ff_n<kPipeThreads>(dsm, reinterpret_cast<float4*>(us), kb1, threadIdx.x, status, M.Dff);
      else
        diag_sweep_smem_n<kPipeThreads>(dsm, kb1, threadIdx.x, status);
      for (int e = threadIdx.x; e < NB * NB; e += kPipeThreads) {
        const int rr = e / NB, c2 = e % NB;
        if (rr >= kb1 || c2 >= kb1) continue;
        const double2 v = (rr >= c2) ? dsm.L[rr][c2] : make_double2(dsm.L[c2][rr].x, -dsm.L[c2][rr].y);
        M.Dinv[rr * NB + c2] = make_double2(-v.x, -v.y);
        if (rr >= c2) M.A[(size_t)(k1 + rr) * ng + k1 + c2] = v;
      }
      __syncthreads();
    }
  }
  // no copies in flight at exit (bounded waits on the last loads issued)
  if (control && lane == 0 && u_loads > 0) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(u_full, (u_loads - 1) & 1) && globaltimer() - t0 < kWaitNs) {
    }
    const uint64_t t2 = globaltimer();
    while (!*abort_flag && !mbar_try_wait(u_empty, (u_loads - 1) & 1) && globaltimer() - t2 < kWaitNs) {
    }
    for (int tt = max(0, vissued - 2); tt < vissued; ++tt) {
      const uint64_t t1 = globaltimer();
      while (!mbar_try_wait(&v_full[tt & 1], (tt >> 1) & 1) && globaltimer() - t1 < kWaitNs) {
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace oz

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode_oz = nullptr;
}  // namespace

// Dynamic shared memory of update_pipe_kernel with SL slices: U, two V
// buffers, alignment slack and the barriers.
size_t pipe_smem(int slices) { return (size_t)slices * (oz::kUTile + 2 * oz::kVTile) + 1024 + 128; }

// State of one batched sweep that uses the tensor-core update.
struct OzPlan {
  bool general = false;   // Gauss-Jordan update (mode 3) of the pivoted inverse
  int slices = 7;         // slices per value the update uses (5 or 7)
  bool ff_chain = false;  // next diagonal block and panel product in double FP32
  bool real_values = false;  // every matrix real (real flavor): only the real-part MMAs
  int bulk_narrow = -1;   // bulk items: -1 SM-count rule, 0 wide, 1 two column tiles
  int nmat = 0;
  int rows_total = 0;
  int max_tiles = 0;
  oz::OzBatch batch;
  CUtensorMap umap, vmap;
  Scratch U, V, sig, tau, dff;
};

int oz_prepare(Ctx* c, int nmat, const int* ng, double2* const* A, const double2* const* C, const double2* const* P,
               double2* const* D, OzPlan* plan, bool general, bool real_values, int slices, bool ff_chain) {
  using namespace oz;
  if (slices != 5 && slices != 7) return fail(c, BGW_EINVAL, "tensor-core inverse: 5 or 7 slices");
  plan->slices = slices;
  plan->ff_chain = ff_chain || slices < 7;   // five slices always use the double-FP32 chain
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
  plan->U.pool = plan->V.pool = plan->sig.pool = plan->tau.pool = plan->dff.pool = &c->pool;
  int rc;
  // two slice buffers: a step may slice while the previous step's update
  // still reads its own
  const size_t sb = (size_t)2 * S * rows * KR * sizeof(__half);
  if ((rc = c->pool.alloc(sb, &plan->U.ptr)) != BGW_OK || (rc = c->pool.alloc(sb, &plan->V.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * rows * sizeof(int), &plan->sig.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * rows * sizeof(int), &plan->tau.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)nmat * NB * NB * sizeof(float4), &plan->dff.ptr)) != BGW_OK)
    return fail(c, rc, "tensor-core inverse: slice buffers (%zu B each) could not be allocated", sb);
  for (int m = 0; m < nmat; ++m) plan->batch.m[m].Dff = plan->dff.as<float4>() + (size_t)m * NB * NB;
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
  // U slices, two V buffers, alignment and barriers: about 170 KiB dynamic (7 slices)
  const size_t psmem = pipe_smem(slices);
#define BGW_PIPE_ATTR(RV, SLC, FF)                                                                        \
  BGW_CUDA(c, cudaFuncSetAttribute(update_pipe_kernel<RV, SLC, FF, false>,                                       \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));                    \
  BGW_CUDA(c, cudaFuncSetAttribute(update_pipe_kernel<RV, SLC, FF, true>,                                        \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem))
  if (slices == 7 && !plan->ff_chain) {
    BGW_PIPE_ATTR(false, 7, false);
    BGW_PIPE_ATTR(true, 7, false);
  } else if (slices == 7) {
    BGW_PIPE_ATTR(false, 7, true);
    BGW_PIPE_ATTR(true, 7, true);
  } else {
    BGW_PIPE_ATTR(false, 5, true);
    BGW_PIPE_ATTR(true, 5, true);
  }
#undef BGW_PIPE_ATTR
  return BGW_OK;
}

// Slices of one pivoted Gauss-Jordan step (column panel and R^H of every matrix) into buffer buf.
int oz_slice(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, cudaStream_t st) {
  using namespace oz;
  const int rpad = (ngmax + BM - 1) / BM * BM;
  if (!plan->general) return fail(c, BGW_EINVAL, "oz_slice: the Hermitian sweep slices in oz_panel_slice");
  slice_general_kernel<<<dim3(rpad / 8, plan->nmat, 2), 256, 0, st>>>(plan->batch, k0, plan->rows_total, buf,
                                                                      plan->U.as<__half>(), plan->V.as<__half>(),
                                                                      plan->sig.as<int>(), plan->tau.as<int>());
  BGW_CUDA(c, cudaGetLastError());
  return BGW_OK;
}

// Panel and slices of one Hermitian sweep step in one launch (buffer buf).
int oz_panel_slice(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, cudaStream_t st) {
  using namespace oz;
  const int rpad = (ngmax + BM - 1) / BM * BM;
  // the look-ahead launches of the double-FP32 chain leave D^-1 as pairs
  // for every step after the first
  if (plan->ff_chain && k0 > 0)
    panel_slice_kernel<true, true><<<dim3(rpad / 8, plan->nmat), 256, 0, st>>>(
        plan->batch, k0, plan->rows_total, buf, plan->U.as<__half>(), plan->V.as<__half>(), plan->sig.as<int>(),
        plan->tau.as<int>());
  else if (plan->ff_chain)
    panel_slice_kernel<true, false><<<dim3(rpad / 8, plan->nmat), 256, 0, st>>>(
        plan->batch, k0, plan->rows_total, buf, plan->U.as<__half>(), plan->V.as<__half>(), plan->sig.as<int>(),
        plan->tau.as<int>());
  else
    panel_slice_kernel<false, false><<<dim3(rpad / 8, plan->nmat), 256, 0, st>>>(
        plan->batch, k0, plan->rows_total, buf, plan->U.as<__half>(), plan->V.as<__half>(), plan->sig.as<int>(),
        plan->tau.as<int>());
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
  // Column tiles per bulk work item: 4 with seven slices, 3 with five; 2
  // where those items would not exceed the SMs (each CTA then pipelines two
  // items instead of running one alone; measured with seven slices: N_G 2120
  // 3.10 -> 2.95 ms per inverse, while at 7180 items of 4 stay best), unless
  // the plan fixes the width (the context's timed choice or its option).
  const int nsm = sm_count(c);
  int wide = plan->slices < 7 ? 3 : kJPI;
  {
    const int nI = (ngmax + BM - 1) / BM, nJ = (ngmax + BN - 1) / BN, k1 = k0 + NB;
    grid = pipe_items(mode, wide, nI, nJ, k1 / BM, k1 < ngmax);
    const bool narrow = plan->bulk_narrow >= 0 ? plan->bulk_narrow == 1 : (long long)grid * plan->nmat <= nsm;
    if (mode != 1 && narrow) {
      wide = 2;
      grid = pipe_items(mode, wide, nI, nJ, k1 / BM, k1 < ngmax);
    }
  }
  if (grid <= 0) return BGW_OK;
  // Bulk launches with more items than SMs run persistent CTAs (items taken
  // round-robin): the next item's copies and MMAs then overlap the last
  // epilogue of the one before, and a CTA's start-up is paid once.  Only when
  // the matrices of the batch share the SMs evenly; the look-ahead launch
  // (on the critical path, few items) keeps one item per CTA.
  if (mode != 1) {
    const int per = nsm / plan->nmat;
    if (per >= 1 && (long long)grid * plan->nmat > nsm && 10 * per * plan->nmat >= 9 * nsm)
      grid = std::min(grid, per);
  }
  const size_t smem = pipe_smem(plan->slices);
  const dim3 g(grid, plan->nmat);
#define BGW_PIPE_LAUNCH(RV, SLC, FF)                                                                          \
  do {                                                                                                         \
    if (wide == 2)                                                                                             \
      update_pipe_kernel<RV, SLC, FF, true><<<g, kPipeThreads, smem, st>>>(                                     \
          plan->umap, plan->vmap, plan->batch, k0, plan->rows_total, buf, mode, plan->sig.as<int>(),           \
          plan->tau.as<int>(), c->d_status);                                                                   \
    else                                                                                                       \
      update_pipe_kernel<RV, SLC, FF, false><<<g, kPipeThreads, smem, st>>>(                                    \
          plan->umap, plan->vmap, plan->batch, k0, plan->rows_total, buf, mode, plan->sig.as<int>(),           \
          plan->tau.as<int>(), c->d_status);                                                                   \
  } while (0)
  const bool rv = plan->real_values;
  if (plan->slices == 7 && !plan->ff_chain) {
    if (rv)
      BGW_PIPE_LAUNCH(true, 7, false);
    else
      BGW_PIPE_LAUNCH(false, 7, false);
  } else if (plan->slices == 7) {
    if (rv)
      BGW_PIPE_LAUNCH(true, 7, true);
    else
      BGW_PIPE_LAUNCH(false, 7, true);
  } else {
    if (rv)
      BGW_PIPE_LAUNCH(true, 5, true);
    else
      BGW_PIPE_LAUNCH(false, 5, true);
  }
#undef BGW_PIPE_LAUNCH
  if (plan->general) {
    const long long ne = (long long)NB * ngmax;
    rows_from_r_kernel<<<dim3((unsigned)((ne + 255) / 256), plan->nmat), 256, 0, st>>>(plan->batch, k0);
  }
  BGW_CUDA(c, cudaGetLastError());
  return BGW_OK;
}

void oz_set_bulk_items(OzPlan* plan, int narrow) { plan->bulk_narrow = narrow < 0 ? -1 : (narrow ? 1 : 0); }

OzPlan* oz_plan_new() { return new OzPlan(); }
void oz_plan_delete(OzPlan* p) { delete p; }

}  // namespace bgw
