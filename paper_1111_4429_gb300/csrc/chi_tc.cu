// Mixed-precision polarizability on the 5th-generation tensor cores (paper,
// Eq. eqn_static_xi as the matrix product of Eq. eqn_static_xi_compact):
//
//   X[p][G] = M[p][G] sqrt|w_p| 2^e        (w_p < 0 always: the sign is pulled out)
//   chi[G][G'] (+)= -(4/Omega) 2^{-2e} sum_p conj(X[p][G]) X[p][G']
//   Re = sum_p xr(G) xr(G') + xi(G) xi(G')          Im = sum_p xr(G) xi(G') - xi(G) xr(G')
//
// Each real part x is split into two 16-bit numbers x = hi + lo (FP16 with a
// power-of-two scale 2^e chosen from max|X|, or BF16 without scale) and every
// real product is taken as hi*hi + hi*lo + lo*hi, so one complex lower-
// triangle tile needs 12 MMAs per K step (6 into Re, 6 into Im, three of them
// with the A operand negated).
//
// GEMM kernel (one CTA = one 128 x BN tile of the lower triangle and one
// segment of KS pairs):
//   * operands: planes P[4][NGpad][Kpad] (xr_hi, xi_hi, xr_lo, xi_lo), K-major,
//     streamed by TMA (SWIZZLE_64B boxes of 32 pairs) through a STAGES-deep
//     shared-memory ring guarded by mbarriers;
//   * one thread issues tcgen05.mma (M = 128, N = BN, K = 16) into four FP32
//     accumulators in tensor memory (Re and Im of the hi*hi products and of
//     the corrections) and tcgen05.commit frees a stage;
//   * four warps drain tensor memory (tcgen05.ld 32x32b) into an FP32
//     workspace W[seg][tile][re|im][128][BN];
//   * every wait on an mbarrier gives up after kWaitNs, records
//     BGW_ETIMEOUT in the status word and lets the CTA release its tensor
//     memory and return.
// A reduce kernel adds the segments (compensated FP32 sums in a fixed order:
// deterministic) and writes both triangles of the FP64 chi.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "runtime.h"
#include "sweep_common.cuh"

namespace bgw {

namespace tc {

constexpr int BM = 128;          // tile rows (G)
constexpr int BK = 32;           // pairs per TMA box / stage (64 B of 16-bit values)
constexpr int kEpiWarps = 8;     // epilogue warps of the GEMM kernel (two per tensor-memory lane quadrant)
constexpr int kThreads = 32 * (kEpiWarps + 2);   // + TMA producer + MMA issuer
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s: default limit of every wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
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
// Bounded wait: false when the barrier did not complete within limit_ns or
// (watch_abort) the CTA is aborting.  A limit of 0 gives up at the first
// failed try.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns = kWaitNs, bool watch_abort = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (watch_abort && *abort_flag) return false;
    if (globaltimer() - t0 >= limit_ns) return false;
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 bytes, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1u << 16;                            // leading byte offset (unused here)
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;       // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1u << 46;                            // descriptor version
  d |= (uint64_t)4u << 61;                            // SWIZZLE_64B
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B FP16 or BF16,
// K-major A and B, optional negation of A.
__host__ __device__ constexpr uint32_t idesc(int n, bool bf16, bool neg_a) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((neg_a ? 1u : 0u) << 13) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int BN, int NP = 4>
struct Layout {
  static constexpr int kATile = BM * BK * 2;    // bytes of one A-side plane tile
  static constexpr int kBTile = BN * BK * 2;    // bytes of one B-side plane tile
  static constexpr int kStage = NP * kATile + NP * kBTile;   // NP planes per operand (4 complex, 2 real)
  // Four FP32 accumulators of BN columns: Re and Im of the hi*hi products
  // (the large values) and of the hi*lo + lo*hi corrections.  Keeping the
  // corrections apart cuts the adds into the large accumulators threefold;
  // the accumulator's rounding error grows with the number of adds.
  static constexpr int kTmemCols = 4 * BN;
};

// grid: ngroups * ntiles CTAs (group-major, so the CTAs that run together
// read the same pairs), block kThreads = 10 warps, dynamic smem STAGES *
// stage + 1 KiB (alignment) + barriers.  One CTA computes one 128 x BN tile
// of the lower triangle over one group of `segs` segments of KS = kb_per_seg
// * BK pairs: each segment is accumulated in FP32 in tensor memory, then
// drained by the eight epilogue warps into FP32 running sums in registers
// (the accumulator's rounding error grows with the number of adds into it,
// so it restarts every segment), and the group's sum is written once as an
// FP32 partial W[group][tile][re|im][128][BN].
//
// Warps 0..7: epilogue (warp w reads tensor-memory lanes 32 (w % 4).. and
// columns (w / 4) BN/2..); warp 8: TMA producer and tensor-memory owner;
// warp 9: MMA issuer.  Barriers: full/empty per stage (TMA <-> MMA), done
// (MMA -> epilogue, one phase per segment), tfree (epilogue -> MMA: tensor
// memory drained, the next segment may start).
//
// Waits: the waits on the pipeline (empty, full, tfree) give up after
// wait_ns, set the abort flag and record BGW_ETIMEOUT.  An MMA issuer that
// gives up first waits (1 s bound) until its issued MMAs have finished, then
// commits `done` once more so that the epilogue (which waits on it with the
// fixed 1 s bound) wakes and stops; the producer waits (1 s bound) for its
// copies in flight.  Only then does the CTA free its tensor memory and exit.
template <int BN, int STAGES, int NP = 4>
__global__ void __launch_bounds__(kThreads, 1)
    chi_tc_kernel(const __grid_constant__ CUtensorMap tmap, int ngpad, int brow, int nkb, int kb_per_seg, int segs,
                  int ntiles, const int2* __restrict__ tiles, int bf16, unsigned long long wait_ns,
                  float* __restrict__ work, int* __restrict__ status) {
  using L = Layout<BN, NP>;
  constexpr int HC = BN / 2;        // columns per epilogue thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * L::kStage);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint64_t* tfree = done + 1;
  uint64_t* mflush = tfree + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mflush + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = blockIdx.x / ntiles, tix = blockIdx.x - grp * ntiles;
  const int2 tile = tiles[tix];
  const int row0 = tile.x * BM, col0 = tile.y * BN;
  const int kb0 = grp * segs * kb_per_seg;
  const int kb1 = min(nkb, kb0 + segs * kb_per_seg);
  const int nk = max(0, kb1 - kb0);
  const int nseg = (nk + kb_per_seg - 1) / kb_per_seg;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    mbar_init(tfree, kEpiWarps);
    mbar_init(mflush, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)L::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_re = tmem, t_im = tmem + BN, t_rec = tmem + 2 * BN, t_imc = tmem + 3 * BN;

  if (warp == kEpiWarps) {
    if (lane == 0) {
      // ---------------- TMA producer
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % STAGES;
        if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) - 1) & 1, abort_flag, wait_ns)) {
          if (!*abort_flag) atomicExch(status, (int)kDevTimeout);
          *abort_flag = 1;
          break;
        }
        unsigned char* st = smem + s * L::kStage;
        mbar_expect_tx(&full[s], L::kStage);
        const int kx = (kb0 + i) * BK;
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) {
          tma_load_2d(st + pl * L::kATile, &tmap, &full[s], kx, pl * ngpad + row0);
          tma_load_2d(st + NP * L::kATile + pl * L::kBTile, &tmap, &full[s], kx, brow + pl * ngpad + col0);
        }
        issued = i + 1;
      }
      // Never leave copies in flight: wait (bounded) until every issued stage
      // has landed before this CTA may exit.
      for (int i = max(0, issued - STAGES); i < issued; ++i) {
        uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[i % STAGES], (i / STAGES) & 1) && globaltimer() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == kEpiWarps + 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t id = idesc(BN, bf16 != 0, false);
      const uint32_t idn = idesc(BN, bf16 != 0, true);
      bool ok = true;
      for (int i = 0; i < nk && ok; ++i) {
        const int s = i % STAGES;
        const int kin = i % kb_per_seg;       // k-block inside the segment
        if (kin == 0 && i > 0) {
          // the previous segment's sums must have left tensor memory
          if (!mbar_wait(tfree, ((i / kb_per_seg) - 1) & 1, abort_flag, wait_ns)) {
            ok = false;
            break;
          }
          fence_after();
        }
        if (!mbar_wait(&full[s], (i / STAGES) & 1, abort_flag, wait_ns)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t base = smem_u32(smem + s * L::kStage);
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint32_t off = ks * 32;  // 16 values x 2 B along K
          const uint32_t first = (kin > 0 || ks > 0) ? 1u : 0u;
          if constexpr (NP == 2) {
            // real flavor: planes (x_hi, x_lo); x x' = hi hi' + (hi lo' + lo hi')
            const uint64_t ah = sdesc(base + off), al = sdesc(base + L::kATile + off);
            const uint64_t bh = sdesc(base + 2 * L::kATile + off), bl = sdesc(base + 2 * L::kATile + L::kBTile + off);
            mma(t_re, ah, bh, id, first);
            mma(t_rec, ah, bl, id, first);
            mma(t_rec, al, bh, id, 1);
            continue;
          }
          const uint64_t arh = sdesc(base + 0 * L::kATile + off), aih = sdesc(base + 1 * L::kATile + off);
          const uint64_t arl = sdesc(base + 2 * L::kATile + off), ail = sdesc(base + 3 * L::kATile + off);
          const uint32_t bb = base + 4 * L::kATile;
          const uint64_t brh = sdesc(bb + 0 * L::kBTile + off), bih = sdesc(bb + 1 * L::kBTile + off);
          const uint64_t brl = sdesc(bb + 2 * L::kBTile + off), bil = sdesc(bb + 3 * L::kBTile + off);
          // Re += xr xr' + xi xi': hi*hi into t_re, hi*lo + lo*hi into t_rec
          mma(t_re, arh, brh, id, first);
          mma(t_re, aih, bih, id, 1);
          mma(t_rec, arh, brl, id, first);
          mma(t_rec, arl, brh, id, 1);
          mma(t_rec, aih, bil, id, 1);
          mma(t_rec, ail, bih, id, 1);
          // Im += xr xi' - xi xr': hi*hi into t_im, corrections into t_imc
          mma(t_im, arh, bih, id, first);
          mma(t_im, aih, brh, idn, 1);
          mma(t_imc, arh, bil, id, first);
          mma(t_imc, arl, bih, id, 1);
          mma(t_imc, aih, brl, idn, 1);
          mma(t_imc, ail, brh, idn, 1);
        }
        mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
        if (kin == kb_per_seg - 1 || i == nk - 1) mma_commit(done);   // the segment's sums are complete
      }
      if (!ok) {
        // Let every MMA issued so far finish (the tensor memory is freed
        // after this thread reaches the final barrier), then wake the
        // epilogue: it sees the abort flag and stops.
        mma_commit(mflush);
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(mflush, 0) && globaltimer() - t0 < kWaitNs) {
        }
        if (!*abort_flag) atomicExch(status, (int)kDevTimeout);
        *abort_flag = 1;
        mma_commit(done);
      }
    }
  } else {
    // ---------------- epilogue: tensor memory -> FP32 running sums
    const int q = warp & 3, h = warp >> 2;
    const uint32_t lane_off = ((uint32_t)(q * 32) << 16) + (uint32_t)(h * HC);
    float acc_re[HC], acc_im[HC];
#pragma unroll
    for (int j = 0; j < HC; ++j) acc_re[j] = acc_im[j] = 0.f;
    bool have = nseg > 0;
    for (int sg = 0; sg < nseg; ++sg) {
      bool got = mbar_wait(done, sg & 1, abort_flag, kWaitNs, false);
      got = __all_sync(0xffffffffu, got) != 0;   // tcgen05.ld needs the whole warp
      if (!got) {
        if (lane == 0 && !*abort_flag) atomicExch(status, (int)kDevTimeout);
        *abort_flag = 1;
      }
      if (!got || __any_sync(0xffffffffu, *abort_flag != 0)) {
        have = false;
        break;
      }
      fence_after();
#pragma unroll
      for (int c0 = 0; c0 < HC; c0 += 8) {
        uint32_t a[8], b[8], ac[8], bc[8];
        tmem_ld8(t_re + lane_off + c0, a);
        tmem_ld8(t_rec + lane_off + c0, ac);
        if constexpr (NP != 2) {
          tmem_ld8(t_im + lane_off + c0, b);
          tmem_ld8(t_imc + lane_off + c0, bc);
        }
        tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          acc_re[c0 + k] += __uint_as_float(a[k]) + __uint_as_float(ac[k]);
          if constexpr (NP != 2) acc_im[c0 + k] += __uint_as_float(b[k]) + __uint_as_float(bc[k]);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tfree);   // this warp's share of tensor memory is free again
    }
    if (have) {
      const int row = q * 32 + lane;
      float* wre = work + ((size_t)grp * ntiles + tix) * 2 * BM * BN + (size_t)row * BN + h * HC;
      float* wim = wre + BM * BN;
#pragma unroll
      for (int c = 0; c < HC; c += 4) {
        *reinterpret_cast<float4*>(wre + c) = make_float4(acc_re[c], acc_re[c + 1], acc_re[c + 2], acc_re[c + 3]);
        *reinterpret_cast<float4*>(wim + c) = make_float4(acc_im[c], acc_im[c + 1], acc_im[c + 2], acc_im[c + 3]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == kEpiWarps) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)L::kTmemCols)
                 : "memory");
  }
}

// max |Re|, |Im| of M[p][g] sqrt|w_p| over all p, g (as float bits: the
// values are >= 0 so integer order is float order).
// Per-pair FP32 factors of a weight row, converted once: sqrt|w_p| (the
// Hermitian and real products) or the complex w_p (the general product).
// The conversions run on the SM's slow FP64-conversion path, so they are
// taken once per pair instead of once per element.
__global__ void pair_factors_kernel(const double* __restrict__ w, const double2* __restrict__ wc, long long K,
                                    float2* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < K; p += (long long)gridDim.x * blockDim.x)
    out[p] = wc ? make_float2((float)wc[p].x, (float)wc[p].y) : make_float2(sqrtf(fabsf((float)w[p])), 0.f);
}

// max over the pairs p and G of max(|Re|, |Im|) M[p][G] sqrt|w_p| (float
// bits into out; values >= 0).  A block takes whole rows (the row's factor
// once, coalesced loads); max(|v|) s equals max(|v| s) for s >= 0, rounding
// included.
__global__ void maxabs_kernel(const float2* __restrict__ M, const float2* __restrict__ f, long long K, int ng,
                              unsigned int* __restrict__ out) {
  float m = 0.f;
  for (long long p = blockIdx.x; p < K; p += gridDim.x) {
    const float2* row = M + p * ng;
    float mr = 0.f;
    if ((ng & 1) == 0 && !(reinterpret_cast<uintptr_t>(M) & 15u)) {   // rows 16-byte aligned: two values per load
      const float4* r4 = reinterpret_cast<const float4*>(row);
      for (int g = threadIdx.x; g < ng / 2; g += blockDim.x) {
        const float4 v = r4[g];
        mr = fmaxf(mr, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
    } else {
      for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const float2 v = row[g];
        mr = fmaxf(mr, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
    m = fmaxf(m, mr * f[p].x);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Power-of-two scale exponent e with max|X| 2^e in [2^13, 2^14) for FP16
// (largest |hi * hi| products stay far below the FP16 and FP32 limits); 0 for BF16.
__device__ __forceinline__ int scale_exp(const unsigned int* maxbits, int bf16) {
  if (bf16) return 0;
  const float m = __uint_as_float(*maxbits);
  if (!(m > 0.f) || !isfinite(m)) return 0;
  int ex;
  frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
  return 14 - ex;
}

// planes[pl][g][p] for g < ngpad, p < kpad (zero padded), from M[p0 + p][g]
// for the K pairs of one chunk:
// x = M sqrt|w_p| 2^e split into hi + lo.  32 x 32 transposing tiles.
template <typename H>
__global__ void split_kernel(const float2* __restrict__ M, const float2* __restrict__ f, long long p0, long long K,
                             int ng, int ngpad, int kpad, const unsigned int* __restrict__ maxbits, int bf16,
                             H* __restrict__ planes) {
  __shared__ float2 t[32][33];
  const long long pc0 = (long long)blockIdx.x * 32;
  const int g0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const float sc = ldexpf(1.f, scale_exp(maxbits, bf16));
  for (int r = ty; r < 32; r += 8) {
    const long long p = pc0 + r;   // pair inside the chunk
    const int g = g0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (p < K && g < ng) {
      v = M[(p0 + p) * ng + g];
      const float s = f[p0 + p].x * sc;
      v.x *= s;
      v.y *= s;
    }
    t[r][tx] = v;
  }
  __syncthreads();
  // two adjacent pairs per thread and row: paired conversions (one
  // instruction rounds two values) and 4-byte stores
  const size_t plane = (size_t)ngpad * kpad;
  const int q = ty * 32 + tx, pp = 2 * (q & 15);
#pragma unroll
  for (int gr = q >> 4; gr < 32; gr += 16) {
    const float2 a = t[pp][gr], b = t[pp + 1][gr];
    const size_t o = (size_t)(g0 + gr) * kpad + pc0 + pp;   // even: 4-byte aligned (kpad is even)
    if constexpr (std::is_same<H, __half>::value) {
      const __half2 rh = __floats2half2_rn(a.x, b.x), ih = __floats2half2_rn(a.y, b.y);
      const float2 rf = __half22float2(rh), jf = __half22float2(ih);
      const __half2 rl = __floats2half2_rn(a.x - rf.x, b.x - rf.y), il = __floats2half2_rn(a.y - jf.x, b.y - jf.y);
      *reinterpret_cast<__half2*>(planes + o) = rh;
      *reinterpret_cast<__half2*>(planes + plane + o) = ih;
      *reinterpret_cast<__half2*>(planes + 2 * plane + o) = rl;
      *reinterpret_cast<__half2*>(planes + 3 * plane + o) = il;
    } else {
      const __nv_bfloat162 rh = __floats2bfloat162_rn(a.x, b.x), ih = __floats2bfloat162_rn(a.y, b.y);
      const float2 rf = __bfloat1622float2(rh), jf = __bfloat1622float2(ih);
      const __nv_bfloat162 rl = __floats2bfloat162_rn(a.x - rf.x, b.x - rf.y),
                           il = __floats2bfloat162_rn(a.y - jf.x, b.y - jf.y);
      *reinterpret_cast<__nv_bfloat162*>(planes + o) = rh;
      *reinterpret_cast<__nv_bfloat162*>(planes + plane + o) = ih;
      *reinterpret_cast<__nv_bfloat162*>(planes + 2 * plane + o) = rl;
      *reinterpret_cast<__nv_bfloat162*>(planes + 3 * plane + o) = il;
    }
  }
}

// Real flavor: X[p][G] = M[p][G] sqrt|w_p| 2^e with real M, two planes
// (hi, lo) per operand, chi real symmetric.
__global__ void maxabs_real_kernel(const float* __restrict__ M, const float2* __restrict__ f, long long K, int ng,
                                   unsigned int* __restrict__ out) {
  float m = 0.f;
  for (long long p = blockIdx.x; p < K; p += gridDim.x) {
    const float* row = M + p * ng;
    float mr = 0.f;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) mr = fmaxf(mr, fabsf(row[g]));
    m = fmaxf(m, mr * f[p].x);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

template <typename H>
__global__ void split_real_kernel(const float* __restrict__ M, const float2* __restrict__ f, long long p0,
                                  long long K, int ng, int ngpad, int kpad, const unsigned int* __restrict__ maxbits,
                                  int bf16, H* __restrict__ planes) {
  __shared__ float t[32][33];
  const long long pc0 = (long long)blockIdx.x * 32;
  const int g0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const float sc = ldexpf(1.f, scale_exp(maxbits, bf16));
  for (int r = ty; r < 32; r += 8) {
    const long long p = pc0 + r;
    const int g = g0 + tx;
    float v = 0.f;
    if (p < K && g < ng) v = M[(p0 + p) * ng + g] * (f[p0 + p].x * sc);
    t[r][tx] = v;
  }
  __syncthreads();
  const size_t plane = (size_t)ngpad * kpad;
  for (int r = ty; r < 32; r += 8) {
    const size_t o = (size_t)(g0 + r) * kpad + pc0 + tx;
    const float v = t[tx][r];
    H h, l;
    if constexpr (std::is_same<H, __half>::value) {
      h = __float2half_rn(v);
      l = __float2half_rn(v - __half2float(h));
    } else {
      h = __float2bfloat16_rn(v);
      l = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    planes[o] = h;
    planes[plane + o] = l;
  }
}

// chi[g][g'] (+)= factor 2^{-2e} sum_seg W_re, lower triangle, mirrored (real symmetric).
template <int BN>
__global__ void reduce_real_kernel(const float* __restrict__ work, int nseg, int ntiles,
                                   const int2* __restrict__ tiles, int ng, double factor,
                                   const unsigned int* __restrict__ maxbits, int bf16, int accumulate,
                                   double* __restrict__ chi) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)BM * BN;
  if (e >= per * ntiles) return;
  const int tix = (int)(e / per);
  const int r = (int)((e - (long long)tix * per) / BN), c = (int)(e % BN);
  const int2 tl = tiles[tix];
  const int g = tl.x * BM + r, gp = tl.y * BN + c;
  if (g >= ng || gp >= ng || gp > g) return;
  float re = 0.f, rel = 0.f;
  for (int s = 0; s < nseg; ++s) {
    const float a = work[((size_t)s * ntiles + tix) * 2 * per + r * BN + c];
    const float t = __fadd_rn(re, a);
    const float z = __fsub_rn(t, re);
    rel = __fadd_rn(rel, __fadd_rn(__fsub_rn(re, __fsub_rn(t, z)), __fsub_rn(a, z)));
    re = t;
  }
  double v = ((double)re + (double)rel) * (factor * ldexp(1.0, -2 * scale_exp(maxbits, bf16)));
  double* lo = chi + (size_t)g * ng + gp;
  if (accumulate) v += *lo;
  *lo = v;
  if (g != gp) chi[(size_t)gp * ng + g] = v;
}

// Real-axis operands: X = M 2^eX and Y = (w_p M) 2^eY with complex w_p.
// out[0] = max|Re,Im| of M, out[1] = that of w M (float bits, values >= 0).
__global__ void maxabs_general_kernel(const float2* __restrict__ M, const float2* __restrict__ f, long long K,
                                      int ng, unsigned int* __restrict__ out) {
  float mx = 0.f, my = 0.f;
  for (long long p = blockIdx.x; p < K; p += gridDim.x) {
    const float2* row = M + p * ng;
    const float wr = f[p].x, wi = f[p].y;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
      const float2 v = row[g];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      my = fmaxf(my, fmaxf(fabsf(fmaf(wr, v.x, -wi * v.y)), fabsf(fmaf(wr, v.y, wi * v.x))));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(mx));
    atomicMax(out + 1, __float_as_uint(my));
  }
}

template <typename H>
__device__ __forceinline__ void split4(float2 v, H* planes, size_t plane, size_t o) {
  H rh, ih, rl, il;
  if constexpr (std::is_same<H, __half>::value) {
    rh = __float2half_rn(v.x);
    ih = __float2half_rn(v.y);
    rl = __float2half_rn(v.x - __half2float(rh));
    il = __float2half_rn(v.y - __half2float(ih));
  } else {
    rh = __float2bfloat16_rn(v.x);
    ih = __float2bfloat16_rn(v.y);
    rl = __float2bfloat16_rn(v.x - __bfloat162float(rh));
    il = __float2bfloat16_rn(v.y - __bfloat162float(ih));
  }
  planes[o] = rh;
  planes[plane + o] = ih;
  planes[2 * plane + o] = rl;
  planes[3 * plane + o] = il;
}

// planes[0..3] <- X = M 2^eX, planes[4..7] <- Y = w M 2^eY, transposed to
// [plane][g][p] like split_kernel.
template <typename H>
__global__ void split_general_kernel(const float2* __restrict__ M, const float2* __restrict__ f, long long p0,
                                     long long K, int ng, int ngpad, int kpad,
                                     const unsigned int* __restrict__ maxbits, int bf16, H* __restrict__ planes) {
  __shared__ float2 tx_[32][33];
  __shared__ float2 ty_[32][33];
  const long long pc0 = (long long)blockIdx.x * 32;
  const int g0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const float sx = ldexpf(1.f, scale_exp(maxbits, bf16)), sy = ldexpf(1.f, scale_exp(maxbits + 1, bf16));
  for (int r = ty; r < 32; r += 8) {
    const long long p = pc0 + r;
    const int g = g0 + tx;
    float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
    if (p < K && g < ng) {
      const float2 v = M[(p0 + p) * ng + g];
      const float wr = f[p0 + p].x, wi = f[p0 + p].y;
      x = make_float2(v.x * sx, v.y * sx);
      y = make_float2(fmaf(wr, v.x, -wi * v.y) * sy, fmaf(wr, v.y, wi * v.x) * sy);
    }
    tx_[r][tx] = x;
    ty_[r][tx] = y;
  }
  __syncthreads();
  const size_t plane = (size_t)ngpad * kpad;
  for (int r = ty; r < 32; r += 8) {
    const int g = g0 + r;
    const long long p = pc0 + tx;
    const size_t o = (size_t)g * kpad + p;
    split4<H>(tx_[tx][r], planes, plane, o);
    split4<H>(ty_[tx][r], planes + 4 * plane, plane, o);
  }
}

// General (non-Hermitian) reduce: every element of every tile, factor
// 2^{-(eX + eY)}, no mirroring.
template <int BN>
__global__ void reduce_general_kernel(const float* __restrict__ work, int nseg, int ntiles,
                                      const int2* __restrict__ tiles, int ng, double factor,
                                      const unsigned int* __restrict__ maxbits, int bf16, int accumulate,
                                      double2* __restrict__ chi) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)BM * BN;
  if (e >= per * ntiles) return;
  const int tix = (int)(e / per);
  const int r = (int)((e - (long long)tix * per) / BN), c = (int)(e % BN);
  const int2 tl = tiles[tix];
  const int g = tl.x * BM + r, gp = tl.y * BN + c;
  if (g >= ng || gp >= ng) return;
  float re = 0.f, rel = 0.f, im = 0.f, iml = 0.f;
  for (int s = 0; s < nseg; ++s) {
    const float* w = work + ((size_t)s * ntiles + tix) * 2 * per;
    const float a = w[r * BN + c], b = w[per + r * BN + c];
    float t = __fadd_rn(re, a);
    float z = __fsub_rn(t, re);
    rel = __fadd_rn(rel, __fadd_rn(__fsub_rn(re, __fsub_rn(t, z)), __fsub_rn(a, z)));
    re = t;
    t = __fadd_rn(im, b);
    z = __fsub_rn(t, im);
    iml = __fadd_rn(iml, __fadd_rn(__fsub_rn(im, __fsub_rn(t, z)), __fsub_rn(b, z)));
    im = t;
  }
  const double f = factor * ldexp(1.0, -(scale_exp(maxbits, bf16) + scale_exp(maxbits + 1, bf16)));
  double2 v = make_double2(((double)re + (double)rel) * f, ((double)im + (double)iml) * f);
  double2* dst = chi + (size_t)g * ng + gp;
  if (accumulate) {
    const double2 o = *dst;
    v.x += o.x;
    v.y += o.y;
  }
  *dst = v;
}

// chi[g][g'] (+)= factor 2^{-2e} sum_seg W, lower triangle of every tile,
// mirrored (conjugated) into the upper triangle.  One thread per tile element.
template <int BN>
__global__ void reduce_kernel(const float* __restrict__ work, int nseg, int ntiles, const int2* __restrict__ tiles,
                              int ng, double factor, const unsigned int* __restrict__ maxbits, int bf16,
                              int accumulate, double2* __restrict__ chi) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)BM * BN;
  if (e >= per * ntiles) return;
  const int tix = (int)(e / per);
  const int r = (int)((e - (long long)tix * per) / BN), c = (int)(e % BN);
  const int2 tl = tiles[tix];
  const int g = tl.x * BM + r, gp = tl.y * BN + c;
  if (g >= ng || gp >= ng || gp > g) return;
  // compensated FP32 sum of the segments (two-sum; the FP64 pipe is far
  // slower on this part), converted to FP64 once
  float re = 0.f, rel = 0.f, im = 0.f, iml = 0.f;
  for (int s = 0; s < nseg; ++s) {
    const float* w = work + ((size_t)s * ntiles + tix) * 2 * per;
    const float a = w[r * BN + c], b = w[per + r * BN + c];
    float t = __fadd_rn(re, a);
    float z = __fsub_rn(t, re);
    rel = __fadd_rn(rel, __fadd_rn(__fsub_rn(re, __fsub_rn(t, z)), __fsub_rn(a, z)));
    re = t;
    t = __fadd_rn(im, b);
    z = __fsub_rn(t, im);
    iml = __fadd_rn(iml, __fadd_rn(__fsub_rn(im, __fsub_rn(t, z)), __fsub_rn(b, z)));
    im = t;
  }
  // the pairs to FP64 with the scale 2^-2e applied in the integer pipe: the
  // FP64 pipe keeps one multiply by the factor and one add per word
  const int ex = -2 * scale_exp(maxbits, bf16);
  double2 v = make_double2(ff_to_scaled_any(re, rel, ex) * factor, ff_to_scaled_any(im, iml, ex) * factor);
  double2* lo = chi + (size_t)g * ng + gp;
  if (accumulate) {
    const double2 o = *lo;
    v.x += o.x;
    v.y += o.y;
  }
  if (g == gp) v.y = 0.0;
  *lo = v;
  if (g != gp) chi[(size_t)gp * ng + g] = make_double2(v.x, neg_bits(v.y));
}

// Row-major operands of a general product C = X^H-row Y-row (the Sigma
// quadratic forms): planes[pl][r][k] from src[r][k], no transpose.  max|.|
// of an operand (conj does not change it) into *out.
template <typename S2>
__global__ void maxabs_rows_kernel(const S2* __restrict__ src, long long n, unsigned int* __restrict__ out) {
  float m = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf((float)src[e].x), fabsf((float)src[e].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// planes[0..3][r][k] <- (conj ? conj(src) : src)[r][k] 2^e split hi/lo, rows
// r < R of K values each; padding rows and columns zero.  grid (kpad/32, Rpad/8), block (32, 8).
template <typename H, typename S2>
__global__ void split_rows_kernel(const S2* __restrict__ src, int R, int K, int kpad, size_t plane, int conj,
                                  const unsigned int* __restrict__ maxbits, int bf16, H* __restrict__ planes) {
  const int k = blockIdx.x * 32 + threadIdx.x;
  const int r = blockIdx.y * 8 + threadIdx.y;
  const float sc = ldexpf(1.f, scale_exp(maxbits, bf16));
  float2 v = make_float2(0.f, 0.f);
  if (r < R && k < K) {
    const S2 x = src[(size_t)r * K + k];
    v = make_float2((float)x.x * sc, (conj ? -(float)x.y : (float)x.y) * sc);
  }
  split4<H>(v, planes, plane, (size_t)r * kpad + k);
}

// C[p][g] = 2^{-(eX + eY)} sum_seg W for p < R1, g < R2 (row stride R2).
template <int BN>
__global__ void reduce_rows_kernel(const float* __restrict__ work, int nseg, int ntiles,
                                   const int2* __restrict__ tiles, int R1, int R2,
                                   const unsigned int* __restrict__ maxbits, int bf16, double2* __restrict__ C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)BM * BN;
  if (e >= per * ntiles) return;
  const int tix = (int)(e / per);
  const int r = (int)((e - (long long)tix * per) / BN), cc = (int)(e % BN);
  const int2 tl = tiles[tix];
  const int p = tl.x * BM + r, g = tl.y * BN + cc;
  if (p >= R1 || g >= R2) return;
  float re = 0.f, rel = 0.f, im = 0.f, iml = 0.f;
  for (int s = 0; s < nseg; ++s) {
    const float* w = work + ((size_t)s * ntiles + tix) * 2 * per;
    const float a = w[r * BN + cc], b = w[per + r * BN + cc];
    float t = __fadd_rn(re, a);
    float z = __fsub_rn(t, re);
    rel = __fadd_rn(rel, __fadd_rn(__fsub_rn(re, __fsub_rn(t, z)), __fsub_rn(a, z)));
    re = t;
    t = __fadd_rn(im, b);
    z = __fsub_rn(t, im);
    iml = __fadd_rn(iml, __fadd_rn(__fsub_rn(im, __fsub_rn(t, z)), __fsub_rn(b, z)));
    im = t;
  }
  const double f = ldexp(1.0, -(scale_exp(maxbits, bf16) + scale_exp(maxbits + 1, bf16)));
  C[(size_t)p * R2 + g] = make_double2(((double)re + (double)rel) * f, ((double)im + (double)iml) * f);
}

}  // namespace tc

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

int get_encode(Ctx* c) {
  if (g_encode) return BGW_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return fail(c, BGW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  return BGW_OK;
}

constexpr int kBN = 128;
constexpr int kStages = 3;
// Default pairs per K segment (FP32 accumulation span before the FP64 sum).
constexpr int kSegPairsDefault = 512;
}  // namespace

// Bound of the operand planes of one chunk of pairs (as large as the chunk's
// complex64 M); larger calls are processed chunk by chunk, each chunk's FP64
// sum added into chi.
constexpr size_t kChunkBytes = size_t(4) << 30;

namespace {

// Segments per CTA for nseg segments over ntiles tiles: the fewest groups of
// segments (one FP32 partial per tile and group) whose grid of groups x
// tiles CTAs fills the SMs in nearly whole waves (at least 90 % of the last
// wave busy), else the grid with the best wave efficiency.
int segs_per_cta(long long nseg, int ntiles, int nsm) {
  if (nseg <= 1) return 1;
  int best = (int)nseg;
  double best_eff = -1.0;
  for (long long gc = 1; gc <= nseg; ++gc) {
    const long long per = (nseg + gc - 1) / gc;
    const long long groups = (nseg + per - 1) / per;
    const double waves = (double)(groups * ntiles) / nsm;
    const double eff = waves / std::ceil(waves);
    if (eff >= 0.9) return (int)per;
    if (eff > best_eff) {
      best_eff = eff;
      best = (int)per;
    }
  }
  return best;
}

// Both products: the Hermitian one (wr: real weights, X = Y = M sqrt|w|,
// lower tiles, mirrored) and the general one (wc: complex weights, X = M,
// Y = w M, all tiles).
int chi_tc_run(Ctx* c, int prec, long long K, int ng, const void* M, const double* wr, const double2* wc, int nrow,
               double scale, int accumulate, void* chi, cudaStream_t st, bool real = false) {
  using namespace tc;
  const bool general = wc != nullptr;
  int rc;
  if ((rc = get_encode(c)) != BGW_OK) return rc;
  const int bf16 = prec == BGW_PREC_MIX_BF16;
  const int ntr = (ng + BM - 1) / BM, ntc = (ng + kBN - 1) / kBN;
  const int ngpad = std::max(ntr * BM, ntc * kBN);
  const int nplanes = general ? 8 : (real ? 2 : 4);
  const int seg_pairs_opt = c->chi_segment_pairs > 0 ? c->chi_segment_pairs : kSegPairsDefault;
  const int kb_per_seg = std::max(1, seg_pairs_opt / BK);
  const long long seg_pairs = (long long)kb_per_seg * BK;
  std::vector<int2> tl;
  for (int I = 0; I < ntr; ++I)
    for (int J = 0; J < ntc; ++J)
      if (general || J * kBN <= I * BM + BM - 1) tl.push_back(make_int2(I, J));
  const int ntiles = (int)tl.size();
  const size_t part_bytes = (size_t)ntiles * 2 * BM * kBN * sizeof(float);   // one FP32 partial per tile
  const long long segs_per_chunk =
      std::max<long long>(1, (long long)(kChunkBytes / (2ull * nplanes * ngpad * seg_pairs)));
  long long kchunk = std::min<long long>(segs_per_chunk * seg_pairs, (K + BK - 1) / BK * BK);
  if (c->chi_chunk_pairs > 0) kchunk = std::max<long long>(BK, (long long)c->chi_chunk_pairs / BK * BK);
  const long long kcpad = (kchunk + BK - 1) / BK * BK;
  const int nsm = sm_count(c);
  // groups of segments per chunk (a shorter last chunk may take more groups)
  auto groups_of = [&](long long kc) {
    const long long nseg = ((kc + BK - 1) / BK + kb_per_seg - 1) / kb_per_seg;
    const int per = segs_per_cta(nseg, ntiles, nsm);
    return std::make_pair(per, (nseg + per - 1) / per);
  };
  const long long last = K - (K - 1) / kchunk * kchunk;
  const long long ngroups_max = std::max(groups_of(std::min(kchunk, K)).second, groups_of(last).second);
  const void* d_tiles;
  if ((rc = upload_cached(c, tl.data(), tl.size() * sizeof(int2), st, &d_tiles)) != BGW_OK) return rc;
  Scratch planes, work, mx, fac;
  planes.pool = work.pool = mx.pool = fac.pool = &c->pool;
  const size_t plane_bytes = (size_t)nplanes * ngpad * kcpad * 2;
  const size_t work_bytes = (size_t)ngroups_max * part_bytes;
  if ((rc = c->pool.alloc(plane_bytes, &planes.ptr)) != BGW_OK || (rc = c->pool.alloc(work_bytes, &work.ptr)) != BGW_OK ||
      (rc = c->pool.alloc(2 * sizeof(unsigned int), &mx.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)K * sizeof(float2), &fac.ptr)) != BGW_OK)
    return fail(c, rc, "bgw_chi_sum (mixed): scratch allocation failed (planes %zu B, workspace %zu B)", plane_bytes,
                work_bytes);
  CUtensorMap tmap;
  cuuint64_t gdim[2] = {(cuuint64_t)kcpad, (cuuint64_t)nplanes * ngpad};
  cuuint64_t gstride[1] = {(cuuint64_t)kcpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  // One map serves both operands: the B box has kBN rows; with kBN == BM the
  // same box height applies.
  static_assert(kBN == BM, "one tensor map per operand height");
  CUresult cr = g_encode(&tmap, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                         planes.ptr, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(c, BGW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  const size_t smem = (size_t)kStages * (real ? Layout<kBN, 2>::kStage : Layout<kBN>::kStage) + 1024 + 256;
  if (real)
    BGW_CUDA(c, cudaFuncSetAttribute(chi_tc_kernel<kBN, kStages, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  else
    BGW_CUDA(c, cudaFuncSetAttribute(chi_tc_kernel<kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const int brow = general ? 4 * ngpad : 0;
  for (int f = 0; f < nrow; ++f) {
    const double* wf = general ? nullptr : wr + (size_t)f * K;
    const double2* wcf = general ? wc + (size_t)f * K : nullptr;
    {
      TimedScope ts(c, kTChiSplit, st);
      BGW_CUDA(c, cudaMemsetAsync(mx.ptr, 0, 2 * sizeof(unsigned int), st));
      pair_factors_kernel<<<(unsigned)std::min<long long>((K + 255) / 256, (long long)nsm * 4), 256, 0, st>>>(
          wf, wcf, K, fac.as<float2>());
      const unsigned mb = (unsigned)std::min<long long>(K, (long long)nsm * 8);
      if (general)
        maxabs_general_kernel<<<mb, 256, 0, st>>>(static_cast<const float2*>(M), fac.as<float2>(), K, ng,
                                                  mx.as<unsigned int>());
      else if (real)
        maxabs_real_kernel<<<mb, 256, 0, st>>>(static_cast<const float*>(M), fac.as<float2>(), K, ng,
                                               mx.as<unsigned int>());
      else
        maxabs_kernel<<<mb, 256, 0, st>>>(static_cast<const float2*>(M), fac.as<float2>(), K, ng,
                                          mx.as<unsigned int>());
      c->launches += 2;
    }
    for (long long p0 = 0; p0 < K; p0 += kchunk) {
      const long long kc = std::min(kchunk, K - p0);
      const long long kpad = (kc + BK - 1) / BK * BK;
      const int nkb = (int)(kpad / BK);
      const auto grp = groups_of(kc);
      const int per = grp.first, ngroups = (int)grp.second;
      {
        TimedScope ts(c, kTChiSplit, st);
        dim3 sg((unsigned)(kpad / 32), (unsigned)(ngpad / 32));
        // rows of the planes are kcpad long (the tensor map's stride); a
        // shorter last chunk fills the first kpad of each row, and the GEMM
        // reads no further than nkb = kpad / BK k-blocks
        const unsigned int* mb = mx.as<unsigned int>();
        if (real && bf16)
          split_real_kernel<__nv_bfloat16><<<sg, dim3(32, 8), 0, st>>>(static_cast<const float*>(M), fac.as<float2>(), p0, kc, ng,
                                                                       ngpad, (int)kcpad, mb, 1,
                                                                       planes.as<__nv_bfloat16>());
        else if (real)
          split_real_kernel<__half><<<sg, dim3(32, 8), 0, st>>>(static_cast<const float*>(M), fac.as<float2>(), p0, kc, ng, ngpad,
                                                                (int)kcpad, mb, 0, planes.as<__half>());
        else if (general && bf16)
          split_general_kernel<__nv_bfloat16><<<sg, dim3(32, 8), 0, st>>>(
              static_cast<const float2*>(M), fac.as<float2>(), p0, kc, ng, ngpad, (int)kcpad, mb, 1, planes.as<__nv_bfloat16>());
        else if (general)
          split_general_kernel<__half><<<sg, dim3(32, 8), 0, st>>>(static_cast<const float2*>(M), fac.as<float2>(), p0, kc, ng,
                                                                   ngpad, (int)kcpad, mb, 0, planes.as<__half>());
        else if (bf16)
          split_kernel<__nv_bfloat16><<<sg, dim3(32, 8), 0, st>>>(static_cast<const float2*>(M), fac.as<float2>(), p0, kc, ng,
                                                                  ngpad, (int)kcpad, mb, 1,
                                                                  planes.as<__nv_bfloat16>());
        else
          split_kernel<__half><<<sg, dim3(32, 8), 0, st>>>(static_cast<const float2*>(M), fac.as<float2>(), p0, kc, ng, ngpad,
                                                           (int)kcpad, mb, 0, planes.as<__half>());
      }
      {
        TimedScope ts(c, kTChiTc, st);
        if (real)
          chi_tc_kernel<kBN, kStages, 2><<<(unsigned)((long long)ngroups * ntiles), kThreads, smem, st>>>(
              tmap, ngpad, brow, nkb, kb_per_seg, per, ntiles, static_cast<const int2*>(d_tiles), bf16, c->wait_ns,
              work.as<float>(), c->d_status);
        else
          chi_tc_kernel<kBN, kStages><<<(unsigned)((long long)ngroups * ntiles), kThreads, smem, st>>>(
              tmap, ngpad, brow, nkb, kb_per_seg, per, ntiles, static_cast<const int2*>(d_tiles), bf16, c->wait_ns,
              work.as<float>(), c->d_status);
      }
      {
        TimedScope ts(c, kTChiReduce, st);
        const long long ne = (long long)ntiles * BM * kBN;
        double2* cf = static_cast<double2*>(chi) + (size_t)f * ng * ng;
        const int acc = (accumulate || p0 > 0) ? 1 : 0;
        if (real)
          reduce_real_kernel<kBN><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
              work.as<float>(), ngroups, ntiles, static_cast<const int2*>(d_tiles), ng, -scale, mx.as<unsigned int>(),
              bf16, acc, static_cast<double*>(chi) + (size_t)f * ng * ng);
        else if (general)
          reduce_general_kernel<kBN><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
              work.as<float>(), ngroups, ntiles, static_cast<const int2*>(d_tiles), ng, scale, mx.as<unsigned int>(),
              bf16, acc, cf);
        else
          reduce_kernel<kBN><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
              work.as<float>(), ngroups, ntiles, static_cast<const int2*>(d_tiles), ng, -scale, mx.as<unsigned int>(),
              bf16, acc, cf);
      }
      BGW_CUDA(c, cudaGetLastError());
      c->launches += 3;
    }
  }
  return BGW_OK;
}

}  // namespace

int chi_mixed_run(Ctx* c, int prec, long long K, int ng, const void* M, const double* w, int nrow, double scale,
                  int accumulate, void* chi, cudaStream_t st, bool real) {
  return chi_tc_run(c, prec, K, ng, M, w, nullptr, nrow, scale, accumulate, chi, st, real);
}

// C[p][g] = sum_k X[p][k] Y[g][k] on the tensor cores for a complex64 X
// [R1][K] and a complex128 Y [R2][K] (both row-major), FP16 (or BF16) hi/lo
// splits with their own power-of-two scales, FP32 segment sums, FP64 result
// [R1][R2].  The general chi kernel computes sum_k conj(A[p][k]) B[g][k]:
// A = conj(X), B = Y.
int tc_rows_gemm(Ctx* c, int prec, int R1, int R2, int K, const void* X, const void* Y, void* C, cudaStream_t st) {
  using namespace tc;
  int rc;
  if ((rc = get_encode(c)) != BGW_OK) return rc;
  const int bf16 = prec == BGW_PREC_MIX_BF16;
  const int rpad = (std::max(R1, R2) + BM - 1) / BM * BM;
  const int kpad = (K + BK - 1) / BK * BK;
  const int ntr = (R1 + BM - 1) / BM, ntc = (R2 + kBN - 1) / kBN;
  std::vector<int2> tl;
  for (int I = 0; I < ntr; ++I)
    for (int J = 0; J < ntc; ++J) tl.push_back(make_int2(I, J));
  const int ntiles = (int)tl.size();
  const int kb_per_seg = std::max(1, kSegPairsDefault / BK);
  const int nkb = kpad / BK;
  const int nseg = (nkb + kb_per_seg - 1) / kb_per_seg;
  const int per = segs_per_cta(nseg, ntiles, sm_count(c));
  const int ngroups = (nseg + per - 1) / per;
  const size_t plane = (size_t)rpad * kpad;
  const void* d_tiles;
  if ((rc = upload_cached(c, tl.data(), tl.size() * sizeof(int2), st, &d_tiles)) != BGW_OK) return rc;
  Scratch planes, work, mx;
  planes.pool = work.pool = mx.pool = &c->pool;
  const size_t work_bytes = (size_t)ngroups * ntiles * 2 * BM * kBN * sizeof(float);
  if ((rc = c->pool.alloc(8 * plane * 2, &planes.ptr)) != BGW_OK || (rc = c->pool.alloc(work_bytes, &work.ptr)) != BGW_OK ||
      (rc = c->pool.alloc(2 * sizeof(unsigned int), &mx.ptr)) != BGW_OK)
    return fail(c, rc, "tensor-core product: scratch allocation failed");
  CUtensorMap tmap;
  cuuint64_t gdim[2] = {(cuuint64_t)kpad, (cuuint64_t)8 * rpad};
  cuuint64_t gstride[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = g_encode(&tmap, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                         planes.ptr, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(c, BGW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  const size_t smem = (size_t)kStages * Layout<kBN>::kStage + 1024 + 256;
  BGW_CUDA(c, cudaFuncSetAttribute(chi_tc_kernel<kBN, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  unsigned int* mb = mx.as<unsigned int>();
  BGW_CUDA(c, cudaMemsetAsync(mb, 0, 2 * sizeof(unsigned int), st));
  {
    TimedScope ts(c, kTChiSplit, st);
    const long long n1 = (long long)R1 * K, n2 = (long long)R2 * K;
    maxabs_rows_kernel<float2><<<(unsigned)std::min<long long>((n1 + 255) / 256, 152LL * 8), 256, 0, st>>>(
        static_cast<const float2*>(X), n1, mb);
    maxabs_rows_kernel<double2><<<(unsigned)std::min<long long>((n2 + 255) / 256, 152LL * 8), 256, 0, st>>>(
        static_cast<const double2*>(Y), n2, mb + 1);
    // X rows fill the planes' rpad rows; Y's tiles read no row past ntc * BN
    dim3 g((unsigned)(kpad / 32), (unsigned)(rpad / 8)), g2((unsigned)(kpad / 32), (unsigned)(ntc * kBN / 8)), b(32, 8);
    if (bf16) {
      split_rows_kernel<__nv_bfloat16, float2><<<g, b, 0, st>>>(static_cast<const float2*>(X), R1, K, kpad, plane, 1,
                                                                 mb, 1, planes.as<__nv_bfloat16>());
      split_rows_kernel<__nv_bfloat16, double2><<<g2, b, 0, st>>>(static_cast<const double2*>(Y), R2, K, kpad, plane,
                                                                   0, mb + 1, 1, planes.as<__nv_bfloat16>() + 4 * plane);
    } else {
      split_rows_kernel<__half, float2><<<g, b, 0, st>>>(static_cast<const float2*>(X), R1, K, kpad, plane, 1, mb, 0,
                                                          planes.as<__half>());
      split_rows_kernel<__half, double2><<<g2, b, 0, st>>>(static_cast<const double2*>(Y), R2, K, kpad, plane, 0,
                                                            mb + 1, 0, planes.as<__half>() + 4 * plane);
    }
  }
  {
    TimedScope ts(c, kTChiTc, st);
    chi_tc_kernel<kBN, kStages><<<(unsigned)((long long)ngroups * ntiles), kThreads, smem, st>>>(
        tmap, rpad, 4 * rpad, nkb, kb_per_seg, per, ntiles, static_cast<const int2*>(d_tiles), bf16, c->wait_ns,
        work.as<float>(), c->d_status);
  }
  {
    TimedScope ts(c, kTChiReduce, st);
    const long long ne = (long long)ntiles * BM * kBN;
    reduce_rows_kernel<kBN><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
        work.as<float>(), ngroups, ntiles, static_cast<const int2*>(d_tiles), R1, R2, mb, bf16,
        static_cast<double2*>(C));
  }
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 7;
  return BGW_OK;
}

int chi_real_mixed_run(Ctx* c, int prec, long long K, int ng, const void* M, const double2* w, int nrow,
                       double scale, int accumulate, void* chi, cudaStream_t st) {
  return chi_tc_run(c, prec, K, ng, M, nullptr, w, nrow, scale, accumulate, chi, st);
}

}  // namespace bgw
