// General (non-Hermitian) dielectric matrix and its inverse, for the real-axis
// response of Eq. retarded_advanced_epsilon: with complex pair weights chi is
// no longer Hermitian, eps~ = I - V^1/2 chi V^1/2 is a general complex matrix,
// and its inverse needs pivoting (the paper inverts with ZGESV, an LU with
// partial pivoting).
//
// Blocked Gauss-Jordan elimination with row interchanges, 32 columns a step:
//   1. pivot rows for the block's columns among the rows not yet used, chosen
//      by tournament pivoting: CTAs run a partial-pivoting LU on 256-row
//      slices of the column panel and keep 32 candidates each; merge rounds
//      run the same LU on up to 8 candidate sets at a time until 32 rows
//      remain (the selection of a partial-pivoting LU of the panel when one
//      slice holds every row, a tournament among slices otherwise).  The
//      selection LUs run in FP32: they only choose rows;
//   2. the chosen rows are swapped into the block's rows (whole rows of the
//      working matrix: row operations on the augmented system), the
//      interchanges recorded LAPACK-style (ipiv[j] >= j);
//   3. one Gauss-Jordan block step without further pivoting (the block's
//      diagonal block is the chosen rows, eliminated in their selection order).
// After the last step the working matrix holds the inverse with permuted
// columns; undoing the interchanges on the columns in reverse order gives
// eps~^-1.
#include <algorithm>
#include <memory>
#include <vector>

#include "runtime.h"

namespace bgw {

namespace {

constexpr int kPB = 32;      // block width of the Gauss-Jordan step
constexpr int kTRows = 256;  // rows per selection CTA (one per thread)
constexpr int kSwapCols = 64;
constexpr int kGB = 16;      // matrices of one size stepped together (grid.y / grid.z = matrix)

struct GenPtrs {
  double2* A[kGB];
};

__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }

// Partial-pivoting LU of nr (<= 256) rows x kb columns held in P; thread t
// owns row t.  Picks, column by column, the active row of largest |Re|+|Im|
// (ties: smallest global row), eliminates that column from the other active
// rows.  Writes the global rows in selection order to sel and returns their
// number (min(nr, kb)).  The selection runs in FP32: it only orders the rows
// (the elimination itself is the FP64 Gauss-Jordan step that follows), and
// FP32 runs at 64 times the FP64 rate of one SM.
__device__ __forceinline__ float cabs1f(float2 z) { return fabsf(z.x) + fabsf(z.y); }

__device__ int select_rows(float2 (*P)[kPB + 1], const int* gid, int nr, int kb, int* sel) {
  __shared__ float wv[kTRows / 32];
  __shared__ int wg[kTRows / 32], wl[kTRows / 32];
  __shared__ int win;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  bool active = t < nr;
  const int cnt = min(nr, kb);
  for (int j = 0; j < cnt; ++j) {
    float v = active ? cabs1f(P[t][j]) : -1.f;
    int g = active ? gid[t] : 0x7fffffff, l = t;
    for (int o = 16; o > 0; o >>= 1) {
      const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int g2 = __shfl_xor_sync(0xffffffffu, g, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
      if (v2 > v || (v2 == v && g2 < g)) {
        v = v2;
        g = g2;
        l = l2;
      }
    }
    if (lane == 0) {
      wv[warp] = v;
      wg[warp] = g;
      wl[warp] = l;
    }
    __syncthreads();
    if (t == 0) {
      float bv = wv[0];
      int bg = wg[0], bl = wl[0];
      for (int w = 1; w < kTRows / 32; ++w)
        if (wv[w] > bv || (wv[w] == bv && wg[w] < bg)) {
          bv = wv[w];
          bg = wg[w];
          bl = wl[w];
        }
      win = bl;
      sel[j] = bg;
    }
    __syncthreads();
    const int w = win;
    if (t == w) active = false;
    const float2 pv = P[w][j];
    const float m2 = pv.x * pv.x + pv.y * pv.y;
    if (active && m2 > 0.f) {
      const float2 a = P[t][j];
      const float2 l = make_float2((a.x * pv.x + a.y * pv.y) / m2, (a.y * pv.x - a.x * pv.y) / m2);
      for (int c = j + 1; c < kb; ++c) {
        const float2 u = P[w][c];
        P[t][c] = make_float2(P[t][c].x - (l.x * u.x - l.y * u.y), P[t][c].y - (l.x * u.y + l.y * u.x));
      }
    }
    __syncthreads();
  }
  return cnt;
}

// FP32 copy of a panel entry.  The values are eps~ entries (finite, far
// inside the FP32 range); a zero pivot column stays zero.
__device__ __forceinline__ float2 to_f2(double2 z) { return make_float2((float)z.x, (float)z.y); }

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// FP64 LU (without further pivoting) of the block D = A[sel][K], the chosen
// rows in selection order: lu[r][c] holds L below the diagonal (unit
// diagonal implied) and U on and above it, lu[NB*NB + s] = 1/U_ss.  Run by
// the CTA that makes the final choice, before the rows are swapped; the
// buffer P (no longer needed) holds D.
__device__ void factor_block(const double2* __restrict__ A, int ng, int k0, int kb, const int* sel, void* scratch,
                             double2* __restrict__ lu, int* __restrict__ status) {
  double2 (*D)[kPB + 1] = reinterpret_cast<double2 (*)[kPB + 1]>(scratch);
  __shared__ double2 rinv[kPB];
  const int tid = threadIdx.x;
  for (int e = tid; e < kPB * kPB; e += blockDim.x) {
    const int r = e / kPB, c = e % kPB;
    D[r][c] = (r < kb && c < kb) ? A[(size_t)sel[r] * ng + k0 + c] : make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  for (int s = 0; s < kb; ++s) {
    __syncthreads();
    if (tid == 0) {
      const double2 p = D[s][s];
      const double m2 = p.x * p.x + p.y * p.y;
      if (!(m2 > 0.0) || !isfinite(m2)) {
        atomicExch(status, (int)kDevZeroPivot);
        rinv[s] = make_double2(0.0, 0.0);
      } else {
        const double q = 1.0 / m2;
        rinv[s] = make_double2(p.x * q, -p.y * q);
      }
    }
    __syncthreads();
    for (int r = s + 1 + tid; r < kb; r += blockDim.x) D[r][s] = cmul2(D[r][s], rinv[s]);
    __syncthreads();
    const int w = kb - 1 - s;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int r = s + 1 + e / w, c = s + 1 + e % w;
      const double2 t = cmul2(D[r][s], D[s][c]);
      D[r][c] = make_double2(D[r][c].x - t.x, D[r][c].y - t.y);
    }
  }
  __syncthreads();
  for (int e = tid; e < kPB * kPB; e += blockDim.x) lu[e] = D[e / kPB][e % kPB];
  for (int e = tid; e < kPB; e += blockDim.x) lu[kPB * kPB + e] = e < kb ? rinv[e] : make_double2(1.0, 0.0);
}

// Row panel R = D^-1 A_K,: from the factors (after the swap, row k0 + r is
// the r-th chosen row): each CTA solves L U x = b for 16 columns of A_K,:,
// the block's own columns replaced by identity columns (R = D^-1 there).
// blockIdx.y >= 1 copies the column panel Cp = A_:,K (ld NB).  256 threads:
// 16 columns x 16 row groups (rows g, g + 16).
__global__ void __launch_bounds__(256) solve_panels_kernel(const __grid_constant__ GenPtrs P, int ng, int k0,
                                                           int kb, const double2* __restrict__ lu_all,
                                                           double2* __restrict__ R_all, double2* __restrict__ C_all) {
  const int tid = threadIdx.x;
  const int m = blockIdx.z;
  const double2* __restrict__ A = P.A[m];
  const double2* __restrict__ lu = lu_all + (size_t)m * kPB * (kPB + 1);
  double2* __restrict__ R = R_all + (size_t)m * kPB * ng;
  double2* __restrict__ C = C_all + (size_t)m * kPB * ng;
  if (blockIdx.y > 0) {
    const int i = (blockIdx.y - 1) * 256 + tid;
    if (blockIdx.x != 0 || i >= ng) return;
    for (int s = 0; s < kb; ++s) C[(size_t)i * kPB + s] = A[(size_t)i * ng + k0 + s];
    return;
  }
  __shared__ double2 D[kPB][kPB + 1];
  __shared__ double2 B[kPB][17];
  __shared__ double2 rinv[kPB];
  const int j0 = blockIdx.x * 16;
  for (int e = tid; e < kPB * kPB; e += 256) D[e / kPB][e % kPB] = lu[e];
  if (tid < kPB) rinv[tid] = lu[kPB * kPB + tid];
  for (int e = tid; e < kPB * 16; e += 256) {
    const int r = e / 16, jj = e % 16, j = j0 + jj;
    double2 v = make_double2(0.0, 0.0);
    if (r < kb && j < ng)
      v = (j >= k0 && j < k0 + kb) ? make_double2(j - k0 == r ? 1.0 : 0.0, 0.0) : A[(size_t)(k0 + r) * ng + j];
    B[r][jj] = v;
  }
  const int col = tid & 15, g = tid >> 4;
  for (int s = 0; s < kb; ++s) {   // unit lower factor
    __syncthreads();
    const double2 y = B[s][col];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = g + 16 * h;
      if (r > s && r < kb) {
        const double2 t = cmul2(D[r][s], y);
        B[r][col] = make_double2(B[r][col].x - t.x, B[r][col].y - t.y);
      }
    }
  }
  for (int s = kb - 1; s >= 0; --s) {   // upper factor
    __syncthreads();
    if (g == (s & 15)) B[s][col] = cmul2(B[s][col], rinv[s]);
    __syncthreads();
    const double2 x = B[s][col];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = g + 16 * h;
      if (r < s) {
        const double2 t = cmul2(D[r][s], x);
        B[r][col] = make_double2(B[r][col].x - t.x, B[r][col].y - t.y);
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < kPB * 16; e += 256) {
    const int r = e / 16, jj = e % 16, j = j0 + jj;
    if (r < kb && j < ng) R[(size_t)r * ng + j] = B[r][jj];
  }
}

// Leaf round: CTA b takes rows k0 + 256 b ... of the panel.
__global__ void __launch_bounds__(kTRows) pivot_leaf_kernel(const __grid_constant__ GenPtrs Pm, int ng, int k0,
                                                            int kb, int* __restrict__ out_all, int cstride,
                                                            double2* __restrict__ lu_all, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.y;
  const double2* __restrict__ A = Pm.A[m];
  int* __restrict__ out = out_all + (size_t)m * cstride;
  int* __restrict__ cnt = out + (cstride / (kPB + 1)) * kPB;
  double2* __restrict__ lu = lu_all + (size_t)m * kPB * (kPB + 1);
  float2 (*P)[kPB + 1] = reinterpret_cast<float2 (*)[kPB + 1]>(smem_raw);
  __shared__ int gid[kTRows];
  __shared__ int sel[kPB];
  const int r0 = k0 + blockIdx.x * kTRows;
  const int nr = min(kTRows, ng - r0);
  const int t = threadIdx.x;
  gid[t] = r0 + t;
  if (t < nr)
    for (int c = 0; c < kb; ++c) P[t][c] = to_f2(A[(size_t)(r0 + t) * ng + k0 + c]);
  __syncthreads();
  const int n = select_rows(P, gid, nr, kb, sel);
  __syncthreads();
  if (t < n) out[blockIdx.x * kPB + t] = sel[t];
  if (t == 0) cnt[blockIdx.x] = n;
  if (gridDim.x == 1) factor_block(A, ng, k0, kb, sel, smem_raw, lu, status);   // the final choice
}

// Merge round: CTA m takes candidate sets 8m .. 8m+7 (of ngroups).
__global__ void __launch_bounds__(kTRows) pivot_merge_kernel(const __grid_constant__ GenPtrs Pm, int ng, int k0,
                                                             int kb, const int* __restrict__ in_all,
                                                             int ngroups, int* __restrict__ out_all, int cstride,
                                                             double2* __restrict__ lu_all, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.y;
  const double2* __restrict__ A = Pm.A[m];
  const int* __restrict__ in = in_all + (size_t)m * cstride;
  const int* __restrict__ cin = in + (cstride / (kPB + 1)) * kPB;
  int* __restrict__ out = out_all + (size_t)m * cstride;
  int* __restrict__ cout = out + (cstride / (kPB + 1)) * kPB;
  double2* __restrict__ lu = lu_all + (size_t)m * kPB * (kPB + 1);
  float2 (*P)[kPB + 1] = reinterpret_cast<float2 (*)[kPB + 1]>(smem_raw);
  __shared__ int gid[kTRows];
  __shared__ int sel[kPB];
  __shared__ int nr_s;
  const int t = threadIdx.x;
  if (t == 0) {
    int n = 0;
    for (int g = blockIdx.x * 8; g < min(ngroups, blockIdx.x * 8 + 8); ++g)
      for (int i = 0; i < cin[g]; ++i) gid[n++] = in[g * kPB + i];
    nr_s = n;
  }
  __syncthreads();
  const int nr = nr_s;
  if (t < nr)
    for (int c = 0; c < kb; ++c) P[t][c] = to_f2(A[(size_t)gid[t] * ng + k0 + c]);
  __syncthreads();
  const int n = select_rows(P, gid, nr, kb, sel);
  __syncthreads();
  if (t < n) out[blockIdx.x * kPB + t] = sel[t];
  if (t == 0) cout[blockIdx.x] = n;
  if (gridDim.x == 1) factor_block(A, ng, k0, kb, sel, smem_raw, lu, status);   // the final choice
}

// Brings row sel[j] to row k0 + j for j < kb by successive interchanges
// (recorded in ipiv[k0 + j]).  Every CTA replays the interchanges on the set
// of affected rows (at most 64) and moves its 64 columns of them.
__global__ void __launch_bounds__(256) pivot_swap_kernel(const __grid_constant__ GenPtrs Pm, int ng, int k0, int kb,
                                                         const int* __restrict__ sel_all, int cstride,
                                                         int* __restrict__ ipiv_all) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.y;
  double2* __restrict__ A = Pm.A[m];
  const int* __restrict__ sel = sel_all + (size_t)m * cstride;
  int* __restrict__ ipiv = ipiv_all + (size_t)m * ng;
  double2 (*buf)[kSwapCols] = reinterpret_cast<double2 (*)[kSwapCols]>(smem_raw);
  __shared__ int pos[2 * kPB];   // positions of the affected rows
  __shared__ int from[2 * kPB];  // original row that ends at pos[i]
  __shared__ int ns;
  const int t = threadIdx.x;
  if (t == 0) {
    int n = 0;
    for (int j = 0; j < kb; ++j) pos[n++] = k0 + j;
    for (int j = 0; j < kb; ++j)
      if (sel[j] >= k0 + kb) pos[n++] = sel[j];
    for (int i = 0; i < n; ++i) from[i] = pos[i];
    for (int j = 0; j < kb; ++j) {
      int cur = -1;   // slot currently holding original row sel[j]
      for (int i = 0; i < n; ++i)
        if (from[i] == sel[j]) cur = i;
      const int tmp = from[j];
      from[j] = from[cur];
      from[cur] = tmp;
      if (blockIdx.x == 0) ipiv[k0 + j] = pos[cur];
    }
    ns = n;
  }
  __syncthreads();
  const int n = ns;
  const int c0 = blockIdx.x * kSwapCols;
  for (int e = t; e < n * kSwapCols; e += 256) {
    const int i = e / kSwapCols, cc = e % kSwapCols;
    if (c0 + cc < ng && from[i] != pos[i]) buf[i][cc] = A[(size_t)from[i] * ng + c0 + cc];
  }
  __syncthreads();
  for (int e = t; e < n * kSwapCols; e += 256) {
    const int i = e / kSwapCols, cc = e % kSwapCols;
    if (c0 + cc < ng && from[i] != pos[i]) A[(size_t)pos[i] * ng + c0 + cc] = buf[i][cc];
  }
}

// Column j of the inverse is column src[j] of the working matrix: the
// interchanges undone on the columns, last first.
__global__ void colperm_build_kernel(const int* __restrict__ ipiv_all, int ng, int* __restrict__ src_all) {
  if (threadIdx.x != 0) return;
  const int* __restrict__ ipiv = ipiv_all + (size_t)blockIdx.x * ng;
  int* __restrict__ src = src_all + (size_t)blockIdx.x * ng;
  for (int j = 0; j < ng; ++j) src[j] = j;
  for (int j = ng - 1; j >= 0; --j) {
    const int p = ipiv[j];
    const int tmp = src[j];
    src[j] = src[p];
    src[p] = tmp;
  }
}

__global__ void __launch_bounds__(256) colperm_apply_kernel(const __grid_constant__ GenPtrs Pm, int ng,
                                                            const int* __restrict__ src_all) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* row = reinterpret_cast<double2*>(smem_raw);
  double2* a = Pm.A[blockIdx.y] + (size_t)blockIdx.x * ng;
  const int* __restrict__ src = src_all + (size_t)blockIdx.y * ng;
  for (int j = threadIdx.x; j < ng; j += 256) row[j] = a[j];
  __syncthreads();
  for (int j = threadIdx.x; j < ng; j += 256) a[j] = row[src[j]];
}

}  // namespace

int epsinv_general_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells, const int32_t* const* d_geps,
                       const void* const* chi, void* const* eps, void* const* epsinv, cudaStream_t st,
                       bool tc_update) {
  int ngmax = 0;
  for (int m = 0; m < nmat; ++m) ngmax = std::max(ngmax, ng[m]);
  const int nleaf_max = (ngmax + kTRows - 1) / kTRows;
  const int cstride = nleaf_max * (kPB + 1);   // candidates then counts, per matrix
  Scratch sv, lu, R, Cp, cand, ipiv;
  sv.pool = lu.pool = R.pool = Cp.pool = cand.pool = ipiv.pool = &c->pool;
  int rc;
  if ((rc = c->pool.alloc((size_t)ngmax * sizeof(double), &sv.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)kGB * kPB * (kPB + 1) * sizeof(double2), &lu.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)kGB * kPB * ngmax * sizeof(double2), &R.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)kGB * kPB * ngmax * sizeof(double2), &Cp.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * kGB * cstride * sizeof(int), &cand.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * kGB * ngmax * sizeof(int), &ipiv.ptr)) != BGW_OK)
    return fail(c, rc, "general inverse: scratch allocation failed");
  const size_t psmem = sizeof(float2) * kTRows * (kPB + 1);
  const size_t ssmem = sizeof(double2) * 2 * kPB * kSwapCols;
  BGW_CUDA(c, cudaFuncSetAttribute(pivot_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  BGW_CUDA(c, cudaFuncSetAttribute(pivot_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  BGW_CUDA(c, cudaFuncSetAttribute(pivot_swap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem));
  BGW_CUDA(c, cudaFuncSetAttribute(colperm_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(double2) * ngmax)));
  int* cbuf[2] = {cand.as<int>(), cand.as<int>() + (size_t)kGB * cstride};
  // Matrices of equal size are stepped together, up to kGB at a time: every
  // launch below serves the whole group.
  for (int m0 = 0; m0 < nmat;) {
    const int n = ng[m0];
    int nb = 1;
    while (m0 + nb < nmat && nb < kGB && ng[m0 + nb] == n) ++nb;
    GenPtrs P = {};
    for (int k = 0; k < nb; ++k) {
      const int m = m0 + k;
      P.A[k] = static_cast<double2*>(epsinv[m]);
      if ((rc = eps_form_run(c, cells[m], d_geps[m], n, chi[m], sv.as<double>(), P.A[k], eps ? eps[m] : nullptr,
                             st)) != BGW_OK)
        return rc;
    }
    TimedScope ts(c, kTInverse, st);
    std::unique_ptr<OzPlan, void (*)(OzPlan*)> oz(nullptr, oz_plan_delete);
    if (tc_update) {
      oz.reset(oz_plan_new());
      std::vector<int> ngs(nb, n);
      std::vector<double2*> As(nb);
      std::vector<const double2*> Rs(nb), Cs(nb);
      for (int k = 0; k < nb; ++k) {
        As[k] = P.A[k];
        Rs[k] = R.as<double2>() + (size_t)k * kPB * n;
        Cs[k] = Cp.as<double2>() + (size_t)k * kPB * n;
      }
      if ((rc = oz_prepare(c, nb, ngs.data(), As.data(), Rs.data(), Cs.data(), nullptr, oz.get(), true, false,
                           c->run_slices, c->run_ff_chain)) != BGW_OK)
        return rc;
      oz_set_bulk_items(oz.get(), c->update_items);   // the option's width, else the SM-count rule
    }
    int* piv = ipiv.as<int>();
    int* src = piv + (size_t)kGB * ngmax;
    for (int k0 = 0; k0 < n; k0 += kPB) {
      const int kb = std::min(kPB, n - k0);
      int groups = (n - k0 + kTRows - 1) / kTRows;
      int cur = 0;
      {
        TimedScope tp(c, kTPivot, st);
        pivot_leaf_kernel<<<dim3(groups, nb), kTRows, psmem, st>>>(P, n, k0, kb, cbuf[0], cstride, lu.as<double2>(),
                                                                   c->d_status);
        c->launches += 1;
        while (groups > 1) {
          const int next = (groups + 7) / 8;
          pivot_merge_kernel<<<dim3(next, nb), kTRows, psmem, st>>>(P, n, k0, kb, cbuf[cur], groups, cbuf[1 - cur],
                                                                    cstride, lu.as<double2>(), c->d_status);
          c->launches += 1;
          cur = 1 - cur;
          groups = next;
        }
        pivot_swap_kernel<<<dim3((n + kSwapCols - 1) / kSwapCols, nb), 256, ssmem, st>>>(P, n, k0, kb, cbuf[cur],
                                                                                         cstride, piv);
        c->launches += 1;
        BGW_CUDA(c, cudaGetLastError());
      }
      {
        TimedScope tg(c, kTSweepChain, st);
        solve_panels_kernel<<<dim3((n + 15) / 16, 1 + (n + 255) / 256, nb), 256, 0, st>>>(
            P, n, k0, kb, lu.as<double2>(), R.as<double2>(), Cp.as<double2>());
        c->launches += 1;
        BGW_CUDA(c, cudaGetLastError());
      }
      if (!tc_update) {
        for (int k = 0; k < nb; ++k)
          if ((rc = gj_update_run(c, P.A[k], n, k0, kb, R.as<double2>() + (size_t)k * kPB * n,
                                  Cp.as<double2>() + (size_t)k * kPB * n, st)) != BGW_OK)
            return rc;
      } else {
        TimedScope tu(c, kTOzUpdate, st);
        if ((rc = oz_slice(c, oz.get(), k0, n, 0, st)) != BGW_OK || (rc = oz_update(c, oz.get(), k0, n, 0, 0, st)) != BGW_OK)
          return rc;
        c->launches += 3;
      }
    }
    colperm_build_kernel<<<nb, 1, 0, st>>>(piv, n, src);
    colperm_apply_kernel<<<dim3(n, nb), 256, sizeof(double2) * n, st>>>(P, n, src);
    BGW_CUDA(c, cudaGetLastError());
    c->launches += 2;
    m0 += nb;
  }
  return BGW_OK;
}

}  // namespace bgw
