/*
 * bgw.h -- C ABI of the GB300 library for the RPA epsilon hot path of one
 * q-point: plane-wave matrix elements, the Adler-Wiser polarizability chi,
 * the symmetrized dielectric matrix eps~ and its inverse.
 *
 * Source of every operation: the BerkeleyGW paper, Section "RPA Dielectric
 * Matrix: epsilon" (Eqs. eqn_matrix_elem, eqn_static_xi,
 * eqn_static_xi_compact, epsilon, untruncated_bare_coulomb,
 * screened_interaction, retarded_advanced_epsilon) and its Appendix
 * "Specification of file formats" for the input conventions.
 *
 * Conventions shared by all calls
 * -------------------------------
 *  - G vectors are int32 triples (x,y,z) in reciprocal-lattice units, listed
 *    as full spheres (Appendix); components must lie in [-n/2, n/2) for the
 *    FFT grid n.  G lists are HOST arrays (read during the call, copied into
 *    a device-side plan cached by content).
 *  - Wavefunction coefficients are band-major [nbands][npw] complex128
 *    (interleaved re,im doubles), normalized to sum |c|^2 = 1 per band.
 *  - The occupied (valence) band sits on the q-shifted sphere (k+q), the
 *    empty (conduction) band at k = 0.  Pair index p = v * nc + c.
 *  - Energies are in Hartree; cutoffs in Ry (|k|^2 in bohr^-2); v(q+G) =
 *    4 pi / |q+G|^2 (Hartree atomic units).
 *  - Complex outputs are row-major, interleaved.  c128 = 2 doubles,
 *    c64 = 2 floats.
 *  - Bulk arrays (coefficients, M, chi, eps) are DEVICE pointers owned by
 *    the caller unless a call says otherwise; host arrays are marked "host".
 *  - Every call enqueues its work on `stream` (a cudaStream_t passed as
 *    void*; NULL = legacy default stream) and returns before the work is
 *    done.  A context serves one host thread and one stream at a time:
 *    its scratch memory is reused by the next call in stream order.
 *  - Every call returns an int status (BGW_OK = 0).  Arguments are checked
 *    before any launch, so nothing is written when a call returns
 *    BGW_EINVAL.  Errors raised inside kernels (a zero or non-finite pivot)
 *    are recorded in a device status word and returned by bgw_sync().
 *    Outputs are undefined after any non-OK status.  bgw_last_error()
 *    returns a message for the last failure.  No C++ exception crosses the
 *    ABI.
 */
#ifndef BGW_H
#define BGW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BGW_OK = 0,
  BGW_EINVAL = 1,    /* bad sizes/pointers, G outside [-n/2,n/2), aliasing,
                        q+G = 0, unsorted energies, Delta >= 0           */
  BGW_ENOMEM = 2,    /* over the context's HBM budget or allocation failed */
  BGW_ECUDA = 3,     /* a CUDA runtime call failed                        */
  BGW_ETIMEOUT = 4,  /* a bounded device wait gave up                     */
  BGW_ENUMERIC = 5,  /* non-finite value or zero pivot in the inversion   */
  BGW_EBUSY = 6,
  BGW_ECANCELED = 7,
  BGW_EUNSUPPORTED = 8 /* valid request outside what this build implements
                          (e.g. an FFT grid size without a kernel)        */
};

/* Precision of a call.
 *  BGW_PREC_FP64     : every step in FP64 / complex128 (the plain path).
 *  BGW_PREC_MIX_FP16 : M in complex64 (FP32 FFTs); chi on the tensor cores
 *                      as split FP16 (hi*hi + hi*lo + lo*hi) products with
 *                      FP32 accumulation, flushed into an FP64 chi per call;
 *                      eps~ and its inverse in FP64.
 *  BGW_PREC_MIX_BF16 : as MIX_FP16 with BF16 splits.                      */
enum { BGW_PREC_FP64 = 0, BGW_PREC_MIX_FP16 = 1, BGW_PREC_MIX_BF16 = 2 };

/* Real flavor (Section "Real and complex flavors"): with inversion and
 * time-reversal symmetry the coefficients can be chosen real, and then M,
 * chi, eps~ and eps~^-1 are real (M_vc(G) = sum c_v(G+G') c_c(G')).  OR this
 * flag into the precision of bgw_mtxel, bgw_chi_sum and bgw_epsilon: the
 * coefficients are double [nb][npw], M is double (FP64) or float (mixed)
 * [nv*nc][ng], chi, eps~ and eps~^-1 are double [..][ng][ng] (symmetric,
 * both triangles).  chi is a real SYRK (a quarter of the complex flops; the
 * mixed precisions split hi/lo into two planes and take 3 MMAs per K step
 * instead of 12); the inverse runs on the complex embedding of the real
 * matrix (its imaginary parts stay exactly zero).  EUNSUPPORTED with the
 * real-axis entry points (complex chi) and bgw_epsilon_batch.             */
enum { BGW_FLAVOR_REAL = 0x100 };

typedef struct bgw_ctx bgw_ctx;

/* Coulomb interaction v(k), k = (q + G) B in bohr^-1, Hartree units
 * (Section "Coulomb Interaction"):
 *  BGW_COULOMB_BULK   v = 4 pi / k^2 (Eq. untruncated_bare_coulomb);
 *                     k = 0 is rejected (EINVAL).
 *  BGW_COULOMB_SPHERE v = 4 pi / k^2 (1 - cos(k r_c)), the interaction cut
 *                     off beyond a sphere of radius r_c = coulomb_cut; finite
 *                     at k = 0, where it takes its limit 2 pi r_c^2.
 *  BGW_COULOMB_SLAB   v = 4 pi / k^2 (1 - exp(-k_xy z_c) cos(k_z z_c)), cut off
 *                     beyond |z| = z_c = coulomb_cut along Cartesian z (the
 *                     slab normal), k_xy = (k_x^2 + k_y^2)^{1/2}; k = 0 is
 *                     rejected (the slab form diverges there as 1/k).
 * Both truncated forms are evaluated as 2 sin^2(k r_c / 2) and
 * -expm1(-k_xy z_c) + exp(-k_xy z_c) 2 sin^2(k_z z_c / 2), which equal the
 * brackets above and lose no digits at small k.                            */
enum { BGW_COULOMB_BULK = 0, BGW_COULOMB_SPHERE = 1, BGW_COULOMB_SLAB = 2 };

/* Cell and q-point.  bvec rows are the reciprocal lattice vectors b1,b2,b3
 * in bohr^-1 (Appendix: reciprocal lattice vectors); omega is the cell volume
 * in bohr^3; q_frac is q in crystal coordinates; fft is the FFT grid.  This
 * build requires a cubic grid fft[0] = fft[1] = fft[2] = n with n in
 * {8,10,12,16,20,24,30,32,36,40,48,50,60,64}.  coulomb selects v (a
 * zero-filled cell is the bulk interaction); coulomb_cut is r_c or z_c in
 * bohr, finite and > 0 for the truncated forms, ignored for bulk.  EINVAL
 * for another model or a bad cut length.                                   */
typedef struct bgw_cell {
  double bvec[3][3];
  double omega;
  double q_frac[3];
  int fft[3];
  int coulomb;
  double coulomb_cut;
} bgw_cell;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the library itself allocates (scratch, plans, cached
 * uploads); 0 = no bound.  On success *ctx is owned by the caller and must
 * be released with bgw_destroy.                                             */
int bgw_create(bgw_ctx** ctx, int device, uint64_t hbm_budget_bytes);
int bgw_destroy(bgw_ctx* ctx);

/* Message for the last failing call on ctx (static storage inside ctx;
 * valid until the next call).  Never NULL.                                  */
const char* bgw_last_error(bgw_ctx* ctx);

/* Wait for the work enqueued on `stream` and return (then clear) the device
 * status word: BGW_OK, BGW_ENUMERIC or BGW_ETIMEOUT; BGW_ECUDA if the
 * stream itself failed.                                                     */
int bgw_sync(bgw_ctx* ctx, void* stream);

/* Bytes the library currently holds on the device, and the high-water mark. */
int bgw_mem_stats(bgw_ctx* ctx, uint64_t* in_use, uint64_t* high_water);

/* Number of kernels this context has launched since it was created (a CUDA
 * graph replay counts the kernels the graph holds).                        */
int bgw_launch_count(bgw_ctx* ctx, uint64_t* launches);

/* CUDA graphs the context holds (bgw_epsinv, bgw_epsilon and
 * bgw_epsilon_batch capture one per argument set on capturable streams, up
 * to 8 per context; each keeps the pool blocks it uses until
 * bgw_destroy; the server's slot contexts capture none) and how many times
 * they have been replayed.  A replay reads and writes the buffers at the
 * captured addresses: its key matches only calls with the same pointers.   */
int bgw_graph_stats(bgw_ctx* ctx, uint64_t* graphs, uint64_t* replays);

/* Tuning options of a context (EINVAL for an unknown option or value).
 *  BGW_OPT_CHI_SEGMENT_PAIRS: mixed-precision chi accumulates the products
 *    of this many pairs in FP32 in tensor memory, restarting every segment
 *    (rounded down to a multiple of 32; 0 restores the default, 512); the
 *    segments of a tile are added in FP32 registers and the tiles' partial
 *    sums in FP64.  Shorter segments lower the FP32 accumulation error and
 *    cost more drains of tensor memory.                                      */
/*  BGW_OPT_AUTOTUNE: 1 (default) lets the context time the candidate tile
 *    shapes of the pair transform (pairs per block, or a warp per pair) the
 *    first time it meets a (grid, precision, epsilon-sphere shape) and keep
 *    the fastest; 0 uses the fixed default for shapes not yet tuned.       */
/*  BGW_OPT_CHI_CHUNK_PAIRS: mixed-precision chi converts and sums the pairs
 *    in chunks of this many pairs (rounded down to a multiple of 32), each
 *    chunk's FP64 sum added into chi; 0 (default) sizes chunks so that their
 *    operand planes (as large as the chunk's complex64 M) stay within 4 GiB. */
/*  BGW_OPT_INVERSE: how the sweep's trailing updates run.  -1 (default):
 *    bgw_epsilon, bgw_epsilon_batch and the server use the tensor cores for
 *    the mixed precisions and FP64 FMA for BGW_PREC_FP64, bgw_epsinv uses
 *    FP64 FMA; 0: FP64 FMA everywhere; 1: the tensor cores everywhere.  The
 *    tensor-core update splits P and C into 8-bit slices held exactly in
 *    FP16 (seven or five, BGW_OPT_UPDATE_SLICES), accumulates every slice
 *    product exactly in FP32 and combines them in double-FP32 before the
 *    FP64 subtraction: with seven its error is near 2^-48 of the update's
 *    scale (FP64 FMA: 2^-53).                                              */
/*  BGW_OPT_HEAD: the q0 head of the mixed precisions.  At a small q0 the
 *    head column M_vc(G = 0) is O(|q0|) while v(q0) = 4 pi / |q0|^2, so the
 *    FP32 FFTs' absolute error on it (near 2^-24 |M|) becomes a relative
 *    error near 2^-24 / |q0| in v chi_00, the macroscopic response.  With
 *    the head on, bgw_epsilon, bgw_epsilon_batch and the server compute
 *    M_vc(0) = sum_G conj(c_v(G)) c_c(G) as an FP64 dot product, leave it out
 *    of the tensor-core sum and add row and column G = 0 of chi in FP64.
 *    -1 (default): on when the epsilon list holds G = 0, the interaction is
 *    bulk or slab and |q| < 0.02 min_i |b_i|; 0: off; 1: on whenever G = 0
 *    is in the list.  No effect on BGW_PREC_FP64 or on bgw_chi_sum.         */
/*  BGW_OPT_SIGMA_DENSITY: how bgw_sigma_cohsex forms the band densities
 *    rho_n(D) of the closed-form Coulomb hole.  -1 (default) and 1: as the
 *    matrix element M_nn(D) of the band with itself, by the pruned product
 *    transform on the smallest supported grid that aliases neither the
 *    difference box nor the product's spectrum, else (no such grid up to 64)
 *    as 0; 0: the direct sum over the outer sphere, O(box x npw) per band.
 *    Both are FP64.                                                         */
/*  BGW_OPT_UPDATE_SLICES: slices per value of the tensor-core update.  0
 *    (default) and 7: error near 2^-48 of the update's scale (FP64-level
 *    inverse); 5: near 2^-34 with 15 slice products per tile instead of 28
 *    (implies BGW_OPT_DOUBLE_FP32).  For inputs whose own errors are far
 *    larger and ε̃ that is well conditioned.                                 */
/*  BGW_OPT_DOUBLE_FP32: the tensor-core sweep's critical chain -- the next
 *    32 x 32 diagonal block's sweep and the panel product P = C D^-1 -- in
 *    double-FP32 arithmetic (value = hi + lo, about 2^-46 per operation,
 *    the FP64-level class of the seven-slice update) on the FP32 pipe, which
 *    on GB300 issues 64 times the FP64 pipe's operations.  -1 (default): on
 *    in bgw_epsilon, bgw_epsilon_real, bgw_epsilon_batch and the server for
 *    the mixed precisions, off for FP64 inputs and for bgw_epsinv*; 0: off;
 *    1: on.                                                                */
/*  BGW_OPT_PAIR_KERNEL: which kernel runs the pair transform's y and x
 *    passes.  -1 (default): the autotuner's choice (or the fixed default
 *    while BGW_OPT_AUTOTUNE is 0); 0: one (pair block, plane) per CTA with
 *    the default pairs per block; 1: one warp per pair, where every kept
 *    frequency lies in |k| < N/4 (elsewhere 0 runs).  The results agree to
 *    rounding; the choice only changes the speed.                          */
/*  BGW_OPT_UPDATE_ITEMS: column tiles per work item of the tensor-core
 *    sweep's bulk update launches.  -1 (default): the SM-count rule, items
 *    of 2 tiles where the wider items would number no more than the SMs
 *    (a CTA then pipelines two items instead of running one alone); 0: the
 *    wider items (4 column tiles with seven slices, 3 with five); 1: items
 *    of 2 tiles.  Every tile's arithmetic is the same: the results are
 *    bit-identical, only the speed changes.                                */
/*  BGW_OPT_WAIT_LIMIT_NS: how long (nanoseconds, 0 .. 10^10; default 10^9)
 *    a wait of the tensor-core chi kernels on its pipeline (a copy landing,
 *    an MMA stage finishing, tensor memory being drained) may last before
 *    the kernel gives up: it then lets its copies and MMAs in flight finish
 *    (within 1 s), frees its tensor memory, returns, and the next bgw_sync
 *    (or call that synchronizes) reports BGW_ETIMEOUT; the outputs of that
 *    call are undefined, the context stays usable.  0 gives up at the first
 *    wait that is not already complete (a test of that path).              */
enum { BGW_OPT_CHI_SEGMENT_PAIRS = 1, BGW_OPT_TIMING = 2, BGW_OPT_AUTOTUNE = 3, BGW_OPT_CHI_CHUNK_PAIRS = 4,
       BGW_OPT_INVERSE = 5, BGW_OPT_HEAD = 6, BGW_OPT_SIGMA_DENSITY = 7, BGW_OPT_UPDATE_SLICES = 8,
       BGW_OPT_DOUBLE_FP32 = 9, BGW_OPT_WAIT_LIMIT_NS = 10, BGW_OPT_PAIR_KERNEL = 11, BGW_OPT_UPDATE_ITEMS = 12 };
int bgw_set_option(bgw_ctx* ctx, int option, int64_t value);

/* With BGW_OPT_TIMING = 1 the context records CUDA events around its main
 * kernel groups (band transform, pair passes, chi kernels, eps~ formation,
 * the inverse).  bgw_timing_report waits for the recorded events, adds them
 * to running totals and writes the totals as a JSON object
 * {"name": [launches, milliseconds], ...} into buf (NUL-terminated,
 * truncated to len).  reset = 1 clears the totals afterwards.             */
int bgw_timing_report(bgw_ctx* ctx, char* buf, size_t len, int reset);

/* ------------------------------------------------------------------------
 * bgw_mtxel -- plane-wave matrix elements (Eq. eqn_matrix_elem), computed as
 * the FFT of the real-space product of the two bands (paper's equation
 * M = FFT^-1(phi*_{n,k+q}(r) phi_{n',k}(r))):
 *   u_b(r_j)   = sum_G c_b(G) exp(+2 pi i G.j/n)
 *   M[p][iG]   = (1/n^3) sum_j conj(u_v(r_j)) u_c(r_j) exp(+2 pi i G_iG.j/n)
 *              = sum_{G2} conj(c_v(G_iG + G2)) c_c(G2)
 *   gv   host int32 [npw_v][3]  valence (q-shifted) sphere
 *   cv   device c128 [nv][npw_v]
 *   gc   host int32 [npw_c][3]  conduction sphere
 *   cc   device c128 [nc][npw_c]
 *   geps host int32 [ng][3]     epsilon sphere (output order)
 *   M    device, pair-major [nv*nc][ng]: c128 for BGW_PREC_FP64, c64 for
 *        the mixed precisions.
 * EINVAL when a G component lies outside [-n/2, n/2), when a list holds a
 * duplicate G, or when the grid aliases: n <= max|Gv_d| + max|Gc_d| +
 * max|Geps_d| on some axis d.                                              */
int bgw_mtxel(bgw_ctx* ctx, const bgw_cell* cell,
              int nv, int npw_v, const int32_t* gv, const void* cv,
              int nc, int npw_c, const int32_t* gc, const void* cc,
              int ng, const int32_t* geps, int prec, void* M, void* stream);

/* ------------------------------------------------------------------------
 * bgw_chi_sum -- polarizability (Eq. eqn_static_xi as the single matrix
 * product of Eq. eqn_static_xi_compact):
 *   chi_f[G][G'] (+)= (4/Omega) sum_p w_p(f) conj(M[p][G]) M[p][G']
 *   static (nfreq = 0): w_p = 1/Delta_p, Delta_p = E_v - E_c < 0
 *   imaginary axis:      w_p = Delta_p / (Delta_p^2 + omega_f^2)
 *                        (Eq. retarded_advanced_epsilon at E = i omega_f)
 *   M     device [nv*nc][ng], c128 (prec FP64) or c64 (mixed precisions)
 *   ev,ec host double [nv], [nc] in Ha, each ascending, every ec > every ev
 *   omega host double [nfreq] in Ha (ignored when nfreq = 0)
 *   chi   device c128 [max(1,nfreq)][ng][ng], Hermitian, both triangles
 *         written.  accumulate = 1 adds into chi (stream conduction chunks:
 *         call once per chunk with that chunk's M, ec and nc).
 * The mixed precisions accumulate each call's contribution in FP32 on the
 * tensor cores and add it to the FP64 chi once per call.                   */
int bgw_chi_sum(bgw_ctx* ctx, const bgw_cell* cell, int nv, int nc, int ng,
                const void* M, const double* ev, const double* ec,
                int nfreq, const double* omega, int prec, int accumulate,
                void* chi, void* stream);

/* ------------------------------------------------------------------------
 * bgw_epsinv -- symmetrized dielectric matrix and its inverse (Eq. epsilon
 * with the symmetric Coulomb form v^{1/2}(q+G) v^{1/2}(q+G')):
 *   eps~[G][G'] = delta_GG' - sqrt(v_G) chi[G][G'] sqrt(v_G'),
 *   v_G = v((q + G) B) of the cell's Coulomb model (4 pi / |(q + G) B|^2
 *   for bulk),  then epsinv = (eps~)^-1   (FP64 always).
 * Batched over nmat independent matrices of sizes ng[i] (may differ):
 *   cells[i]  host, q and bvec of matrix i
 *   geps[i]   host int32 [ng[i]][3]
 *   chi[i]    device c128 [ng[i]][ng[i]] (read only)
 *   eps[i]    device c128 [ng[i]][ng[i]] or NULL (eps~ is also written
 *             there when non-NULL; the array `eps` itself may be NULL)
 *   epsinv[i] device c128 [ng[i]][ng[i]]
 * eps~ is Hermitian positive definite (chi <= 0 makes eps~ >= I); the
 * inverse is a blocked sweep (Gauss-Jordan without pivoting in its
 * Hermitian form) that reads and updates only the lower triangle of chi's
 * Hermitian eps~, then writes both triangles of epsinv.  Elimination without
 * pivoting is backward stable for such matrices.
 * EINVAL if some |q+G| = 0 under the bulk or slab interaction.  A zero or
 * non-finite pivot sets BGW_ENUMERIC, reported by bgw_sync.                */
int bgw_epsinv(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng,
               const int32_t* const* geps, const void* const* chi,
               void* const* eps, void* const* epsinv, void* stream);

/* ------------------------------------------------------------------------
 * bgw_screened_w -- the screened Coulomb interaction (Eq.
 * screened_interaction), W_GG' = eps^-1_GG' v(q+G'), from the symmetrized
 * inverse bgw_epsinv returns: since eps~ = v^{-1/2} eps v^{1/2},
 *   W[G][G'] = sqrt(v_G) epsinv[G][G'] sqrt(v_G'),
 * with v of the cell's Coulomb model (see bgw_cell).  W is Hermitian.
 * Batched over nmat matrices like bgw_epsinv:
 *   cells[i]  host, q, bvec and Coulomb model of matrix i
 *   geps[i]   host int32 [ng[i]][3]
 *   epsinv[i] device c128 [ng[i]][ng[i]] (read)
 *   W[i]      device c128 [ng[i]][ng[i]] (written; may equal epsinv[i]
 *             for an in-place update, must not overlap it otherwise)
 * One pass over HBM: 16 B read and 16 B written per element.
 * EINVAL on NULL pointers, bad sizes or |q+G| = 0 where v diverges;
 * EUNSUPPORTED for ng > 65535.                                           */
int bgw_screened_w(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng,
                   const int32_t* const* geps, const void* const* epsinv,
                   void* const* W, void* stream);

/* bgw_epsinv_rflavor -- bgw_epsinv for the real flavor (Section "Real and
 * complex flavors": with inversion and time-reversal symmetry the
 * coefficients, M, chi and eps are real; Eq. epsilon as for bgw_epsinv):
 * chi[i], eps[i] (or NULL) and epsinv[i] are real double [ng[i]][ng[i]],
 * symmetric.  Errors as bgw_epsinv.                                        */
int bgw_epsinv_rflavor(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng,
                       const int32_t* const* geps, const void* const* chi,
                       void* const* eps, void* const* epsinv, void* stream);

/* ------------------------------------------------------------------------
 * bgw_sigma_cohsex -- diagonal static COHSEX and bare-exchange self-energy
 * for one q (Section "The Self-Energy": Eqs. cohsex-sx, cohsex-ch-sum,
 * cohsex-ch-exact, hf-x), from this path's symmetrized eps~^-1 at that q:
 *   m_{n''n}(G) = M_{n''n}(k, -q, -G) = sum_{G2} conj(c_n''(G2 - G)) c_n(G2)
 *   W = eps^-1 v = V^1/2 eps~^-1 V^1/2   (the cell's Coulomb model)
 *   sigma[0][n] X        = -(1/Omega) sum_{n'' < nocc} sum_G |m(G)|^2 v(q+G)
 *   sigma[1][n] SX       = -(1/Omega) sum_{n'' < nocc} m^H W m
 *   sigma[2][n] CH       = (1/(2 Omega)) sum_{n'' < ni} m^H (W - V) m
 *   sigma[3][n] CH exact = (1/(2 Omega)) sum_{G G'} <n|e^{i(G-G').r}|n> (W - V)_{G G'}
 * (1/Omega: one q point of a q sum; Hartree.  The closed form is the sum
 * form over a complete set of inner bands.)
 *   co  device c128 [no][npw_o], outer bands n at k on the G list go (host)
 *   ci  device c128 [ni][npw_i], inner bands n'' at k - q on gi (host); the
 *       first nocc are occupied
 *   geps host int32 [ng][3], the eps sphere of q; epsinv device c128
 *       [ng][ng] (bgw_epsinv of the same cell and list)
 *   prec BGW_PREC_FP64: FP64 throughout.  BGW_PREC_MIX_FP16 / _BF16: m from
 *        the FP32 matrix-element path and W m on the tensor cores (split
 *        operands, FP32 segment sums, FP64 result); the quadratic forms,
 *        the sums and the closed form in FP64.
 *   sigma host double [4][no]; the call returns after it is written.
 * EINVAL as bgw_mtxel for the lists and grid (n > max|Gi| + max|Go| +
 * max|Geps| per axis, and -G inside [-n/2, n/2)), for non-device arrays or
 * nocc outside [0, ni].                                                     */
int bgw_sigma_cohsex(bgw_ctx* ctx, const bgw_cell* cell,
                     int no, int npw_o, const int32_t* go, const void* co,
                     int ni, int npw_i, const int32_t* gi, const void* ci,
                     int nocc, int ng, const int32_t* geps, const void* epsinv,
                     int prec, double* sigma, void* stream);

/* bgw_real_coefficients -- real-flavor coefficients from complex ones (host
 * arrays), as the paper prescribes: bands whose energies (ascending) differ
 * by at most tol from their neighbour form a degenerate subspace of n
 * states; the 2n vectors Re c_1, Im c_1, Re c_2, ... are orthonormalized in
 * that order by modified Gram-Schmidt (a remainder below 1e-8 of the
 * vector's norm is dropped) and the first n kept, so a non-degenerate
 * state loses its global phase.
 *   c   host c128 [nb][npw];  energies host double [nb];  out host double
 *       [nb][npw].
 * ENUMERIC if a subspace gives fewer than n real directions (no inversion
 * and time-reversal symmetry).  Host only, no context.                    */
int bgw_real_coefficients(int nb, int npw, const void* c, const double* energies, double tol, double* out);

/* ------------------------------------------------------------------------
 * bgw_epsinv_noalloc -- bgw_epsinv for one matrix without any device
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc, such as an application whose own
 * allocator has already reserved the device memory it may use (a serving
 * engine or framework holding the GPU's memory in its caching pool), or a
 * loop that cannot accept the device-wide synchronization an allocation may
 * cause.  It needs no bgw_ctx and runs on the caller's current device.
 *   cell, ng, geps  as bgw_epsinv (geps host int32 [ng][3])
 *   chi     device c128 [ng][ng] (read only)
 *   eps     device c128 [ng][ng] or NULL (eps~ is also written there)
 *   epsinv  device c128 [ng][ng]
 * Scratch: one fixed file-scope device array of about 4.1 MiB inside the
 * library, which every GPU that loads the library holds until the process
 * exits; it bounds ng <= 4096 (larger ng returns BGW_EINVAL before any
 * work is queued).  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current) and caches it with
 * the id of the current CUDA context; a call made in another context of the
 * device (after cudaDeviceReset, or under a driver-API context the caller
 * made current) looks it up again.  Make the first call on a device before
 * any stream capture.  All calls share the array and it keeps the last
 * call's contents (each call clears what must start at zero), so calls whose
 * work overlaps on the GPU (other streams, other host threads) race:
 * serialize them.  Returns BGW_EINVAL for bad arguments or |q+G| = 0,
 * BGW_ECUDA when one of this call's CUDA calls or launches fails.  A zero or
 * non-finite pivot is not reported (there is no context to carry the status
 * word); the result is then meaningless.                                   */
int bgw_epsinv_noalloc(const bgw_cell* cell, int ng, const int32_t* geps,
                       const void* chi, void* eps, void* epsinv, void* stream);

/* ------------------------------------------------------------------------
 * bgw_epsilon_batch -- independent q-points, each at the same nfreq
 * imaginary frequencies (nfreq = 0: static), as one stream of work: per
 * q-point the matrix elements are computed once and serve every frequency
 * (the paper's observation that the summation, not the matrix elements,
 * repeats per frequency), then chi for each frequency and the batched
 * inverses of all frequencies.  The q-points' epsilon spheres may differ in
 * size (uneven N_G).
 *   problems[q]  one q-point; all bulk arrays (cv, cc) are DEVICE arrays,
 *                G lists and energies host arrays (as in the single calls)
 *   omega        host double [nfreq] (Ha)
 *   epsinv[q]    device c128 [max(1,nfreq)][ng_q][ng_q]
 * On a stream other than the legacy default stream the first call with a
 * given argument set runs the work directly and also captures it into a
 * CUDA graph; later calls with the same arguments (same pointers, sizes and
 * host-array contents) replay that graph with one launch.  Device array
 * contents may change between calls.  The library's scratch memory used by
 * a captured graph stays reserved until the context is destroyed.          */
typedef struct bgw_problem {
  bgw_cell cell;
  int nv, npw_v;
  const int32_t* gv;
  const void* cv;
  const double* ev;
  int nc, npw_c;
  const int32_t* gc;
  const void* cc;
  const double* ec;
  int ng;
  const int32_t* geps;
} bgw_problem;

int bgw_epsilon_batch(bgw_ctx* ctx, int nq, const bgw_problem* problems,
                      int nfreq, const double* omega, int prec,
                      void* const* epsinv, void* stream);

/* ------------------------------------------------------------------------
 * Serving: a stream of independent eps~^-1 requests of different sizes.
 * Each request is one q-point's whole path; the paper notes that Eq.
 * eqn_static_xi separates in q, so q-points run as independent epsilon
 * calculations (Section "Parallelization and Performance", epsilon), and
 * that each run estimates the memory its largest arrays need against what
 * is available (Section "Memory estimation"): the server admits a request
 * against such an estimate.  The server keeps max_slots requests in flight, each on its own CUDA
 * stream and context; a request waiting in the FIFO is admitted as soon as
 * a slot is free and its device-memory estimate fits in what the HBM budget
 * has left, so its work overlaps with the requests already running
 * (continuous batching across streams).  Inputs are copied into pinned host
 * memory at submit time, so the caller's arrays may be reused immediately.
 * Every request runs the whole path (bgw_epsilon) in opts->prec.
 * Thread safety: submit, poll and cancel may be called from any thread.
 *
 *   ctx                    the context whose device serves the requests;
 *                          the server gives every slot a context of its own
 *                          on that device (a slot's pool, plans and streams
 *                          must not be shared with other slots or with the
 *                          caller's own calls), so ctx is only read at open
 *                          and may be used or destroyed independently
 *   opts.hbm_budget_bytes  bound on the sum of the estimates of admitted
 *                          requests (0 = 90 % of the free device memory at
 *                          open); a request whose estimate exceeds it alone
 *                          completes with BGW_ENOMEM
 *   opts.max_slots         1..64 requests in flight
 *   request.problem        one q-point; cv, cc are HOST arrays here
 *   request.epsinv_out     host c128 [ng][ng]; written before the request
 *                          completes; must stay valid until then
 *   bgw_serve_poll         waits up to timeout_ms; BGW_EBUSY if the request
 *                          is still pending, else fills *out and forgets the
 *                          ticket (out->status is the request's own status)
 *   bgw_serve_cancel       removes a request that has not been admitted
 *                          (BGW_EBUSY once it runs); its status becomes
 *                          BGW_ECANCELED
 *   bgw_serve_close        cancels waiting requests, lets running ones
 *                          finish, and frees the server                    */
typedef struct bgw_serve_opts {
  uint64_t hbm_budget_bytes;
  int max_slots;
  int prec;
} bgw_serve_opts;

typedef struct bgw_request {
  bgw_problem problem;
  void* epsinv_out;
} bgw_request;

typedef struct bgw_result {
  int status;
  double latency_ms;   /* submit -> eps~^-1 on the host */
  double queue_ms;     /* submit -> admission */
  uint64_t hbm_bytes;  /* admission estimate */
} bgw_result;

typedef struct bgw_server bgw_server;

int bgw_serve_open(bgw_ctx* ctx, const bgw_serve_opts* opts, bgw_server** out);
int bgw_serve_submit(bgw_server* srv, const bgw_request* req, uint64_t* ticket);
int bgw_serve_poll(bgw_server* srv, uint64_t ticket, int timeout_ms, bgw_result* out);
int bgw_serve_cancel(bgw_server* srv, uint64_t ticket);
int bgw_serve_close(bgw_server* srv);

/* ------------------------------------------------------------------------
 * bgw_epsilon -- the whole path for one q-point and nfreq frequencies
 * (nfreq = 0: static), the three steps of Section "RPA Dielectric Matrix:
 * epsilon" (Eqs. eqn_matrix_elem, eqn_static_xi / eqn_static_xi_compact,
 * epsilon): bgw_mtxel, bgw_chi_sum over conduction chunks of at
 * most `nc_chunk` bands (0 = all at once), then bgw_epsinv per frequency.
 * Bulk inputs (cv, cc) and outputs (chi, epsinv) may be host or device
 * memory (detected per pointer); host buffers are copied inside the call
 * and the call then returns after the results are back on the host.
 *   chi     c128 [max(1,nfreq)][ng][ng] or NULL (not returned)
 *   epsinv  c128 [max(1,nfreq)][ng][ng]
 * The library holds M and the chi accumulator in its own scratch memory.
 * Errors as the three calls it makes.                                      */
int bgw_epsilon(bgw_ctx* ctx, const bgw_cell* cell,
                int nv, int npw_v, const int32_t* gv, const void* cv,
                const double* ev,
                int nc, int npw_c, const int32_t* gc, const void* cc,
                const double* ec,
                int ng, const int32_t* geps, int nfreq, const double* omega,
                int prec, int nc_chunk, void* chi, void* epsinv, void* stream);

/* ------------------------------------------------------------------------
 * Real axis ("full frequency"): the retarded or advanced response of Eq.
 * retarded_advanced_epsilon at real frequencies E_f with broadening delta,
 *   chi_f[G][G'] (+)= (4/Omega) sum_p w_p(E_f) conj(M[p][G]) M[p][G'],
 *   w_p(E) = (1/2) [1/(D_p - E - s i delta) + 1/(D_p + E + s i delta)],
 * D_p = E_v - E_c, s = +1 retarded (advanced = 0), -1 advanced (advanced =
 * 1).  The weights are complex, so chi is not Hermitian (chi^a = (chi^r)^H);
 * every element is computed.  At E = 0 the weight is D/(D^2 + delta^2), the
 * imaginary-axis weight at omega = delta.
 *   energy host double [nfreq] (Ha, finite), delta > 0 (Ha)
 *   M, prec, accumulate, chi as bgw_chi_sum (chi [nfreq][ng][ng], both
 *   triangles).  The mixed precisions split X = M and Y = w M (two operand
 *   sets) and run every 128 x 128 tile on the tensor cores.
 * EINVAL for nfreq < 1, a non-finite energy, delta <= 0 or advanced not 0/1. */
int bgw_chi_sum_real(bgw_ctx* ctx, const bgw_cell* cell, int nv, int nc, int ng,
                     const void* M, const double* ev, const double* ec,
                     int nfreq, const double* energy, double delta, int advanced,
                     int prec, int accumulate, void* chi, void* stream);

/* bgw_epsinv_general -- eps~ = I - sqrt(v_G) chi sqrt(v_G') for a general
 * (non-Hermitian) chi, and its inverse by blocked Gauss-Jordan elimination
 * with partial pivoting (pivot rows of each 32-column block chosen by a
 * tournament of partial-pivoting LUs over 256-row slices; the paper inverts
 * with ZGESV).  Arguments as bgw_epsinv; every element of chi is read.
 * EUNSUPPORTED for ng > 14336; a zero pivot (singular eps~) sets
 * BGW_ENUMERIC, reported by bgw_sync.                                      */
int bgw_epsinv_general(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng,
                       const int32_t* const* geps, const void* const* chi,
                       void* const* eps, void* const* epsinv, void* stream);

/* bgw_epsilon_real -- bgw_epsilon on the real axis (Eq.
 * retarded_advanced_epsilon): bgw_mtxel, bgw_chi_sum_real over conduction
 * chunks, bgw_epsinv_general per frequency.
 * chi and epsinv are c128 [nfreq][ng][ng]; other arguments as bgw_epsilon
 * and bgw_chi_sum_real.                                                    */
int bgw_epsilon_real(bgw_ctx* ctx, const bgw_cell* cell,
                     int nv, int npw_v, const int32_t* gv, const void* cv, const double* ev,
                     int nc, int npw_c, const int32_t* gc, const void* cc, const double* ec,
                     int ng, const int32_t* geps, int nfreq, const double* energy,
                     double delta, int advanced, int prec, int nc_chunk,
                     void* chi, void* epsinv, void* stream);

/* bgw_frequency_grid -- the real-frequency grid of the paper's full-frequency
 * calculation (Fig. frequency_grid): 0, spacing, 2 spacing, ... while
 * <= low_cutoff; after the last uniform point each step is `increment`
 * longer than the one before, while the frequency stays <= high_cutoff (a
 * relative slack of 1e-12 absorbs rounding at both cutoffs).  Writes up to
 * max_points values to out (host, may be NULL to count) and the number of
 * points to *npoints.  EINVAL for spacing <= 0, increment < 0, low < 0,
 * high < low or more than 2^24 points; ENOMEM when out is too short (the
 * count is still written).  Host only, no context.                        */
int bgw_frequency_grid(double spacing, double low_cutoff, double high_cutoff, double increment,
                       int max_points, double* out, int* npoints);

#ifdef __cplusplus
}
#endif
#endif /* BGW_H */
