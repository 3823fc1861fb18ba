// Internal runtime of the library: context, device-memory pool with a
// budget, content-keyed caches of uploaded host arrays and plans, error
// state.  Not part of the ABI (include/bgw.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/bgw.h"

namespace bgw {

// Device status word values written by kernels (read by bgw_sync).
enum DevStatus : int { kDevOk = 0, kDevZeroPivot = 1, kDevTimeout = 2 };

struct Block {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Caching device allocator.  Blocks are rounded up to 2 MiB (small ones to
// 256 B multiples of 64 KiB) and kept on per-size free lists after release;
// every byte obtained from cudaMalloc counts against the budget until the
// context is destroyed or trim() runs.  Reuse is stream-ordered: a context
// runs on one stream at a time.
class Pool {
 public:
  explicit Pool(uint64_t budget) : budget_(budget) {}
  ~Pool();
  // Returns BGW_OK / BGW_ENOMEM / BGW_ECUDA.
  int alloc(size_t bytes, void** out);
  // For blocks kept for the context's life (uploaded inputs, plans): never
  // a block pinned by a captured graph.  A pinned block on the free list is
  // safe for a later call's scratch (stream order puts it after the graph's
  // replays), but a replay would overwrite anything kept in it.
  int alloc_keep(size_t bytes, void** out);
  void release(void* p);
  void trim();  // cudaFree every cached free block not pinned by a graph
  // While pinning is on, every block handed out is marked pinned: a CUDA
  // graph captured meanwhile refers to it, so trim() must never free it.
  // A capture that fails unpins what it pinned (abandon_pins).
  void set_pinning(bool on) {
    pinning_ = on;
    if (on) capture_pins_.clear();
  }
  void abandon_pins() {
    for (void* p : capture_pins_) pinned_.erase(p);
    capture_pins_.clear();
  }
  void unpin_all() { pinned_.clear(); }
  uint64_t in_use() const { return in_use_; }
  uint64_t reserved() const { return reserved_; }
  uint64_t high_water() const { return high_water_; }

 private:
  static size_t round(size_t b);
  int alloc_impl(size_t bytes, void** out, bool keep);
  uint64_t budget_;
  uint64_t reserved_ = 0;   // bytes obtained from cudaMalloc
  uint64_t in_use_ = 0;     // bytes handed out
  uint64_t high_water_ = 0;
  std::multimap<size_t, void*> free_;
  std::unordered_map<void*, size_t> live_;
  std::unordered_map<void*, size_t> pinned_;
  std::vector<void*> capture_pins_;   // blocks pinned by the capture in progress
  bool pinning_ = false;
};

// RAII scratch handle released to the pool at scope exit (stream order).
struct Scratch {
  Pool* pool = nullptr;
  void* ptr = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() { if (pool && ptr) pool->release(ptr); }
  template <typename T> T* as() const { return reinterpret_cast<T*>(ptr); }
};

// Plan of the two pruned 3D transforms for one (G list, grid) pair.
struct BandPlan {        // band transform of one wavefunction sphere
  int n = 0, npw = 0, ncol = 0, nxs = 0;
  int* d_ent_col = nullptr;    // [npw] local column of coefficient slot i (entries sorted by column)
  int* d_ent_z = nullptr;      // [npw] gz mod n
  int* d_ent_idx = nullptr;    // [npw] coefficient index in the caller's order
  int* d_col_start = nullptr;  // [ncol+1] entry range per column
  int* d_col_xy = nullptr;     // [ncol] (gy mod n) * n + (gx mod n)
  int* d_xslot = nullptr;      // [nxs] distinct gx mod n
};
struct PairPlan {        // pruned product transform onto the epsilon sphere
  int n = 0, ng = 0, ncol = 0, nys = 0;
  bool lowband = false;         // every kept k (all three axes) in k < n/4 or k >= 3n/4
  int* d_yslot_of_k = nullptr;  // [n] ky-slot of FFT index k along y, or -1
  int* d_colmap = nullptr;      // [n][nys] column of (kx=k, ky=slot) or -1 (k-major)
  int* d_zmap = nullptr;        // [n][ncol] G index of (column, kz=k) or -1 (k-major)
};

// Optional CUDA-event timing of named kernel groups (BGW_OPT_TIMING).
struct Timing {
  bool on = false;
  struct Rec { int name; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> free_events;
  std::map<int, std::pair<long long, double>> acc;  // name -> (launches, ms)
};
enum TimedName { kTBand = 0, kTPairYX, kTPairZ, kTChiF64, kTChiSplit, kTChiTc, kTChiReduce, kTEpsForm, kTInverse,
                 kTOzUpdate, kTSweepChain, kTHeadDot, kTHeadWings, kTScreenedW, kTPivot, kTSigmaForms, kTSigmaExact, kTOzAhead, kTNumNames };
const char* timed_name(int n);

// A captured batch (bgw_epsilon_batch) replayed while its key is unchanged.
constexpr size_t kMaxGraphs = 8;   // graphs one context keeps (each pins the pool blocks it uses)
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;   // kernel launches the graph holds (added to the launch count per replay)
};

struct Ctx {
  int device = 0;
  Timing timing;
  std::unordered_map<uint64_t, BatchGraph> graphs;
  uint64_t graph_replays = 0;
  bool use_graphs = true;          // false in the server's slot contexts (one-shot buffers per request)
  std::map<std::tuple<int, int, int, int>, int> tuned_ppb;  // (n, prec, nys, ncol) -> pairs per CTA
  bool autotune = true;
  int pair_kernel = -1;      // pair transform y,x kernel: -1 autotuned, 0 block, 1 warp per pair
  int update_items = -1;     // bulk update items: -1 the SM-count rule, 0 wide, 1 two column tiles
  cudaStream_t side = nullptr;     // high-priority stream of the sweep's look-ahead chain
  cudaEvent_t la_ev[4] = {};       // look-ahead dependencies (fork, slice, rest x2)
  cudaStream_t copy_st = nullptr;  // host-to-device copies of bgw_epsilon's conduction chunks
  cudaEvent_t copy_ev[3] = {};     // fork, and the chunk copies (ping-pong)
  int inverse_mode = -1;     // -1: tensor-core update for the mixed precisions; 0: FP64 FMA; 1: tensor cores
  int head_mode = -1;        // mixed chi head/wings in FP64: -1 automatic at small q, 0 off, 1 on
  int sigma_density = -1;    // Sigma band densities: -1/1 product transform where alias-free, 0 direct sum
  int update_slices = 0;     // tensor-core update slices: 0 automatic (7), 5 or 7
  int double_fp32 = -1;      // double-FP32 sweep chain: -1 automatic (mixed precisions), 0 off, 1 on
  int run_slices = 7;        // slices of the call in progress (set by each entry point)
  bool run_ff_chain = false; // double-FP32 chain for the call in progress (mixed precisions)
  std::unordered_map<uint64_t, const int32_t*> head_maps;  // conduction G -> valence index (head dot products)
  Pool pool;
  std::string err;
  int* d_status = nullptr;   // device status word
  bool twiddles_ready = false;
  bool chi_tc_ready = false;
  uint64_t launches = 0;     // kernels launched by this context
  int chi_segment_pairs = 0; // mixed chi: pairs per FP32 accumulation segment (0 = default)
  int chi_chunk_pairs = 0;   // mixed chi: pairs per chunk of operand planes (0 = sized to 4 GiB)
  unsigned long long wait_ns = 1000000000ull;  // limit of the tensor-core chi kernels' pipeline waits
  // Content-keyed caches (hash_bytes over the bytes plus sizes).
  std::unordered_map<uint64_t, void*> uploads;           // small host arrays
  std::unordered_map<uint64_t, std::unique_ptr<BandPlan>> band_plans;
  std::unordered_map<uint64_t, std::unique_ptr<PairPlan>> pair_plans;
  explicit Ctx(uint64_t budget) : pool(budget) {}
};

uint64_t hash_bytes(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull);

// Records CUDA events around its scope on `st` when timing is enabled.
class TimedScope {
 public:
  TimedScope(Ctx* c, int name, cudaStream_t st);
  ~TimedScope();

 private:
  Ctx* c_;
  int name_;
  cudaStream_t st_;
  cudaEvent_t a_ = nullptr;
};
// Collects the finished records (synchronizing on their events).
void timing_collect(Ctx* c);

// Errors: set ctx->err and return the code.
int fail(Ctx* c, int code, const char* fmt, ...);
int cuda_fail(Ctx* c, cudaError_t e, const char* what);
// Streaming multiprocessors of the context's device (152 if the query fails).
int sm_count(Ctx* c);
#define BGW_CUDA(c, expr)                                    \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::bgw::cuda_fail((c), _e, #expr); \
  } while (0)

// Copy a small host array to device memory on stream `st`, cached by content
// for the life of the context (only the first call with given content copies).
int upload_cached(Ctx* c, const void* host, size_t bytes, cudaStream_t st, const void** dev);

// Plans (mtxel.cu); built on the host, uploaded on `st`, cached by content.
int get_band_plan(Ctx* c, int n, int npw, const int32_t* g, cudaStream_t st, const BandPlan** out);
int get_pair_plan(Ctx* c, int n, int ng, const int32_t* geps, cudaStream_t st, const PairPlan** out);
bool fft_size_supported(int n);

// One matrix-element evaluation with its scratch (see mtxel_kernels.cuh).
// Codes of the pair transform's y,x kernel in the tuned-shape table: a
// positive number below kPairWarpCode is the block kernel's pairs per block.
constexpr int kPairWarpCode = 1000;     // one warp per pair (low-band grids)

struct MtxelExec {
  int n = 0, nv = 0, nc = 0;
  const BandPlan* bpv = nullptr;
  const BandPlan* bpc = nullptr;
  const PairPlan* pp = nullptr;
  const void* cv = nullptr;      // c128 [nb][npw], or double when real
  const void* cc = nullptr;
  int real = 0;                  // real flavor: real coefficients in, real M out
  void* uv = nullptr;   // [nv][n^3]
  void* uc = nullptr;   // [nc][n^3]
  void* U1 = nullptr;   // [max(nv,nc)][n][max ncol]
  void* T = nullptr;    // [pair_block][n][pp->ncol]
  int pair_block = 0;
  void* M = nullptr;
  cudaStream_t st = nullptr;
  uint64_t* launches = nullptr;  // incremented per kernel launch
  Ctx* ctx = nullptr;            // for optional event timing
  int* tuned_ppb = nullptr;      // in/out: pairs per pair_yxpass CTA (0 = tune now)
};
cudaError_t mtxel_exec_f64(const MtxelExec& x);
cudaError_t mtxel_exec_f32(const MtxelExec& x);
cudaError_t mtxel_init_f64();
cudaError_t mtxel_init_f32();

// Launchers (each enqueues on `st`; return BGW_OK or an error code).
// real = true: the real flavor (real coefficients, real M of the precision's
// scalar type).
int mtxel_run(Ctx* c, int n, int prec, int nv, const BandPlan* bpv, const void* cv,
              int nc, const BandPlan* bpc, const void* cc, const PairPlan* pp,
              void* M, cudaStream_t st, bool real = false);
// FP64 head of the mixed precisions at a small q (head.cu).  g0 < 0: not used.
struct HeadPlan {
  int g0 = -1;                   // index of G = 0 in the epsilon list
  int npw_c = 0;
  const int32_t* d_map = nullptr;  // [npw_c] valence index of each conduction G, or -1
};
int head_prepare(Ctx* c, const bgw_cell* cell, int npw_v, const int32_t* gv, int npw_c, const int32_t* gc, int ng,
                 const int32_t* geps, int prec, cudaStream_t st, HeadPlan* out);
// h[p] = M_p(G = 0) in FP64 for the nv x nc pairs; zeroes column g0 of the FP32 M.
int head_dot(Ctx* c, const HeadPlan* hp, int nv, const void* cv, int npw_v, int nc, const void* cc, int ng,
             void* M, double2* h, cudaStream_t st);
// Adds row and column g0 of chi from h and M (weights w[nrow][K]).
int head_wings(Ctx* c, const HeadPlan* hp, long long K, int ng, const void* M, const double2* h, const double* w,
               int nrow, double scale, void* chi, cudaStream_t st);
// hp/h: when hp->g0 >= 0 the mixed precisions add the FP64 head and wings
// (column g0 of M must have been zeroed by head_dot).
// real = true: the real flavor (real M, real symmetric chi of doubles).
int chi_run(Ctx* c, int prec, int nv, int nc, int ng, const void* M, const double* d_ev,
            const double* d_ec, int nfreq, const double* d_omega, double scale, int accumulate,
            void* chi, cudaStream_t st, const HeadPlan* hp = nullptr, const double2* h = nullptr,
            bool real = false);
// eps~ and its inverse for nmat matrices (per-matrix size, cell and q).
// tc_update: the sweep's trailing updates run on the tensor cores with
// FP64-level accuracy (sweep_tc.cu) instead of FP64 FMA.
int epsinv_batch_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells,
                     const int32_t* const* d_geps, const void* const* chi, void* const* eps, void* const* epsinv,
                     cudaStream_t st, bool tc_update, bool real_values = false);
// eps~ = I - sv chi sv of one matrix into A (and eps when non-NULL), sv from
// the cell's Coulomb model (epsinv.cu).
int eps_form_run(Ctx* c, const bgw_cell* cell, const int32_t* d_geps, int ng, const void* chi, double* sv,
                 double2* A, void* eps, cudaStream_t st);
// FP64 FMA trailing update of one general Gauss-Jordan step on columns
// k0..k0+kb (kb <= 32): rows of K become R [32][ng], the others
// A_ij = (j in K ? 0 : A_ij) - (Cp R)_ij with Cp [ng][32].
int gj_update_run(Ctx* c, double2* A, int ng, int k0, int kb, const double2* R, const double2* Cp,
                  cudaStream_t st);
// General (non-Hermitian) eps~ and its inverse with partial pivoting
// (epsinv_general.cu), one matrix after the other.
// tc_update: the trailing updates on the tensor cores (Ozaki split, FP64-level
// accuracy) instead of FP64 FMA.
int epsinv_general_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells, const int32_t* const* d_geps,
                       const void* const* chi, void* const* eps, void* const* epsinv, cudaStream_t st,
                       bool tc_update = false);
constexpr int kGeneralMaxNg = 14336;   // row of the column unscramble in shared memory
// Real-axis chi (chi.cu): complex weights of Eq. retarded_advanced_epsilon.
int chi_real_run(Ctx* c, int prec, int nv, int nc, int ng, const void* M, const double* d_ev, const double* d_ec,
                 int nfreq, const double* d_energy, double delta, int advanced, double scale, int accumulate,
                 void* chi, cudaStream_t st);
// Real flavor: eps~ and its inverse of real symmetric chi (doubles in and
// out) through the Hermitian sweep on the complex embedding, whose imaginary
// parts stay exactly zero.
int epsinv_rflavor_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells, const int32_t* const* d_geps,
                       const void* const* chi, void* const* eps, void* const* epsinv, cudaStream_t st,
                       bool tc_update);
// sv = v(q+G)^1/2 of the cell's Coulomb model.
int coulomb_sqrt_run(Ctx* c, const bgw_cell* cell, const int32_t* d_geps, int ng, double* sv, cudaStream_t st);
// Diagonal static COHSEX and bare exchange for one q (sigma.cu); pp_neg is the
// pair plan of the negated epsilon list; sigma_host [4][no].
int sigma_run(Ctx* c, const bgw_cell* cell, int n, int no, const BandPlan* bpo, const int32_t* go, const void* co,
              int ni, const BandPlan* bpi, const void* ci, int nocc, int ng, const int32_t* geps_host,
              const int32_t* d_geps, const PairPlan* pp_neg, const void* epsinv, int prec, double* sigma_host,
              cudaStream_t st);
// C[p][g] = sum_k X[p][k] Y[g][k] on the tensor cores (chi_tc.cu): X complex64
// [R1][K], Y complex128 [R2][K], C complex128 [R1][R2].
int tc_rows_gemm(Ctx* c, int prec, int R1, int R2, int K, const void* X, const void* Y, void* C, cudaStream_t st);
// W = v^1/2 epsinv v^1/2 for nmat matrices (bgw_screened_w).
int screened_w_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells, const int32_t* const* d_geps,
                   const void* const* epsinv, void* const* W, cudaStream_t st);
// Host check of a cell's Coulomb model against its G list: BGW_OK, or
// BGW_EINVAL with *what = 1 (unknown model), 2 (bad cut length) or
// 3 (v diverges at geps[*bad]).
int coulomb_check(const bgw_cell* cell, int ng, const int32_t* geps, int* what, int* bad);

// Tensor-core trailing update of the sweep (sweep_tc.cu).
struct OzPlan;
OzPlan* oz_plan_new();
void oz_plan_delete(OzPlan* p);
// general = false: the Hermitian sweep's update (C, P: [ng][32] panels, D
// the next diagonal inverse).  general = true: the pivoted Gauss-Jordan
// update A -= P R with P the column panel [ng][32] and C = R [32][ng].
// real_values: every matrix is real (the real flavor's embedding), so only
// the real-part products are formed.
// slices: 7 (update error near 2^-48 of its scale) or 5 (near 2^-34).
// ff_chain: the next diagonal block and the panel product in double FP32
// (about 2^-46), the FP64-level class of the seven-slice update, on the
// FP32 pipe (GB300's FP64 pipe is 64 times slower); five slices imply it.
int oz_prepare(Ctx* c, int nmat, const int* ng, double2* const* A, const double2* const* C, const double2* const* P,
               double2* const* D, OzPlan* plan, bool general, bool real_values, int slices, bool ff_chain);
// epsinv_batch_run with real_values: the matrices are real (imaginary parts zero).
// Slices of one pivoted Gauss-Jordan step (general plans).
int oz_slice(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, cudaStream_t st);
// The Hermitian sweep's panel (C, P = C D^-1, A_RK <- P) and its slices in one launch.
int oz_panel_slice(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, cudaStream_t st);
int oz_update(Ctx* c, OzPlan* plan, int k0, int ngmax, int buf, int mode, cudaStream_t st);
// Column tiles per work item of the bulk update launches (modes 0, 2, 3)
// that follow: -1 the SM-count rule (items of 2 tiles where the slice
// count's wider items would number no more than the SMs), 0 the wider
// items, 1 items of 2 tiles.  Every tile's arithmetic is the same either
// way (bit-identical results); only the speed changes.
void oz_set_bulk_items(OzPlan* plan, int narrow);

}  // namespace bgw

struct bgw_ctx {
  bgw::Ctx impl;
  explicit bgw_ctx(uint64_t budget) : impl(budget) {}
};
