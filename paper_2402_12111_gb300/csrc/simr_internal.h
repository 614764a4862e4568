// simr_internal.h -- host-side launch descriptors shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "simr.h"
#include "simr_device.cuh"

namespace simr {

// Accumulator slot of each Greek bit, in bit order (slot 0 = sum f, 1 = sum f^2).
constexpr int kMaxGreeks = 9;
constexpr int kMaxResim = 6;  // vega, theta, kappa, long-run var, vol-of-vol, correlation

// Everything one launch of the fused path kernel needs, passed by value
// (kernel parameter space; all of it is uniform over the grid).
struct PathLaunch {
  uint32_t rk[10][2];     // Philox round keys
  uint64_t path_begin;    // first path index
  uint64_t path_count;    // paths in this launch
  uint32_t steps;
  uint32_t option_index;  // fourth counter word
  int32_t n_scen;         // simulated scenarios (base first)
  int32_t n_strikes;
  int32_t nk_pad;         // strikes rounded up to the tile width (1 or multiple of 32)
  int32_t n_acc;          // accumulators per strike = 2 + number of Greeks
  int32_t is_put;
  uint32_t greek_mask;
  float S0;
  float h_s;              // relative S0 bump (delta, gamma)
  double rho_em;          // e^{-h_r T}: strike factor of the r-up revaluation
  double rho_w;           // e^{h_r T} - e^{-h_r T} = 2 sinh(h_r T): band width factor
  int32_t resim_up[kMaxResim], resim_dn[kMaxResim];  // scenario of each re-simulated Greek
  ScenConst sc[kMaxScen];
  ScenConst2 pair2[kMaxScen / 2];  // scenarios (2k + 1, 2k + 2): their constants (deltas) lane by lane
  FirstConst f0[kMaxScen];  // step-0 constants (used when first_split != 0)
  int32_t first_split;      // 1: step 0 of every scenario through step0_crn
  int32_t n_v0_scen;        // 2: scenarios 1 and 2 are the up/down v0 bumps (no constant deltas)
  // finalisation (FP64)
  double disc;            // e^{-rT}
  double paths_total;     // denominator of the mean
  double denom[kMaxGreeks];  // per Greek: bump denominator (sign folded in)
  int32_t raw_sums;       // 1: write raw sums instead of normalised results
  int32_t scheme;         // 0: QE; 1: QE-M
  QemConst qm;            // QE-M constants of the base scenario
  QemConst qmd[kMaxScen]; // QE-M: the bumped scenarios' constant deltas to qm (qmd[0] zero)
  QemConst2 qmd2[kMaxScen / 2];  // QE-M: scenarios (2k + 1, 2k + 2): their deltas lane by lane
};

// Counters of the generator's raw words: paths [path_begin, path_begin + n_paths)
// x step pairs [pair_begin, pair_begin + n_pairs) of option option_index.
struct DrawLaunch {
  uint32_t rk[10][2];
  uint64_t path_begin, n_paths;
  uint32_t pair_begin, n_pairs, option_index;
};

struct PathOutputs {
  double* price;   // [n_strikes]
  double* stderr_; // [n_strikes] or null
  double* greeks;  // [n_strikes][n_greeks] or null
  double* sums;    // raw mode: [n_strikes][n_acc]
  int* status;     // device status word: bit 0 = invalid strike seen
};

// Constants of the adjoint kernel: checkpointing, and the FP64-derived
// derivatives of the per-step constants with respect to the parameters.
// The map from the sweep's sums to the parameters runs once per path in FP64:
// the kappa sensitivity, for one, is a small residual of much larger terms.
struct AdjConst {
  int32_t ckpt_every;  // even, >= 2
  int32_t n_seg;       // ceil(steps / ckpt_every)
  float theta, invS0, T;
  double dE_dk, omE, dc1_dk, dc2_dk, dc2_dth;
  double dCd_dk, dCdl_dk, N_Cd;
  double two_over_sigma, c1, c2, Cd_over_sigma, Cdl_over_sigma;
  double D_over_sigma, B_over_sigma, dsK3_drho;
  // QE-M (scheme 1): the log-spot step r dt - qa (v + m) - lam(A) + K2 (v' - m) + sK3 sqrt(v + v') Z_X
  // on the steps where the correction exists, the plain step on the others; derivatives of
  // qa = dt (1 - rho^2)/4, K2 and A = K2 + qa with respect to kappa, sigma, rho, and Cd for the
  // plain steps' C0 = r dt + Cd theta
  int32_t qem;
  double Cd, dqa_drho, dK2_dk, dK2_ds, dK2_dr, dA_dk, dA_ds, dA_dr;
};

// Shared floats per thread of the per-path adjoint with checkpoints in shared
// memory: n_seg checkpoints and a segment buffer of 3 k floats (state, branch
// draw, Z_X) per path.
__host__ __device__ inline int adjoint_thread_floats(int n_seg, int k, int ppt) { return (n_seg + 3 * k) * ppt; }

struct AdjOutputs {
  double* price;    // [n_strikes]
  double* stderr_;  // [n_strikes] or null
  double* grad;     // [n_strikes][7]: S0, v0, kappa, theta, sigma, rho, r
  int* status;
};

// One option of a batched book (device table, longest first).
struct BatchOption {
  ScenConst sc;             // base scenario constants
  AdjConst A;               // adjoint constants (adjoint books)
  QemConst qm;              // QE-M constants (books under scheme QE-M)
  float S0, K, invS0, T;
  int32_t is_put;
  uint32_t steps;
  uint32_t option_index;    // position in the caller's array: output slot and Philox counter word
  uint32_t item_begin, item_count;
  uint32_t pad;
  uint64_t paths;
  double disc;
};

// A work item: `count` consecutive paths of one option, for one warp.
struct BatchItem {
  uint32_t option;  // index into the BatchOption table
  uint32_t count;
  uint64_t path_begin;
};

struct BatchLaunch {
  uint32_t rk[10][2];
  uint32_t n_items, n_opts;
  int32_t adjoint;
  int32_t ckpt_rows;  // adjoint: checkpoint rows per thread column (max over options of n_seg - 1), even
  int32_t seg_rows;   // adjoint: rows of each segment array (max over options of ckpt_every)
  float* gseg;        // adjoint with one segment per path: [3 seg_rows][grid threads] in global memory, else null
  size_t gseg_floats;  // its capacity
  int32_t tpb, ppt, unroll;  // the kernel's shape (batch_variant)
  int32_t qem;               // 1: the options' log-spot steps under QE-M
};

struct BatchOutputs {
  double* price;    // [n_opts] in the caller's order
  double* stderr_;  // [n_opts] or null
  double* grad;     // [n_opts][7] or null
};

struct Scratch {
  double* partials;      // [grid][n_acc * nk_pad]
  unsigned int* ticket;  // zero between launches
  size_t partial_doubles;
  float* ckpt = nullptr;  // adjoint checkpoints in global memory
  size_t ckpt_floats = 0;
  float* gseg = nullptr;  // adjoint segment buffers in global memory (segments too long for shared memory)
  size_t gseg_floats = 0;
};

// Host-side fault injection (simr_inject_fault): true when this request of the
// given kind is the one armed to fail (and disarms it).
bool take_fault(int what);

// Launch the fused price / Greeks kernel; returns a cudaError_t.
cudaError_t launch_paths(const PathLaunch& L, const double* strikes_dev, const PathOutputs& out,
                         const Scratch& s, int num_sms, cudaStream_t stream, int* grid_used);

// Upper bound of the partial-sum doubles launch_paths needs for this shape.
size_t paths_scratch_doubles(const PathLaunch& L, int num_sms);

// Normalise combined raw sums [n_strikes][n_acc] into the outputs.
cudaError_t launch_finalize(const PathLaunch& L, const double* sums, const PathOutputs& out, cudaStream_t stream);

// Pathwise adjoint Greeks (price + 7 sensitivities per strike).
cudaError_t launch_adjoint(const PathLaunch& L, const AdjConst& A, const double* strikes, const AdjOutputs& out,
                           const Scratch& s, int num_sms, cudaStream_t stream);
size_t adjoint_scratch_doubles(const PathLaunch& L, int num_sms);
size_t adjoint_smem_bytes(const PathLaunch& L, const AdjConst& A);
// Dynamic shared memory one block of an adjoint kernel may ask for.
constexpr size_t kAdjMaxSmem = 200 * 1024;
// Largest global segment buffer of the per-strike adjoint (8 GB), and the
// largest the automatic interval takes (4 GB).
constexpr size_t kAdjMaxGsegFloats = (size_t)1 << 31;
constexpr size_t kAdjAutoGsegFloats = (size_t)1 << 30;
// The largest even checkpoint interval (at most steps_cap, rounded up to even)
// at which the per-strike adjoint kernel for L's strike count keeps the blocks
// per SM it has at interval 2 (its register limit): each thread's segment
// buffer is 3 k floats of shared memory.
cudaError_t adjoint_max_ckpt_every(const PathLaunch& L, int steps_cap, int* k_max);
size_t adjoint_ckpt_scratch_floats(const AdjConst& A, int num_sms);
// Floats of the global segment buffers the per-strike adjoint launch needs (0
// when its segments fit in shared memory): 3 k per thread of its grid.
cudaError_t adjoint_gseg_floats(const PathLaunch& L, const AdjConst& A, int num_sms, size_t* floats);
// Per-path x_T and d x_T / d(v0, kappa, theta, sigma, rho) ([n][5]).
cudaError_t launch_paths_adjoint(const PathLaunch& L, const AdjConst& A, float* x_T, float* grad, cudaStream_t stream);

// Batched book: queue counter reset, persistent kernel, per-option reduction.
cudaError_t launch_batch(const BatchLaunch& B, const BatchOption* opts, const BatchItem* items, unsigned int* counter,
                         double* partials, const BatchOutputs& out, int num_sms, cudaStream_t stream);
cudaError_t prepare_batch(const BatchLaunch& B);  // kernel attributes (outside any stream capture)
// Threads of the adjoint book kernel's grid when its segments are in global
// memory (the largest over the kernel shapes).
cudaError_t batch_gseg_threads(int num_sms, size_t* threads);
// Kernel shape v of a book, v in [0, kBatchVariants): threads per block 128 /
// 256 (bit 0); price books: paths per thread 2 / 1 (bit 1), step-pair loop
// unrolled 1 / 2 times (bit 2); adjoint books use bit 0 only.
constexpr int kBatchVariants = 8;
void batch_variant(int v, bool adjoint, BatchLaunch* B);  // reads B->qem

// Terminal (x_T, v_T) per path of scenario 0.
cudaError_t launch_terminal(const PathLaunch& L, float* x_T, float* v_T, cudaStream_t stream);
cudaError_t launch_philox_words(const DrawLaunch& D, uint32_t* words, cudaStream_t stream);
cudaError_t launch_normals(const uint32_t* words, uint64_t n, float* z, float* zp, cudaStream_t stream);

// Longstaff-Schwartz (simr_lsm.cu).  Exercise dates t_j = (j + 1) every dt,
// j = 0 .. n_ex - 1; per-path states at the dates in [date][path] arrays.
struct LsmLaunch {
  uint32_t rk[10][2];
  ScenConst sc;        // base scenario constants (v0 included)
  float S0, K;         // spot, strike
  int32_t is_put, n_ex, every, min_itm;
  uint32_t steps, option_index;
  uint64_t paths;
  uint64_t pitch;      // floats per date row of the states: paths rounded up to a multiple of 4 (16 bytes)
  double disc0;        // e^{-r t_0}
  double Kd, wd;       // strike and basis scale w in FP64 (coefficient conversion)
  int32_t scheme;      // 0: QE; 1: QE-M
  QemConst qm;
  int32_t barrier_extra;  // 0; 1 (fault injection): the sweep's first grid barrier waits for a block too many
};

struct LsmBuffers {
  float* S;            // [n_ex][pitch], the first `paths` of each row used
  float* V;            // [n_ex][pitch]
  float* cash;         // [paths] payoff at the exercise date (0: never exercised)
  int32_t* stop;       // [paths] exercise date, -1 = never
  double* beta;        // [n_ex][6] in the basis (1, x, x^2, y, xy, y^2); NaN row = no regression
  double* beta_t;      // [n_ex][6] the same fit in the date's scaled basis (what the kernels use)
  const float4* xform; // [n_ex] scaled coordinates of date j: xs = a S + b, ys = p v + q
  const float* dpow;   // [n_ex] e^{-r k (t_1 - t_0)}, k = 0 .. n_ex - 1
  double* partials;    // [grid][21] (cooperative sweep: [2][grid][21] double-float pairs)
  unsigned int* ticket;  // last-block ticket; words 4 and 8 after it: sweep barrier count, generation
  int* status;         // bit 1 set when a sweep barrier wait timed out
  double* price;       // [1]
  double* stderr_;     // [1] or null
};

// All launches of one Longstaff-Schwartz valuation on `stream`: the path
// kernel, then the backward induction as one cooperative launch (or, where
// that is not possible, one kernel per exercise date; the last reduces the price).
cudaError_t launch_lsm(const LsmLaunch& L, const LsmBuffers& B, int num_sms, cudaStream_t stream);
size_t lsm_partial_doubles(int num_sms);

// simr_rates.cu: throughput of the FP32 FMA (scalar, packed), MUFU rsqrt,
// 32 x 32 -> 64 multiply and FP64 FMA units, then the elapsed ms (rates[6]).
cudaError_t measure_unit_rates(int num_sms, float* scratch, cudaStream_t st, double* rates);
size_t unit_rates_scratch_floats(int num_sms);

// Basket options on correlated assets (simr_basket.cu).
constexpr int kMaxAssets = 16;

struct BasketLaunch {
  uint32_t rk[10][2];
  ScenConst sc[kMaxAssets];                          // per asset (v0 included)
  ScenConst2 pk[kMaxAssets / 2];                     // assets (2q, 2q + 1) packed lane by lane
  float Lc[kMaxAssets * (kMaxAssets + 1) / 2];       // lower Cholesky factor, rows packed
  float S0w[kMaxAssets];                             // S0_k w_k
  int32_t n_assets, n_strikes, nk_pad, is_put;
  uint32_t steps;
  int32_t scheme;                                    // 0: QE; 1: QE-M
  uint64_t paths;
  double disc, paths_total;
  QemConst qm[kMaxAssets];                           // QE-M constants per asset
  QemConst2 qk[kMaxAssets / 2];                      // the same, assets (2q, 2q + 1) packed lane by lane
};

struct BasketOutputs {
  double* price;    // [n_strikes]
  double* stderr_;  // [n_strikes] or null
  int* status;      // bit 0: a device strike was not finite and >= 0
};

cudaError_t launch_basket(const BasketLaunch& L, const double* strikes, const BasketOutputs& out, double* partials,
                          size_t partial_doubles, unsigned int* ticket, int num_sms, cudaStream_t stream);
size_t basket_partial_doubles(const BasketLaunch& L, int num_sms);

// Validation and launch building of the C ABI (simr_api.cu), for the other
// entry points of the library.  They set the thread-local error message.
int internal_fail(int code, const char* message);
int internal_cuda_fail(cudaError_t e, const char* what);
int internal_check_price_args(const simr_heston* model, const double* strikes, int n_strikes, int max_strikes,
                              uint32_t steps, uint64_t paths);
bool internal_is_device_ptr(const void* p);
int internal_build_price_launch(const simr_heston* model, int n_strikes, int is_put, uint32_t steps, uint64_t paths,
                                uint64_t seed, uint32_t option_index, PathLaunch* L);

}  // namespace simr
