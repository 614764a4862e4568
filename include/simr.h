/*
 * simr.h -- C ABI of the GB300 Heston Monte Carlo pricing library (libsimr.so).
 *
 * The library implements the data-parallel hot path of the SIMR (STAC-A2
 * inspired market risk) workload studied in "Evaluating Versal AI Engines for
 * option price discovery in market risk analysis" (Klaisoongnoen et al.,
 * FPGA'24): per path and per time step the VariancePathQE stage (Sec. 4), the
 * LogPricePathQE and AssetPathExponential stages (Sec. 5, Fig. 1), and the
 * reduction over paths (Sec. 6), over the assets x timesteps x paths loop nest
 * of Sec. 5.1 (Listing 2) with the per-path state carried between timesteps.
 * The paper names the stages but prints no formula; the scheme is the
 * Quadratic-Exponential (QE) discretisation of L. Andersen (J. Comput. Finance
 * 11(3), 2008) of the Heston (1993) model under the risk-neutral measure with a
 * constant rate r and no dividends: psi_c = 1.5, gamma1 = gamma2 = 1/2.
 * The paper's random inputs V and Z (Sec. 3, Table 1: two FP32 data points per
 * element) are generated in-kernel by Philox4x32-10 (Salmon et al., SC'11):
 *   key     = (seed mod 2^32, seed >> 32)
 *   counter = (step / 2, path mod 2^32, path >> 32, option_index)
 *   words 0,1 drive even steps and words 2,3 odd steps: (U_V, U_X)
 *   u       = ((word >> 9) + 1/2) * 2^-23, Z = Phi^-1(u).
 * A result therefore depends only on (seed, option, path, step), never on the
 * launch configuration, and shards of a path range agree with the whole.
 * Path arithmetic is FP32 (the paper's SIMR precision, Sec. 3); sums over paths
 * and the final normalisation are FP64.
 *
 * Conventions for every entry point:
 *  - Return 0 (SIMR_OK) or a negative simr_status; simr_last_error() gives a
 *    thread-local message for the last failure on the calling thread.
 *  - Arguments are validated on the host before anything is launched; an
 *    invalid argument returns SIMR_EINVAL and writes nothing.  The one
 *    exception is a strike array in device memory, which the kernel checks:
 *    a strike that is not finite and > 0 yields NaN results for that strike
 *    and sets a device status that simr_sync returns as SIMR_EINVAL.
 *  - Array arguments are plain pointers to caller-owned memory, either device
 *    memory of the context's device or host memory (detected per pointer).
 *    With device pointers the call is asynchronous on `stream` (a
 *    cudaStream_t passed as void*, NULL = legacy default stream) and the
 *    caller synchronises.  If any output pointer is host memory the call
 *    copies results back and synchronises `stream` before returning.
 *  - The library never frees caller memory.  Its own device scratch belongs to
 *    the context; calls on one context must not run concurrently on different
 *    streams (they share that scratch).
 *  - Model validity: S0, K, T > 0; v0, theta >= 0; kappa > 0; sigma > 0 (the
 *    log-spot coefficients divide by sigma); rho in [-1, 1]; all finite;
 *    steps >= 1; paths >= 1.
 *  - Every compute entry point opens an NVTX range named after itself.
 *
 * Environment read at run time: SIMR_AUTOTUNE=0 (books run without the
 * first-call search of simr_batch_submit), SIMR_TUNE_CACHE=<file> (its tuned
 * choices persist there), SIMR_LSM_SWEEP=0 (simr_lsm_price runs one kernel per
 * exercise date instead of the cooperative sweep).  At build time
 * (paper_2402_12111_gb300/build.py): SIMR_IEEE=1 builds the error-study
 * library, with correctly rounded division, square roots and log2 in place of
 * the special-function unit's approximations.
 */
#ifndef SIMR_H
#define SIMR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SIMR_API __attribute__((visibility("default")))
#else
#define SIMR_API
#endif

typedef enum {
  SIMR_OK = 0,
  SIMR_EINVAL = -1,      /* invalid argument (nothing launched)                 */
  SIMR_ENOMEM = -2,      /* device or host allocation failed                    */
  SIMR_ECUDA = -3,       /* a CUDA runtime call failed (message has the reason) */
  SIMR_ETIMEOUT = -4,    /* a device-side bounded wait gave up                  */
  SIMR_EUNSUPPORTED = -5 /* size or feature beyond what this build supports     */
} simr_status;

/* Opaque context bound to one CUDA device; owns scratch memory. */
typedef struct simr_ctx simr_ctx;

/* Model and market inputs (the paper's problem statement per asset). */
typedef struct {
  double S0;    /* spot                          */
  double r;     /* continuously compounded rate  */
  double T;     /* maturity in years             */
  double v0;    /* initial variance              */
  double kappa; /* mean-reversion speed          */
  double theta; /* long-run variance             */
  double sigma; /* volatility of variance        */
  double rho;   /* spot/variance correlation     */
} simr_heston;

/* One option of a batched book (simr_batch_submit). */
typedef struct {
  simr_heston m;   /* model and market                */
  double K;        /* strike                           */
  int32_t is_put;  /* 0 call, 1 put                    */
  uint32_t steps;  /* time steps                       */
  uint64_t paths;  /* Monte Carlo paths                */
} simr_option;

/* simr_batch_submit flags */
/* Log-spot schemes (simr_set_scheme). */
#define SIMR_SCHEME_QE 0   /* Andersen's QE, central weights, no martingale correction (default) */
#define SIMR_SCHEME_QEM 1  /* QE with Andersen's martingale correction                          */

#define SIMR_BATCH_ADJOINT (1u << 0)      /* also the 7 pathwise sensitivities per option       */
#define SIMR_BATCH_GRAPH (1u << 1)        /* capture the launch in a CUDA graph; replay on repeat */
#define SIMR_BATCH_NO_AUTOTUNE (1u << 2)  /* skip the first-call kernel-shape and chunk search   */
/* Run kernel shape v (0-7) instead of the tuned one (no search): threads per
 * block 128 / 256 (bit 0); price books: paths per thread 2 / 1 (bit 1) and the
 * step-pair loop unrolled 1 / 2 times (bit 2); adjoint books: bit 0 only (v < 2).
 * Every shape gives the same results bit for bit. */
#define SIMR_BATCH_VARIANT(v) ((((uint32_t)(v) & 7u) + 1u) << 8)

/* Greek selection bits for simr_greeks_fd; output columns follow bit order. */
#define SIMR_G_DELTA (1u << 0)  /* d/dS0, analytic S-bump on the same path   */
#define SIMR_G_GAMMA (1u << 1)  /* d2/dS0^2, same path                       */
#define SIMR_G_VEGA (1u << 2)   /* d/dv0, re-simulated                       */
#define SIMR_G_THETA (1u << 3)  /* -d/dT (calendar theta), re-simulated      */
#define SIMR_G_RHO (1u << 4)    /* d/dr, exact r-shift of the same path      */
#define SIMR_G_KAPPA (1u << 5)  /* d/dkappa, re-simulated                    */
#define SIMR_G_LRVAR (1u << 6)  /* d/dtheta (long-run variance), re-simulated */
#define SIMR_G_VOLVOL (1u << 7) /* d/dsigma, re-simulated                    */
#define SIMR_G_CORR (1u << 8)   /* d/drho, re-simulated                      */
#define SIMR_G_ALL 0x1FFu

/* Create a context on CUDA device `device`.  *out is set on success. */
SIMR_API int simr_create(simr_ctx** out, int device);

/* Destroy a context (NULL allowed).  Synchronises the device first. */
SIMR_API void simr_destroy(simr_ctx* ctx);

/* Thread-local message describing the last failure on this thread ("" if none). */
SIMR_API const char* simr_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
SIMR_API int simr_version(void);

/*
 * European price of one asset on a strike grid by Monte Carlo over paths
 * [0, paths): the stages VariancePathQE, LogPricePathQE, AssetPathExponential
 * (paper Sec. 4-5) and the reduction over paths (Sec. 6).
 *   strikes[n_strikes] (FP64)   in   strike grid, each K > 0
 *   is_put                      in   0 call, 1 put (payoff zero at S_T = K)
 *   price[n_strikes]            out  e^{-rT} mean_p f_k(S_T)
 *   stderr_out[n_strikes]       out  e^{-rT} sqrt((mean f^2 - mean(f)^2)/(paths-1)); may be NULL
 * n_strikes in [1, 1024].  option_index is the fourth Philox counter word (use 0
 * for a single asset; distinct assets of one book use distinct indices).
 */
SIMR_API int simr_price(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes,
               int is_put, uint32_t steps, uint64_t paths, uint64_t seed, uint32_t option_index,
               double* price, double* stderr_out, void* stream);

/*
 * Bump-and-revalue Greeks with common random numbers: every scenario reuses the
 * Philox counters of the base paths.  Central differences with bump
 * h = rel_bump * |value| (rel_bump itself when the value is 0; rho is bumped by
 * rel_bump in absolute terms); where the down-bump leaves the domain (v0 or theta
 * below 0, rho outside [-1, 1]) the one-sided difference is used.
 * Delta and gamma re-value the same path at S0(1 +- h) (x_T does not depend on
 * S0); rho shifts x_T by the exact r-dependence of the log-spot step (+- h T)
 * and the discount; vega, theta, kappa, long-run variance, vol-of-vol and
 * correlation re-simulate every step with the bumped constants.
 *   greek_mask   in   SIMR_G_* bits, at least one
 *   price[n_strikes]                out  base price
 *   greeks[n_strikes * n_greeks]    out  row-major [strike][greek], greeks in bit order
 * n_strikes in [1, 256].
 */
SIMR_API int simr_greeks_fd(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes,
                   int is_put, uint32_t steps, uint64_t paths, uint64_t seed, uint32_t option_index,
                   double rel_bump, uint32_t greek_mask, double* price, double* greeks,
                   void* stream);

/*
 * Pathwise adjoint (reverse-mode) Greeks: the price and its sensitivities to
 * (S0, v0, kappa, theta, sigma, rho, r) per strike from ONE kernel launch.  Per
 * path, a forward pass (the paper's VariancePathQE and LogPricePathQE stages,
 * Sec. 4-5) keeps the variance every ckpt_every steps; a reverse sweep
 * recomputes each segment from its checkpoint (regenerating the segment's
 * Philox draws) and differentiates the steps backwards with the forward
 * branches held fixed.  dP/dq = e^{-rT} mean[f'(S_T) S_T dx_T/dq] with
 * f' = 1{S_T > K} (call) or -1{S_T < K} (put); dP/dS0 = e^{-rT} mean[f' S_T/S0];
 * dP/dr = e^{-rT} mean[f' S_T T] - T P.  Pathwise derivatives miss the jump of
 * the QE map where a bump would switch a path's branch, so they differ from
 * bump-and-revalue by that (small) term.
 *   ckpt_every   in   even number of steps per checkpoint segment, in [2, 1024];
 *                     values above steps act as steps (rounded up to even): one
 *                     segment, no forward pass.  Each resident thread keeps
 *                     steps/ckpt_every checkpoints in a context-owned device
 *                     buffer (at most 2^30 floats in all) and a segment buffer
 *                     of 3 ckpt_every floats: in shared memory while a
 *                     128-thread block's buffers and accumulators fit 200 KB,
 *                     else in a context-owned device buffer (at most 2^31
 *                     floats in all; SIMR_EUNSUPPORTED beyond).
 *                     0 = the library's choice for speed (the forward pass runs
 *                     all segments but the last): one segment of the whole
 *                     path when its buffer fits shared memory or 2^30 floats of
 *                     device memory; else, among the even intervals whose
 *                     shared memory keeps the kernel's blocks per SM (found
 *                     once per context by the occupancy API), the one with the
 *                     longest last segment.
 *   price[n_strikes], stderr_out[n_strikes] (nullable)   out
 *   grad[n_strikes * 7]   out  row-major [strike][S0, v0, kappa, theta, sigma, rho, r]
 * n_strikes in [1, 256].  The rho column is NaN when |rho| = 1 (the pathwise
 * derivative of sqrt(1 - rho^2) does not exist there).
 */
SIMR_API int simr_greeks_adjoint(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes,
                                 int is_put, uint32_t steps, uint64_t paths, uint64_t seed,
                                 uint32_t option_index, uint32_t ckpt_every, double* price, double* stderr_out,
                                 double* grad, void* stream);

/*
 * Fault injection, for tests of the error paths.  On the host (nothing reaches
 * the GPU): the after-th next request of this process for context scratch memory
 * (what = SIMR_FAULT_ALLOC; allocated or reused) or for a kernel launch (what =
 * SIMR_FAULT_LAUNCH) fails as if the CUDA call had failed -- the entry point that
 * meets it returns SIMR_ENOMEM or SIMR_ECUDA and leaves the context usable.
 * what = SIMR_FAULT_BARRIER: the after-th next cooperative Longstaff-Schwartz
 * sweep waits at its first grid barrier for one block more than its grid holds,
 * so that bounded wait runs out (0.25 s); the sweep's blocks leave, the device
 * status reports SIMR_ETIMEOUT (simr_sync, or the call itself with host outputs)
 * and the context stays usable.  No memory access changes; a valuation that runs
 * per-date launches instead of the sweep consumes the injection unaffected.
 * what = 0 disarms.  after in [1, 2^30].  SIMR_EINVAL otherwise.
 */
#define SIMR_FAULT_ALLOC 1
#define SIMR_FAULT_LAUNCH 2
#define SIMR_FAULT_BARRIER 3
SIMR_API int simr_inject_fault(int what, int after);

/*
 * The checkpoint interval simr_greeks_adjoint takes for ckpt_every = 0 with
 * n_strikes strikes (in [1, 256]) and `steps` time steps, in *ckpt_every.
 */
SIMR_API int simr_adjoint_interval(simr_ctx* ctx, int n_strikes, uint32_t steps, uint32_t* ckpt_every);

/*
 * A heterogeneous book of European options in one persistent launch: every
 * option has its own model, strike, steps and paths; option i uses Philox
 * counter word 3 = i (so its paths are those of simr_price with option_index i).
 * The library cuts each option's paths into work items of `chunk` paths,
 * longest options first; the kernel's warps take items from an atomic queue
 * (the paper's multi-CU replication, Sec. 6, as dynamic load balancing over one
 * GPU's SMs) and a second kernel sums each option's item rows in a fixed order.
 *   opts[n_opts]   in   HOST array; n_opts in [1, 2^22]
 *   flags          in   SIMR_BATCH_* (0 = prices only)
 *   price[n_opts], stderr_out[n_opts] (nullable)   out, caller's order
 *   grad[n_opts * 7]   out (SIMR_BATCH_ADJOINT): d/d{S0, v0, kappa, theta, sigma, rho, r}
 * The kernel's shape and the chunk are chosen by timing on the first submission
 * of each book shape (a book's size class): first the eight kernel shapes of
 * SIMR_BATCH_VARIANT (two for adjoint books) at the default chunk, then, with
 * the fastest shape, four chunks: 1024/4096/16384 paths (256/1024/4096 with the
 * adjoint) and the size that gives about two items per resident warp -- that
 * first call prices the book up to twelve more times.  The choice is cached in
 * the context and, when the environment variable SIMR_TUNE_CACHE names a file,
 * appended there as a JSON line {"gpu", "key", "chunk", "variant", ...} and read
 * back by later processes on a GPU of the same name.  Without tuning: shape 0
 * and the smaller of 4096 (1024) and that size.  Adjoint books keep every
 * path whole (one segment, no forward pass) in a context-owned device buffer of 3 x (the longest
 * option's steps) floats per resident thread when the longest option has at most 1,024 steps and the
 * buffer fits 2^30 floats; otherwise checkpoints and segments in shared memory as simr_paths_adjoint
 * chooses them.  With SIMR_BATCH_GRAPH the upload-free part
 * of the call (queue reset, batch kernel, reduction) is captured once per
 * (book, seed, flags, output buffers) and replayed afterwards.
 */
SIMR_API int simr_batch_submit(simr_ctx* ctx, const simr_option* opts, int n_opts, uint64_t seed, uint32_t flags,
                               double* price, double* stderr_out, double* grad, void* stream);

/*
 * Per-path pathwise derivatives: for paths [path_begin, path_begin + n_paths),
 * x_T[i] = ln(S_T/S0) and grad[i * 5 + j] = d x_T / d(v0, kappa, theta, sigma,
 * rho)[j] (FP32), by the same forward pass and reverse sweep as
 * simr_greeks_adjoint (dx_T/dS0 = 0 and dx_T/dr = T need no sweep).  Custom
 * payoffs g(S_T) get dE[g]/dq = E[g'(S_T) S_T dx_T/dq].  Device pointers only.
 * ckpt_every as in simr_greeks_adjoint, except that 0 = the even interval near
 * sqrt(steps / 3), the one that needs the least shared memory: here the
 * checkpoints too are kept there (steps/ckpt_every + 3 ckpt_every floats per
 * thread, at most 200 KB per 128-thread block).
 */
SIMR_API int simr_paths_adjoint(simr_ctx* ctx, const simr_heston* model, uint32_t steps, uint64_t path_begin,
                                uint64_t n_paths, uint64_t seed, uint32_t option_index, uint32_t ckpt_every,
                                float* x_T, float* grad, void* stream);

/*
 * Basket option on n_assets correlated Heston assets: e^{-rT} mean of
 * max(+-(B_T - K), 0), B_T = sum_k weights[k] S_T,k, per strike.  Each asset runs
 * the QE scheme of simr_price with its own model and the Philox counters of
 * option index k (so with the identity correlation asset k's path is simr_price's
 * path of option k), except that its log-spot normal is
 * z_k = sum_{j <= k} Lc[k][j] eps_j, eps_j = Phi^-1(U_X) of asset j, Lc the lower
 * Cholesky factor of corr; the variance drivers stay independent.  The paper's A
 * assets (Sec. 5, Table 1) are the independent case.
 *   assets[n_assets]        in  host; all share r and T; n_assets in [1, 16]
 *   corr[n_assets^2]        in  host, row-major correlation of the spot drivers:
 *                                symmetric, unit diagonal, positive definite
 *   weights[n_assets]       in  host, finite (negative allowed: spreads, exchange)
 *   strikes[n_strikes]      in  host or device, finite and >= 0; n_strikes <= 1024
 *   price, stderr_out (nullable)  out  [n_strikes], host or device
 * Under SIMR_SCHEME_QEM each asset takes the QE-M log-spot step with its own
 * martingale correction.
 */
SIMR_API int simr_basket_price(simr_ctx* ctx, const simr_heston* assets, int n_assets, const double* corr,
                               const double* weights, const double* strikes, int n_strikes, int is_put,
                               uint32_t steps, uint64_t paths, uint64_t seed, double* price, double* stderr_out,
                               void* stream);

/*
 * Select the log-spot scheme of the context's later path simulations.
 *   SIMR_SCHEME_QE   Andersen (2008) QE, psi_c = 1.5, gamma1 = gamma2 = 1/2 (the
 *                    stages VariancePathQE / LogPricePathQE of the paper, Sec. 4-5).
 *   SIMR_SCHEME_QEM  the same variance step; the log-spot step with Andersen's
 *                    martingale correction: K0 - r dt replaced by
 *                    K0* = -ln M - (K1 + K3/2) v, M = E[exp(A v(t+dt)) | v(t)],
 *                    A = K2 + K4/2 (the plain step where M does not exist), so
 *                    that the discounted spot is an exact martingale of the scheme.
 * QE-M applies to simr_price, simr_paths_terminal, simr_lsm_price,
 * simr_greeks_fd / simr_path_sums (every Greek: each re-simulated scenario takes
 * the QE-M step on its own moments and A, the deltas of its constants to the base
 * scenario's entering as separate sums as under QE, step 0 on FP64 first-step
 * constants r dt - qa (v0 + m0) - lam(v0)), simr_greeks_adjoint /
 * simr_paths_adjoint (the reverse step also differentiates lam = ln M - A m and
 * the constants qa = dt (1 - rho^2)/4, K2 and A) and simr_batch_submit (price
 * books then have two kernel shapes, SIMR_BATCH_VARIANT 0 and 1: two paths per
 * thread, no unrolling) and simr_basket_price (each asset its own correction:
 * its log-spot normal is independent of its own variance path).
 * simr_price_noalloc is always QE.  SIMR_EINVAL for an unknown scheme.
 */
SIMR_API int simr_set_scheme(simr_ctx* ctx, int scheme);

/*
 * Longstaff-Schwartz (least-squares Monte Carlo) price of a Bermudan call or
 * put on paths [0, paths) of the simulation of simr_price (same seed,
 * option_index and Philox counters) -- the paper's writeLongstaffSchwartzPath and
 * longstaffSchwartzPathReduction stages (Sec. 5, Fig. 1; a reduction across
 * paths with dependencies between them, Sec. 6), with the method of Longstaff
 * and Schwartz (2001):
 *   exercise dates t_j = (j + 1) exercise_every dt, j = 0 .. n_ex - 1,
 *   n_ex = steps / exercise_every (none at t = 0; the last is the maturity);
 *   backwards from t_{n_ex-2}: over the paths with a positive payoff h at t_j,
 *   least squares of the cash flow they realise later, discounted to t_j, on
 *   the basis (1, x, x^2, y, x y, y^2), x = S/K - 1, y = v/w - 1,
 *   w = (v0 + theta)/2 (1 if 0), fitted in per-date standardised coordinates
 *   (the same quadratics with order-one Gram entries): normal equations by FP32
 *   Cholesky with one step of refinement against an FP64 residual, a basis
 *   function left out when its pivot is not above 1e-5 of its diagonal entry
 *   (FP32's resolution; non-degenerate fits have pivots near 0.05 or above);
 *   fewer than 12 such paths: no exercise at that date; a path
 *   exercises where h > the fitted continuation value (FP32);
 *   price = mean of e^{-r t_stop} h(t_stop) (0 if never exercised).
 *   K, is_put         in   strike (finite, > 0), 0 = call
 *   exercise_every    in   >= 1, divides steps; n_ex <= 8192
 *   paths             in   [2, 2^31]; n_ex * paths * 8 bytes of states <= 64 GiB
 *   price[1], stderr_out[1] (nullable)    out  FP64
 *   beta[n_ex * 6] (nullable)    out  coefficients per date, row-major; NaN rows
 *                                     where no regression ran (the maturity's)
 *   stop[paths] (nullable)       out  int32 exercise date per path, -1 = never
 * Outputs may be host or device pointers (host: the call synchronises).  The
 * context owns the per-path states (8 n_ex bytes per path) between calls.
 * The backward induction runs as one cooperative launch where the GPU keeps
 * enough blocks resident (otherwise one launch per date); its grid barriers and
 * state copies are bounded waits (0.25 s): one that runs out invalidates the
 * results and is reported as SIMR_ETIMEOUT by this call (host outputs) or the
 * next simr_sync.
 */
SIMR_API int simr_lsm_price(simr_ctx* ctx, const simr_heston* model, double K, int is_put, uint32_t steps,
                            uint32_t exercise_every, uint64_t paths, uint64_t seed, uint32_t option_index,
                            double* price, double* stderr_out, double* beta, int32_t* stop, void* stream);

/*
 * The random inputs the path kernels draw -- the paper's V and Z, which it
 * streams from the host (Sec. 3 Table 1, Sec. 4) -- computed by the kernels' own
 * device functions, for checking the generator word by word.
 *
 * simr_philox_words: Philox4x32-10 (Salmon et al., SC'11; 10 rounds, multipliers
 * 0xD2511F53, 0xCD9E8D57, Weyl key increments 0x9E3779B9, 0xBB67AE85) of the
 * counters the path kernels use, (pair, path mod 2^32, path >> 32, option_index)
 * under the key (seed mod 2^32, seed >> 32): step pair `pair` of a path gives
 * words 0, 1 (U_V, U_X of step 2 pair) and 2, 3 (those of step 2 pair + 1).
 *   paths [path_begin, path_begin + n_paths), pairs [pair_begin, pair_begin +
 *   n_pairs) (pair_begin + n_pairs <= 2^32); n_paths * n_pairs in [1, 2^28].
 *   words   out   DEVICE pointer, uint32 [n_paths][n_pairs][4].
 *
 * simr_normals: the FP32 standard normal of each 32-bit word w, as the path
 * kernels form it: x = 2u - 1 with u = ((w >> 9) + 1/2) 2^-23 (exact), then
 * Z = Phi^-1(u) by M. Giles' single-precision erfinv approximation (GPU
 * Computing Gems, 2011) with the special-function unit's logarithm and square
 * root.
 *   words[n] in (DEVICE), n in [1, 2^31]; z[n] out (DEVICE): one word at a time;
 *   z_paired[n] out (DEVICE, nullable): words 2j, 2j + 1 through the packed
 *   two-lane form (the same values, bit for bit, by construction).
 * Both: SIMR_EINVAL for host pointers, NULLs or sizes out of range; asynchronous
 * on `stream`.
 */
SIMR_API int simr_philox_words(simr_ctx* ctx, uint64_t seed, uint32_t option_index, uint64_t path_begin,
                               uint64_t n_paths, uint32_t pair_begin, uint32_t n_pairs, uint32_t* words,
                               void* stream);
SIMR_API int simr_normals(simr_ctx* ctx, const uint32_t* words, uint64_t n, float* z, float* z_paired,
                          void* stream);

/*
 * Measured throughput of the execution units the path kernels use -- the
 * roofline's denominators on the GPU in use (no counterpart in the paper).
 * Kernels that run one operation in long dependent chains (eight independent
 * chains per thread, 2,048 threads per SM), timed with CUDA events on `stream`
 * (which the call synchronises; about 0.1 s in all):
 *   rates[0]  FP32 FMA, scalar fma.rn.f32            TFLOP/s (2 flops per FMA)
 *   rates[1]  FP32 FMA, packed fma.rn.f32x2          TFLOP/s (4 flops per instruction)
 *   rates[2]  special-function unit, rsqrt.approx    T operations/s
 *   rates[3]  32 x 32 -> 64-bit multiply (mul.wide)  T operations/s (Philox's products)
 *   rates[4]  FP64 FMA                               TFLOP/s
 *   rates[5]  elapsed time of the whole measurement  ms
 * rates: HOST array of 6 doubles.  SIMR_EINVAL for NULL or device pointers.
 */
SIMR_API int simr_unit_rates(simr_ctx* ctx, double* rates, void* stream);

/*
 * Terminal state of paths [path_begin, path_begin + n_paths): x_T = ln(S_T/S0)
 * and v_T per path, FP32, the state the paper's writeLongstaffSchwartzPath stage
 * writes out (Sec. 5).  x_T[n_paths], v_T[n_paths] out; v_T may be NULL.
 */
SIMR_API int simr_paths_terminal(simr_ctx* ctx, const simr_heston* model, uint32_t steps,
                        uint64_t path_begin, uint64_t n_paths, uint64_t seed,
                        uint32_t option_index, float* x_T, float* v_T, void* stream);

/*
 * Raw (undiscounted) per-strike path sums over paths [path_begin, path_begin +
 * path_count) for a sharded run: sums[k * n_acc + a] with n_acc = 2 + number of
 * Greeks, a = 0: sum f, 1: sum f^2, then one sum per Greek of the per-path
 * difference the FD estimator averages.  Combine shards by adding sums, then
 * call simr_finalize_sums.  FP64 throughout the accumulation.
 */
SIMR_API int simr_path_sums(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes,
                   int is_put, uint32_t steps, uint64_t path_begin, uint64_t path_count,
                   uint64_t seed, uint32_t option_index, double rel_bump, uint32_t greek_mask,
                   double* sums, void* stream);

/*
 * Normalise combined sums (from simr_path_sums over a total of `paths` paths)
 * into price[n_strikes], stderr_out[n_strikes] (nullable) and
 * greeks[n_strikes * n_greeks] (nullable when greek_mask is 0).
 */
SIMR_API int simr_finalize_sums(simr_ctx* ctx, const simr_heston* model, const double* strikes,
                       int n_strikes, int is_put, uint32_t steps, uint64_t paths, double rel_bump,
                       uint32_t greek_mask, const double* sums, double* price, double* stderr_out,
                       double* greeks, void* stream);

/*
 * simr_price without any allocation: the paper has no counterpart to this entry
 * point.  It is for callers that cannot let a library allocate device memory --
 * serving loops that must never block on the allocator (cudaMalloc can
 * synchronise the device), and host applications that hand out all device
 * memory themselves.  It needs no context and calls no cudaMalloc, cudaFree or
 * allocating library routine: its reduction scratch is one file-scope device
 * array of 1 MiB + 256 B, which every GPU that loads libsimr holds until the
 * process exits.
 *   strikes[n_strikes], price[n_strikes], stderr_out[n_strikes] (nullable):
 *   DEVICE (or managed) pointers of the current device only (host pointers or
 *   another GPU's memory: SIMR_EINVAL);
 *   n_strikes in [1, 32] (larger: SIMR_EINVAL).  Arguments and results are
 *   those of simr_price with the same seed, option_index and sizes.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset on a device it no longer names the array, so a process that
 * resets a device must not call simr_price_noalloc on it again.  Calls on one device share the array, which keeps the last call's
 * contents (each call clears the words that must start at zero): calls that
 * overlap on the GPU -- on different streams, or from several host threads --
 * race and must be serialised by the caller.  A device strike that is not
 * finite and > 0 gives NaN results for that strike.  Asynchronous on `stream`.
 */
SIMR_API int simr_price_noalloc(const simr_heston* model, const double* strikes, int n_strikes, int is_put,
                                uint32_t steps, uint64_t paths, uint64_t seed, uint32_t option_index,
                                double* price, double* stderr_out, void* stream);

/*
 * Wait for `stream` and report any asynchronous device error as a status; also
 * reports (and clears) a device-side argument error such as a device-resident
 * strike that is not finite and > 0 (SIMR_EINVAL).
 */
SIMR_API int simr_sync(simr_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SIMR_H */
