/*
 * simr_oracle.c -- plain FP64 CPU oracle for Heston QE Monte Carlo option pricing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs load this library.  The product path (the CUDA
 * library behind include/simr.h) never links, loads or calls it, and this file
 * shares no code, header, constant table or helper with it.
 *
 * What it computes (the SIMR stages of the paper, Sec. 4 and Sec. 5 / Fig. 1):
 *   VariancePathQE         -> oracle_qe_variance_step   (Andersen 2008 QE step)
 *   LogPricePathQE         -> log-spot update in simulate_path
 *   AssetPathExponential   -> S_T = S0 * exp(x_N) in the payoff functions
 *   reduction over paths   -> oracle_price (Sec. 6: paths reduced with a cross-path sum)
 *   QE-M variant           -> oracle_set_scheme(1) (Andersen's martingale correction)
 *   writeLongstaffSchwartzPath -> oracle_states (per-path states at the exercise
 *                             dates; the regression itself is in lsm.py)
 * The per-path state is carried from timestep to timestep exactly as in the
 * paper's asset/timestep/path loop nest (Sec. 5.1, Listing 2): here the path is
 * the outer loop and the timestep the inner one, which changes nothing in the
 * arithmetic of any single path.
 *
 * The paper itself prints no model formula.  Its stage names ("...QE") identify
 * the Quadratic-Exponential scheme of L. Andersen, "Simple and efficient
 * simulation of the Heston stochastic volatility model", J. Comput. Finance 11(3),
 * 2008 (critical psi_c = 1.5, central weights gamma1 = gamma2 = 1/2, no martingale
 * correction), for the Heston (1993) model under the risk-neutral measure with a
 * constant short rate r and no dividends.  The random inputs V and Z of the paper
 * (Sec. 3, Table 1 caption) are produced by Philox4x32-10 (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) from a counter that
 * depends only on (step, path, option) and mapped to normals by the inverse CDF
 * (Wichura, "Algorithm AS 241", Applied Statistics 37(3), 1988).
 *
 * Everything is FP64, serial per path; OpenMP only spreads independent paths
 * over host threads, each writing its own output slot, and every cross-path sum
 * is a serial loop in path order, so the results do not depend on the thread
 * count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double S0, r, T, v0, kappa, theta, sigma, rho;
} oracle_heston;

/* QE scheme settings (Andersen 2008): switching level and central discretisation. */
static const double PSI_C = 1.5;
static const double GAMMA1 = 0.5;
static const double GAMMA2 = 0.5;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. SC'11): 10 rounds of the 4x32 Philox S-box,   */
/* Weyl key schedule between rounds.                                           */
/* ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t prod0 = (uint64_t)mult0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)mult1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 23-bit open-interval uniform: u = (floor(w / 2^9) + 1/2) * 2^-23, in (0, 1). */
double oracle_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/*
 * The two uniforms (U_V, U_X) of one time step.  Counter = (step/2, path low
 * word, path high word, option index), key = (seed low word, seed high word).
 * Even steps take output words 0 and 1, odd steps words 2 and 3.
 */
void oracle_step_uniforms(uint64_t seed, uint32_t option_index, uint64_t path, uint32_t step,
                          double* u_v, double* u_x) {
  uint32_t ctr[4] = {step >> 1, (uint32_t)path, (uint32_t)(path >> 32), option_index};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  oracle_philox4x32_10(ctr, key, w);
  if ((step & 1u) == 0) {
    *u_v = oracle_uniform(w[0]);
    *u_x = oracle_uniform(w[1]);
  } else {
    *u_v = oracle_uniform(w[2]);
    *u_x = oracle_uniform(w[3]);
  }
}

/* ------------------------------------------------------------------------- */
/* Inverse standard normal CDF, Wichura's AS 241 (PPND16), ~1e-16 relative.    */
/* ------------------------------------------------------------------------- */
static double poly7(const double* c, double x) {
  double s = c[7];
  for (int i = 6; i >= 0; --i) s = s * x + c[i];
  return s;
}

double oracle_norminv(double p) {
  static const double a[8] = {3.3871328727963666080e0,  1.3314166789178437745e+2,
                              1.9715909503065514427e+3, 1.3731693765509461125e+4,
                              4.5921953931549871457e+4, 6.7265770927008700853e+4,
                              3.3430575583588128105e+4, 2.5090809287301226727e+3};
  static const double b[8] = {1.0,
                              4.2313330701600911252e+1, 6.8718700749205790830e+2,
                              5.3941960214247511077e+3, 2.1213794301586595867e+4,
                              3.9307895800092710610e+4, 2.8729085735721942674e+4,
                              5.2264952788528545610e+3};
  static const double c[8] = {1.42343711074968357734e0,  4.63033784615654529590e0,
                              5.76949722146069140550e0,  3.64784832476320460504e0,
                              1.27045825245236838258e0,  2.41780725177450611770e-1,
                              2.27238449892691845833e-2, 7.74545014278341407640e-4};
  static const double d[8] = {1.0,
                              2.05319162663775882187e0,  1.67638483018380384940e0,
                              6.89767334985100004550e-1, 1.48103976427480074590e-1,
                              1.51986665636164571966e-2, 5.47593808499534494600e-4,
                              1.05075007164441684324e-9};
  static const double e[8] = {6.65790464350110377720e0,  5.46378491116411436990e0,
                              1.78482653991729133580e0,  2.96560571828504891230e-1,
                              2.65321895265761230930e-2, 1.24266094738807843860e-3,
                              2.71155556874348757815e-5, 2.01033439929228813265e-7};
  static const double f[8] = {1.0,
                              5.99832206555887937690e-1, 1.36929880922735805310e-1,
                              1.48753612908506148525e-2, 7.86869131145613259100e-4,
                              1.84631831751005468180e-5, 1.42151175831644588870e-7,
                              2.04426310338993978564e-15};
  double q = p - 0.5;
  if (fabs(q) <= 0.425) {
    double r = 0.180625 - q * q;
    return q * poly7(a, r) / poly7(b, r);
  }
  double r = (q < 0.0) ? p : 1.0 - p;
  r = sqrt(-log(r));
  double val;
  if (r <= 5.0) {
    r -= 1.6;
    val = poly7(c, r) / poly7(d, r);
  } else {
    r -= 5.0;
    val = poly7(e, r) / poly7(f, r);
  }
  return (q < 0.0) ? -val : val;
}

void oracle_norminv_array(const double* u, double* z, int64_t n) {
  for (int64_t i = 0; i < n; ++i) z[i] = oracle_norminv(u[i]);
}

/* ------------------------------------------------------------------------- */
/* Per-option constants of the QE scheme (Andersen 2008), at step dt = T/N.    */
/* out = {dt, E, c1, c2, K0, K1, K2, K3, K4}                                   */
/*   E  = exp(-kappa dt)                                                       */
/*   c1 = sigma^2 E (1-E) / kappa          (s^2 = v c1 + c2)                   */
/*   c2 = theta sigma^2 (1-E)^2 / (2 kappa)                                    */
/*   K0 = -rho kappa theta dt / sigma + r dt                                   */
/*   K1 = gamma1 dt (kappa rho / sigma - 1/2) - rho / sigma                    */
/*   K2 = gamma2 dt (kappa rho / sigma - 1/2) + rho / sigma                    */
/*   K3 = gamma1 dt (1 - rho^2),  K4 = gamma2 dt (1 - rho^2)                   */
/* ------------------------------------------------------------------------- */
void oracle_qe_constants(const oracle_heston* m, uint32_t steps, double out[9]) {
  double dt = m->T / (double)steps;
  double E = exp(-m->kappa * dt);
  double s2 = m->sigma * m->sigma;
  out[0] = dt;
  out[1] = E;
  out[2] = s2 * E * (1.0 - E) / m->kappa;
  out[3] = m->theta * s2 * (1.0 - E) * (1.0 - E) / (2.0 * m->kappa);
  out[4] = -m->rho * m->kappa * m->theta * dt / m->sigma + m->r * dt;
  out[5] = GAMMA1 * dt * (m->kappa * m->rho / m->sigma - 0.5) - m->rho / m->sigma;
  out[6] = GAMMA2 * dt * (m->kappa * m->rho / m->sigma - 0.5) + m->rho / m->sigma;
  out[7] = GAMMA1 * dt * (1.0 - m->rho * m->rho);
  out[8] = GAMMA2 * dt * (1.0 - m->rho * m->rho);
}

/*
 * One QE variance step (the paper's VariancePathQE stage, Sec. 4; formulas of
 * Andersen 2008).  Returns v(t+dt) given v(t) and the step's variance uniform.
 *   m = theta + (v - theta) E,  s^2 = v c1 + c2,  psi = s^2 / m^2
 *   psi <= psi_c : b^2 = 2/psi - 1 + sqrt(2/psi) sqrt(2/psi - 1), a = m / (1 + b^2),
 *                  v' = a (b + Z_V)^2 with Z_V = Phi^-1(U_V)
 *   psi >  psi_c : p = (psi - 1)/(psi + 1), beta = (1 - p)/m,
 *                  v' = 0 if U_V <= p, else ln((1 - p)/(1 - U_V)) / beta
 * *branch receives 0 (quadratic), 1 (exponential, v' > 0), 2 (exponential, v' = 0)
 * or 3 (m = 0: zero mean and variance, v' = 0).  *margin receives the distance of
 * the branch decisions from their thresholds: |psi - psi_c| / psi_c, and in the
 * exponential branch also |U_V - p|.  *cond (may be NULL) receives, in the
 * quadratic branch, |b + Z_V| / (1 + b): small values mean v' = a (b + Z_V)^2 is
 * a cancellation that a lower-precision evaluation resolves poorly (diagnostic
 * only, +inf in the other branches).
 */
double oracle_qe_variance_step(double v, double u_v, const double* k, int* branch, double* margin,
                               double* cond) {
  if (cond) *cond = INFINITY;
  const double theta_ = k[9];  /* theta is appended after the 9 constants */
  double E = k[1], c1 = k[2], c2 = k[3];
  double m = theta_ + (v - theta_) * E;
  double s2 = v * c1 + c2;
  if (m <= 0.0) {
    *branch = 3;
    *margin = INFINITY;
    return 0.0;
  }
  double psi = s2 / (m * m);
  double mg = fabs(psi - PSI_C) / PSI_C;
  if (psi <= PSI_C) {
    double two_over_psi = 2.0 / psi;
    double b2 = two_over_psi - 1.0 + sqrt(two_over_psi) * sqrt(two_over_psi - 1.0);
    double a = m / (1.0 + b2);
    double b = sqrt(b2);
    double zv = oracle_norminv(u_v);
    *branch = 0;
    *margin = mg;
    if (cond) *cond = fabs(b + zv) / (1.0 + b);
    return a * (b + zv) * (b + zv);
  }
  double p = (psi - 1.0) / (psi + 1.0);
  double beta = (1.0 - p) / m;
  double mu = fabs(u_v - p);
  *margin = (mu < mg) ? mu : mg;
  if (u_v <= p) {
    *branch = 2;
    return 0.0;
  }
  *branch = 1;
  return log((1.0 - p) / (1.0 - u_v)) / beta;
}

/*
 * Log-spot scheme: 0 = QE as above; 1 = QE-M, Andersen's martingale correction
 * (Andersen 2008, the martingale-correction section): with A = K2 + K4/2 the
 * constant K0 - r dt of the log-spot step is replaced by
 *   K0* = -ln M - (K1 + K3/2) v,   M = E[exp(A v(t+dt)) | v(t)] under the QE step,
 *   quadratic branch:    ln M = A b^2 a / (1 - 2 A a) - (1/2) ln(1 - 2 A a)   (needs 2 A a < 1)
 *   exponential branch:  M = p + beta (1 - p) / (beta - A)                    (needs A < beta)
 * so that E[exp(x(t+dt) - x(t) - r dt) | v(t)] = 1; where the condition fails
 * the step keeps K0.  Set for the whole library by oracle_set_scheme (test
 * infrastructure: read-only while a computation runs).
 */
static int g_scheme = 0;

void oracle_set_scheme(int scheme) { g_scheme = scheme; }

/* ln M of the QE-M correction at state v (k: the 9 constants + theta); *ok = 0
 * where the correction does not exist.  m = 0 gives v' = 0, M = 1. */
static double qem_log_m_branch(double v, const double* k, int quad_forced, int* ok) {
  const double theta_ = k[9], E = k[1], c1 = k[2], c2 = k[3];
  const double A = k[6] + 0.5 * k[8];
  const double m = theta_ + (v - theta_) * E;
  const double s2 = v * c1 + c2;
  *ok = 1;
  if (m <= 0.0) return 0.0;
  const double psi = s2 / (m * m);
  if (quad_forced >= 0 ? quad_forced : psi <= PSI_C) {
    const double two_over_psi = 2.0 / psi;
    const double b2 = two_over_psi - 1.0 + sqrt(two_over_psi) * sqrt(two_over_psi - 1.0);
    const double a = m / (1.0 + b2);
    if (!(2.0 * A * a < 1.0)) {
      *ok = 0;
      return 0.0;
    }
    return A * b2 * a / (1.0 - 2.0 * A * a) - 0.5 * log(1.0 - 2.0 * A * a);
  }
  const double p = (psi - 1.0) / (psi + 1.0);
  const double beta = (1.0 - p) / m;
  if (!(A < beta)) {
    *ok = 0;
    return 0.0;
  }
  return log(p + beta * (1.0 - p) / (beta - A));
}

/* ln M in the branch the variance step takes. */
static double qem_log_m(double v, const double* k, int* ok) { return qem_log_m_branch(v, k, -1, ok); }

/*
 * The constant term of a log-spot step from state v (r dt included): K0 (k[4])
 * under QE; under QE-M, where M exists, K0* + r dt = r dt - ln M - (K1 + K3/2) v
 * with ln M in the branch quad_forced imposes (-1: the step's own).
 */
static double step_k0(const oracle_heston* m, const double* k, double v, int quad_forced) {
  if (g_scheme != 1) return k[4];
  int ok;
  const double lnM = qem_log_m_branch(v, k, quad_forced, &ok);
  if (!ok) return k[4];
  return m->r * k[0] - lnM - (k[5] + 0.5 * k[7]) * v;
}

/*
 * The adjoint of -ln M at the state with mean m and variance s2 (A = K2 + K4/2),
 * where the correction exists: adds to *bar_A, *bar_m, *bar_s2 the derivatives of
 * -ln M in the branch the variance step takes (quad_forced 1 or 0: the quadratic
 * or the exponential branch imposed; -1: the step's own).

 *   quadratic: ln M = A b^2 a / D - ln(D)/2, D = 1 - 2 A a, a = m / (1 + b^2),
 *              b^2 = t - 1 + sqrt(t (t - 1)), t = 2 m^2 / s2;
 *   exponential: ln M = ln((1 - q) + beta q / (beta - A)), q = 1 - p = 2 m^2 / (m^2 + s2),
 *              beta = q / m.
 */
static void qem_log_m_adjoint(double m, double s2, double A, int quad_forced, double* bar_A, double* bar_m,
                              double* bar_s2) {
  if (m <= 0.0) return;
  const double psi = s2 / (m * m);
  if (quad_forced >= 0 ? quad_forced : psi <= PSI_C) {
    const double t = 2.0 / psi;
    const double root = sqrt(t) * sqrt(t - 1.0);
    const double b2 = t - 1.0 + root;
    const double a = m / (1.0 + b2);
    const double D = 1.0 - 2.0 * A * a;
    const double dA = b2 * a / D + A * b2 * a * 2.0 * a / (D * D) + a / D;
    const double da = A * b2 / D + A * b2 * a * 2.0 * A / (D * D) + A / D;
    const double db2 = A * a / D;
    const double ba = -da;                                  /* bar a of -ln M */
    const double bb2 = -db2 + ba * (-m / ((1.0 + b2) * (1.0 + b2)));
    const double bt = bb2 * (1.0 + (2.0 * t - 1.0) / (2.0 * root));
    *bar_A += -dA;
    *bar_m += ba / (1.0 + b2) + bt * 4.0 * m / s2;
    *bar_s2 += -bt * t / s2;
    return;
  }
  const double den = m * m + s2;
  const double q = 2.0 * m * m / den;
  const double beta = q / m;
  const double M = (1.0 - q) + beta * q / (beta - A);
  const double bM = -1.0 / M;
  const double bbeta = bM * (-A * q / ((beta - A) * (beta - A)));
  const double bq = bM * (-1.0 + beta / (beta - A)) + bbeta / m;
  *bar_A += bM * beta * q / ((beta - A) * (beta - A));
  *bar_m += bbeta * (-q / (m * m)) + bq * 4.0 * m * s2 / (den * den);
  *bar_s2 += bq * (-2.0 * m * m / (den * den));
}

/* Constants array used by the step: the 9 QE constants followed by theta. */
static void step_constants(const oracle_heston* m, uint32_t steps, double k[10]) {
  oracle_qe_constants(m, steps, k);
  k[9] = m->theta;
}

/*
 * Simulate one path for `steps` steps from v = v0, x = ln(S/S0) = 0.
 * Writes x_N, v_N and the smallest decision margin met on the path; with
 * every > 0 it also records (x, v) after steps every, 2 every, ... into
 * x_rec[], v_rec[] (the states at a Bermudan option's exercise dates).
 */
static void simulate_path_rec(const oracle_heston* m, const double* k, uint32_t steps, uint64_t seed,
                              uint32_t option_index, uint64_t path, double* x_out, double* v_out,
                              double* margin_out, double* cond_out, uint32_t every, double* x_rec,
                              double* v_rec) {
  double v = m->v0, x = 0.0, min_margin = INFINITY, min_cond = INFINITY;
  for (uint32_t n = 0; n < steps; ++n) {
    double u_v, u_x;
    oracle_step_uniforms(seed, option_index, path, n, &u_v, &u_x);
    int branch;
    double mg, cd;
    double v_next = oracle_qe_variance_step(v, u_v, k, &branch, &mg, &cd);
    if (mg < min_margin) min_margin = mg;
    if (cd < min_cond) min_cond = cd;
    /* LogPricePathQE: x += K0 + K1 v + K2 v' + sqrt(K3 v + K4 v') Z_X */
    double z_x = oracle_norminv(u_x);
    const double k0 = step_k0(m, k, v, -1);
    x += k0 + k[5] * v + k[6] * v_next + sqrt(k[7] * v + k[8] * v_next) * z_x;
    v = v_next;
    if (every && (n + 1) % every == 0) {
      x_rec[(n + 1) / every - 1] = x;
      v_rec[(n + 1) / every - 1] = v;
    }
  }
  *x_out = x;
  *v_out = v;
  if (margin_out) *margin_out = min_margin;
  if (cond_out) *cond_out = min_cond;
}

static void simulate_path(const oracle_heston* m, const double* k, uint32_t steps, uint64_t seed,
                          uint32_t option_index, uint64_t path, double* x_out, double* v_out,
                          double* margin_out, double* cond_out) {
  simulate_path_rec(m, k, steps, seed, option_index, path, x_out, v_out, margin_out, cond_out, 0, NULL, NULL);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/*
 * Terminal states of paths [path_begin, path_begin + n_paths): x_T = ln(S_T/S0)
 * and v_T per path, plus the smallest branch-decision margin of each path
 * (margin may be NULL).
 */
int oracle_terminal(const oracle_heston* m, uint32_t steps, uint64_t seed, uint32_t option_index,
                    uint64_t path_begin, int64_t n_paths, double* x_T, double* v_T, double* margin) {
  if (steps == 0 || n_paths < 0) return -1;
  double k[10];
  step_constants(m, steps, k);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_paths; ++i) {
    simulate_path(m, k, steps, seed, option_index, path_begin + (uint64_t)i, &x_T[i], &v_T[i],
                  margin ? &margin[i] : NULL, NULL);
  }
  return 0;
}

/* As oracle_terminal, plus the per-path conditioning diagnostic cond (the
 * smallest |b + Z_V| / (1 + b) over the path's quadratic-branch steps). */
int oracle_terminal_diag(const oracle_heston* m, uint32_t steps, uint64_t seed, uint32_t option_index,
                         uint64_t path_begin, int64_t n_paths, double* x_T, double* v_T, double* margin,
                         double* cond) {
  if (steps == 0 || n_paths < 0) return -1;
  double k[10];
  step_constants(m, steps, k);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_paths; ++i) {
    simulate_path(m, k, steps, seed, option_index, path_begin + (uint64_t)i, &x_T[i], &v_T[i], &margin[i],
                  &cond[i]);
  }
  return 0;
}

/*
 * States at the exercise dates of a Bermudan option, for the Longstaff-Schwartz
 * regression (the paper's longstaffSchwartzPathReduction stage consumes the
 * per-path states that writeLongstaffSchwartzPath writes out, Sec. 5): dates
 * t_j = (j + 1) every dt, j = 0 .. n_ex - 1 with n_ex = steps / every (every
 * must divide steps, so the last date is the maturity).  S[i * n_ex + j] =
 * S0 exp(x) and v[i * n_ex + j] for path path_begin + i.
 */
int oracle_states(const oracle_heston* m, uint32_t steps, uint32_t every, uint64_t seed, uint32_t option_index,
                  uint64_t path_begin, int64_t n_paths, double* S, double* v) {
  if (steps == 0 || every == 0 || steps % every != 0 || n_paths < 0) return -1;
  const int64_t n_ex = steps / every;
  double k[10];
  step_constants(m, steps, k);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_paths; ++i) {
    double xT, vT;
    double* xs = &S[i * n_ex];
    simulate_path_rec(m, k, steps, seed, option_index, path_begin + (uint64_t)i, &xT, &vT, NULL, NULL, every, xs,
                      &v[i * n_ex]);
    for (int64_t j = 0; j < n_ex; ++j) xs[j] = m->S0 * exp(xs[j]);
  }
  return 0;
}

/*
 * Terminal log-spots of A correlated assets (basket options): asset k runs the
 * single-asset scheme with its own model and the Philox counters of option
 * index k, except that its log-spot normal is z_k = sum_{j <= k} Lc[k][j] eps_j,
 * where eps_j = Phi^-1(U_X) of asset j and Lc is the lower Cholesky factor of
 * the correlation of the spot drivers (row-major A x A; computed by the caller).
 * The variance drivers stay independent across assets.  Under QE-M each asset
 * takes its own martingale correction: z_k is a standard normal independent of
 * the asset's own variance path, so M is the single-asset one.  x[i * A + k] =
 * ln(S_T / S0) of asset k on path path_begin + i; margin[i] (may be NULL) the
 * smallest branch-decision margin over the path's assets and steps.
 */
int oracle_basket_terminal(const oracle_heston* models, int n_assets, const double* Lc, uint32_t steps,
                           uint64_t seed, uint64_t path_begin, int64_t n_paths, double* x_out, double* margin) {
  if (steps == 0 || n_assets < 1 || n_assets > 64 || n_paths < 0) return -1;
  const int A = n_assets;
  double* k = (double*)malloc(sizeof(double) * 10 * (size_t)A);
  if (!k) return -2;
  for (int a = 0; a < A; ++a) step_constants(&models[a], steps, &k[10 * a]);
  int rc = 0;
#pragma omp parallel
  {
    double* v = (double*)malloc(sizeof(double) * (size_t)A);
    double* x = (double*)malloc(sizeof(double) * (size_t)A);
    double* uv = (double*)malloc(sizeof(double) * (size_t)A);
    double* eps = (double*)malloc(sizeof(double) * (size_t)A);
    if (!v || !x || !uv || !eps) {
#pragma omp atomic write
      rc = -2;
    } else {
#pragma omp for schedule(static)
      for (int64_t i = 0; i < n_paths; ++i) {
        const uint64_t path = path_begin + (uint64_t)i;
        double min_mg = INFINITY;
        for (int a = 0; a < A; ++a) {
          v[a] = models[a].v0;
          x[a] = 0.0;
        }
        for (uint32_t n = 0; n < steps; ++n) {
          for (int a = 0; a < A; ++a) {
            double u_x;
            oracle_step_uniforms(seed, (uint32_t)a, path, n, &uv[a], &u_x);
            eps[a] = oracle_norminv(u_x);
          }
          for (int a = 0; a < A; ++a) {
            const double* ka = &k[10 * a];
            double z = 0.0;
            for (int j = 0; j <= a; ++j) z += Lc[a * A + j] * eps[j];
            int br;
            double mg;
            const double vn = oracle_qe_variance_step(v[a], uv[a], ka, &br, &mg, NULL);
            if (mg < min_mg) min_mg = mg;
            x[a] += step_k0(&models[a], ka, v[a], -1) + ka[5] * v[a] + ka[6] * vn + sqrt(ka[7] * v[a] + ka[8] * vn) * z;
            v[a] = vn;
          }
        }
        for (int a = 0; a < A; ++a) x_out[i * A + a] = x[a];
        if (margin) margin[i] = min_mg;
      }
    }
    free(v);
    free(x);
    free(uv);
    free(eps);
  }
  free(k);
  return rc;
}

/*
 * E[exp(x(t+dt) - x(t) - r dt) | v(t) = v] of one step under the library's
 * scheme: the normal Z_X integrated exactly (E exp(s Z) = exp(s^2/2)) and the
 * variance uniform summed over its whole lattice u = (j + 1/2) 2^-23, the set
 * of values the generator produces, each equally likely -- so this is the
 * scheme's exact one-step expectation.  1 for a martingale scheme.
 */
double oracle_step_exp_mean(const oracle_heston* m, uint32_t steps, double v) {
  double k[10];
  step_constants(m, steps, k);
  const double k0 = step_k0(m, k, v, -1) - m->r * k[0];
  const int64_t n = (int64_t)1 << 23;
  double sum = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    const double u = ((double)j + 0.5) * 0x1p-23;
    int br;
    double mg;
    const double vn = oracle_qe_variance_step(v, u, k, &br, &mg, NULL);
    sum += exp(k0 + k[5] * v + k[6] * vn + 0.5 * (k[7] * v + k[8] * vn));
  }
  return sum / (double)n;
}

/* European payoff of a call (is_put = 0) or put; zero at S_T = K. */
static double payoff(double s_T, double K, int is_put) {
  double d = is_put ? (K - s_T) : (s_T - K);
  return d > 0.0 ? d : 0.0;
}

/*
 * Discounted Monte Carlo price and standard error per strike over paths
 * [0, paths):  price_k = e^{-rT} mean_p f_k(S_T,p),
 * stderr_k = e^{-rT} sqrt((mean f^2 - mean(f)^2) / (paths - 1)).
 * The cross-path sums run serially in path order.
 */
int oracle_price(const oracle_heston* m, const double* strikes, int n_strikes, int is_put,
                 uint32_t steps, int64_t paths, uint64_t seed, uint32_t option_index,
                 double* price, double* stderr_out) {
  if (paths <= 0 || n_strikes <= 0 || steps == 0) return -1;
  double* x = (double*)malloc(sizeof(double) * (size_t)paths);
  double* v = (double*)malloc(sizeof(double) * (size_t)paths);
  if (!x || !v) {
    free(x);
    free(v);
    return -2;
  }
  oracle_terminal(m, steps, seed, option_index, 0, paths, x, v, NULL);
  double disc = exp(-m->r * m->T);
  for (int j = 0; j < n_strikes; ++j) {
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < paths; ++i) {
      double f = payoff(m->S0 * exp(x[i]), strikes[j], is_put);
      s1 += f;
      s2 += f * f;
    }
    double mean = s1 / (double)paths;
    price[j] = disc * mean;
    if (stderr_out) {
      double var = (paths > 1) ? (s2 / (double)paths - mean * mean) / (double)(paths - 1) : 0.0;
      stderr_out[j] = disc * sqrt(var > 0.0 ? var : 0.0);
    }
  }
  free(x);
  free(v);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Bump-and-revalue Greeks with common random numbers: every scenario is a     */
/* full re-simulation with the same Philox counters; central differences.      */
/* ------------------------------------------------------------------------- */
enum {
  G_DELTA = 1u << 0,   /* d/dS0                     */
  G_GAMMA = 1u << 1,   /* d2/dS0^2                  */
  G_VEGA = 1u << 2,    /* d/dv0                     */
  G_THETA = 1u << 3,   /* -d/dT (calendar)          */
  G_RHO = 1u << 4,     /* d/dr                      */
  G_KAPPA = 1u << 5,   /* d/dkappa                  */
  G_LRVAR = 1u << 6,   /* d/dtheta (long-run var.)  */
  G_VOLVOL = 1u << 7,  /* d/dsigma                  */
  G_CORR = 1u << 8     /* d/drho                    */
};

static int scenario_price(const oracle_heston* m, const double* strikes, int n_strikes, int is_put,
                          uint32_t steps, int64_t paths, uint64_t seed, uint32_t option_index,
                          double* out) {
  return oracle_price(m, strikes, n_strikes, is_put, steps, paths, seed, option_index, out, NULL);
}

/*
 * Central difference of the price in one parameter.  The bump is rel_bump*|value|
 * (rel_bump itself when the value is zero); for rho it is rel_bump in absolute
 * terms.  Where the down-bumped value would leave the domain (v0 or theta below
 * zero, rho outside [-1, 1]) the one-sided difference on the valid side is used.
 * `which` selects the field; `sign` = -1 turns d/dT into theta = -d/dT.
 */
static int fd_one(const oracle_heston* base, int which, double rel_bump, double sign,
                  const double* strikes, int n_strikes, int is_put, uint32_t steps, int64_t paths,
                  uint64_t seed, uint32_t option_index, const double* p0, double* out, double* tmp_up,
                  double* tmp_dn) {
  oracle_heston up = *base, dn = *base;
  double* fld_up = &((double*)&up)[which];
  double* fld_dn = &((double*)&dn)[which];
  double value = ((const double*)base)[which];
  double h = (which == 7) ? rel_bump : rel_bump * fabs(value);
  if (h == 0.0) h = rel_bump;
  *fld_up = value + h;
  *fld_dn = value - h;
  int up_ok = 1, dn_ok = 1;
  if ((which == 3 || which == 5) && *fld_dn < 0.0) dn_ok = 0;  /* v0, theta >= 0 */
  if (which == 7 && *fld_dn < -1.0) dn_ok = 0;                 /* rho >= -1 */
  if (which == 7 && *fld_up > 1.0) up_ok = 0;                  /* rho <= 1 */
  if (up_ok && scenario_price(&up, strikes, n_strikes, is_put, steps, paths, seed, option_index, tmp_up))
    return -1;
  if (dn_ok && scenario_price(&dn, strikes, n_strikes, is_put, steps, paths, seed, option_index, tmp_dn))
    return -1;
  for (int j = 0; j < n_strikes; ++j) {
    double d;
    if (up_ok && dn_ok) d = (tmp_up[j] - tmp_dn[j]) / (2.0 * h);
    else if (up_ok) d = (tmp_up[j] - p0[j]) / h;
    else d = (p0[j] - tmp_dn[j]) / h;
    out[j] = sign * d;
  }
  return 0;
}

/*
 * greeks[j * n_out + g] for strike j and the g-th set bit of greek_mask, in bit
 * order.  price receives the base-scenario price.  Returns the number of Greeks.
 * Gamma uses the three-point second difference (S0(1+h), S0, S0(1-h)).
 */
int oracle_greeks_fd(const oracle_heston* m, const double* strikes, int n_strikes, int is_put,
                     uint32_t steps, int64_t paths, uint64_t seed, uint32_t option_index,
                     double rel_bump, uint32_t greek_mask, double* price, double* greeks) {
  if (rel_bump <= 0.0 || n_strikes <= 0) return -1;
  int n_out = 0;
  for (int b = 0; b < 9; ++b) n_out += (greek_mask >> b) & 1u;
  double* up = (double*)malloc(sizeof(double) * (size_t)n_strikes);
  double* dn = (double*)malloc(sizeof(double) * (size_t)n_strikes);
  double* g = (double*)malloc(sizeof(double) * (size_t)n_strikes);
  if (!up || !dn || !g) {
    free(up);
    free(dn);
    free(g);
    return -2;
  }
  int rc = scenario_price(m, strikes, n_strikes, is_put, steps, paths, seed, option_index, price);
  int col = 0;
  /* field index into oracle_heston: S0=0 r=1 T=2 v0=3 kappa=4 theta=5 sigma=6 rho=7 */
  static const int field[9] = {0, 0, 3, 2, 1, 4, 5, 6, 7};
  for (int b = 0; b < 9 && rc == 0; ++b) {
    if (!((greek_mask >> b) & 1u)) continue;
    if ((1u << b) == G_GAMMA) {
      oracle_heston su = *m, sd = *m;
      double h = rel_bump * m->S0;
      su.S0 = m->S0 + h;
      sd.S0 = m->S0 - h;
      rc |= scenario_price(&su, strikes, n_strikes, is_put, steps, paths, seed, option_index, up);
      rc |= scenario_price(&sd, strikes, n_strikes, is_put, steps, paths, seed, option_index, dn);
      for (int j = 0; j < n_strikes; ++j) g[j] = (up[j] - 2.0 * price[j] + dn[j]) / (h * h);
    } else {
      double sign = ((1u << b) == G_THETA) ? -1.0 : 1.0;
      rc |= fd_one(m, field[b], rel_bump, sign, strikes, n_strikes, is_put, steps, paths, seed,
                   option_index, price, g, up, dn);
    }
    for (int j = 0; j < n_strikes; ++j) greeks[(size_t)j * n_out + col] = g[j];
    ++col;
  }
  free(up);
  free(dn);
  free(g);
  return rc ? rc : n_out;
}

/* ------------------------------------------------------------------------- */
/* Pathwise derivatives of x_T = ln(S_T/S0) with respect to                    */
/* (v0, kappa, theta, sigma, rho), branch decisions held fixed.                */
/* ------------------------------------------------------------------------- */

/*
 * Reverse mode (hand-written adjoint).  The forward sweep records v_n and the
 * branch of every step; the reverse sweep runs the steps backwards,
 * accumulating the adjoints of v and of the per-option constants (E, c1, c2,
 * K0..K4 and theta as it enters m), then maps those onto the parameters.
 * grad5 = {dx/dv0, dx/dkappa, dx/dtheta, dx/dsigma, dx/drho}; dx/dr = T exactly.
 */
static double qe_step_forced(double v, double u_v, const double* k, int f_kind, int f_value);

static void path_adjoint_forced(const oracle_heston* m, const double* k, uint32_t steps, uint64_t seed,
                                uint32_t option_index, uint64_t path, double* v_hist, double* x_out,
                                double grad5[5], int64_t f_step, int f_kind, int f_value) {
  double v = m->v0, x = 0.0;
  v_hist[0] = v;
  for (uint32_t n = 0; n < steps; ++n) {
    double u_v, u_x, mg;
    int br;
    oracle_step_uniforms(seed, option_index, path, n, &u_v, &u_x);
    double vn = ((int64_t)n == f_step) ? qe_step_forced(v, u_v, k, f_kind, f_value)
                                       : oracle_qe_variance_step(v, u_v, k, &br, &mg, NULL);
    const double k0 = step_k0(m, k, v, ((int64_t)n == f_step && f_kind == 1) ? f_value : -1);
    x += k0 + k[5] * v + k[6] * vn + sqrt(k[7] * v + k[8] * vn) * oracle_norminv(u_x);
    v = vn;
    v_hist[n + 1] = v;
  }
  *x_out = x;

  const double dt = k[0], E = k[1], c1 = k[2], c2 = k[3];
  const double K1 = k[5], K2 = k[6], K3 = k[7], K4 = k[8], th = m->theta;
  double bar_E = 0, bar_c1 = 0, bar_c2 = 0, bar_th = 0;
  double bar_K0 = 0, bar_K1 = 0, bar_K2 = 0, bar_K3 = 0, bar_K4 = 0;
  double bar_vnext = 0.0; /* adjoint of v_{n+1} */
  for (int64_t n = (int64_t)steps - 1; n >= 0; --n) {
    double u_v, u_x;
    oracle_step_uniforms(seed, option_index, path, (uint32_t)n, &u_v, &u_x);
    double z_x = oracle_norminv(u_x);
    double vc = v_hist[n], vn = v_hist[n + 1];
    /* x_{n+1} = x_n + K0 + K1 vc + K2 vn + sqrt(K3 vc + K4 vn) z_x,  xbar = 1 */
    double w = K3 * vc + K4 * vn;
    double dsq = (w > 0.0) ? z_x / (2.0 * sqrt(w)) : 0.0; /* d sqrt(w) z / dw */
    double bar_vcur = K1 + K3 * dsq;
    bar_vnext += K2 + K4 * dsq;
    bar_K2 += vn;
    bar_K3 += vc * dsq;
    bar_K4 += vn * dsq;
    /* v_{n+1} = QE(v_n): adjoints of m and s^2 */
    double mm = th + (vc - th) * E;
    double s2 = vc * c1 + c2;
    double bar_m = 0.0, bar_s2 = 0.0;
    int qem_ok = 0;
    const int quad_forced = (n == f_step && f_kind == 1) ? f_value : -1;
    if (g_scheme == 1) (void)qem_log_m_branch(vc, k, quad_forced, &qem_ok);
    if (qem_ok) {
      /* QE-M: K0 + K1 v is replaced by r dt - ln M(v) - (K1 + K3/2) v + K1 v, so K0 and
       * K1 drop out, K3 gains -v/2 and v gains -(K1 + K3/2); ln M adds its own adjoint
       * (bar ln M = -1) to A = K2 + K4/2 and to m and s^2 (qem_log_m_adjoint). */
      bar_vcur -= K1 + 0.5 * K3;
      bar_K3 -= 0.5 * vc;
      double bar_A = 0.0;
      qem_log_m_adjoint(mm, s2, K2 + 0.5 * K4, quad_forced, &bar_A, &bar_m, &bar_s2);
      bar_K2 += bar_A;
      bar_K4 += 0.5 * bar_A;
    } else {
      bar_K0 += 1.0;
      bar_K1 += vc;
    }
    if (mm > 0.0) {
      double psi = s2 / (mm * mm);
      int quad = psi <= PSI_C;
      if (n == f_step && f_kind == 1) quad = f_value;
      if (quad) {
        double t = 2.0 / psi; /* = 2 m^2 / s^2 */
        double root = sqrt(t) * sqrt(t - 1.0);
        double b2 = t - 1.0 + root;
        double b = sqrt(b2);
        double a = mm / (1.0 + b2);
        double zv = oracle_norminv(u_v);
        double bar_a = bar_vnext * (b + zv) * (b + zv);
        double bar_b = bar_vnext * 2.0 * a * (b + zv);
        double bar_b2 = bar_b / (2.0 * b) - bar_a * mm / ((1.0 + b2) * (1.0 + b2));
        double bar_t = bar_b2 * (1.0 + (2.0 * t - 1.0) / (2.0 * root));
        bar_m += bar_a / (1.0 + b2) + bar_t * 4.0 * mm / s2;
        bar_s2 += -bar_t * t / s2;
      } else {
        double p = (psi - 1.0) / (psi + 1.0);
        int pos = u_v > p;
        if (n == f_step && f_kind == 2) pos = f_value;
        if (pos) {
          double q = 2.0 * mm * mm / (mm * mm + s2); /* 1 - p */
          double L = log(q / (1.0 - u_v));
          double dv_dm = L / q;
          double dv_dq = (mm / (q * q)) * (1.0 - L);
          double den = (mm * mm + s2) * (mm * mm + s2);
          double dq_dm = 4.0 * mm * s2 / den;
          double dq_ds2 = -2.0 * mm * mm / den;
          bar_m += bar_vnext * (dv_dm + dv_dq * dq_dm);
          bar_s2 += bar_vnext * dv_dq * dq_ds2;
        }
      }
    }
    bar_vcur += bar_m * E + bar_s2 * c1;
    bar_E += bar_m * (vc - th);
    bar_th += bar_m * (1.0 - E);
    bar_c1 += bar_s2 * vc;
    bar_c2 += bar_s2;
    bar_vnext = bar_vcur;
  }
  /* map constant adjoints onto the parameters */
  const double kap = m->kappa, sig = m->sigma, rho = m->rho;
  const double dE_dk = -dt * E;
  const double s2g = sig * sig;
  const double dc1_dk = s2g * ((1.0 - 2.0 * E) * dE_dk / kap - E * (1.0 - E) / (kap * kap));
  const double dc2_dk = th * s2g * (-2.0 * (1.0 - E) * dE_dk / (2.0 * kap) -
                                    (1.0 - E) * (1.0 - E) / (2.0 * kap * kap));
  const double dc2_dth = s2g * (1.0 - E) * (1.0 - E) / (2.0 * kap);
  grad5[0] = bar_vnext;
  grad5[1] = bar_E * dE_dk + bar_c1 * dc1_dk + bar_c2 * dc2_dk + bar_K0 * (-rho * th * dt / sig) +
             bar_K1 * (GAMMA1 * dt * rho / sig) + bar_K2 * (GAMMA2 * dt * rho / sig);
  grad5[2] = bar_th + bar_c2 * dc2_dth + bar_K0 * (-rho * kap * dt / sig);
  grad5[3] = bar_c1 * 2.0 * c1 / sig + bar_c2 * 2.0 * c2 / sig +
             bar_K0 * (rho * kap * th * dt / (sig * sig)) +
             bar_K1 * (-GAMMA1 * dt * kap * rho / (sig * sig) + rho / (sig * sig)) +
             bar_K2 * (-GAMMA2 * dt * kap * rho / (sig * sig) - rho / (sig * sig));
  grad5[4] = bar_K0 * (-kap * th * dt / sig) + bar_K1 * (GAMMA1 * dt * kap / sig - 1.0 / sig) +
             bar_K2 * (GAMMA2 * dt * kap / sig + 1.0 / sig) + bar_K3 * (-2.0 * GAMMA1 * dt * rho) +
             bar_K4 * (-2.0 * GAMMA2 * dt * rho);
}

static void path_adjoint(const oracle_heston* m, const double* k, uint32_t steps, uint64_t seed,
                         uint32_t option_index, uint64_t path, double* v_hist, double* x_out,
                         double grad5[5]) {
  path_adjoint_forced(m, k, steps, seed, option_index, path, v_hist, x_out, grad5, -1, 0, 0);
}

/*
 * The other side of a branch decision.  A pathwise derivative holds every
 * branch decision of the path fixed; where a lower-precision evaluation of the
 * same path can take the other side of a decision that sits close to its
 * threshold, the derivative it computes is that of the path with the decision
 * taken the other way.  qe_step_forced is the QE variance step of
 * oracle_qe_variance_step with one decision imposed: f_kind 1 the branch
 * (f_value 1 quadratic, 0 exponential; the quadratic formulas need psi <= 2,
 * the exponential ones psi > -1 -- both hold near psi_c), f_kind 2 the
 * exponential branch's atom (f_value 1: v' = ln((1-p)/(1-U_V))/beta, its
 * continuation below U_V = p held at 0 -- the value and one-sided derivative
 * at the boundary; 0: v' = 0).
 */
static double qe_step_forced(double v, double u_v, const double* k, int f_kind, int f_value) {
  const double theta_ = k[9], E = k[1], c1 = k[2], c2 = k[3];
  const double mean = theta_ + (v - theta_) * E;
  const double var = v * c1 + c2;
  if (mean <= 0.0) return 0.0;
  const double ps = var / (mean * mean);
  int quad = ps <= PSI_C;
  if (f_kind == 1) quad = f_value;
  if (quad) { /* v' = a (b + Z_V)^2 */
    const double t2 = 2.0 / ps;
    const double bb = t2 - 1.0 + sqrt(t2) * sqrt(t2 - 1.0);
    const double aa = mean / (1.0 + bb);
    const double bz = sqrt(bb) + oracle_norminv(u_v);
    return aa * bz * bz;
  }
  const double pp = (ps - 1.0) / (ps + 1.0); /* atom probability */
  int pos = u_v > pp;
  if (f_kind == 2) pos = f_value;
  if (!pos) return 0.0;
  const double vn = log((1.0 - pp) / (1.0 - u_v)) * mean / (1.0 - pp);
  return vn > 0.0 ? vn : 0.0;
}

/* The decision of a path closest to its threshold: its step, kind (1 the
 * branch, 2 the atom) and margin (|psi - psi_c| / psi_c, or |U_V - p|), and the
 * value the decision takes there. */
static void closest_decision(const oracle_heston* m, const double* k, uint32_t steps, uint64_t seed,
                             uint32_t option_index, uint64_t path, int64_t* step, int* kind, int* value,
                             double* margin) {
  double v = m->v0;
  *step = -1;
  *kind = 0;
  *value = 0;
  *margin = INFINITY;
  const double theta_ = k[9], E = k[1], c1 = k[2], c2 = k[3];
  for (uint32_t n = 0; n < steps; ++n) {
    double u_v, u_x, mg;
    int br;
    oracle_step_uniforms(seed, option_index, path, n, &u_v, &u_x);
    double mm = theta_ + (v - theta_) * E;
    double s2 = v * c1 + c2;
    if (mm > 0.0) {
      double psi = s2 / (mm * mm);
      double mpsi = fabs(psi - PSI_C) / PSI_C;
      if (mpsi < *margin) {
        *margin = mpsi;
        *step = n;
        *kind = 1;
        *value = psi <= PSI_C;
      }
      if (psi > PSI_C) {
        double p = (psi - 1.0) / (psi + 1.0);
        if (fabs(u_v - p) < *margin) {
          *margin = fabs(u_v - p);
          *step = n;
          *kind = 2;
          *value = u_v > p;
        }
      }
    }
    v = oracle_qe_variance_step(v, u_v, k, &br, &mg, NULL);
  }
}

/*
 * Per path: the reverse-mode gradient with the path's closest decision taken
 * the other way where its margin is below margin_below (flip_step[i] = its
 * step, flip_kind[i] its kind, flip_value[i] the value imposed), else the plain
 * gradient (flip_step[i] = -1); x_T and grad[i*5 + j] as
 * oracle_path_grad_reverse.
 */
int oracle_path_grad_flip(const oracle_heston* m, uint32_t steps, uint64_t seed, uint32_t option_index,
                          uint64_t path_begin, int64_t n_paths, double margin_below, double* x_T, double* grad,
                          int64_t* flip_step, int32_t* flip_kind, int32_t* flip_value) {
  if (steps == 0 || n_paths < 0) return -1;
  double k[10];
  step_constants(m, steps, k);
  int rc = 0;
#pragma omp parallel
  {
    double* hist = (double*)malloc(sizeof(double) * ((size_t)steps + 1));
    if (!hist) {
#pragma omp atomic write
      rc = -2;
    } else {
#pragma omp for schedule(static)
      for (int64_t i = 0; i < n_paths; ++i) {
        const uint64_t path = path_begin + (uint64_t)i;
        int64_t st;
        int kind, value;
        double mg;
        closest_decision(m, k, steps, seed, option_index, path, &st, &kind, &value, &mg);
        if (!(mg < margin_below)) st = -1;
        flip_step[i] = st;
        flip_kind[i] = st >= 0 ? kind : 0;
        flip_value[i] = st >= 0 ? !value : 0;
        path_adjoint_forced(m, k, steps, seed, option_index, path, hist, &x_T[i], &grad[i * 5], st, kind,
                            !value);
      }
    }
    free(hist);
  }
  return rc;
}

/* x_T of one path with one decision imposed (f_step < 0: none) -- the forward
 * simulation of path_adjoint_forced, for finite-difference checks of it. */
double oracle_terminal_forced(const oracle_heston* m, uint32_t steps, uint64_t seed, uint32_t option_index,
                              uint64_t path, int64_t f_step, int f_kind, int f_value) {
  double k[10];
  step_constants(m, steps, k);
  double v = m->v0, x = 0.0;
  for (uint32_t n = 0; n < steps; ++n) {
    double u_v, u_x, mg;
    int br;
    oracle_step_uniforms(seed, option_index, path, n, &u_v, &u_x);
    double vn = ((int64_t)n == f_step) ? qe_step_forced(v, u_v, k, f_kind, f_value)
                                       : oracle_qe_variance_step(v, u_v, k, &br, &mg, NULL);
    const double k0 = step_k0(m, k, v, ((int64_t)n == f_step && f_kind == 1) ? f_value : -1);
    x += k0 + k[5] * v + k[6] * vn + sqrt(k[7] * v + k[8] * vn) * oracle_norminv(u_x);
    v = vn;
  }
  return x;
}

/* One QE variance step for a model and step count (the step function above with
 * the model's constants), for unit tests of the step in isolation. */
double oracle_qe_step(const oracle_heston* m, uint32_t steps, double v, double u_v, int* branch) {
  double k[10], mg;
  step_constants(m, steps, k);
  return oracle_qe_variance_step(v, u_v, k, branch, &mg, NULL);
}

/* The step applied to one variance v and many uniforms (moment checks). */
void oracle_qe_step_array(const oracle_heston* m, uint32_t steps, double v, const double* u_v,
                          double* v_next, int64_t n) {
  double k[10];
  step_constants(m, steps, k);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int br;
    double mg;
    v_next[i] = oracle_qe_variance_step(v, u_v[i], k, &br, &mg, NULL);
  }
}

/* Per-path reverse-mode gradients: grad[i*5 + j], plus x_T per path. */
int oracle_path_grad_reverse(const oracle_heston* m, uint32_t steps, uint64_t seed,
                             uint32_t option_index, uint64_t path_begin, int64_t n_paths,
                             double* x_T, double* grad) {
  if (steps == 0 || n_paths < 0) return -1;
  double k[10];
  step_constants(m, steps, k);
  int rc = 0;
#pragma omp parallel
  {
    double* hist = (double*)malloc(sizeof(double) * ((size_t)steps + 1));
    if (!hist) {
#pragma omp atomic write
      rc = -2;
    } else {
#pragma omp for schedule(static)
      for (int64_t i = 0; i < n_paths; ++i)
        path_adjoint(m, k, steps, seed, option_index, path_begin + (uint64_t)i, hist, &x_T[i],
                     &grad[i * 5]);
    }
    free(hist);
  }
  return rc;
}

/* ---- forward mode with dual numbers (5 tangent directions), independent of the above ---- */
typedef struct {
  double v;
  double d[5];
} dual5;

static dual5 dconst(double c) {
  dual5 r;
  r.v = c;
  for (int i = 0; i < 5; ++i) r.d[i] = 0.0;
  return r;
}
static dual5 dseed(double c, int dir) {
  dual5 r = dconst(c);
  r.d[dir] = 1.0;
  return r;
}
static dual5 dadd(dual5 a, dual5 b) {
  dual5 r;
  r.v = a.v + b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
static dual5 dsub(dual5 a, dual5 b) {
  dual5 r;
  r.v = a.v - b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
static dual5 dmul(dual5 a, dual5 b) {
  dual5 r;
  r.v = a.v * b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
static dual5 ddiv(dual5 a, dual5 b) {
  dual5 r;
  r.v = a.v / b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
static dual5 dscale(dual5 a, double s) {
  for (int i = 0; i < 5; ++i) a.d[i] *= s;
  a.v *= s;
  return a;
}
static dual5 dsqrt(dual5 a) {
  dual5 r;
  r.v = sqrt(a.v);
  for (int i = 0; i < 5; ++i) r.d[i] = (r.v > 0.0) ? a.d[i] / (2.0 * r.v) : 0.0;
  return r;
}
static dual5 dexp(dual5 a) {
  dual5 r;
  r.v = exp(a.v);
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] * r.v;
  return r;
}
static dual5 dlog(dual5 a) {
  dual5 r;
  r.v = log(a.v);
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] / a.v;
  return r;
}

/*
 * Per-path forward-mode tangents d x_T / d(v0, kappa, theta, sigma, rho): the
 * constants and every step are evaluated on dual numbers seeded with the
 * parameters.  Branch decisions are taken on the primal values.
 */
int oracle_path_grad_forward(const oracle_heston* m, uint32_t steps, uint64_t seed,
                             uint32_t option_index, uint64_t path_begin, int64_t n_paths,
                             double* x_T, double* grad) {
  if (steps == 0 || n_paths < 0) return -1;
  const double dt = m->T / (double)steps;
  dual5 v0 = dseed(m->v0, 0), kap = dseed(m->kappa, 1), th = dseed(m->theta, 2);
  dual5 sig = dseed(m->sigma, 3), rho = dseed(m->rho, 4);
  dual5 one = dconst(1.0), half = dconst(0.5);
  dual5 E = dexp(dscale(kap, -dt));
  dual5 sig2 = dmul(sig, sig);
  dual5 omE = dsub(one, E);
  dual5 c1 = ddiv(dmul(dmul(sig2, E), omE), kap);
  dual5 c2 = ddiv(dmul(dmul(th, sig2), dmul(omE, omE)), dscale(kap, 2.0));
  dual5 rho_sig = ddiv(rho, sig);
  dual5 K0 = dadd(dscale(ddiv(dmul(dmul(rho, kap), th), sig), -dt), dconst(m->r * dt));
  dual5 kr = dsub(dmul(kap, rho_sig), half);
  dual5 K1 = dsub(dscale(kr, GAMMA1 * dt), rho_sig);
  dual5 K2 = dadd(dscale(kr, GAMMA2 * dt), rho_sig);
  dual5 om_r2 = dsub(one, dmul(rho, rho));
  dual5 K3 = dscale(om_r2, GAMMA1 * dt);
  dual5 K4 = dscale(om_r2, GAMMA2 * dt);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_paths; ++i) {
    uint64_t path = path_begin + (uint64_t)i;
    dual5 v = v0, x = dconst(0.0);
    for (uint32_t n = 0; n < steps; ++n) {
      double u_v, u_x;
      oracle_step_uniforms(seed, option_index, path, n, &u_v, &u_x);
      dual5 mm = dadd(th, dmul(dsub(v, th), E));
      dual5 s2 = dadd(dmul(v, c1), c2);
      dual5 vn;
      /* QE-M: ln M of this step's branch (Andersen's martingale correction), where it exists */
      const dual5 Aq = dadd(K2, dscale(K4, 0.5));
      dual5 lnM = dconst(0.0);
      int ok = 1;
      if (mm.v <= 0.0) {
        vn = dconst(0.0);
      } else {
        dual5 psi = ddiv(s2, dmul(mm, mm));
        if (psi.v <= PSI_C) {
          dual5 tp = ddiv(dconst(2.0), psi);
          dual5 b2 = dadd(dsub(tp, one), dmul(dsqrt(tp), dsqrt(dsub(tp, one))));
          dual5 a = ddiv(mm, dadd(one, b2));
          dual5 bz = dadd(dsqrt(b2), dconst(oracle_norminv(u_v)));
          vn = dmul(a, dmul(bz, bz));
          dual5 D = dsub(one, dscale(dmul(Aq, a), 2.0));
          ok = D.v > 0.0;
          if (ok) lnM = dsub(ddiv(dmul(dmul(Aq, b2), a), D), dscale(dlog(D), 0.5));
        } else {
          dual5 p = ddiv(dsub(psi, one), dadd(psi, one));
          dual5 beta = ddiv(dsub(one, p), mm);
          if (u_v <= p.v) {
            vn = dconst(0.0);
          } else {
            vn = ddiv(dlog(ddiv(dsub(one, p), dconst(1.0 - u_v))), beta);
          }
          ok = Aq.v < beta.v;
          if (ok) lnM = dlog(dadd(p, ddiv(dmul(beta, dsub(one, p)), dsub(beta, Aq))));
        }
      }
      dual5 k0 = K0;
      if (g_scheme == 1 && ok)
        k0 = dsub(dsub(dconst(m->r * dt), lnM), dmul(dadd(K1, dscale(K3, 0.5)), v));
      dual5 w = dadd(dmul(K3, v), dmul(K4, vn));
      dual5 inc = dadd(dadd(k0, dmul(K1, v)), dmul(K2, vn));
      inc = dadd(inc, dscale(dsqrt(w), oracle_norminv(u_x)));
      x = dadd(x, inc);
      v = vn;
    }
    x_T[i] = x.v;
    for (int j = 0; j < 5; ++j) grad[i * 5 + j] = x.d[j];
  }
  return 0;
}

/*
 * Pathwise (adjoint) price sensitivities per strike, from the reverse-mode
 * per-path gradients:  dP/dq = e^{-rT} mean[ f'(S_T) S_T dx_T/dq ],
 * f'(S) = 1{S > K} for a call and -1{S < K} for a put; dx_T/dS0 = 1/S0 enters
 * via dS_T/dS0 = S_T/S0; for r, dx_T/dr = T and the discount adds -T * price.
 * grad[j*7 + c], c = {S0, v0, kappa, theta, sigma, rho, r}.
 */
int oracle_adjoint(const oracle_heston* m, const double* strikes, int n_strikes, int is_put,
                   uint32_t steps, int64_t paths, uint64_t seed, uint32_t option_index,
                   double* price, double* grad) {
  if (paths <= 0 || n_strikes <= 0 || steps == 0) return -1;
  double* x = (double*)malloc(sizeof(double) * (size_t)paths);
  double* g = (double*)malloc(sizeof(double) * (size_t)paths * 5);
  if (!x || !g) {
    free(x);
    free(g);
    return -2;
  }
  int rc = oracle_path_grad_reverse(m, steps, seed, option_index, 0, paths, x, g);
  double disc = exp(-m->r * m->T);
  for (int j = 0; j < n_strikes && rc == 0; ++j) {
    double K = strikes[j];
    double sf = 0.0, s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < paths; ++i) {
      double sT = m->S0 * exp(x[i]);
      sf += payoff(sT, K, is_put);
      double fp = is_put ? ((sT < K) ? -1.0 : 0.0) : ((sT > K) ? 1.0 : 0.0);
      if (fp == 0.0) continue;
      double w = fp * sT;
      s[0] += w / m->S0;
      for (int c = 0; c < 5; ++c) s[1 + c] += w * g[i * 5 + c];
      s[6] += w * m->T;
    }
    double inv = 1.0 / (double)paths;
    price[j] = disc * sf * inv;
    for (int c = 0; c < 7; ++c) grad[j * 7 + c] = disc * s[c] * inv;
    grad[j * 7 + 6] -= m->T * price[j];
  }
  free(x);
  free(g);
  return rc;
}
