// simr_api.cu -- the C ABI of include/simr.h: context, validation, per-scenario
// constants (FP64 on the host, rounded once to FP32), launches and host staging.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "simr.h"
#include "simr_internal.h"

using namespace simr;

struct simr_ctx {
  int device = 0;
  int num_sms = 0;
  // path-kernel scratch: partial rows + ticket
  double* partials = nullptr;
  size_t partial_doubles = 0;
  // 256-byte block: ticket word at 0, status word at 64, batch queue counter at
  // 128, Longstaff-Schwartz ticket at 192, its sweep barrier counter at 208
  unsigned int* ticket = nullptr;
  int scheme = SIMR_SCHEME_QE;  // log-spot scheme of the path simulations (simr_set_scheme)
  float* ckpt = nullptr;  // adjoint checkpoints, [slot][resident thread]
  size_t ckpt_floats = 0;
  float* gseg = nullptr;  // adjoint segment buffers too long for shared memory, [3 k][resident thread]
  size_t gseg_floats = 0;
  // Longstaff-Schwartz: states at the exercise dates, per-path cash flows,
  // coefficients, discount table
  float* lsm_S = nullptr;
  size_t lsm_S_cap = 0;
  float* lsm_V = nullptr;
  size_t lsm_V_cap = 0;
  float* lsm_cash = nullptr;
  size_t lsm_cash_cap = 0;
  int32_t* lsm_stop = nullptr;
  size_t lsm_stop_cap = 0;
  double* lsm_beta = nullptr;  // [2][n_ex][6]: reported basis, then the scaled one
  size_t lsm_beta_cap = 0;
  float4* lsm_xform = nullptr;
  size_t lsm_xform_cap = 0;
  float* lsm_dpow = nullptr;
  size_t lsm_dpow_cap = 0;
  int* status = nullptr;
  // staging for host-pointer arguments
  double* dev_strikes = nullptr;
  size_t strikes_cap = 0;
  double* dev_out = nullptr;
  size_t out_cap = 0;
  double* host_out = nullptr;  // pinned: the staged results and the status word on their way back
  size_t host_out_cap = 0;
  float* dev_f32 = nullptr;
  size_t f32_cap = 0;
  // batched book: device tables, per-item partial rows, pinned upload staging
  BatchOption* b_opts = nullptr;
  size_t b_opts_cap = 0;
  BatchItem* b_items = nullptr;
  size_t b_items_cap = 0;
  double* b_partials = nullptr;
  size_t b_partials_cap = 0;
  unsigned char* b_host = nullptr;  // pinned
  size_t b_host_cap = 0;
  cudaEvent_t b_uploaded = nullptr;  // the last upload from b_host has completed
  uint64_t graph_key = 0;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t g_stream = nullptr;  // graphs are captured and launched here (non-blocking)
  cudaEvent_t g_in = nullptr, g_out = nullptr;
  struct Tune {
    uint64_t key;
    uint32_t chunk;
    int32_t variant;  // batch kernel shape (batch_variant)
  };
  std::vector<Tune> tune;
  bool tune_loaded = false;  // $SIMR_TUNE_CACHE read
  char gpu_name[256] = "";
  struct AdjK {  // adjoint_max_ckpt_every per strike tile, found once
    int32_t nk_pad;
    int32_t k_max;
  };
  std::vector<AdjK> adj_k;
};

namespace {

thread_local char g_err[512] = "";

// simr_inject_fault: the armed kind and the requests left until it fires
std::atomic<int> g_fault_what{0}, g_fault_left{0};

// An NVTX range around a C-ABI call (visible to Nsight Systems and Nsight
// Compute's NVTX filters; a no-op without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SIMR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite(double x) { return std::isfinite(x); }

int check_model(const simr_heston* m) {
  if (!m) return fail(SIMR_EINVAL, "model is NULL");
  const double v[8] = {m->S0, m->r, m->T, m->v0, m->kappa, m->theta, m->sigma, m->rho};
  for (double x : v)
    if (!finite(x)) return fail(SIMR_EINVAL, "model has a non-finite value");
  if (!(m->S0 > 0)) return fail(SIMR_EINVAL, "S0 must be > 0");
  if (!(m->T > 0)) return fail(SIMR_EINVAL, "T must be > 0");
  if (!(m->v0 >= 0)) return fail(SIMR_EINVAL, "v0 must be >= 0");
  if (!(m->theta >= 0)) return fail(SIMR_EINVAL, "theta must be >= 0");
  if (!(m->kappa > 0)) return fail(SIMR_EINVAL, "kappa must be > 0");
  if (!(m->sigma > 0)) return fail(SIMR_EINVAL, "sigma must be > 0");
  if (!(m->rho >= -1.0 && m->rho <= 1.0)) return fail(SIMR_EINVAL, "rho must lie in [-1, 1]");
  return SIMR_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
int ensure(T** buf, size_t* cap, size_t n, const char* what) {
  if (take_fault(SIMR_FAULT_ALLOC))
    return fail(SIMR_ENOMEM, "cudaMalloc of %s (%zu bytes) failed: injected fault", what, n * sizeof(T));
  if (*cap >= n) return SIMR_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc((void**)buf, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SIMR_ENOMEM, "cudaMalloc of %s (%zu bytes) failed: %s", what, n * sizeof(T),
                cudaGetErrorString(e));
  }
  *cap = n;
  return SIMR_OK;
}

// FP64 constants of one scenario (formulas in simr_device.cuh), in the order
// E, thE, c1, c2, C0, Cv, Cd, Cdl, sK3.
void scen_const64(const simr_heston& m, uint32_t steps, double out[9]) {
  const double dt = m.T / (double)steps;
  const double kdt = m.kappa * dt;
  const double E = std::exp(-kdt);
  const double omE = -std::expm1(-kdt);
  const double s2 = m.sigma * m.sigma;
  const double rs = m.rho / m.sigma;
  const double Cd = rs * (omE - 0.5 * kdt * (1.0 + E));
  out[0] = E;
  out[1] = m.theta * omE;
  out[2] = s2 * E * omE / m.kappa;
  out[3] = m.theta * s2 * omE * omE / (2.0 * m.kappa);
  out[4] = m.r * dt + Cd * m.theta;
  out[5] = -0.25 * dt;
  out[6] = Cd;
  out[7] = rs * (1.0 + 0.5 * kdt);
  out[8] = std::sqrt(0.5 * dt * (1.0 - m.rho * m.rho));
}

ScenConst pack(const double c[9], double ratio, double v0) {
  ScenConst s;
  s.E = (float)c[0];
  s.thE = (float)c[1];
  s.h1 = (float)(0.5 * c[2]);  // halves of c1, c2: the step carries s^2 / 2
  s.h2 = (float)(0.5 * c[3]);
  s.C0 = (float)c[4];
  s.Cv = (float)c[5];
  s.Cd = (float)c[6];
  s.Cdl = (float)c[7];
  s.sK3 = (float)c[8];
  s.ratio = (float)ratio;
  s.v0 = (float)v0;
  s.pad = 0.0f;
  return s;
}

// Base scenario: full constants.
ScenConst base_const(const simr_heston& m, uint32_t steps) {
  double c[9];
  scen_const64(m, steps, c);
  return pack(c, 1.0, m.v0);
}

// Bumped scenario: the FP64 difference of the exact constants, added in the
// kernel to the base scenario's FP32 constants -- the bumped scenario is the
// base scenario's FP32 model moved by the exact bump (so a v0-only bump has zero
// deltas); v0 is the scenario's own FP32 initial variance.
ScenConst bumped_const(const simr_heston& base, const simr_heston& bumped, uint32_t steps) {
  double cb[9], cs[9], d[9];
  scen_const64(base, steps, cb);
  scen_const64(bumped, steps, cs);
  for (int i = 0; i < 9; ++i) d[i] = cs[i] - cb[i];
  const double ratio_m1 = std::expm1(-bumped.r * bumped.T + base.r * base.T);
  return pack(d, ratio_m1, bumped.v0);
}

// FP64 step-0 quantities of a scenario starting from v0 (formulas in simr_device.cuh):
// out = {a, b, q, C, L, m0, K0p}, returns the branch.
int first_step64(const simr_heston& m, uint32_t steps, double v0, double out[7]) {
  double c[9];
  scen_const64(m, steps, c);
  const double E = c[0], thE = c[1], c1 = c[2], c2 = c[3], C0 = c[4], Cv = c[5], Cd = c[6];
  const double m0 = thE + v0 * E, s20 = v0 * c1 + c2;
  for (int i = 0; i < 7; ++i) out[i] = 0.0;
  out[5] = m0;
  out[6] = C0 + (Cv - Cd) * v0;
  if (!(m0 > 0.0)) return 2;
  const double psi = s20 / (m0 * m0);
  if (psi <= 1.5) {
    const double t = 2.0 / psi;
    const double b2 = t - 1.0 + std::sqrt(t) * std::sqrt(t - 1.0);
    out[0] = m0 / (1.0 + b2);
    out[1] = std::sqrt(b2);
    return 0;
  }
  const double q = 2.0 / (psi + 1.0);
  out[2] = q;
  out[3] = m0 / q;
  out[4] = std::log(q);
  return 1;
}

void philox_round_keys(uint64_t seed, uint32_t rk[10][2]) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int i = 0; i < 10; ++i) {
    rk[i][0] = k0;
    rk[i][1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

int popcount9(uint32_t m) {
  int n = 0;
  for (int b = 0; b < kMaxGreeks; ++b) n += (m >> b) & 1u;
  return n;
}

// Build the launch descriptor: base scenario, re-simulated scenarios per Greek,
// analytic bumps and the FP64 normalisation constants.
int build_launch(const simr_heston* m, int n_strikes, int is_put, uint32_t steps, uint64_t path_begin,
                 uint64_t path_count, uint64_t paths_total, uint64_t seed, uint32_t option_index,
                 double rel_bump, uint32_t mask, PathLaunch* L, simr_heston* scen_out = nullptr) {
  std::memset(L, 0, sizeof(*L));
  philox_round_keys(seed, L->rk);
  L->path_begin = path_begin;
  L->path_count = path_count;
  L->steps = steps;
  L->option_index = option_index;
  L->n_strikes = n_strikes;
  L->nk_pad = n_strikes == 1 ? 1 : ((n_strikes + 31) / 32) * 32;
  L->n_acc = 2 + popcount9(mask);
  L->is_put = is_put ? 1 : 0;
  L->greek_mask = mask;
  L->S0 = (float)m->S0;
  L->h_s = (float)rel_bump;
  L->disc = std::exp(-m->r * m->T);
  L->paths_total = (double)paths_total;
  L->sc[0] = base_const(*m, steps);
  simr_heston scen_model[kMaxScen];
  scen_model[0] = *m;
  int ns = 1, r = 0, g = 0;
  for (int bit = 0; bit < kMaxGreeks; ++bit) {
    if (!((mask >> bit) & 1u)) continue;
    const uint32_t b = 1u << bit;
    double denom = 1.0;
    if (b == SIMR_G_DELTA) {
      denom = 2.0 * rel_bump * m->S0;
    } else if (b == SIMR_G_GAMMA) {
      denom = (rel_bump * m->S0) * (rel_bump * m->S0);
    } else if (b == SIMR_G_RHO) {
      double h = rel_bump * std::fabs(m->r);
      if (h == 0.0) h = rel_bump;
      L->rho_em = std::exp(-h * m->T);
      L->rho_w = 2.0 * std::sinh(h * m->T);
      denom = 2.0 * h;
    } else {
      // re-simulated: field selection
      simr_heston up = *m, dn = *m;
      double* fu;
      double* fd;
      double val;
      bool absolute = false, nonneg = false, unit = false;
      double sign = 1.0;
      if (b == SIMR_G_VEGA) {
        fu = &up.v0; fd = &dn.v0; val = m->v0; nonneg = true;
      } else if (b == SIMR_G_THETA) {
        fu = &up.T; fd = &dn.T; val = m->T; sign = -1.0;
      } else if (b == SIMR_G_KAPPA) {
        fu = &up.kappa; fd = &dn.kappa; val = m->kappa;
      } else if (b == SIMR_G_LRVAR) {
        fu = &up.theta; fd = &dn.theta; val = m->theta; nonneg = true;
      } else if (b == SIMR_G_VOLVOL) {
        fu = &up.sigma; fd = &dn.sigma; val = m->sigma;
      } else {
        fu = &up.rho; fd = &dn.rho; val = m->rho; absolute = true; unit = true;
      }
      double h = absolute ? rel_bump : rel_bump * std::fabs(val);
      if (h == 0.0) h = rel_bump;
      *fu = val + h;
      *fd = val - h;
      bool up_ok = true, dn_ok = true;
      if (nonneg && *fd < 0.0) dn_ok = false;
      if (unit && *fd < -1.0) dn_ok = false;
      if (unit && *fu > 1.0) up_ok = false;
      int iu = 0, id = 0;
      double hu = 0.0, hd = 0.0;
      // v0 is only the initial state: the kernel starts each scenario from its
      // FP32 value, so the realised bump is the difference of those values.
      const double v0f = (double)(float)m->v0;
      if (up_ok) {
        iu = ns;
        scen_model[ns] = up;
        L->sc[ns++] = bumped_const(*m, up, steps);
        hu = (b == SIMR_G_VEGA) ? (double)(float)up.v0 - v0f : h;
      }
      if (dn_ok) {
        id = ns;
        scen_model[ns] = dn;
        L->sc[ns++] = bumped_const(*m, dn, steps);
        hd = (b == SIMR_G_VEGA) ? v0f - (double)(float)dn.v0 : h;
      }
      L->resim_up[r] = iu;
      L->resim_dn[r] = id;
      ++r;
      denom = sign * (hu + hd);
      if (!(denom != 0.0)) return fail(SIMR_EINVAL, "degenerate bump for Greek bit %d", bit);
    }
    L->denom[g++] = denom;
  }
  L->n_scen = ns;
  // the paired steps' operands, packed once here
  for (int k = 0; 2 * k + 1 < ns; ++k)
    L->pair2[k] = pack_const(L->sc[2 * k + 1], L->sc[2 * k + 2 < ns ? 2 * k + 2 : 2 * k + 1]);
  // vega is the first re-simulated Greek in bit order, so its two-sided bump occupies
  // scenarios 1 and 2 when present
  L->n_v0_scen = ((mask & SIMR_G_VEGA) && L->resim_up[0] == 1 && L->resim_dn[0] == 2) ? 2 : 0;
  // step-0 constants: base full values, bumped scenarios the exact differences to them
  double fb[7];
  const int br0 = first_step64(*m, steps, (double)L->sc[0].v0, fb);
  L->first_split = ns > 1 ? 1 : 0;
  for (int s = 0; s < ns; ++s) {
    double f[7];
    const int br = s == 0 ? br0 : first_step64(scen_model[s], steps, (double)L->sc[s].v0, f);
    if (s == 0) {
      for (int i = 0; i < 7; ++i) f[i] = fb[i];
    } else {
      if (br != br0) L->first_split = 0;  // a bump moved step 0 across a branch: plain step 0
      for (int i = 0; i < 7; ++i)
        if (i != 2) f[i] -= fb[i];
    }
    FirstConst& fc = L->f0[s];
    fc.a = (float)f[0];
    fc.b = (float)f[1];
    fc.q = (float)f[2];
    fc.C = (float)f[3];
    fc.L = (float)f[4];
    fc.m0 = (float)f[5];
    fc.K0p = (float)f[6];
    fc.branch = br;
  }
  if (scen_out)
    for (int s = 0; s < ns; ++s) scen_out[s] = scen_model[s];
  return SIMR_OK;
}

// Checkpoint interval and the FP64-derived parameter-map constants of the
// adjoint kernel (formulas beside the kernel in simr_adjoint.cu).
int build_adjoint(const simr_heston& m, uint32_t steps, uint32_t ckpt_every, AdjConst* A) {
  uint32_t k = ckpt_every;
  if (k == 0) {  // the even k near sqrt(steps / 3) that minimises steps / k + 3 k shared floats
    k = 2;
    while (3ull * k * k < steps) k += 2;
  }
  if ((k & 1u) || k < 2 || k > 1024) return fail(SIMR_EINVAL, "ckpt_every must be 0 or an even number in [2, 1024]");
  if (k > steps) k = steps + (steps & 1u);  // one segment either way; size its buffer to the path
  const double dt = m.T / (double)steps, kdt = m.kappa * dt;
  const double E = std::exp(-kdt), omE = -std::expm1(-kdt), s2 = m.sigma * m.sigma, rs = m.rho / m.sigma;
  const double dE_dk = -dt * E;
  const double D = omE - 0.5 * kdt * (1.0 + E);
  const double B = 1.0 + 0.5 * kdt;
  const double sK3 = std::sqrt(0.5 * dt * (1.0 - m.rho * m.rho));
  A->ckpt_every = (int32_t)k;
  A->n_seg = (int32_t)((steps + k - 1) / k);
  A->theta = (float)m.theta;
  A->invS0 = (float)(1.0 / m.S0);
  A->T = (float)m.T;
  A->dE_dk = dE_dk;
  A->omE = omE;
  A->dc1_dk = s2 * ((1.0 - 2.0 * E) * dE_dk / m.kappa - E * omE / (m.kappa * m.kappa));
  A->dc2_dk = m.theta * s2 * (-omE * dE_dk / m.kappa - omE * omE / (2.0 * m.kappa * m.kappa));
  A->dc2_dth = s2 * omE * omE / (2.0 * m.kappa);
  A->dCd_dk = rs * (-dE_dk - 0.5 * dt * (1.0 + E) - 0.5 * kdt * dE_dk);
  A->dCdl_dk = rs * 0.5 * dt;
  A->N_Cd = (double)steps * rs * D;
  A->two_over_sigma = 2.0 / m.sigma;
  A->c1 = s2 * E * omE / m.kappa;
  A->c2 = m.theta * s2 * omE * omE / (2.0 * m.kappa);
  A->Cd_over_sigma = rs * D / m.sigma;
  A->Cdl_over_sigma = rs * B / m.sigma;
  A->D_over_sigma = D / m.sigma;
  A->B_over_sigma = B / m.sigma;
  A->dsK3_drho = sK3 > 0.0 ? -m.rho * dt / (2.0 * sK3) : __builtin_nan("");
  A->qem = 0;  // plain QE unless adjoint_scheme sets QE-M
  A->Cd = A->dqa_drho = A->dK2_dk = A->dK2_ds = A->dK2_dr = A->dA_dk = A->dA_ds = A->dA_dr = 0.0;
  return SIMR_OK;
}

int check_common(simr_ctx* ctx, const simr_heston* m, const double* strikes, int n_strikes, int max_strikes,
                 uint32_t steps, uint64_t paths) {
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  int rc = check_model(m);
  if (rc) return rc;
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be >= 1");
  if (paths < 1) return fail(SIMR_EINVAL, "paths must be >= 1");
  if (!strikes) return fail(SIMR_EINVAL, "strikes is NULL");
  if (n_strikes < 1 || n_strikes > max_strikes)
    return fail(SIMR_EINVAL, "n_strikes must lie in [1, %d]", max_strikes);
  return SIMR_OK;
}

int check_strikes_host(const double* strikes, int n) {
  for (int i = 0; i < n; ++i)
    if (!(strikes[i] > 0) || !finite(strikes[i])) return fail(SIMR_EINVAL, "strike %d must be finite and > 0", i);
  return SIMR_OK;
}

// Return a device pointer to the strikes.  Host strikes are validated here and
// copied to staging; device strikes are validated by the kernel, which sets bit 0
// of the context's status word (reported by simr_sync) and yields NaN results.
int stage_strikes(simr_ctx* ctx, const double* strikes, int n, cudaStream_t st, const double** dev) {
  if (is_device_ptr(strikes)) {
    *dev = strikes;
    return SIMR_OK;
  }
  int rc = check_strikes_host(strikes, n);
  if (rc) return rc;
  rc = ensure(&ctx->dev_strikes, &ctx->strikes_cap, (size_t)n, "strike staging");
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(ctx->dev_strikes, strikes, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copying strikes");
  *dev = ctx->dev_strikes;
  return SIMR_OK;
}

// The device status word h as read from the device: clear it there, report it.
int decode_status(simr_ctx* ctx, int h, cudaStream_t st) {
  cudaError_t e = h ? cudaMemsetAsync(ctx->status, 0, sizeof(int), st) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "clearing the device status");
  if (h & 1) return fail(SIMR_EINVAL, "a device-resident strike was not finite and > 0 (results are NaN)");
  if (h & 2) return fail(SIMR_ETIMEOUT, "a wait of the Longstaff-Schwartz sweep (grid barrier or state copy) timed out (results invalid)");
  return SIMR_OK;
}

// Read and clear the device status word (the stream must be idle).
int take_status(simr_ctx* ctx, cudaStream_t st) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
  return decode_status(ctx, h, st);
}

struct OutStage {
  double* user[3] = {nullptr, nullptr, nullptr};
  double* dev[3] = {nullptr, nullptr, nullptr};
  size_t n[3] = {0, 0, 0};
  bool any_host = false;
};

// Map each output (price, stderr, greeks/sums) to a device pointer; host outputs
// are placed in the context's staging buffer and copied back after the launch.
int stage_outputs(simr_ctx* ctx, OutStage* o) {
  size_t total = 0;
  for (int i = 0; i < 3; ++i)
    if (o->user[i] && !is_device_ptr(o->user[i])) total += o->n[i], o->any_host = true;
  if (o->any_host) {
    int rc = ensure(&ctx->dev_out, &ctx->out_cap, total, "output staging");
    if (rc) return rc;
  }
  size_t off = 0;
  for (int i = 0; i < 3; ++i) {
    if (!o->user[i]) continue;
    if (is_device_ptr(o->user[i])) {
      o->dev[i] = o->user[i];
    } else {
      o->dev[i] = ctx->dev_out + off;
      off += o->n[i];
    }
  }
  return SIMR_OK;
}

// Results for host buffers: the staged block (dev_out, the host outputs in
// order) and the status word come back by two copies into pinned host memory and
// one synchronisation, then go to the caller's buffers on the host.
int finish_outputs(simr_ctx* ctx, const OutStage& o, cudaStream_t st) {
  if (!o.any_host) return SIMR_OK;
  size_t total = 0;
  for (int i = 0; i < 3; ++i)
    if (o.user[i] && o.dev[i] != o.user[i]) total += o.n[i];
  if (ctx->host_out_cap < total + 1) {  // + one double's room for the status word
    cudaError_t e = cudaStreamSynchronize(st);  // (nothing in flight may still target the old buffer)
    if (e != cudaSuccess) return cuda_fail(e, "synchronising the stream");
    if (ctx->host_out) cudaFreeHost(ctx->host_out);
    ctx->host_out = nullptr;
    ctx->host_out_cap = 0;
    e = cudaHostAlloc((void**)&ctx->host_out, (total + 1) * sizeof(double), cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SIMR_ENOMEM, "pinned result staging of %zu bytes: %s", (total + 1) * sizeof(double),
                  cudaGetErrorString(e));
    }
    ctx->host_out_cap = total + 1;
  }
  int* h_status = reinterpret_cast<int*>(ctx->host_out + total);
  cudaError_t e = cudaMemcpyAsync(ctx->host_out, ctx->dev_out, total * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "copying results to the host");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "synchronising the stream");
  size_t off = 0;
  for (int i = 0; i < 3; ++i) {
    if (o.user[i] && o.dev[i] != o.user[i]) {
      std::memcpy(o.user[i], ctx->host_out + off, o.n[i] * sizeof(double));
      off += o.n[i];
    }
  }
  return decode_status(ctx, *h_status, st);
}

int with_device(simr_ctx* ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return SIMR_OK;
}

// QE-M constants in FP64: r dt, qa = dt (1 - rho^2)/4 (= K3/2 = K4/2),
// K2 = dt/2 (kappa rho/sigma - 1/2) + rho/sigma, A = K2 + K4/2 = K2 + qa.
void qem_const64(const simr_heston& m, uint32_t steps, double q[4]) {
  const double dt = m.T / (double)steps;
  const double K2 = 0.5 * dt * (m.kappa * m.rho / m.sigma - 0.5) + m.rho / m.sigma;
  const double qa = 0.25 * dt * (1.0 - m.rho * m.rho);
  q[0] = m.r * dt;
  q[1] = qa;
  q[2] = K2;
  q[3] = K2 + qa;
}

// Two scenarios' (or assets') QE-M constants lane by lane.
QemConst2 pack_qem(const QemConst& a, const QemConst& b) {
  return QemConst2{make_float2(a.rdt, b.rdt), make_float2(a.qa, b.qa), make_float2(a.K2, b.K2),
                   make_float2(a.A, b.A)};
}

QemConst qem_const(const simr_heston& m, uint32_t steps) {
  double q[4];
  qem_const64(m, steps, q);
  return QemConst{(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
}

// The QE-M first-step constant of a scenario starting from v0, in FP64:
// r dt - qa (v0 + m0) - lam(v0), lam = ln M - A m0 in the branch of step 0
// (quadratic: 2 (A a)^2 b^2 / (1 - u) + g(u)/2 with u = 2 A a and
// g(u) = -u - ln(1 - u); exponential: ln(1 + q w / (1 - w)) - q w with
// q = 1 - p, w = A / beta; zero mean: lam = 0).  False where M does not exist.
bool qem_first64(const simr_heston& m, uint32_t steps, double v0, double* K0q) {
  double c[9], q[4];
  scen_const64(m, steps, c);
  qem_const64(m, steps, q);
  const double m0 = c[1] + v0 * c[0], s20 = v0 * c[2] + c[3], A = q[3];
  double lam = 0.0;
  if (m0 > 0.0) {
    const double psi = s20 / (m0 * m0);
    if (psi <= 1.5) {
      const double t = 2.0 / psi;
      const double b2 = t - 1.0 + std::sqrt(t) * std::sqrt(t - 1.0);
      const double a = m0 / (1.0 + b2);
      const double u = 2.0 * A * a;
      if (!(u < 1.0)) return false;
      lam = 0.5 * u * u * b2 / (1.0 - u) + 0.5 * (-u - std::log1p(-u));
    } else {
      const double qq = 2.0 / (psi + 1.0);  // 1 - p
      const double w = A * m0 / qq;         // A / beta, beta = (1 - p) / m0
      if (!(w < 1.0)) return false;
      lam = std::log1p(qq * w / (1.0 - w)) - qq * w;
    }
  }
  *K0q = q[0] - q[1] * (v0 + m0) - lam;
  return true;
}

// The context's scheme on a path launch.  QE-M with bumped scenarios (scen: the
// launch's scenario models, base first) adds each scenario's QE-M constant
// deltas to the base's, in FP64; step 0's split (the CRN first step) takes the
// QE-M first-step constants where M exists at every scenario's v0, and is
// dropped otherwise.
int apply_scheme(const simr_ctx* ctx, const simr_heston& m, uint32_t steps, PathLaunch* L,
                 const simr_heston* scen = nullptr) {
  if (ctx->scheme == SIMR_SCHEME_QE) return SIMR_OK;
  L->scheme = 1;
  L->qm = qem_const(m, steps);
  if (L->n_scen == 1) return SIMR_OK;
  if (!scen) return fail(SIMR_EUNSUPPORTED, "internal: QE-M bumped scenarios without their models");
  double qb[4];
  qem_const64(m, steps, qb);
  L->qmd[0] = QemConst{0.0f, 0.0f, 0.0f, 0.0f};
  for (int s = 1; s < L->n_scen; ++s) {
    double qs[4];
    qem_const64(scen[s], steps, qs);
    L->qmd[s] = QemConst{(float)(qs[0] - qb[0]), (float)(qs[1] - qb[1]), (float)(qs[2] - qb[2]),
                         (float)(qs[3] - qb[3])};
  }
  for (int k = 0; 2 * k + 1 < L->n_scen; ++k)  // the paired steps' operands (as pair2)
    L->qmd2[k] = pack_qem(L->qmd[2 * k + 1], L->qmd[2 * k + 2 < L->n_scen ? 2 * k + 2 : 2 * k + 1]);
  if (L->first_split) {
    double k0b = 0.0;
    bool ok = qem_first64(m, steps, (double)L->sc[0].v0, &k0b);
    double k0s[kMaxScen];
    for (int s = 1; s < L->n_scen && ok; ++s) ok = qem_first64(scen[s], steps, (double)L->sc[s].v0, &k0s[s]);
    if (!ok) {
      L->first_split = 0;
    } else {
      L->f0[0].K0p = (float)k0b;
      for (int s = 1; s < L->n_scen; ++s) L->f0[s].K0p = (float)(k0s[s] - k0b);
    }
  }
  return SIMR_OK;
}

// The FP64 derivatives of the QE-M constants in the adjoint's map (qa, K2 and
// A = K2 + qa in kappa, sigma and rho; Cd theta's coefficient per plain step).
void adjoint_qem_fields(const simr_heston& m, uint32_t steps, AdjConst* A) {
  const double dt = m.T / (double)steps, kdt = m.kappa * dt, E = std::exp(-kdt), omE = -std::expm1(-kdt);
  const double sg = m.sigma, r = m.rho;
  A->qem = 1;
  A->Cd = (r / sg) * (omE - 0.5 * kdt * (1.0 + E));
  A->dqa_drho = -0.5 * dt * r;
  A->dK2_dk = 0.5 * dt * r / sg;
  A->dK2_ds = -0.5 * dt * m.kappa * r / (sg * sg) - r / (sg * sg);
  A->dK2_dr = 0.5 * dt * m.kappa / sg + 1.0 / sg;
  A->dA_dk = A->dK2_dk;
  A->dA_ds = A->dK2_ds;
  A->dA_dr = A->dK2_dr + A->dqa_drho;
}

// The context's scheme on an adjoint launch: under QE-M the launch's scheme and
// QemConst, and the adjoint map's QE-M fields.
void adjoint_scheme(const simr_ctx* ctx, const simr_heston& m, uint32_t steps, PathLaunch* L, AdjConst* A) {
  A->qem = 0;
  if (ctx->scheme != SIMR_SCHEME_QEM) return;
  L->scheme = 1;
  L->qm = qem_const(m, steps);
  adjoint_qem_fields(m, steps, A);
}

int ensure_scratch(simr_ctx* ctx, const PathLaunch& L) {
  return ensure(&ctx->partials, &ctx->partial_doubles, paths_scratch_doubles(L, ctx->num_sms), "reduction scratch");
}

int run_paths(simr_ctx* ctx, const PathLaunch& L, const double* dev_strikes, OutStage& o, cudaStream_t st) {
  int rc = ensure_scratch(ctx, L);
  if (rc) return rc;
  PathOutputs out{};
  out.status = ctx->status;
  if (L.raw_sums) {
    out.sums = o.dev[0];
  } else {
    out.price = o.dev[0];
    out.stderr_ = o.dev[1];
    out.greeks = o.dev[2];
  }
  Scratch s{ctx->partials, ctx->ticket, ctx->partial_doubles};
  int grid = 0;
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_paths(L, dev_strikes, out, s, ctx->num_sms, st, &grid);
  if (e != cudaSuccess) return cuda_fail(e, "launching the path kernel");
  return finish_outputs(ctx, o, st);
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

// Per-option device records (caller's order) and the longest-first order.
int build_batch_options(const simr_option* opts, int n, bool adjoint, bool qem, std::vector<BatchOption>* out,
                        bool one_segment, std::vector<uint32_t>* order, int* ckpt_rows, int* seg_rows) {
  out->resize(n);
  std::vector<double> cost(n);
  int crows = 0, srows = 0;
  for (int i = 0; i < n; ++i) {
    const simr_option& o = opts[i];
    int rc = check_model(&o.m);
    if (rc) {
      char msg[sizeof(g_err)];
      std::strncpy(msg, g_err, sizeof(msg) - 1);
      msg[sizeof(msg) - 1] = 0;
      return fail(SIMR_EINVAL, "option %d: %s", i, msg);
    }
    if (!(o.K > 0.0) || !finite(o.K)) return fail(SIMR_EINVAL, "option %d: strike must be finite and > 0", i);
    if (o.steps < 1 || o.paths < 1) return fail(SIMR_EINVAL, "option %d: steps and paths must be >= 1", i);
    if (o.paths > (1ull << 40)) return fail(SIMR_EINVAL, "option %d: paths beyond 2^40", i);
    BatchOption& b = (*out)[i];
    std::memset(&b, 0, sizeof(b));
    b.sc = base_const(o.m, o.steps);
    if (adjoint) {
      // one segment of the whole path (global segments), or the interval near
      // sqrt(steps / 3) that needs the least shared memory
      if ((rc = build_adjoint(o.m, o.steps, one_segment ? o.steps + (o.steps & 1u) : 0u, &b.A))) return rc;
      crows = std::max(crows, b.A.n_seg - 1);
      srows = std::max(srows, b.A.ckpt_every);
      if (qem) adjoint_qem_fields(o.m, o.steps, &b.A);
    }
    if (qem) b.qm = qem_const(o.m, o.steps);
    b.S0 = (float)o.m.S0;
    b.K = (float)o.K;
    b.invS0 = (float)(1.0 / o.m.S0);
    b.T = (float)o.m.T;
    b.is_put = o.is_put ? 1 : 0;
    b.steps = o.steps;
    b.option_index = (uint32_t)i;
    b.paths = o.paths;
    b.disc = std::exp(-o.m.r * o.m.T);
    cost[i] = (double)o.steps * (double)o.paths;
  }
  order->resize(n);
  std::iota(order->begin(), order->end(), 0u);
  std::stable_sort(order->begin(), order->end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
  *ckpt_rows = crows + (crows & 1);  // even: the segment pairs stay 8-byte aligned
  *seg_rows = srows;
  return SIMR_OK;
}

// Sorted option table and its items of `chunk` paths, in pinned staging, then uploaded.
int upload_batch(simr_ctx* ctx, const std::vector<BatchOption>& opts, const std::vector<uint32_t>& order,
                 uint32_t chunk, cudaStream_t st, uint32_t* n_items_out) {
  const size_t n = opts.size();
  uint64_t n_items = 0;
  for (uint32_t o : order) n_items += (opts[o].paths + chunk - 1) / chunk;
  if (n_items > 0xffffffffull) return fail(SIMR_EUNSUPPORTED, "book needs more than 2^32 work items");
  const size_t bytes = n * sizeof(BatchOption) + n_items * sizeof(BatchItem);
  int rc;
  if (ctx->b_uploaded) {
    cudaError_t e = cudaEventSynchronize(ctx->b_uploaded);  // staging still in use by the last upload?
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the previous upload");
  }
  if (ctx->b_host_cap < bytes) {
    if (ctx->b_host) cudaFreeHost(ctx->b_host);
    ctx->b_host = nullptr;
    ctx->b_host_cap = 0;
    cudaError_t e = cudaHostAlloc((void**)&ctx->b_host, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SIMR_ENOMEM, "pinned staging of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    ctx->b_host_cap = bytes;
  }
  BatchOption* ho = reinterpret_cast<BatchOption*>(ctx->b_host);
  BatchItem* hi = reinterpret_cast<BatchItem*>(ctx->b_host + n * sizeof(BatchOption));
  uint64_t it = 0;
  for (size_t j = 0; j < n; ++j) {
    BatchOption b = opts[order[j]];
    b.item_begin = (uint32_t)it;
    const uint64_t cnt = (b.paths + chunk - 1) / chunk;
    b.item_count = (uint32_t)cnt;
    for (uint64_t q = 0; q < cnt; ++q) {
      const uint64_t pb = q * chunk;
      hi[it + q].option = (uint32_t)j;
      hi[it + q].count = (uint32_t)std::min<uint64_t>(chunk, b.paths - pb);
      hi[it + q].path_begin = pb;
    }
    it += cnt;
    ho[j] = b;
  }
  if ((rc = ensure(&ctx->b_opts, &ctx->b_opts_cap, n, "batch option table"))) return rc;
  if ((rc = ensure(&ctx->b_items, &ctx->b_items_cap, (size_t)n_items, "batch item table"))) return rc;
  cudaError_t e = cudaMemcpyAsync(ctx->b_opts, ho, n * sizeof(BatchOption), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->b_items, hi, (size_t)n_items * sizeof(BatchItem), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !ctx->b_uploaded) e = cudaEventCreateWithFlags(&ctx->b_uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->b_uploaded, st);
  if (e != cudaSuccess) return cuda_fail(e, "uploading the book");
  *n_items_out = (uint32_t)n_items;
  return SIMR_OK;
}

}  // namespace

bool simr::take_fault(int what) {
  if (g_fault_what.load(std::memory_order_relaxed) != what) return false;
  if (g_fault_left.fetch_sub(1) != 1) return false;
  g_fault_what.store(0);
  return true;
}

extern "C" {

int simr_inject_fault(int what, int after) {
  if (what == 0) {
    g_fault_what.store(0);
    return SIMR_OK;
  }
  if ((what != SIMR_FAULT_ALLOC && what != SIMR_FAULT_LAUNCH && what != SIMR_FAULT_BARRIER) || after < 1 ||
      after > (1 << 30))
    return fail(SIMR_EINVAL,
                "simr_inject_fault: what must be 0, SIMR_FAULT_ALLOC, SIMR_FAULT_LAUNCH or SIMR_FAULT_BARRIER, after >= 1");
  g_fault_what.store(0);
  g_fault_left.store(after);
  g_fault_what.store(what);
  return SIMR_OK;
}

int simr_version(void) { return 100; }

const char* simr_last_error(void) { return g_err; }

int simr_create(simr_ctx** out, int device) {
  if (!out) return fail(SIMR_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(SIMR_EINVAL, "device %d out of range (%d devices)", device, n);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  simr_ctx* c = new (std::nothrow) simr_ctx();
  if (!c) return fail(SIMR_ENOMEM, "host allocation failed");
  c->device = device;
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceProp prop;
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "querying the device");
  }
  std::snprintf(c->gpu_name, sizeof(c->gpu_name), "%s", prop.name);
  for (char* q = c->gpu_name; *q; ++q)
    if (*q == '"' || *q == '\\') *q = '_';  // kept out of the cache file's strings
  e = cudaMalloc((void**)&c->ticket, 256);
  if (e == cudaSuccess) e = cudaMemset(c->ticket, 0, 256);
  c->status = reinterpret_cast<int*>(reinterpret_cast<char*>(c->ticket) + 64);
  if (e != cudaSuccess) {
    cudaFree(c->ticket);
    delete c;
    return cuda_fail(e, "allocating the ticket word");
  }
  *out = c;
  return SIMR_OK;
}

void simr_destroy(simr_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->partials);
  cudaFree(ctx->ckpt);
  cudaFree(ctx->gseg);
  cudaFree(ctx->lsm_S);
  cudaFree(ctx->lsm_V);
  cudaFree(ctx->lsm_cash);
  cudaFree(ctx->lsm_stop);
  cudaFree(ctx->lsm_beta);
  cudaFree(ctx->lsm_dpow);
  cudaFree(ctx->lsm_xform);
  cudaFree(ctx->ticket);
  cudaFree(ctx->dev_strikes);
  cudaFree(ctx->dev_out);
  cudaFree(ctx->dev_f32);
  cudaFree(ctx->b_opts);
  cudaFree(ctx->b_items);
  cudaFree(ctx->b_partials);
  if (ctx->b_host) cudaFreeHost(ctx->b_host);
  if (ctx->host_out) cudaFreeHost(ctx->host_out);
  if (ctx->b_uploaded) cudaEventDestroy(ctx->b_uploaded);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->g_in) cudaEventDestroy(ctx->g_in);
  if (ctx->g_out) cudaEventDestroy(ctx->g_out);
  if (ctx->g_stream) cudaStreamDestroy(ctx->g_stream);
  delete ctx;
}

int simr_sync(simr_ctx* ctx, void* stream) {
  const NvtxRange nvtx("simr_sync");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  int rc = with_device(ctx);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "asynchronous error");
  return take_status(ctx, (cudaStream_t)stream);
}

int simr_price(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes, int is_put,
               uint32_t steps, uint64_t paths, uint64_t seed, uint32_t option_index, double* price,
               double* stderr_out, void* stream) {
  const NvtxRange nvtx("simr_price");
  int rc = check_common(ctx, model, strikes, n_strikes, 1024, steps, paths);
  if (rc) return rc;
  if (!price) return fail(SIMR_EINVAL, "price is NULL");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PathLaunch L;
  if ((rc = build_launch(model, n_strikes, is_put, steps, 0, paths, paths, seed, option_index, 1e-4, 0u, &L)))
    return rc;
  if ((rc = apply_scheme(ctx, *model, steps, &L))) return rc;
  const double* ks = nullptr;
  if ((rc = stage_strikes(ctx, strikes, n_strikes, st, &ks))) return rc;
  OutStage o;
  o.user[0] = price;
  o.n[0] = n_strikes;
  o.user[1] = stderr_out;
  o.n[1] = n_strikes;
  if ((rc = stage_outputs(ctx, &o))) return rc;
  return run_paths(ctx, L, ks, o, st);
}

int simr_greeks_fd(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes, int is_put,
                   uint32_t steps, uint64_t paths, uint64_t seed, uint32_t option_index, double rel_bump,
                   uint32_t greek_mask, double* price, double* greeks, void* stream) {
  const NvtxRange nvtx("simr_greeks_fd");
  int rc = check_common(ctx, model, strikes, n_strikes, 256, steps, paths);
  if (rc) return rc;
  if (!(rel_bump > 0.0 && rel_bump < 0.5)) return fail(SIMR_EINVAL, "rel_bump must lie in (0, 0.5)");
  if (greek_mask == 0 || (greek_mask & ~SIMR_G_ALL)) return fail(SIMR_EINVAL, "greek_mask must select Greeks");
  if (!price || !greeks) return fail(SIMR_EINVAL, "price and greeks must be non-NULL");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PathLaunch L;
  simr_heston scen[kMaxScen];
  if ((rc = build_launch(model, n_strikes, is_put, steps, 0, paths, paths, seed, option_index, rel_bump,
                         greek_mask, &L, scen)))
    return rc;
  if ((rc = apply_scheme(ctx, *model, steps, &L, scen))) return rc;
  const double* ks = nullptr;
  if ((rc = stage_strikes(ctx, strikes, n_strikes, st, &ks))) return rc;
  OutStage o;
  o.user[0] = price;
  o.n[0] = n_strikes;
  o.user[2] = greeks;
  o.n[2] = (size_t)n_strikes * popcount9(greek_mask);
  if ((rc = stage_outputs(ctx, &o))) return rc;
  return run_paths(ctx, L, ks, o, st);
}

// The checkpoint interval the per-strike adjoint runs fastest with.  Its
// forward pass runs every segment but the last, (n_seg - 1) k = steps - (the
// last segment's length) steps, while the recompute and reverse passes run all
// steps whatever k is.  So: one segment of the whole path (no forward pass), in
// shared memory if it fits there, else in global memory if its buffer is at
// most kAdjAutoGsegFloats; otherwise, among the even k up to the largest that
// keeps the kernel's blocks per SM, the one with the longest last segment (the
// smallest k on a tie, for the least shared memory).
int fast_ckpt_every(simr_ctx* ctx, const PathLaunch& L, uint32_t steps, uint32_t* k) {
  const uint32_t one = steps + (steps & 1u);
  if (one <= 1024) {
    AdjConst A{};
    A.ckpt_every = (int32_t)one;
    A.n_seg = 1;
    size_t floats = 0;
    cudaError_t e = adjoint_gseg_floats(L, A, ctx->num_sms, &floats);
    if (e != cudaSuccess) return cuda_fail(e, "sizing the adjoint's segment buffers");
    if (floats <= kAdjAutoGsegFloats) {
      *k = one;
      return SIMR_OK;
    }
  }
  int k_max = 0;
  for (const auto& t : ctx->adj_k)
    if (t.nk_pad == L.nk_pad) k_max = t.k_max;
  if (!k_max) {
    cudaError_t e = adjoint_max_ckpt_every(L, 1024, &k_max);
    if (e != cudaSuccess) return cuda_fail(e, "sizing the adjoint's checkpoint interval");
    ctx->adj_k.push_back({L.nk_pad, k_max});
  }
  uint32_t best = 2;
  uint64_t fwd_best = UINT64_MAX;
  for (uint32_t c = 2; c <= (uint32_t)k_max; c += 2) {
    const uint64_t fwd = (uint64_t)((steps + c - 1) / c - 1) * c;
    if (fwd < fwd_best) {
      fwd_best = fwd;
      best = c;
    }
    if (c >= steps) break;  // one segment: no forward pass
  }
  *k = best;
  return SIMR_OK;
}

int simr_adjoint_interval(simr_ctx* ctx, int n_strikes, uint32_t steps, uint32_t* ckpt_every) {
  if (!ctx || !ckpt_every) return fail(SIMR_EINVAL, "ctx and ckpt_every must be non-NULL");
  if (n_strikes < 1 || n_strikes > 256) return fail(SIMR_EINVAL, "n_strikes must be in [1, 256]");
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be positive");
  int rc = with_device(ctx);
  if (rc) return rc;
  PathLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.n_strikes = n_strikes;
  L.nk_pad = n_strikes == 1 ? 1 : ((n_strikes + 31) / 32) * 32;
  L.n_acc = 9;
  uint32_t k = 0;
  if ((rc = fast_ckpt_every(ctx, L, steps, &k))) return rc;
  *ckpt_every = k > steps ? steps + (steps & 1u) : k;
  return SIMR_OK;
}

int simr_greeks_adjoint(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes, int is_put,
                        uint32_t steps, uint64_t paths, uint64_t seed, uint32_t option_index, uint32_t ckpt_every,
                        double* price, double* stderr_out, double* grad, void* stream) {
  const NvtxRange nvtx("simr_greeks_adjoint");
  int rc = check_common(ctx, model, strikes, n_strikes, 256, steps, paths);
  if (rc) return rc;
  if (!price || !grad) return fail(SIMR_EINVAL, "price and grad must be non-NULL");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PathLaunch L;
  if ((rc = build_launch(model, n_strikes, is_put, steps, 0, paths, paths, seed, option_index, 1e-4, 0u, &L)))
    return rc;
  L.n_acc = 9;  // the adjoint's accumulators: f, f^2 and 7 sensitivities per strike
  uint32_t k = ckpt_every;
  if (k == 0 && (rc = fast_ckpt_every(ctx, L, steps, &k))) return rc;
  AdjConst A;
  if ((rc = build_adjoint(*model, steps, k, &A))) return rc;
  adjoint_scheme(ctx, *model, steps, &L, &A);
  if (adjoint_smem_bytes(L, A) > kAdjMaxSmem)
    return fail(SIMR_EUNSUPPORTED, "ckpt_every %d with %u steps needs more shared memory than a block has",
                A.ckpt_every, steps);
  if (adjoint_ckpt_scratch_floats(A, ctx->num_sms) > (1ull << 30))
    return fail(SIMR_EUNSUPPORTED, "ckpt_every %d with %u steps gives more than 2^30 checkpoint floats",
                A.ckpt_every, steps);
  const double* ks = nullptr;
  if ((rc = stage_strikes(ctx, strikes, n_strikes, st, &ks))) return rc;
  OutStage o;
  o.user[0] = price;
  o.n[0] = n_strikes;
  o.user[1] = stderr_out;
  o.n[1] = n_strikes;
  o.user[2] = grad;
  o.n[2] = (size_t)n_strikes * 7;
  if ((rc = stage_outputs(ctx, &o))) return rc;
  if ((rc = ensure(&ctx->partials, &ctx->partial_doubles, adjoint_scratch_doubles(L, ctx->num_sms),
                   "reduction scratch")))
    return rc;
  if ((rc = ensure(&ctx->ckpt, &ctx->ckpt_floats, adjoint_ckpt_scratch_floats(A, ctx->num_sms), "checkpoints")))
    return rc;
  size_t gseg_need = 0;
  cudaError_t eg = adjoint_gseg_floats(L, A, ctx->num_sms, &gseg_need);
  if (eg != cudaSuccess) return cuda_fail(eg, "sizing the adjoint's segment buffers");
  if (gseg_need > kAdjMaxGsegFloats)
    return fail(SIMR_EUNSUPPORTED, "ckpt_every %d with %u steps needs more than 2^31 floats of segment buffers",
                A.ckpt_every, steps);
  if (gseg_need && (rc = ensure(&ctx->gseg, &ctx->gseg_floats, gseg_need, "segment buffers"))) return rc;
  AdjOutputs out{o.dev[0], o.dev[1], o.dev[2], ctx->status};
  Scratch sc{ctx->partials, ctx->ticket, ctx->partial_doubles, ctx->ckpt, ctx->ckpt_floats, ctx->gseg,
             ctx->gseg_floats};
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_adjoint(L, A, ks, out, sc, ctx->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "launching the adjoint kernel");
  return finish_outputs(ctx, o, st);
}

int simr_paths_adjoint(simr_ctx* ctx, const simr_heston* model, uint32_t steps, uint64_t path_begin, uint64_t n_paths,
                       uint64_t seed, uint32_t option_index, uint32_t ckpt_every, float* x_T, float* grad,
                       void* stream) {
  const NvtxRange nvtx("simr_paths_adjoint");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  int rc = check_model(model);
  if (rc) return rc;
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be >= 1");
  if (n_paths < 1 || n_paths > (1ull << 31)) return fail(SIMR_EINVAL, "n_paths must lie in [1, 2^31]");
  if (!x_T || !grad) return fail(SIMR_EINVAL, "x_T and grad must be non-NULL");
  if (!is_device_ptr(x_T) || !is_device_ptr(grad)) return fail(SIMR_EINVAL, "x_T and grad must be device pointers");
  AdjConst A;
  if ((rc = build_adjoint(*model, steps, ckpt_every, &A))) return rc;
  if ((size_t)adjoint_thread_floats(A.n_seg, A.ckpt_every, 1) * 128 * sizeof(float) > kAdjMaxSmem)
    return fail(SIMR_EUNSUPPORTED, "ckpt_every %d with %u steps needs more shared memory than a block has",
                A.ckpt_every, steps);
  if ((rc = with_device(ctx))) return rc;
  PathLaunch L;
  if ((rc = build_launch(model, 1, 0, steps, path_begin, n_paths, n_paths, seed, option_index, 1e-4, 0u, &L)))
    return rc;
  adjoint_scheme(ctx, *model, steps, &L, &A);
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_paths_adjoint(L, A, x_T, grad, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching the per-path adjoint kernel");
  return SIMR_OK;
}

int simr_path_sums(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes, int is_put,
                   uint32_t steps, uint64_t path_begin, uint64_t path_count, uint64_t seed, uint32_t option_index,
                   double rel_bump, uint32_t greek_mask, double* sums, void* stream) {
  const NvtxRange nvtx("simr_path_sums");
  int rc = check_common(ctx, model, strikes, n_strikes, 256, steps, path_count);
  if (rc) return rc;
  if (greek_mask & ~SIMR_G_ALL) return fail(SIMR_EINVAL, "unknown Greek bits");
  if (greek_mask && !(rel_bump > 0.0 && rel_bump < 0.5)) return fail(SIMR_EINVAL, "rel_bump must lie in (0, 0.5)");
  if (!sums) return fail(SIMR_EINVAL, "sums is NULL");
  if (path_begin + path_count < path_begin) return fail(SIMR_EINVAL, "path range overflows");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PathLaunch L;
  simr_heston scen[kMaxScen];
  if ((rc = build_launch(model, n_strikes, is_put, steps, path_begin, path_count, path_count, seed, option_index,
                         greek_mask ? rel_bump : 1e-4, greek_mask, &L, scen)))
    return rc;
  if ((rc = apply_scheme(ctx, *model, steps, &L, scen))) return rc;
  L.raw_sums = 1;
  const double* ks = nullptr;
  if ((rc = stage_strikes(ctx, strikes, n_strikes, st, &ks))) return rc;
  OutStage o;
  o.user[0] = sums;
  o.n[0] = (size_t)n_strikes * L.n_acc;
  if ((rc = stage_outputs(ctx, &o))) return rc;
  return run_paths(ctx, L, ks, o, st);
}

int simr_finalize_sums(simr_ctx* ctx, const simr_heston* model, const double* strikes, int n_strikes, int is_put,
                       uint32_t steps, uint64_t paths, double rel_bump, uint32_t greek_mask, const double* sums,
                       double* price, double* stderr_out, double* greeks, void* stream) {
  const NvtxRange nvtx("simr_finalize_sums");
  int rc = check_common(ctx, model, strikes, n_strikes, 256, steps, paths);
  if (rc) return rc;
  if (!sums || !price) return fail(SIMR_EINVAL, "sums and price must be non-NULL");
  if (greek_mask & ~SIMR_G_ALL) return fail(SIMR_EINVAL, "unknown Greek bits");
  if (greek_mask && !greeks) return fail(SIMR_EINVAL, "greeks is NULL");
  if (greek_mask && !(rel_bump > 0.0 && rel_bump < 0.5)) return fail(SIMR_EINVAL, "rel_bump must lie in (0, 0.5)");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PathLaunch L;
  if ((rc = build_launch(model, n_strikes, is_put, steps, 0, paths, paths, 0, 0, greek_mask ? rel_bump : 1e-4,
                         greek_mask, &L)))
    return rc;
  const size_t ns = (size_t)n_strikes * L.n_acc;
  const double* dsums = sums;
  if (!is_device_ptr(sums)) {
    // sums are staged behind the strike staging area
    if ((rc = ensure(&ctx->dev_strikes, &ctx->strikes_cap, ns, "sum staging"))) return rc;
    cudaError_t e = cudaMemcpyAsync(ctx->dev_strikes, sums, ns * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copying sums");
    dsums = ctx->dev_strikes;
  }
  OutStage o;
  o.user[0] = price;
  o.n[0] = n_strikes;
  o.user[1] = stderr_out;
  o.n[1] = n_strikes;
  o.user[2] = greek_mask ? greeks : nullptr;
  o.n[2] = (size_t)n_strikes * (L.n_acc - 2);
  if ((rc = stage_outputs(ctx, &o))) return rc;
  PathOutputs out{};
  out.price = o.dev[0];
  out.stderr_ = o.dev[1];
  out.greeks = o.dev[2];
  out.status = ctx->status;
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_finalize(L, dsums, out, st);
  if (e != cudaSuccess) return cuda_fail(e, "launching the finalize kernel");
  return finish_outputs(ctx, o, st);
}

// Tuned book shapes across processes: $SIMR_TUNE_CACHE names a file of JSON
// lines {"gpu": name, "key": book size class, "chunk": paths per item,
// "variant": kernel shape, ...}; this GPU's entries are read once per context,
// new ones appended (best effort: an unreadable or unwritable file is ignored).
void load_tune_cache(simr_ctx* ctx) {
  if (ctx->tune_loaded) return;
  ctx->tune_loaded = true;
  const char* path = std::getenv("SIMR_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[1024], gpu[256];
  unsigned long long key = 0;
  unsigned chunk = 0;
  int variant = 0;
  while (std::fgets(line, sizeof(line), f)) {
    if (std::sscanf(line, "{\"gpu\": \"%255[^\"]\", \"key\": %llu, \"chunk\": %u, \"variant\": %d", gpu, &key,
                    &chunk, &variant) != 4)
      continue;
    const bool adj = (key & 1ull) != 0;
    if (std::strcmp(gpu, ctx->gpu_name) != 0 || variant < 0 || variant >= (adj ? 2 : kBatchVariants) ||
        chunk < 32 || chunk > 16384 || chunk % (adj ? 32u : 64u) != 0)
      continue;
    ctx->tune.push_back({(uint64_t)key, (uint32_t)chunk, variant});
  }
  std::fclose(f);
}

void save_tune_entry(const simr_ctx* ctx, const simr_ctx::Tune& t, bool adjoint) {
  const char* path = std::getenv("SIMR_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  BatchLaunch B{};
  batch_variant(t.variant, adjoint, &B);
  std::fprintf(f, "{\"gpu\": \"%s\", \"key\": %llu, \"chunk\": %u, \"variant\": %d, \"tpb\": %d, \"ppt\": %d, "
               "\"unroll\": %d}\n",
               ctx->gpu_name, (unsigned long long)t.key, t.chunk, t.variant, B.tpb, B.ppt, B.unroll);
  std::fclose(f);
}

int simr_batch_submit(simr_ctx* ctx, const simr_option* opts, int n_opts, uint64_t seed, uint32_t flags,
                      double* price, double* stderr_out, double* grad, void* stream) {
  const NvtxRange nvtx("simr_batch_submit");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  if (!opts || n_opts < 1 || n_opts > (1 << 22)) return fail(SIMR_EINVAL, "n_opts must lie in [1, 2^22]");
  if (flags & ~(SIMR_BATCH_ADJOINT | SIMR_BATCH_GRAPH | SIMR_BATCH_NO_AUTOTUNE | (15u << 8)))
    return fail(SIMR_EINVAL, "unknown batch flags");
  const int forced = (int)((flags >> 8) & 15u) - 1;  // SIMR_BATCH_VARIANT(v): v, else -1
  if (forced > 7 || (forced > 1 && (flags & SIMR_BATCH_ADJOINT)))
    return fail(SIMR_EINVAL, "kernel shape out of range for this book");
  if (is_device_ptr(opts)) return fail(SIMR_EINVAL, "the option table must be in host memory");
  const bool adjoint = (flags & SIMR_BATCH_ADJOINT) != 0;
  if (!price) return fail(SIMR_EINVAL, "price is NULL");
  const bool qem = ctx->scheme == SIMR_SCHEME_QEM;
  if (qem && forced > 1 && !adjoint)
    return fail(SIMR_EINVAL, "price books under QE-M have two kernel shapes (SIMR_BATCH_VARIANT 0 or 1)");
  if (adjoint && !grad) return fail(SIMR_EINVAL, "adjoint books need grad");
  int rc = with_device(ctx);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<BatchOption> bo;
  std::vector<uint32_t> order;
  // adjoint books: every option one segment of its whole path in global memory
  // (no forward pass) when the longest fits 1,024 steps and the buffer
  // kAdjAutoGsegFloats; else checkpoints and segments in shared memory
  bool one_segment = false;
  size_t gseg_floats = 0;
  if (adjoint) {
    uint32_t max_steps = 0;
    for (int i = 0; i < n_opts; ++i) max_steps = std::max(max_steps, opts[i].steps);
    if (max_steps >= 1 && max_steps <= 1024) {
      size_t threads = 0;
      cudaError_t eg = batch_gseg_threads(ctx->num_sms, &threads);
      if (eg != cudaSuccess) return cuda_fail(eg, "sizing the book's segment buffers");
      gseg_floats = (size_t)3 * (max_steps + (max_steps & 1u)) * threads;
      one_segment = gseg_floats <= kAdjAutoGsegFloats;
    }
  }
  int ckpt_rows = 0, seg_rows = 0;
  if ((rc = build_batch_options(opts, n_opts, adjoint, qem, &bo, one_segment, &order, &ckpt_rows, &seg_rows)))
    return rc;
  if (!one_segment && (size_t)(ckpt_rows + 3 * seg_rows) * 128 * sizeof(float) > kAdjMaxSmem)
    return fail(SIMR_EUNSUPPORTED, "the book's checkpoints need more shared memory than a block has");
  if (one_segment && (rc = ensure(&ctx->gseg, &ctx->gseg_floats, gseg_floats, "segment buffers"))) return rc;
  BatchLaunch B;
  std::memset(&B, 0, sizeof(B));
  philox_round_keys(seed, B.rk);
  B.n_opts = (uint32_t)n_opts;
  B.adjoint = adjoint ? 1 : 0;
  B.ckpt_rows = ckpt_rows;
  B.seg_rows = seg_rows;
  B.gseg = one_segment ? ctx->gseg : nullptr;
  B.qem = qem ? 1 : 0;
  const int nacc = adjoint ? 9 : 2;
  OutStage o;
  o.user[0] = price;
  o.n[0] = n_opts;
  o.user[1] = stderr_out;
  o.n[1] = n_opts;
  o.user[2] = adjoint ? grad : nullptr;
  o.n[2] = (size_t)n_opts * 7;
  if ((rc = stage_outputs(ctx, &o))) return rc;
  BatchOutputs out{o.dev[0], o.dev[1], o.dev[2]};
  B.gseg_floats = ctx->gseg_floats;
  cudaError_t e = cudaSuccess;

  // kernel shape and chunk (paths per work item): autotuned once per book
  // shape, cached in the context and in $SIMR_TUNE_CACHE
  double total = 0.0;
  for (const BatchOption& b : bo) total += (double)b.steps * (double)b.paths;
  const uint64_t tkey = (adjoint ? 1ull : 0ull) | ((uint64_t)std::max(0.0, std::log2(total + 1.0)) << 1) |
                        ((uint64_t)std::log2((double)n_opts) << 16) | ((qem ? 1ull : 0ull) << 40);
  // a chunk that fills the GPU: about two items per resident warp (the kernel
  // runs ~40 warps per SM), a multiple of the paths a warp takes per pass
  double total_paths = 0.0;
  for (const BatchOption& b : bo) total_paths += (double)b.paths;
  const uint32_t quantum = adjoint ? 32u : 64u;
  const double fill = total_paths / (2.0 * 40.0 * (double)ctx->num_sms);
  const uint32_t balanced =
      (uint32_t)std::min(16384.0, std::max((double)quantum, std::ceil(fill / quantum) * quantum));
  uint32_t chunk = std::min(adjoint ? 1024u : 4096u, balanced);
  int variant = 0;
  load_tune_cache(ctx);
  bool tuned = false;
  for (const auto& t : ctx->tune)
    if (t.key == tkey) chunk = t.chunk, variant = t.variant, tuned = true;
  const char* env = std::getenv("SIMR_AUTOTUNE");
  const bool autotune = forced < 0 && !(flags & SIMR_BATCH_NO_AUTOTUNE) && !(env && env[0] == '0');
  if (forced >= 0) variant = forced;
  if (!tuned && autotune) {
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    uint32_t loaded = 0;  // the chunk the uploaded item table was cut with
    auto time_one = [&](uint32_t ch, int v, float* ms) -> int {
      if (ch != loaded) {
        uint32_t n_items = 0;
        int r = upload_batch(ctx, bo, order, ch, st, &n_items);
        if (r) return r;
        B.n_items = n_items;
        if ((r = ensure(&ctx->b_partials, &ctx->b_partials_cap, (size_t)n_items * nacc, "batch partial rows")))
          return r;
        loaded = ch;
      }
      batch_variant(v, adjoint, &B);
      e = prepare_batch(B);
      if (e == cudaSuccess) e = cudaEventRecord(a, st);
      if (e == cudaSuccess)
        e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_batch(B, ctx->b_opts, ctx->b_items, ctx->ticket + 32, ctx->b_partials, out, ctx->num_sms, st);
      if (e == cudaSuccess) e = cudaEventRecord(b, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
      return SIMR_OK;
    };
    float best = 0.0f;
    const int n_var = (adjoint || qem) ? 2 : kBatchVariants;
    for (int v = 0; v < n_var && e == cudaSuccess && !rc; ++v) {  // the kernel shape at the default chunk
      float ms = 0.0f;
      rc = time_one(chunk, v, &ms);
      if (!rc && e == cudaSuccess && (v == 0 || ms < best)) best = ms, variant = v;
    }
    const uint32_t cands[4] = {adjoint ? 256u : 1024u, adjoint ? 1024u : 4096u, adjoint ? 4096u : 16384u, balanced};
    for (int ci = 0; ci < 4 && e == cudaSuccess && !rc; ++ci) {  // then the chunk
      float ms = 0.0f;
      rc = time_one(cands[ci], variant, &ms);
      if (!rc && e == cudaSuccess && (ci == 0 || ms < best)) best = ms, chunk = cands[ci];
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotuning the batch kernel");
    const simr_ctx::Tune t{tkey, chunk, variant};
    ctx->tune.push_back(t);
    save_tune_entry(ctx, t, adjoint);
  }
  batch_variant(variant, adjoint, &B);
  e = prepare_batch(B);
  if (e != cudaSuccess) return cuda_fail(e, "preparing the batch kernel");

  uint32_t n_items = 0;
  if ((rc = upload_batch(ctx, bo, order, chunk, st, &n_items))) return rc;
  B.n_items = n_items;
  if ((rc = ensure(&ctx->b_partials, &ctx->b_partials_cap, (size_t)n_items * nacc, "batch partial rows"))) return rc;
  unsigned int* counter = ctx->ticket + 32;  // word at byte 128 of the ticket block
  if (flags & SIMR_BATCH_GRAPH) {
    // one captured graph per (book, seed, flags, outputs): repeated submissions replay it.
    // Captured and launched on the context's own stream, ordered after `st` by events
    // (capture is not possible on the legacy default stream).
    if (!ctx->g_stream) {
      e = cudaStreamCreateWithFlags(&ctx->g_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->g_in, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->g_out, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "creating the graph stream");
    }
    cudaStream_t gs = ctx->g_stream;
    e = cudaEventRecord(ctx->g_in, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, ctx->g_in, 0);
    if (e != cudaSuccess) return cuda_fail(e, "ordering the graph stream");
    uint64_t key = fnv1a(bo.data(), bo.size() * sizeof(BatchOption));
    key = fnv1a(&seed, sizeof(seed), key);
    key = fnv1a(&flags, sizeof(flags), key);
    key = fnv1a(&chunk, sizeof(chunk), key);
    key = fnv1a(&variant, sizeof(variant), key);
    key = fnv1a(&B.qem, sizeof(B.qem), key);
    key = fnv1a(&out, sizeof(out), key);
    // the captured launches hold the context's device buffers: a reallocation
    // since the capture makes a new graph
    const void* bufs[4] = {ctx->b_opts, ctx->b_items, ctx->b_partials, B.gseg};
    key = fnv1a(bufs, sizeof(bufs), key);
    if (!(ctx->graph_exec && ctx->graph_key == key)) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_batch(B, ctx->b_opts, ctx->b_items, counter, ctx->b_partials, out, ctx->num_sms, gs);
        e = cudaStreamEndCapture(gs, &g);
        if (le != cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        ctx->graph_exec = nullptr;
        return cuda_fail(e, "capturing the batch graph");
      }
      ctx->graph_key = key;
    }
    e = cudaGraphLaunch(ctx->graph_exec, gs);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->g_out, gs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->g_out, 0);
  } else {
    e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_batch(B, ctx->b_opts, ctx->b_items, counter, ctx->b_partials, out, ctx->num_sms, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "launching the batch");
  return finish_outputs(ctx, o, st);
}

int simr_paths_terminal(simr_ctx* ctx, const simr_heston* model, uint32_t steps, uint64_t path_begin,
                        uint64_t n_paths, uint64_t seed, uint32_t option_index, float* x_T, float* v_T,
                        void* stream) {
  const NvtxRange nvtx("simr_paths_terminal");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  int rc = check_model(model);
  if (rc) return rc;
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be >= 1");
  if (n_paths < 1 || n_paths > (1ull << 31)) return fail(SIMR_EINVAL, "n_paths must lie in [1, 2^31]");
  if (!x_T) return fail(SIMR_EINVAL, "x_T is NULL");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PathLaunch L;
  if ((rc = build_launch(model, 1, 0, steps, path_begin, n_paths, n_paths, seed, option_index, 1e-4, 0u, &L)))
    return rc;
  if ((rc = apply_scheme(ctx, *model, steps, &L))) return rc;
  const bool hx = !is_device_ptr(x_T), hv = v_T && !is_device_ptr(v_T);
  float* dx = x_T;
  float* dv = v_T;
  if (hx || hv) {
    if ((rc = ensure(&ctx->dev_f32, &ctx->f32_cap, 2 * (size_t)n_paths, "terminal staging"))) return rc;
    if (hx) dx = ctx->dev_f32;
    if (hv) dv = ctx->dev_f32 + n_paths;
  }
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_terminal(L, dx, dv, st);
  if (e != cudaSuccess) return cuda_fail(e, "launching the terminal kernel");
  if (hx) e = cudaMemcpyAsync(x_T, dx, n_paths * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hv) e = cudaMemcpyAsync(v_T, dv, n_paths * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && (hx || hv)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "copying terminal states");
  return SIMR_OK;
}

int simr_philox_words(simr_ctx* ctx, uint64_t seed, uint32_t option_index, uint64_t path_begin, uint64_t n_paths,
                      uint32_t pair_begin, uint32_t n_pairs, uint32_t* words, void* stream) {
  const NvtxRange nvtx("simr_philox_words");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  if (!words) return fail(SIMR_EINVAL, "words is NULL");
  if (n_paths < 1 || n_pairs < 1 || n_paths * (uint64_t)n_pairs > (1ull << 28))
    return fail(SIMR_EINVAL, "n_paths * n_pairs must lie in [1, 2^28]");
  if ((uint64_t)pair_begin + n_pairs > (1ull << 32)) return fail(SIMR_EINVAL, "pair_begin + n_pairs exceeds 2^32");
  if (!is_device_ptr(words)) return fail(SIMR_EINVAL, "words must be a device pointer");
  int rc = with_device(ctx);
  if (rc) return rc;
  DrawLaunch D;
  philox_round_keys(seed, D.rk);
  D.path_begin = path_begin;
  D.n_paths = n_paths;
  D.pair_begin = pair_begin;
  D.n_pairs = n_pairs;
  D.option_index = option_index;
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources
                                                : launch_philox_words(D, words, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching the Philox kernel");
  return SIMR_OK;
}

int simr_normals(simr_ctx* ctx, const uint32_t* words, uint64_t n, float* z, float* z_paired, void* stream) {
  const NvtxRange nvtx("simr_normals");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  if (!words || !z) return fail(SIMR_EINVAL, "words and z must be non-NULL");
  if (n < 1 || n > (1ull << 31)) return fail(SIMR_EINVAL, "n must lie in [1, 2^31]");
  if (!is_device_ptr(words) || !is_device_ptr(z) || (z_paired && !is_device_ptr(z_paired)))
    return fail(SIMR_EINVAL, "words, z and z_paired must be device pointers");
  int rc = with_device(ctx);
  if (rc) return rc;
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources
                                                : launch_normals(words, n, z, z_paired, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching the normal kernel");
  return SIMR_OK;
}

int simr_unit_rates(simr_ctx* ctx, double* rates, void* stream) {
  const NvtxRange nvtx("simr_unit_rates");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  if (!rates) return fail(SIMR_EINVAL, "rates is NULL");
  if (is_device_ptr(rates)) return fail(SIMR_EINVAL, "rates must be a host array");
  int rc = with_device(ctx);
  if (rc) return rc;
  if ((rc = ensure(&ctx->dev_f32, &ctx->f32_cap, unit_rates_scratch_floats(ctx->num_sms), "unit-rate scratch")))
    return rc;
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH)
                      ? cudaErrorLaunchOutOfResources
                      : measure_unit_rates(ctx->num_sms, ctx->dev_f32, (cudaStream_t)stream, rates);
  if (e != cudaSuccess) return cuda_fail(e, "measuring the unit rates");
  return SIMR_OK;
}

int simr_basket_price(simr_ctx* ctx, const simr_heston* assets, int n_assets, const double* corr,
                      const double* weights, const double* strikes, int n_strikes, int is_put, uint32_t steps,
                      uint64_t paths, uint64_t seed, double* price, double* stderr_out, void* stream) {
  const NvtxRange nvtx("simr_basket_price");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  if (!assets || !corr || !weights) return fail(SIMR_EINVAL, "assets, corr and weights must be non-NULL");
  if (n_assets < 1 || n_assets > kMaxAssets) return fail(SIMR_EINVAL, "n_assets must lie in [1, %d]", kMaxAssets);
  if (is_device_ptr(assets) || is_device_ptr(corr) || is_device_ptr(weights))
    return fail(SIMR_EINVAL, "assets, corr and weights must be host arrays");
  if (!strikes) return fail(SIMR_EINVAL, "strikes is NULL");
  if (n_strikes < 1 || n_strikes > 1024) return fail(SIMR_EINVAL, "n_strikes must lie in [1, 1024]");
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be >= 1");
  if (paths < 1 || paths > (1ull << 40)) return fail(SIMR_EINVAL, "paths must lie in [1, 2^40]");
  if (!price) return fail(SIMR_EINVAL, "price is NULL");
  int rc = SIMR_OK;
  for (int k = 0; k < n_assets; ++k) {
    if ((rc = check_model(&assets[k]))) {
      char msg[sizeof(g_err)];
      std::strncpy(msg, g_err, sizeof(msg) - 1);
      msg[sizeof(msg) - 1] = 0;
      return fail(SIMR_EINVAL, "asset %d: %s", k, msg);
    }
    if (assets[k].r != assets[0].r || assets[k].T != assets[0].T)
      return fail(SIMR_EINVAL, "all assets of a basket share r and T");
    if (!std::isfinite(weights[k])) return fail(SIMR_EINVAL, "weight %d is not finite", k);
  }
  // lower Cholesky factor of the correlation (FP64), validated on the way
  const int A = n_assets;
  std::vector<double> Lc((size_t)A * A, 0.0);
  for (int i = 0; i < A; ++i) {
    for (int j = 0; j < A; ++j) {
      const double c = corr[i * A + j];
      if (!std::isfinite(c) || c < -1.0 || c > 1.0 || c != corr[j * A + i])
        return fail(SIMR_EINVAL, "corr must be a symmetric matrix of values in [-1, 1]");
    }
    if (corr[i * A + i] != 1.0) return fail(SIMR_EINVAL, "corr must have a unit diagonal");
  }
  for (int i = 0; i < A; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = corr[i * A + j];
      for (int k = 0; k < j; ++k) s -= Lc[i * A + k] * Lc[j * A + k];
      if (i == j) {
        if (!(s > 1e-12)) return fail(SIMR_EINVAL, "corr is not positive definite");
        Lc[i * A + i] = std::sqrt(s);
      } else {
        Lc[i * A + j] = s / Lc[j * A + j];
      }
    }
  }
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  BasketLaunch L;
  std::memset(&L, 0, sizeof(L));
  philox_round_keys(seed, L.rk);
  for (int k = 0; k < A; ++k) {
    L.sc[k] = base_const(assets[k], steps);
    L.S0w[k] = (float)(assets[k].S0 * weights[k]);
    for (int j = 0; j <= k; ++j) L.Lc[k * (k + 1) / 2 + j] = (float)Lc[k * A + j];
  }
  for (int q = 0; 2 * q + 1 < A; ++q) L.pk[q] = pack_const(L.sc[2 * q], L.sc[2 * q + 1]);
  if (ctx->scheme == SIMR_SCHEME_QEM) {  // each asset its own martingale correction
    L.scheme = 1;
    for (int k = 0; k < A; ++k) L.qm[k] = qem_const(assets[k], steps);
    for (int q = 0; 2 * q + 1 < A; ++q) L.qk[q] = pack_qem(L.qm[2 * q], L.qm[2 * q + 1]);
  }
  L.n_assets = A;
  L.n_strikes = n_strikes;
  L.nk_pad = n_strikes == 1 ? 1 : ((n_strikes + 31) / 32) * 32;
  L.is_put = is_put ? 1 : 0;
  L.steps = steps;
  L.paths = paths;
  L.disc = std::exp(-assets[0].r * assets[0].T);
  L.paths_total = (double)paths;
  const double* ks = strikes;
  if (!is_device_ptr(strikes)) {
    for (int k = 0; k < n_strikes; ++k)
      if (!(strikes[k] >= 0.0) || !std::isfinite(strikes[k]))
        return fail(SIMR_EINVAL, "strike %d must be finite and >= 0", k);
    if ((rc = ensure(&ctx->dev_strikes, &ctx->strikes_cap, (size_t)n_strikes, "strike staging"))) return rc;
    cudaError_t e = cudaMemcpyAsync(ctx->dev_strikes, strikes, n_strikes * sizeof(double), cudaMemcpyHostToDevice,
                                    st);
    if (e != cudaSuccess) return cuda_fail(e, "copying strikes");
    ks = ctx->dev_strikes;
  }
  OutStage o;
  o.user[0] = price;
  o.n[0] = n_strikes;
  o.user[1] = stderr_out;
  o.n[1] = n_strikes;
  if ((rc = stage_outputs(ctx, &o))) return rc;
  if ((rc = ensure(&ctx->partials, &ctx->partial_doubles, basket_partial_doubles(L, ctx->num_sms),
                   "reduction scratch")))
    return rc;
  BasketOutputs out{o.dev[0], o.dev[1], ctx->status};
  cudaError_t e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_basket(L, ks, out, ctx->partials, ctx->partial_doubles, ctx->ticket, ctx->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "launching the basket kernel");
  return finish_outputs(ctx, o, st);
}

int simr_set_scheme(simr_ctx* ctx, int scheme) {
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  if (scheme != SIMR_SCHEME_QE && scheme != SIMR_SCHEME_QEM) return fail(SIMR_EINVAL, "unknown scheme %d", scheme);
  ctx->scheme = scheme;
  return SIMR_OK;
}

int simr_lsm_price(simr_ctx* ctx, const simr_heston* model, double K, int is_put, uint32_t steps,
                   uint32_t exercise_every, uint64_t paths, uint64_t seed, uint32_t option_index, double* price,
                   double* stderr_out, double* beta, int32_t* stop, void* stream) {
  const NvtxRange nvtx("simr_lsm_price");
  if (!ctx) return fail(SIMR_EINVAL, "context is NULL");
  int rc = check_model(model);
  if (rc) return rc;
  if (!(K > 0.0) || !std::isfinite(K)) return fail(SIMR_EINVAL, "strike must be finite and > 0");
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be >= 1");
  if (exercise_every < 1 || steps % exercise_every != 0)
    return fail(SIMR_EINVAL, "exercise_every must be >= 1 and divide steps");
  const uint32_t n_ex = steps / exercise_every;
  if (n_ex > 8192) return fail(SIMR_EINVAL, "at most 8192 exercise dates");
  if (paths < 2 || paths > (1ull << 31)) return fail(SIMR_EINVAL, "paths must lie in [2, 2^31]");
  if ((double)n_ex * (double)paths * 8.0 > 64.0 * (1ull << 30))
    return fail(SIMR_EUNSUPPORTED, "the states at the exercise dates would exceed 64 GiB");
  if (!price) return fail(SIMR_EINVAL, "price is NULL");
  if ((rc = with_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t pitch = (paths + 3) & ~3ull;  // 16-byte rows, so that the sweep's bulk copies start aligned
  const size_t nS = (size_t)n_ex * pitch;
  if ((rc = ensure(&ctx->lsm_S, &ctx->lsm_S_cap, nS, "exercise-date spots"))) return rc;
  if ((rc = ensure(&ctx->lsm_V, &ctx->lsm_V_cap, nS, "exercise-date variances"))) return rc;
  if ((rc = ensure(&ctx->lsm_cash, &ctx->lsm_cash_cap, (size_t)paths, "cash flows"))) return rc;
  if ((rc = ensure(&ctx->lsm_stop, &ctx->lsm_stop_cap, (size_t)paths, "exercise dates"))) return rc;
  if ((rc = ensure(&ctx->lsm_beta, &ctx->lsm_beta_cap, (size_t)n_ex * 12, "regression coefficients"))) return rc;
  if ((rc = ensure(&ctx->lsm_dpow, &ctx->lsm_dpow_cap, (size_t)n_ex, "discount table"))) return rc;
  if ((rc = ensure(&ctx->lsm_xform, &ctx->lsm_xform_cap, (size_t)n_ex, "basis scaling"))) return rc;
  if ((rc = ensure(&ctx->partials, &ctx->partial_doubles, lsm_partial_doubles(ctx->num_sms), "reduction scratch")))
    return rc;
  OutStage o;
  o.user[0] = price;
  o.n[0] = 1;
  o.user[1] = stderr_out;
  o.n[1] = 1;
  o.user[2] = beta;
  o.n[2] = (size_t)n_ex * 6;
  if ((rc = stage_outputs(ctx, &o))) return rc;

  const double dt_ex = model->T / (double)n_ex;
  std::vector<float> dpow(n_ex);
  for (uint32_t k = 0; k < n_ex; ++k) dpow[k] = (float)std::exp(-model->r * dt_ex * (double)k);
  // per date: xs = (S - F)/sd_S and ys = (v - E v)/sd_v from the model's forward
  // F = S0 e^{rt}, log-spot spread sqrt(vbar t) (vbar: mean expected variance over
  // [0, t]) and the CIR mean and variance of v_t
  std::vector<float4> xf(n_ex);
  const double kap = model->kappa, th = model->theta, v0 = model->v0, s2 = model->sigma * model->sigma;
  for (uint32_t j = 0; j < n_ex; ++j) {
    const double t = dt_ex * (double)(j + 1), E = std::exp(-kap * t), omE = -std::expm1(-kap * t);
    const double F = model->S0 * std::exp(model->r * t);
    const double vbar = th + (v0 - th) * omE / (kap * t);
    const double sdS = F * std::sqrt(std::max(vbar * t, 1e-12));
    const double Ev = th + (v0 - th) * E;
    const double varv = v0 * s2 * E * omE / kap + th * s2 * omE * omE / (2.0 * kap);
    const double sdv = std::max(std::sqrt(std::max(varv, 0.0)), 1e-6 * (Ev + 0.5 * (v0 + th)) + 1e-300);
    xf[j] = make_float4((float)(1.0 / sdS), (float)(-F / sdS), (float)(1.0 / sdv), (float)(-Ev / sdv));
  }
  cudaError_t e = cudaMemcpyAsync(ctx->lsm_dpow, dpow.data(), n_ex * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->lsm_xform, xf.data(), n_ex * sizeof(float4), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables go out of scope
  // rows of dates without a regression stay NaN; the maturity row never gets one
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->lsm_beta, 0xff, (size_t)n_ex * 12 * sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(e, "preparing the Longstaff-Schwartz tables");

  LsmLaunch L;
  std::memset(&L, 0, sizeof(L));
  philox_round_keys(seed, L.rk);
  L.sc = base_const(*model, steps);
  L.S0 = (float)model->S0;
  L.K = (float)K;
  const double w = 0.5 * (model->v0 + model->theta);
  L.is_put = is_put ? 1 : 0;
  L.n_ex = (int32_t)n_ex;
  L.every = (int32_t)exercise_every;
  L.min_itm = 12;
  L.steps = steps;
  L.option_index = option_index;
  L.paths = paths;
  L.pitch = pitch;
  L.disc0 = std::exp(-model->r * dt_ex);
  L.Kd = K;
  L.wd = w > 0.0 ? w : 1.0;
  L.scheme = ctx->scheme == SIMR_SCHEME_QEM ? 1 : 0;
  L.qm = qem_const(*model, steps);
  LsmBuffers B{ctx->lsm_S,
               ctx->lsm_V,
               ctx->lsm_cash,
               ctx->lsm_stop,
               o.dev[2] ? o.dev[2] : ctx->lsm_beta,
               ctx->lsm_beta + (size_t)n_ex * 6,
               ctx->lsm_xform,
               ctx->lsm_dpow,
               ctx->partials,
               ctx->ticket + 48,
               ctx->status,
               o.dev[0],
               o.dev[1]};
  if (o.dev[2]) e = cudaMemsetAsync(o.dev[2], 0xff, (size_t)n_ex * 6 * sizeof(double), st);
  L.barrier_extra = take_fault(SIMR_FAULT_BARRIER) ? 1 : 0;
  if (e == cudaSuccess) e = take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : launch_lsm(L, B, ctx->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "launching the Longstaff-Schwartz kernels");
  if (stop) {
    e = cudaMemcpyAsync(stop, ctx->lsm_stop, (size_t)paths * sizeof(int32_t), cudaMemcpyDefault, st);
    if (e == cudaSuccess && !is_device_ptr(stop)) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copying the exercise dates");
  }
  return finish_outputs(ctx, o, st);
}

}  // extern "C"

// Helpers shared with other translation units of the library (simr_internal.h).
namespace simr {

int internal_fail(int code, const char* message) { return fail(code, "%s", message); }

int internal_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }

int internal_check_price_args(const simr_heston* model, const double* strikes, int n_strikes, int max_strikes,
                              uint32_t steps, uint64_t paths) {
  int rc = check_model(model);
  if (rc) return rc;
  if (steps < 1) return fail(SIMR_EINVAL, "steps must be >= 1");
  if (paths < 1) return fail(SIMR_EINVAL, "paths must be >= 1");
  if (!strikes) return fail(SIMR_EINVAL, "strikes is NULL");
  if (n_strikes < 1 || n_strikes > max_strikes)
    return fail(SIMR_EINVAL, "n_strikes must lie in [1, %d]", max_strikes);
  return SIMR_OK;
}

bool internal_is_device_ptr(const void* p) { return is_device_ptr(p); }

int internal_build_price_launch(const simr_heston* model, int n_strikes, int is_put, uint32_t steps, uint64_t paths,
                                uint64_t seed, uint32_t option_index, PathLaunch* L) {
  return build_launch(model, n_strikes, is_put, steps, 0, paths, paths, seed, option_index, 1e-4, 0u, L);
}

}  // namespace simr
