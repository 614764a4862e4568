"""GB300-native Heston QE Monte Carlo pricing: the SIMR hot path of arXiv:2402.12111.

Public API (torch tensors for device memory and streams; all arithmetic runs in
libsimr.so's sm_103a kernels behind the C ABI of include/simr.h):

  price(model, strikes, ...)            -> (price, stderr)      simr_price
  greeks_fd(model, strikes, ...)        -> (price, greeks)      simr_greeks_fd
  greeks_adjoint(model, strikes, ...)   -> (price, se, grad)    simr_greeks_adjoint
  heston_price(params, strikes, T, ...) differentiable price    torch.autograd.Function over the adjoint
  paths_terminal(model, steps, ...)     -> (x_T, v_T)           simr_paths_terminal
  paths_adjoint(model, steps, ...)      -> (x_T, dx_T/dparams)  simr_paths_adjoint
  batch(options, seed, adjoint, graph)  -> (price, se, grad)    simr_batch_submit (heterogeneous book)
  lsm_price(model, K, ...)              -> (price, se, beta, stop) simr_lsm_price (Longstaff-Schwartz)
  basket_price(models, corr, weights, K) -> (price, se)          simr_basket_price (correlated assets)
  set_scheme("qe" | "qem") / scheme(...)                        simr_set_scheme (QE-M martingale correction)
  path_sums / finalize_sums                                     sharded runs
  sharded.price_greeks(...)             multi-rank path sharding (torch.distributed)
  adjoint_interval(n_strikes, steps)    the checkpoint interval greeks_adjoint takes by default
  inject_fault("alloc" | "launch", n)   host-side fault injection (tests of failure handling)
  sync(device)                          simr_sync: device-side status of the calls on a stream
  philox_words(seed, option, ...)       the generator's raw words   simr_philox_words
  normals(words)                        -> (z, z_paired)        simr_normals (the kernels' FP32 normals)

``model`` is a dict (or Heston struct) with S0, r, T, v0, kappa, theta, sigma, rho.
Tensors on a CUDA device give an asynchronous call on the current stream; CPU
tensors or sequences give a synchronous call with host buffers.
"""
from .api import (ADJOINT_COLUMNS, HestonAdjoint, adjoint_interval, basket_price, batch, finalize_sums,  # noqa: F401
                  greeks_adjoint, greeks_fd, heston_price, inject_fault, lsm_price, normals, path_sums,
                  paths_adjoint, paths_terminal, philox_words, price, scheme, set_scheme, sync, unit_rates)
from ._simr import (G_ALL, G_CORR, G_DELTA, G_GAMMA, G_KAPPA, G_LRVAR, G_RHO, G_THETA, G_VEGA,  # noqa: F401
                    G_VOLVOL, GREEK_BITS, Heston, SimrError, greek_mask, load)

__all__ = ["price", "greeks_fd", "greeks_adjoint", "heston_price", "HestonAdjoint", "ADJOINT_COLUMNS",
           "adjoint_interval", "paths_terminal", "paths_adjoint", "batch", "lsm_price", "basket_price",
           "set_scheme", "scheme", "path_sums", "finalize_sums", "sync", "inject_fault", "philox_words", "normals",
           "Heston", "SimrError",
           "greek_mask", "load", "GREEK_BITS"]
