"""simr_price_noalloc: the pricing entry point for callers that cannot allocate.

Serving loops that must never block on the allocator, and hosts that own all
device memory, cannot let a library call cudaMalloc.  simr_price_noalloc keeps
its scratch in a static device array instead; called through the C ABI it must
give what simr_price gives, bit for bit (the same kernel, constants and launch
shape), call after call.  (Collected last: a failure here leaves every other
test already run.)
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    return simr, simr.load()


def _call(L, simr, model, K, is_put, steps, paths, seed, p, se):
    st = torch.cuda.current_stream().cuda_stream
    return L.simr_price_noalloc(ctypes.byref(simr.Heston(**model)), ctypes.c_void_p(K.data_ptr()), K.numel(),
                                int(is_put), steps, paths, seed, 0, ctypes.c_void_p(p.data_ptr()),
                                ctypes.c_void_p(se.data_ptr() if se is not None else None), ctypes.c_void_p(st))


@pytest.mark.parametrize("K_np,is_put,steps,paths,seed", [
    (workloads.strike_grid(), False, 64, 100_003, 7),
    (np.array([100.0]), True, 33, 4097, 11),
])
def test_noalloc_matches_simr_price_on_two_calls(lib, K_np, is_put, steps, paths, seed):
    simr, L = lib
    model = dict(workloads.BASE_MODEL)
    K = torch.as_tensor(K_np, dtype=torch.float64, device="cuda")
    p_ref, se_ref = simr.price(model, K, is_put, steps, paths, seed)
    torch.cuda.synchronize()
    for _ in range(2):
        p = torch.full_like(p_ref, float("nan"))
        se = torch.full_like(p_ref, float("nan"))
        rc = _call(L, simr, model, K, is_put, steps, paths, seed, p, se)
        assert rc == 0, L.simr_last_error()
        torch.cuda.synchronize()
        # the same kernel, constants and launch shape as simr_price: the same bits
        torch.testing.assert_close(p, p_ref, rtol=0, atol=0)
        torch.testing.assert_close(se, se_ref, rtol=0, atol=0)


def test_noalloc_leaves_device_memory_unchanged(lib):
    # after a first call (the symbol lookup), a call takes no device memory: the
    # device's free memory and torch's allocator are the same before and after
    simr, L = lib
    model = dict(workloads.BASE_MODEL)
    K = torch.as_tensor(workloads.strike_grid(), dtype=torch.float64, device="cuda")
    p = torch.empty_like(K)
    se = torch.empty_like(K)
    assert _call(L, simr, model, K, False, 16, 50_000, 3, p, se) == 0, L.simr_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for seed in (4, 5):
        assert _call(L, simr, model, K, False, 16, 50_000, seed, p, se) == 0, L.simr_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.isfinite(p).all() and torch.isfinite(se).all()


def test_noalloc_rejects_sizes_and_host_pointers(lib):
    simr, L = lib
    model = dict(workloads.BASE_MODEL)
    K = torch.full((33,), 100.0, dtype=torch.float64, device="cuda")
    p = torch.empty(33, dtype=torch.float64, device="cuda")
    assert _call(L, simr, model, K, False, 8, 1000, 1, p, None) == -1
    assert b"[1, 32]" in L.simr_last_error()
    Kh = torch.full((4,), 100.0, dtype=torch.float64)
    ph = torch.empty(4, dtype=torch.float64)
    assert _call(L, simr, model, Kh, False, 8, 1000, 1, ph, None) == -1
    assert b"device pointers" in L.simr_last_error()


def test_noalloc_rejects_another_gpus_memory(lib):
    # host-side pointer check only: no kernel is launched for a refused call
    simr, L = lib
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no other device's memory to pass")
    model = dict(workloads.BASE_MODEL)
    K = torch.full((4,), 100.0, dtype=torch.float64, device="cuda:1")
    p = torch.empty(4, dtype=torch.float64, device="cuda:1")
    with torch.cuda.device(0):
        assert _call(L, simr, model, K, False, 8, 1000, 1, p, None) == -1
    assert b"current device" in L.simr_last_error()
