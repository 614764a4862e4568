"""The generator and the normal transform on the GPU, draw by draw, through the C ABI.

The paper streams pre-generated random inputs V and Z from the host (Sec. 3
Table 1, Sec. 4); here every path kernel draws them itself, and
simr_philox_words / simr_normals expose the kernels' own device functions.

  * Philox4x32-10: every word equals the oracle's Philox (which is pinned to
    Triton's library generator in the CPU suite), bit for bit, for counters that
    cross the path word's 2^32 boundary, large step pairs, option indices and
    64-bit seeds.
  * Normals: the FP32 transform of every point of the 2^23-point uniform lattice
    u = (k + 1/2) 2^-23 -- both tails' polynomial (|x| > 0.9966, 0.3% of the
    lattice) and the extreme points u = 2^-24, 1 - 2^-24 included -- against
    AS 241 (Wichura 1988, the oracle's FP64 inverse CDF).  Bound:
    |Z_gpu - Z| <= 1e-6 |Z| + 5e-7.  Giles' approximation with every FP32
    operation rounded once and the logarithm exact stays within 3.7e-7 |Z| and
    8.3e-7 (a float32 emulation on the CPU); the special-function unit's
    logarithm (absolute error near 2^-22.6) adds about 1e-7.  The one-at-a-time
    and packed two-lane forms agree bit for bit, and the transform is odd:
    Z(1 - u) = -Z(u) exactly, since x(1 - u) = -x(u) exactly.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

N_LATTICE = 1 << 23


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


@pytest.mark.parametrize("seed,option,path_begin,n_paths,pair_begin,n_pairs", [
    (1, 0, 0, 64, 0, 3),
    ((7 << 32) | 0xDEADBEEF, 5, (1 << 32) - 3, 7, 0, 2),        # path crosses the counter's word boundary
    (0xFFFFFFFFFFFFFFFF, (1 << 31) + 9, 12345, 5, (1 << 31) - 1, 4),
    (42, 1023, (3 << 32) + 17, 3, (1 << 32) - 2, 2),             # the last step pairs of the counter word
])
def test_philox_words_equal_the_oracle(simr, seed, option, path_begin, n_paths, pair_begin, n_pairs):
    w = simr.philox_words(seed, option, path_begin, n_paths, pair_begin, n_pairs)
    torch.cuda.synchronize()
    got = w.cpu().numpy().view(np.uint32)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(n_paths):
        p = path_begin + i
        for j in range(n_pairs):
            want = oracle.philox4x32_10((pair_begin + j, p & 0xFFFFFFFF, p >> 32, option), key)
            np.testing.assert_array_equal(got[i, j], want, err_msg=f"path {p} pair {pair_begin + j}")


def test_normals_over_the_whole_uniform_lattice(simr):
    k = torch.arange(N_LATTICE, dtype=torch.int64, device="cuda")
    words = (k << 9).to(torch.int32)  # w >> 9 = k: u = (k + 1/2) 2^-23
    z, zp = simr.normals(words)
    torch.cuda.synchronize()
    z, zp = z.cpu().numpy(), zp.cpu().numpy()
    np.testing.assert_array_equal(z, zp)  # packed lanes: the scalar function's values
    np.testing.assert_array_equal(z, -z[::-1])  # odd: Z(1 - u) = -Z(u)
    u = (np.arange(N_LATTICE, dtype=np.float64) + 0.5) * 2.0 ** -23
    zo = oracle.norminv(u)
    err = np.abs(z.astype(np.float64) - zo)
    bad = err > 1e-6 * np.abs(zo) + 5e-7
    assert not bad.any(), (np.flatnonzero(bad)[:10], err[bad][:10], zo[bad][:10])
    # the extreme lattice points and both tails are in the check above; spot them too
    for i in (0, 1, N_LATTICE // 2 - 1, N_LATTICE // 2, N_LATTICE - 1):
        assert abs(z[i] - zo[i]) <= 1e-6 * abs(zo[i]) + 5e-7, (i, z[i], zo[i])
    tail = np.abs(2 * u - 1) > 0.9966
    assert 0.002 < tail.mean() < 0.004 and err[tail].max() <= 1e-6 * 5.3 + 5e-7


def test_normals_of_drawn_words_match_the_oracle_normals(simr):
    # the words of real counters through the kernels' transform, against the
    # oracle's uniforms and AS 241 for the same counters (steps 0 and 1 of a pair)
    seed, option = 9, 3
    w = simr.philox_words(seed, option, 1000, 256, 0, 4)  # steps 0 .. 7 of paths 1000 .. 1255
    z, _ = simr.normals(w)
    torch.cuda.synchronize()
    z = z.cpu().numpy().reshape(256, 4, 4)
    for i in range(0, 256, 17):
        for n in range(8):
            u_v, u_x = oracle.step_uniforms(seed, option, 1000 + i, n)
            zv, zx = oracle.norminv([u_v, u_x])
            pair, half = divmod(n, 2)
            gv, gx = z[i, pair, 2 * half], z[i, pair, 2 * half + 1]
            assert abs(gv - zv) <= 1e-6 * abs(zv) + 5e-7 and abs(gx - zx) <= 1e-6 * abs(zx) + 5e-7


def test_generator_entry_points_refuse_bad_arguments(simr):
    # through the C ABI with a small device buffer: the sizes are refused on the
    # host before anything is launched or written
    import ctypes

    from paper_2402_12111_gb300 import _simr as S

    L = S.load()
    ctx = S.context(0)
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    zf = torch.zeros(64, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.simr_philox_words(ctx, 1, 0, 0, 1 << 20, 0, 1 << 9, p, st) == S.SIMR_EINVAL  # 2^29 counters
    assert L.simr_philox_words(ctx, 1, 0, 0, 1, (1 << 32) - 1, 2, p, st) == S.SIMR_EINVAL  # past the last pair
    assert L.simr_philox_words(ctx, 1, 0, 0, 0, 0, 1, p, st) == S.SIMR_EINVAL  # no paths
    host = np.zeros(64, dtype=np.uint32)
    assert L.simr_philox_words(ctx, 1, 0, 0, 1, 0, 1, host.ctypes.data_as(ctypes.c_void_p), st) == S.SIMR_EINVAL
    assert L.simr_normals(ctx, p, 0, ctypes.c_void_p(zf.data_ptr()), None, st) == S.SIMR_EINVAL
    assert L.simr_normals(ctx, host.ctypes.data_as(ctypes.c_void_p), 4, ctypes.c_void_p(zf.data_ptr()), None,
                          st) == S.SIMR_EINVAL
    torch.cuda.synchronize()
    assert not zf.any()
