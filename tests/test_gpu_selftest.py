"""The warp kernels' numerical building blocks against exact host references:
Newton reciprocals against correctly rounded 1/x, the integer-pipe FP64->FP32
rounding against NumPy's IEEE conversion (bitwise), and the integer-pipe
segment sum against the exactly rounded sum (math.fsum)."""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(op, x, lanes=1):
    import torch
    from paper_2405_17363_gb300 import camp
    f = camp._lib.camp_selftest
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p]
    xin = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    out = torch.empty_like(xin)
    assert f(op, xin.numel(), xin.data_ptr(), out.data_ptr(), lanes,
             torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _sample(n, lo=-300, hi=300, seed=0):
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], n) * (1 + rng.random(n)) * np.exp2(rng.integers(lo, hi, n))


def test_recip_two_steps_within_one_ulp(cuda):
    x = _sample(1 << 18)
    y = _run(0, x)
    ref = 1.0 / x
    ulp = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 1.0
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 2.0, 0.5])
    ys = _run(0, sp)
    assert ys[0] == np.inf and ys[1] == -np.inf and ys[2] == 0.0 and ys[3] == 0.0
    assert np.isnan(ys[4]) and ys[5] == 0.5 and ys[6] == 2.0


def test_recip_one_step_relative_error(cuda):
    x = _sample(1 << 18)
    y = _run(1, x)
    assert np.max(np.abs(y * x - 1.0)) <= 2.0 ** -43


def test_fp32_rounding_is_ieee(cuda):
    rng = np.random.default_rng(1)
    x = _sample(1 << 18, -120, 120, seed=2)
    # exact ties and values one ulp off a tie
    base = rng.random(4096).astype(np.float32).astype(np.float64)
    half = np.spacing(base.astype(np.float32)).astype(np.float64) / 2
    x = np.concatenate([x, base + half, base - half, base + half * (1 + 2 ** -30)])
    y = _run(2, x)
    np.testing.assert_array_equal(y, x.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("lanes", [2, 8, 16, 32])
def test_integer_segment_sum_is_exact_to_one_rounding(cuda, lanes):
    rng = np.random.default_rng(lanes)
    n = 32 * 2048
    x = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n))
    # a cancelling block and zeros
    x[:32] = np.r_[[1e10, -1e10, 3.0, -3.0] * 8]
    x[32:64] = 0.0
    y = _run(3, x, lanes)
    for s in range(0, n, lanes):
        seg = x[s:s + lanes]
        exact = math.fsum(seg)
        bound = np.spacing(abs(exact)) + lanes * np.abs(seg).max() * 2.0 ** -57
        assert np.all(y[s:s + lanes] == y[s]), "every lane gets the same bits"
        assert abs(y[s] - exact) <= bound
    # the full-warp redux form gives the same bits, NaN and Inf included
    x2 = x.copy()
    x2[64:96] = np.r_[[np.inf, 1.0, np.nan, -2.0] * 8]
    x2[96:128] = np.ldexp(rng.standard_normal(32), -1060)
    np.testing.assert_array_equal(_run(5, x2, lanes).view(np.int64), _run(3, x2, lanes).view(np.int64))
    # the FP64 shuffle tree meets the classic pairwise-summation bound
    tree = _run(4, x, lanes)
    levels = int(np.log2(lanes))
    for s in range(0, n, lanes):
        seg = x[s:s + lanes]
        exact = math.fsum(seg)
        assert abs(tree[s] - exact) <= levels * 2.0 ** -53 * np.abs(seg).sum() * 1.0001 + 1e-300


def test_fp64_rate_probe_computes_its_chains(cuda):
    """op 6 (the FP64 rate probe timed by bench.py) runs four chains
    a <- a*m + q per thread; its output matches the chains' closed form."""
    steps = 1000
    x = np.random.default_rng(6).random(32 * 64)
    y = _run(6, x, steps)
    m, q = 0.999999999, 1e-9
    ms = m ** steps
    chain = lambda a0: ms * a0 + q * (1 - ms) / (1 - m)
    expect = chain(x) + chain(x + 1) + chain(x + 2) + chain(x + 3)
    np.testing.assert_allclose(y, expect, rtol=1e-12)
