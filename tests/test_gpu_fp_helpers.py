"""The hand-written double-precision helpers of the kernels against CUDA's own operations.

The FP64 form replaces the compiler's divide and square roots by float-seeded Newton/Householder
corrections (rcp_d, rsqrt_d, sqrt_d, ratio_t), converts between double and float with integer
operations (d2f, f2d) and halves by lowering the exponent field (half_exact).  A small harness
(tests/cuda/fp_helpers.cu, built here with nvcc) evaluates each helper and the matching CUDA
operation on the same inputs:

- reciprocal and square root within 1 ulp of the correctly rounded result, reciprocal square root
  within 1 ulp of the exact value (computed in long double on the host), the ratio within 2 ulp,
  in every band of binades of the seeded range [2^-100, 2^101) and at its edges;
- outside that range (zero, subnormals, huge values, infinity, NaN) and for negative operands of
  the roots, bit-identical to CUDA's operation, which the helpers fall back to there;
- d2f bit-identical to the hardware conversion wherever the result is a normal float, including
  round-to-nearest-even ties; f2d bit-identical to the hardware widening of normal floats;
- half_exact bit-identical to x * 0.5 for every finite double, subnormals and their ties included.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
N_PER_BAND = 2_000_000
BANDS = [(-100, -80), (-80, -40), (-40, -10), (-10, 10), (10, 40), (40, 80), (80, 101)]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out = str(tmp_path_factory.mktemp("fp") / "libfp.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-o", out, os.path.join(HERE, "cuda", "fp_helpers.cu")]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = C.CDLL(out)
    lib.fp_run.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]

    def run(kind, x, y=None):
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        yd = torch.tensor(x if y is None else y, dtype=torch.float64, device="cuda")
        od = torch.empty(4 * len(x), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert lib.fp_run(kind, xd.data_ptr(), yd.data_ptr(), od.data_ptr(), len(x)) == 0
        o = od.cpu().numpy().reshape(-1, 4)
        return o[:, 0].copy(), o[:, 1].copy()
    return run


def band_samples(lo, hi, n, seed, signed=False):
    rng = np.random.default_rng(seed)
    x = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(lo, hi, n).astype(float))
    if signed:
        x *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return x


def ulp_dist(a, b):
    """|a - b| in units of the last place (same-sign finite doubles)."""
    ia, ib = a.view(np.int64), b.view(np.int64)
    assert np.all(np.sign(a) == np.sign(b))
    return np.abs(ia - ib)


EDGES = np.array([2.0 ** -100, np.nextafter(2.0 ** -100, 0), np.nextafter(2.0 ** -100, 1), 2.0 ** 101,
                  np.nextafter(2.0 ** 101, 0), 1.0, np.nextafter(1.0, 2), np.nextafter(1.0, 0), 3.0, 0.1])
OUTSIDE = np.array([0.0, -0.0, 5e-324, 2.2e-308, 1e-310, 2.0 ** -101, 1e-200, 1e200, 2.0 ** 102, 1.7e308,
                    np.inf, -np.inf, np.nan, -1e-310, -1e300])


def same_bits(a, b):
    both_nan = np.isnan(a) & np.isnan(b)
    return np.all(both_nan | (a.view(np.int64) == b.view(np.int64)))


@pytest.mark.parametrize("kind,name", [(0, "rcp_d"), (1, "sqrt_d")])
def test_reciprocal_and_sqrt_within_one_ulp(harness, kind, name):
    worst = 0
    for i, (lo, hi) in enumerate(BANDS):
        x = band_samples(lo, hi, N_PER_BAND, 100 + i, signed=(kind == 0))
        x = np.concatenate([x, EDGES, -EDGES] if kind == 0 else [x, EDGES])
        got, ieee = harness(kind, x)
        d = ulp_dist(got, ieee)
        worst = max(worst, int(d.max()))
        assert d.max() <= 1, (name, lo, hi, x[d.argmax()])
    print(f"{name}: at most {worst} ulp from the correctly rounded result")


def test_rsqrt_within_one_ulp_of_exact(harness):
    assert np.finfo(np.longdouble).nmant >= 63
    for i, (lo, hi) in enumerate(BANDS):
        x = np.concatenate([band_samples(lo, hi, N_PER_BAND // 4, 200 + i), EDGES])
        got, _ = harness(2, x)
        exact = 1.0 / np.sqrt(x.astype(np.longdouble))
        err = np.abs(got.astype(np.longdouble) - exact)
        assert np.all(err <= np.spacing(got).astype(np.longdouble)), (lo, hi)


def test_ratio_within_two_ulp(harness):
    for i, (lo, hi) in enumerate(BANDS):
        b = band_samples(lo, hi, N_PER_BAND // 2, 300 + i)
        a = b * np.random.default_rng(400 + i).uniform(1e-3, 1.0, len(b))  # the limiter's 0 <= a <= b
        got, ieee = harness(3, b, a)
        assert ulp_dist(got, ieee).max() <= 2, (lo, hi)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_outside_the_seeded_range_equals_cuda(harness, kind):
    x = OUTSIDE.copy()
    if kind == 0:
        x = np.concatenate([x, -OUTSIDE])
    else:  # negative operands of the roots take CUDA's operation too
        x = np.concatenate([x, -band_samples(-10, 10, 1000, 7)])
    got, ref = harness(kind, x)
    assert same_bits(got, ref)


def test_d2f_matches_hardware_in_float_normal_range(harness):
    rng = np.random.default_rng(5)
    x = band_samples(-126, 128, N_PER_BAND, 6, signed=True)
    x = x[(np.abs(x) >= 2.0 ** -126) & (np.abs(x) < np.finfo(np.float32).max)]
    # exact ties: halfway between two consecutive normal floats, both parities of the lower one
    f = rng.uniform(1.0, 2.0, 200_000).astype(np.float32) * np.exp2(rng.integers(-120, 120, 200_000)).astype(np.float32)
    f = f[np.isfinite(f) & (f > 0)]
    ties = f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2.0
    assert np.all(np.float32(ties - np.spacing(f).astype(np.float64) / 2.0) == f)
    x = np.concatenate([x, ties, -ties, [0.0, -0.0, np.inf, -np.inf, 3.0e38]])
    got, hw = harness(4, x)
    assert same_bits(got, hw)
    assert (f.view(np.int32) & 1).any() and ((f.view(np.int32) & 1) == 0).any()  # both parities tested


def test_f2d_matches_hardware_for_normal_floats(harness):
    x = band_samples(-126, 127, N_PER_BAND, 8, signed=True)
    x = np.concatenate([x, [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0]])
    got, hw = harness(5, x)
    assert same_bits(got, hw)


def test_half_exact_is_x_times_half(harness):
    rng = np.random.default_rng(9)
    bits = rng.integers(0, 2 ** 63 - 1, N_PER_BAND, dtype=np.int64)
    x = bits.view(np.float64)
    x = x[np.isfinite(x)] * np.where(rng.random(np.isfinite(x).sum()) < 0.5, -1.0, 1.0)
    sub = (rng.integers(0, 2 ** 52, 200_000, dtype=np.int64)).view(np.float64)  # subnormals, both parities
    x = np.concatenate([x, sub, -sub, [5e-324, -5e-324, 1.5e-323, 2.0 ** -1022, 2.0 ** -1021, 0.0, -0.0,
                                       np.inf, -np.inf, np.nan, 1.7976931348623157e308]])
    got, ref = harness(6, x)
    assert same_bits(got, ref)
