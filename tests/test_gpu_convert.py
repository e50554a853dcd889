"""FP32 -> scaled FP64 conversion on the integer pipe (tensor-core GEMM epilogue).

The GEMM epilogue widens every FP32 accumulator to FP64 (a factor 1 + q 2^-46 is supported, the
epilogue uses 1) by integer operations on the IEEE-754 encodings instead of GB300's slow FP64
arithmetic. The checks below
compare it with IEEE 754 itself (numpy's exact widening and correctly rounded products) and with
CUDA's own conversion, over every binary32 exponent (zero and subnormals, normals, infinities and
NaNs), both signs, and factors of either sign around 1.
"""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf


def test_convert_rejects_bad_arguments():
    x = np.zeros(4, np.float32)
    out = np.zeros(4, np.float64)
    P = ajf._ptr
    assert ajf.lib().ajf_selftest_convert(0, None, P(out), 4, 1.0) == ajf.AJF_E_ARG
    assert ajf.lib().ajf_selftest_convert(0, P(x), None, 4, 1.0) == ajf.AJF_E_ARG
    assert ajf.lib().ajf_selftest_convert(0, P(x), P(out), -1, 1.0) == ajf.AJF_E_ARG
    assert ajf.lib().ajf_selftest_convert(0, P(x), P(out), 4, 1.01) == ajf.AJF_E_ARG  # |s - 1| >= 2^-10
    assert ajf.lib().ajf_selftest_convert(0, P(x), P(out), 4, float("nan")) == ajf.AJF_E_ARG
    assert ajf.lib().ajf_selftest_convert(0, P(x), P(out), 0, 1.0) == ajf.AJF_OK      # nothing to do


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _f32_inputs(seed=0):
    """Every binary32 exponent (0 = zero/subnormal, 255 = inf/NaN) with 64 fractions each
    (including all-zero and all-one fractions), both signs."""
    rng = np.random.default_rng(seed)
    e = np.arange(256, dtype=np.uint32)
    frac = rng.integers(0, 1 << 23, size=(256, 64), dtype=np.uint32)
    frac[:, 0] = 0
    frac[:, 1] = (1 << 23) - 1
    bits = ((e[:, None] << 23) | frac).ravel()
    return np.concatenate([bits, bits | np.uint32(0x80000000)]).view(np.float32)


def _same(a, b):
    """Bitwise equality, NaN matching any NaN."""
    nan = np.isnan(a) & np.isnan(b)
    w = a.dtype.itemsize
    ia = a.view(np.uint32 if w == 4 else np.uint64)
    ib = b.view(np.uint32 if w == 4 else np.uint64)
    return (ia == ib) | nan


@pytest.mark.gpu
def test_f32_to_f64_exact_without_scale(gpu):
    import torch
    x = _f32_inputs()
    got = ajf.ajf_selftest_convert(0, x, 1.0)
    assert _same(got, x.astype(np.float64)).all()
    assert _same(got, torch.from_numpy(x).cuda().double().cpu().numpy()).all()


@pytest.mark.gpu
@pytest.mark.parametrize("q", [round(7.02e-8 * 2 ** 46) * k // 5 for k in (2, 3, 4, 5)] +
                         [round(8.69e-8 * 2 ** 46), -round(3e-7 * 2 ** 46), 2 ** 35, -(2 ** 35), 1])
def test_f32_to_f64_scaled(gpu, q):
    """x * (1 + q 2^-46) within 2 units in the last place of the exact product (3 of its
    rounded value): the de-biasing factors of the tensor-core GEMM and factors of either sign."""
    scale = 1.0 + q * 2.0 ** -46  # exact in binary64, so the library uses this q
    x = _f32_inputs(seed=q & 0xFFFF)
    got = ajf.ajf_selftest_convert(0, x, scale)
    ref = x.astype(np.float64) * scale
    fin = np.isfinite(ref)
    ulp = np.spacing(np.abs(ref[fin]))
    err = np.abs(got[fin] - ref[fin])
    assert (err <= 3 * ulp).all(), float(np.max(err / np.maximum(ulp, 1e-320)))
    assert _same(got[~fin], ref[~fin]).all()
    zero = x == 0
    assert _same(got[zero], x[zero].astype(np.float64)).all()  # signed zeros
