"""The tcgen05 tensor-core GEMM alone (C = sum_{i+j<T} A_i B_j^T over split terms), against float64
products of the same, exactly representable inputs. TF32 and bf16 products of representable inputs
are exact in FP32, so the only error is the FP32 accumulation: |dC| <= c K 2^-24 sum |a||b|."""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def tf32(x):
    """Round float32 to TF32 (10 explicit mantissa bits), nearest-even on the bit pattern."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0xFFF + ((b >> 13) & 1)) & ~np.uint64(0x1FFF)
    return b.astype(np.uint32).view(np.float32)


def bf16_bits(x):
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def bits_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def split_ref(A, B):
    T = A.shape[0]
    ref = sum(A[i] @ B[j].T for i in range(T) for j in range(T) if i + j < T)
    bound = sum(np.abs(A[i]) @ np.abs(B[j]).T for i in range(T) for j in range(T) if i + j < T)
    return ref, bound


SHAPES = [(128, 32, 32, 1), (128, 64, 64, 1), (256, 128, 128, 2), (128, 256, 64, 2), (512, 512, 256, 3),
          (1024, 256, 512, 1), (512, 1024, 128, 2),
          # tiles overhanging M, N or K (TMA zero fill, guarded stores)
          (32, 16, 16, 1), (64, 512, 16, 2), (32, 1024, 8, 1), (128, 16, 64, 3)]


@pytest.mark.parametrize("M,N,K,T", SHAPES)
def test_tf32_gemm(M, N, K, T):
    rng = np.random.default_rng(M + N + K + T)
    A = tf32(rng.standard_normal((T, M, K)).astype(np.float32))
    B = tf32(rng.standard_normal((T, N, K)).astype(np.float32))
    C = ajf.ajf_selftest_gemm(0, 0, A, B, M, N, K)
    ref, bound = split_ref(A.astype(np.float64), B.astype(np.float64))
    assert np.all(np.abs(C - ref) <= 4 * K * 2.0 ** -23 * bound + 1e-30)


@pytest.mark.parametrize("M,N,K,T", [(128, 32, 64, 1), (256, 128, 128, 2), (512, 256, 256, 3), (128, 64, 1024, 3),
                                     (64, 512, 32, 2), (32, 16, 16, 2), (512, 65536 // 64, 32, 2)])
def test_bf16_gemm(M, N, K, T):
    rng = np.random.default_rng(7 * M + N + K)
    A = bf16_bits(rng.standard_normal((T, M, K)))
    B = bf16_bits(rng.standard_normal((T, N, K)))
    C = ajf.ajf_selftest_gemm(0, 1, A, B, M, N, K)
    ref, bound = split_ref(bits_to_f64(A), bits_to_f64(B))
    assert np.all(np.abs(C - ref) <= 4 * K * 2.0 ** -23 * bound + 1e-30)


@pytest.mark.parametrize("K", [256, 4096, 16384])
def test_split_tf32_has_no_k_growing_bias(K):
    """Positive operands make truncation bias visible: a plain TMEM accumulation over K drifts by
    about -(K/8) 2^-24 relative (measured); with per-block promotion to round-to-nearest FP32 the
    mean relative error of the three-product split must stay below 2e-7 whatever K is."""
    rng = np.random.default_rng(K)
    A = rng.random((128, K)).astype(np.float32)
    B = rng.random((64, K)).astype(np.float32)
    Ah, Bh = tf32(A), tf32(B)
    Al, Bl = tf32(A - Ah), tf32(B - Bh)
    C = ajf.ajf_selftest_gemm(0, 0, np.stack([Ah, Al]), np.stack([Bh, Bl]), 128, 64, K)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    rel = (C - ref) / ref
    assert abs(rel.mean()) < 2e-7
    assert np.abs(rel).max() < 3e-6


def test_bounded_waits_report_timeout_and_device_stays_usable():
    """Failure detection without a GPU fault: the producer issues no loads, so the MMA and epilogue
    waits expire after 50 ms; the kernel reports which wait gave up (codes 12-14), frees its TMEM and
    returns. A normal GEMM in the same process then still works."""
    st, code = ajf.ajf_selftest_wait_timeout(0, 50.0)
    assert st == ajf.AJF_E_TIMEOUT
    assert code in (12, 13, 14)
    rng = np.random.default_rng(0)
    A = tf32(rng.standard_normal((1, 128, 64)).astype(np.float32))
    B = tf32(rng.standard_normal((1, 64, 64)).astype(np.float32))
    C = ajf.ajf_selftest_gemm(0, 0, A, B, 128, 64, 64)
    ref, bound = split_ref(A.astype(np.float64), B.astype(np.float64))
    assert np.all(np.abs(C - ref) <= 4 * 64 * 2.0 ** -23 * bound + 1e-30)


def test_unsupported_shape_is_reported():
    A = np.zeros((1, 16, 32), dtype=np.float32)
    B = np.zeros((1, 32, 32), dtype=np.float32)
    with pytest.raises(ajf.AjfError) as e:
        ajf.ajf_selftest_gemm(0, 0, A, B, 16, 32, 32)
    assert e.value.status == ajf.AJF_E_UNSUPPORTED


@pytest.mark.parametrize("M,N,K,T", [(128, 64, 16384, 3), (256, 32, 8192, 2), (1024, 512, 2048, 1)])
def test_k_split_gemm(M, N, K, T):
    """Few tiles and long K: the GEMM splits K over CTAs (FP64 partial tiles summed in order)."""
    rng = np.random.default_rng(7 + M + K)
    A = bf16_bits(rng.standard_normal((T, M, K)).astype(np.float32))
    B = bf16_bits(rng.standard_normal((T, N, K)).astype(np.float32))
    C = ajf.ajf_selftest_gemm(0, 1, A, B, M, N, K)
    ref, bound = split_ref(bits_to_f64(A), bits_to_f64(B))
    # per split at most 4096 K elements are summed in FP32; the splits add in FP64
    assert np.all(np.abs(C - ref) <= 4 * 4096 * 2.0 ** -23 * bound + 1e-30)


# --------------------------------------------------------------------------- through the operand split
# ajf_selftest_split_gemm runs the path's own gather (k_perm; in the six-product split it quantises
# each leading term to a fixed-point multiple of a power of two per row and 128-byte K block) and
# the tensor-core GEMM.

SPLIT_MODES = ["bf16x6", "f16x3", "tf32x3", "bf16x3"]


@pytest.mark.parametrize("precision", SPLIT_MODES)
@pytest.mark.parametrize("K", [64, 256])
def test_split_gemm_exact_on_small_integers(precision, K):
    """Integers |x| <= 127, scaled per row by powers of two: every term and every partial sum is
    exactly representable, so the whole path (split, exact leading partial, correction partial,
    FP32 promotion, FP64 store) must return the exact product, bit for bit."""
    rng = np.random.default_rng(K + len(precision))
    M, N = 64, 128
    A = rng.integers(-127, 128, (M, K)).astype(np.float64) * np.exp2(rng.integers(-12, 12, (M, 1)))
    B = rng.integers(-127, 128, (N, K)).astype(np.float64) * np.exp2(rng.integers(-12, 12, (N, 1)))
    C = ajf.ajf_selftest_split_gemm(0, precision, A, B)
    np.testing.assert_array_equal(C, A @ B.T)


@pytest.mark.parametrize("precision", ["bf16x6", "f16x3"])
@pytest.mark.parametrize("K", [256, 4096, 16384])
def test_split_gemm_has_no_truncation_bias(precision, K):
    """Positive operands make a truncating accumulation visible: a plain TMEM sum drifts by about
    -(K/8) 2^-24 relative, and one promoted K block at a time still loses about 7e-8 (all errors of
    one sign, so the mean relative error is as large as the typical one). In the six-product split
    the leading product accumulates exactly and only the small correction partial truncates: the
    mean relative error must be rounding noise -- below 1e-8 and below a tenth of the RMS error --
    with no correction factor anywhere."""
    rng = np.random.default_rng(K)
    A = rng.random((64, K))
    B = rng.random((128, K))
    C = ajf.ajf_selftest_split_gemm(0, precision, A, B)
    ref = A @ B.T
    rel = (C - ref) / ref
    rms = float(np.sqrt(np.mean(rel ** 2)))
    print(f"{precision} K={K}: mean {rel.mean():.2e} rms {rms:.2e} max {np.abs(rel).max():.2e}")
    assert abs(rel.mean()) < 1e-8
    assert abs(rel.mean()) < 0.1 * rms + 1e-10
    assert np.abs(rel).max() < 1e-6


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_two_term_splits_are_bounded(precision):
    """The two-term splits keep a floating leading term, so their leading partial truncates once
    per promoted K block: on positive operands the mean relative error is a small negative bias
    (bounded modes), far below the K-growing drift of an unpromoted accumulation."""
    K = 4096
    rng = np.random.default_rng(K + 1)
    A = rng.random((64, K))
    B = rng.random((128, K))
    C = ajf.ajf_selftest_split_gemm(0, precision, A, B)
    rel = (C - A @ B.T) / (A @ B.T)
    print(f"{precision}: mean {rel.mean():.2e} max {np.abs(rel).max():.2e}")
    assert -5e-7 < rel.mean() < 1e-8
    assert np.abs(rel).max() < {"tf32x3": 2e-6, "bf16x3": 2e-5}[precision]


@pytest.mark.parametrize("precision", SPLIT_MODES)
@pytest.mark.parametrize("M,N,K", [(64, 64, 64), (128, 512, 1024), (16, 1024, 32), (512, 64, 8192)])
def test_split_gemm_random_signs(precision, M, N, K):
    """Random-sign Gaussian operands against the FP64 product: the error is bounded by the split's
    representation error (bf16x6: 2^-26 of each row block's largest entry; f16x3: 2^-22 of it, with
    the dropped low-term products at 2^-20; tf32x3 and bf16x3: 2^-22 and 2^-17 of each entry) plus
    FP32 promotion."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = ajf.ajf_selftest_split_gemm(0, precision, A, B)
    ref = A @ B.T
    absprod = np.abs(A) @ np.abs(B).T
    bits = {"bf16x6": 22, "f16x3": 19, "tf32x3": 18, "bf16x3": 15}[precision]
    assert np.all(np.abs(C - ref) <= 2.0 ** -bits * absprod * 8)


@pytest.mark.parametrize("K", [8, 16, 32, 64, 128])
def test_f16x3_scales_follow_each_row(K):
    """Scaled fp16: rows and columns of wildly different magnitudes (2^-40 .. 2^40) keep their
    accuracy relative to their own largest entries, because each row's K block carries its own
    power-of-two scale; K below one 128-byte block (8-32 complex elements) shares one scale between
    the real and imaginary halves."""
    rng = np.random.default_rng(K)
    A = rng.standard_normal((32, K)) * np.exp2(rng.integers(-40, 40, (32, 1)))
    B = rng.standard_normal((64, K)) * np.exp2(rng.integers(-40, 40, (64, 1)))
    C = ajf.ajf_selftest_split_gemm(0, "f16x3", A, B)
    ref = A @ B.T
    # block floating point: each entry is kept to ~2^-22 of its row block's largest entry, so the
    # bound pairs one operand's row maximum with the other's absolute row sum
    bound = np.abs(A).max(axis=1)[:, None] * np.abs(B).sum(axis=1)[None, :] + \
        np.abs(A).sum(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(C - ref) <= 2.0 ** -19 * bound)


@pytest.mark.parametrize("precision", ["bf16x6", "tf32x3"])
def test_split_gemm_k_sweep(precision):
    """A sweep over the K mixes the contractions produce -- gate absorptions (K = 8, 16, 32 complex,
    one K block or less) up to the K = 524,288 split-K contractions of Alg. I networks -- through the
    path's operand split and GEMM, against the FP64 product. bf16x6 keeps every entry within
    1e-6 relative of the exact product and shows no bias on positive operands; tf32x3 (a bounded
    mode) stays within its bound, its floating leading term biased low by a K-independent ~1e-7."""
    rng = np.random.default_rng(99)
    for K in (8, 16, 32, 64, 256, 2048, 16384, 131072, 524288):
        M, N = (16, 16) if K >= 131072 else (32, 64)
        A = rng.random((M, K)) + 0.5
        B = rng.random((N, K)) + 0.5
        C = ajf.ajf_selftest_split_gemm(0, precision, A, B)
        ref = A @ B.T
        rel = (C - ref) / ref
        print(f"{precision} K={K}: mean {rel.mean():.2e} max {np.abs(rel).max():.2e}")
        if precision == "bf16x6":
            assert np.abs(rel).max() < 3e-7
            assert abs(rel.mean()) < 2e-8
        else:
            assert np.abs(rel).max() < 1e-6
            assert -3e-7 < rel.mean() < 1e-8
