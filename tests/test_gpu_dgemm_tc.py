"""FP64 products on the tensor cores (tgba_dgemm_tc: BF16 slices of the FP64 operands, tcgen05
MMAs, exact FP32 sums of the leading digit diagonals per chunk of 256 K values, 48-bit running
sums) through the C ABI.

* Exactness of the tensor cores' FP32 accumulation: integer operands of at most 14 bits have
  two base-256 digits, hence only the digit diagonals 0..2, which the design sums exactly, so C
  must equal the integer product bit for bit (K = 4096: 16 chunks, sums up to 2^38).
* Accuracy: random operands whose rows span six decades, ragged sizes (M, N, K not multiples
  of the 128 x 128 x 32 tiles), against an extended-precision reference: error <= 1e-12 of
  sum_k |A_ik B_jk|, and against cuBLAS FP64.  The FP32 rounding of the accumulator shared by
  the digit diagonals 3..5 dominates: a chunk of 128 K values takes 120 MMA additions (15 slice
  pairs x 8 MMAs of K = 16), each rounded to 2^-25 of its magnitude (at most 3/4 of a
  leading-digit unit), against a chunk sum of about 4e5 such units for normal rows (mean |digit|
  58 of 256): a random walk gives ~6e-13 (measured up to 3.9e-13, at K = 100); the worst case,
  all roundings of one sign, is ten times that.  A longer chunk does not raise the relative
  error of its own sum (the rounding noise and the sum both grow), and more chunks average it
  down, so a single short chunk is the worst case.
* The work split: the chunks (256 K values of one tile) of all tiles are cut evenly over the
  SMs, so a tile may be summed by several CTAs (partials added by the last to finish).  The
  shapes cover tiles split over many CTAs at uneven boundaries, whole tiles only, and a mix;
  two calls give bit-identical results (the partials are added in a fixed order).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2410_04204_gb300 import inputs, tgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def dgemm_tc(A, B):
    """C = A B^T through the C ABI (A [M][K], B [N][K] row-major numpy float64)."""
    M, K = A.shape
    N = B.shape[0]
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    c = torch.empty(N, M, dtype=torch.float64, device="cuda")      # column-major M x N
    tgba.tgba_dgemm_tc(M, N, K, a, K, b, K, c, M)
    torch.cuda.synchronize()
    return c.cpu().numpy().T


def test_integer_products_are_exact():
    g = inputs.rng(31)
    M, N, K = 200, 70, 4096
    A = g.integers(-2 ** 13, 2 ** 13 + 1, (M, K)).astype(np.float64)
    B = g.integers(-2 ** 13, 2 ** 13 + 1, (N, K)).astype(np.float64)
    exact = (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float64)    # |C| < 2^38: exact
    C = dgemm_tc(A, B)
    assert np.array_equal(C, exact), np.abs(C - exact).max()


@pytest.mark.parametrize("M,N,K", [(300, 100, 1000), (128, 64, 32), (1, 1, 1), (257, 17, 777),
                                   (700, 300, 5000), (1000, 200, 100), (2000, 129, 700)])
def test_accuracy_against_extended_precision(M, N, K):
    g = inputs.rng(32 + M)
    A = g.standard_normal((M, K)) * 10.0 ** g.uniform(-3, 3, (M, 1))
    B = g.standard_normal((N, K)) * 10.0 ** g.uniform(-3, 3, (N, 1))
    C = dgemm_tc(A, B)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble).T)
    scale = np.abs(A) @ np.abs(B).T
    err = np.abs(C.astype(np.longdouble) - ref) / scale
    assert float(err.max()) <= 1e-12, float(err.max())
    Ct = (torch.from_numpy(A).cuda() @ torch.from_numpy(B).cuda().T).cpu().numpy()
    assert np.all(np.abs(C - Ct) <= 1.1e-12 * scale)


def test_argument_errors():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(tgba.TgbaError) as e:
        tgba.tgba_dgemm_tc(0, 1, 1, x, 1, x, 1, x, 1)
    assert e.value.code == tgba.TGBA_EINVAL


def test_split_tiles_are_deterministic():
    # 6 x 3 tiles of 40 chunks over the SMs: every tile is split, at uneven chunk boundaries
    g = inputs.rng(40)
    A = g.standard_normal((700, 5000))
    B = g.standard_normal((300, 5000))
    C1 = dgemm_tc(A, B)
    C2 = dgemm_tc(A, B)
    assert np.array_equal(C1, C2)
