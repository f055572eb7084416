"""The paper-literal evaluation of X (tgba_x_direct: one complex Pfaffian of size 2L + M_a + M_b
per element, Eq. S1-S2, a warp per element) against the reduced form on the GPU (tgba_x_pairs)
and against the oracle's direct Pfaffians, up to the paper's L = 60."""
import numpy as np
import pytest
import torch

from oracle import elements as oel
from paper_2410_04204_gb300 import inputs, tgba
from tests.gpu_helpers import GpuSector, x_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _both(b, s, pairs):
    p = torch.tensor(pairs, dtype=torch.int32, device="cuda")
    xd = torch.empty(len(pairs), dtype=torch.complex128, device="cuda")
    xr = torch.empty(len(pairs), dtype=torch.complex128, device="cuda")
    tgba.tgba_x_direct(b, s, p, xd)
    tgba.tgba_x_pairs(b, s, p, xr)
    return xd.cpu().numpy(), xr.cpu().numpy()


@pytest.mark.parametrize("L,h,m,mq,cut,count", [(12, 1.0, 0, 12, None, 600), (10, 0.6, 3, 10, None, 400),
                                                (24, 1.0, 7, 6, 11.925, 1500), (60, 1.0, 0, 4, 3.0, 300)])
def test_direct_equals_reduced_and_oracle(L, h, m, mq, cut, count):
    b = tgba.tgba_build_basis(L, h, [m], mq, -1.0 if cut is None else cut)
    try:
        tgba.tgba_compute_x(b)
        g = GpuSector(b, 0, mq)
        pairs = inputs.sample_pairs(g.n_ns, g.n_r, count, tag=L + m)
        pairs[0] = (0, 0)                                  # the vacuum element
        xd, xr = _both(b, 0, pairs)
        ok, worst = x_close(xd, xr, rel=1e-9)
        assert ok, worst
        # a few elements against the oracle's direct Pfaffians of the same strings
        sub = pairs[:24]
        sel = [(g.keys[a][1], g.keys[g.n_ns + c][1]) for a, c in sub]
        xo = oel.x_elements(L, h, sel)
        ok, worst = x_close(xd[:24], xo, rel=1e-9)
        assert ok, worst
    finally:
        tgba.tgba_basis_free(b)


def test_direct_rejects_too_long_strings_and_bad_indices():
    b = tgba.tgba_build_basis(80, 1.0, [0], 2, 3.0)       # string of 164 operators: too big for one warp's triangle
    try:
        tgba.tgba_compute_x(b)
        p = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
        out = torch.empty(1, dtype=torch.complex128, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_x_direct(b, 0, p, out)
        assert e.value.code == tgba.TGBA_EINVAL
    finally:
        tgba.tgba_basis_free(b)
    b = tgba.tgba_build_basis(10, 1.0, [0], 4)
    try:
        tgba.tgba_compute_x(b)
        p = torch.tensor([[0, 0], [10 ** 6, 0]], dtype=torch.int32, device="cuda")
        out = torch.empty(2, dtype=torch.complex128, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_x_direct(b, 0, p, out)
        assert e.value.code == tgba.TGBA_EINVAL
        good = torch.tensor([[0, 0]], dtype=torch.int32, device="cuda")
        tgba.tgba_x_direct(b, 0, good, out[:1])          # the handle stays usable
        assert np.isfinite(out[0].item())
    finally:
        tgba.tgba_basis_free(b)
