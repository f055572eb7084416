"""Same-parity elements of sigma^x_1 sigma^x_{j+1} in the reduced form (tgba_z_elements: both
vacua contracted once into a table, then one Pfaffian of size M_a + 2j + M_b per element)
against the oracle's direct Pfaffians of the whole string (size 2L + M_a + M_b + 2j), and
pinned by j = 0 (the overlaps <phi_a|phi_b> = delta_ab) and by Hermiticity, up to L = 60."""
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


def _z(b, parity, j, pairs):
    p = torch.tensor(np.asarray(pairs, dtype=np.int32).reshape(-1, 2), dtype=torch.int32, device="cuda")
    out = torch.empty(len(pairs), dtype=torch.complex128, device="cuda")
    tgba.tgba_z_elements(b, 0, parity, j, p, out)
    return out.cpu().numpy()


def _modes(g, parity, i):
    return g.keys[(g.n_ns if parity else 0) + i][1]


@pytest.mark.parametrize("L,h,m,mq,cut,js,count", [(10, 1.0, 0, 10, None, (1, 2, 5), 120),
                                                   (12, 0.6, 5, 12, None, (1, 3), 120),
                                                   (24, 1.0, 0, 6, 11.925, (1, 4, 11), 48),
                                                   (60, 1.0, 0, 4, 3.0, (2, 9), 12)])
def test_reduced_equals_oracle_direct(L, h, m, mq, cut, js, count):
    b = tgba.tgba_build_basis(L, h, [m], mq, -1.0 if cut is None else cut)
    try:
        g = GpuSector(b, 0, mq)
        for parity, n in ((0, g.n_ns), (1, g.n_r)):
            if n == 0:
                continue
            pairs = inputs.sample_pairs(n, n, count, tag=L + 7 * parity + m)
            pairs[0] = (0, 0)
            for j in js:
                z = _z(b, parity, j, pairs)
                zo = oel.z_elements(L, h, parity, j, [(_modes(g, parity, a), _modes(g, parity, c)) for a, c in pairs])
                ok, worst = x_close(z, zo, rel=1e-9)
                assert ok, (parity, j, worst)
    finally:
        tgba.tgba_basis_free(b)


@pytest.mark.parametrize("L,mq,cut", [(24, 6, 11.925), (60, 4, 3.0)])
def test_j0_is_the_identity_and_z_is_hermitian(L, mq, cut):
    b = tgba.tgba_build_basis(L, 1.0, [0], mq, cut)
    try:
        g = GpuSector(b, 0, mq)
        for parity, n in ((0, g.n_ns), (1, g.n_r)):
            k = min(n, 24)
            pairs = [(a, c) for a in range(k) for c in range(k)]
            z0 = _z(b, parity, 0, pairs).reshape(k, k)
            assert np.abs(z0 - np.eye(k)).max() < 1e-12
            z = _z(b, parity, 5, pairs).reshape(k, k)
            assert np.abs(z - z.conj().T).max() < 1e-12 * max(1.0, np.abs(z).max())
    finally:
        tgba.tgba_basis_free(b)


def test_rejects_bad_arguments():
    b = tgba.tgba_build_basis(12, 1.0, [0], 4)
    try:
        p = torch.tensor([[0, 10 ** 6]], dtype=torch.int32, device="cuda")
        out = torch.empty(1, dtype=torch.complex128, device="cuda")
        for parity, j in ((2, 1), (0, -1), (0, 12)):
            with pytest.raises(tgba.TgbaError) as e:
                tgba.tgba_z_elements(b, 0, parity, j, p, out)
            assert e.value.code == tgba.TGBA_EINVAL
        with pytest.raises(tgba.TgbaError) as e:                # index outside the sector
            tgba.tgba_z_elements(b, 0, 0, 1, p, out)
        assert e.value.code == tgba.TGBA_EINVAL
        assert np.isnan(out.cpu().numpy()[0].real)
        ok = torch.tensor([[0, 0]], dtype=torch.int32, device="cuda")
        tgba.tgba_z_elements(b, 0, 0, 0, ok, out)               # the handle stays usable
        assert abs(out.cpu().numpy()[0] - 1.0) < 1e-12
    finally:
        tgba.tgba_basis_free(b)
