"""Edge cases of the GPU path: degenerate truncations, the smallest chain, Pfaffian sizes of
every kernel class (up to n = 32), ragged tiles, bad pair indices, and agreement of the
pair kernel with the tiled kernel."""
import numpy as np
import pytest
import torch

from oracle import basis as obs
from oracle import elements as oel
from paper_2410_04204_gb300 import inputs, tgba
from tests.gpu_helpers import GpuSector, x_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def run(L, h, sectors, mq, cut=-1.0, cap=0):
    b = tgba.tgba_build_basis(L, h, sectors, mq, cut, cap)
    tgba.tgba_compute_x(b)
    return b


def test_vacua_only():
    """max_qp = 0: one NS and one R state, X = <0_NS|sigma|0_R> = C0."""
    b = run(10, 0.7, [0], 0)
    try:
        g = GpuSector(b, 0, 0)
        assert (g.n_ns, g.n_r) == (1, 1)
        c0 = tgba.tgba_table(b)
        want = oel.vacuum_sigma(10, 0.7)
        assert abs(g.x()[0, 0] - want) < 1e-13 and abs(c0 - want) < 1e-13
    finally:
        tgba.tgba_basis_free(b)


def test_empty_parity_and_empty_x():
    """Paramagnet (h = 1.5): a cutoff of 0.5 keeps only the NS vacuum, so X is empty and
    H_eff is the NS diagonal."""
    L, h = 12, 1.5
    b = run(L, h, [0], 4, 0.5)
    try:
        g = GpuSector(b, 0, 4)
        ns, r = obs.sector_basis(L, h, 0, 4, 0.5)
        assert (g.n_ns, g.n_r) == (len(ns), len(r)) and len(r) == 0
        n = g.n_ns + g.n_r
        ev = torch.empty(n, dtype=torch.float64, device="cuda")
        tgba.tgba_eigvals(b, 0.2, ev)
        assert np.allclose(np.sort(ev.cpu().numpy()), np.sort([s.E for s in ns + r]), atol=1e-12)
    finally:
        tgba.tgba_basis_free(b)


def test_smallest_chain_all_sectors():
    b = run(4, 1.3, [0, 1, 2, 3], 4)
    try:
        for s in range(4):
            g = GpuSector(b, s, 4)
            ns, r = obs.sector_basis(4, 1.3, s, 4)
            pa, pb = g.perm_to(ns, r)
            if len(ns) and len(r):
                ok, worst = x_close(g.x(), oel.x_block(4, 1.3, ns, r)[np.ix_(pa, pb)])
                assert ok, worst
    finally:
        tgba.tgba_basis_free(b)


@pytest.mark.parametrize("L,mq,m", [(16, 16, 0), (16, 12, 3)])
def test_large_pfaffians_every_class(L, mq, m):
    """Full bases of L = 16 reach n = M + M' up to 30 at k = 0: every register class (n <= 14)
    and every shared-memory class (n <= 16, 20, 24, 32), with ragged last tiles."""
    b = run(L, 1.0, [m], mq)
    try:
        g = GpuSector(b, 0, mq)
        ns, r = obs.sector_basis(L, 1.0, m, mq)
        X = g.x()
        pa, pb = g.perm_to(ns, r)
        inv_a = np.argsort(pa)
        inv_b = np.argsort(pb)
        # all pairs of the largest n, plus a seeded sample of the rest
        big = [(a, c) for a in range(len(ns)) for c in range(len(r)) if ns[a].M + r[c].M >= 24]
        big.sort(key=lambda p: -(ns[p[0]].M + r[p[1]].M))
        sample = [tuple(x) for x in inputs.sample_pairs(len(ns), len(r), 300, tag=L * 100 + m)]
        pairs = sorted(set(big[:400] + sample))
        want = oel.x_elements(L, 1.0, [(ns[a].modes, r[c].modes) for a, c in pairs])
        got = np.array([X[inv_a[a], inv_b[c]] for a, c in pairs])
        scale = np.abs(want).max()
        assert np.all(np.abs(got - want) <= 1e-10 * (np.abs(want) + 1e-3 * scale))
        sizes = {ns[a].M + r[c].M for a, c in pairs}
        assert max(sizes) >= (24 if mq == 12 else 30)
    finally:
        tgba.tgba_basis_free(b)


def test_pairs_kernel_matches_tiles_bit_exactly():
    b = run(14, 1.0, [0], 8)
    try:
        g = GpuSector(b, 0, 8)
        X = g.x()
        pairs = inputs.sample_pairs(g.n_ns, g.n_r, 4000, tag=3).astype(np.int32)
        out = torch.empty(len(pairs), dtype=torch.complex128, device="cuda")
        tgba.tgba_x_pairs(b, 0, torch.from_numpy(pairs).cuda(), out)
        assert np.array_equal(out.cpu().numpy(), X[pairs[:, 0], pairs[:, 1]])
    finally:
        tgba.tgba_basis_free(b)


def test_bad_pair_index_is_rejected():
    b = run(10, 1.0, [0], 4)
    try:
        g = GpuSector(b, 0, 4)
        bad = torch.tensor([[0, 0], [g.n_ns, 0], [0, -1]], dtype=torch.int32, device="cuda")
        out = torch.empty(3, dtype=torch.complex128, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_x_pairs(b, 0, bad, out)
        assert e.value.code == tgba.TGBA_EINVAL
        # the handle stays usable
        good = torch.tensor([[0, 0]], dtype=torch.int32, device="cuda")
        tgba.tgba_x_pairs(b, 0, good, out)
        assert np.isfinite(out[0].item())
    finally:
        tgba.tgba_basis_free(b)


def test_argument_errors_with_device():
    b = run(10, 1.0, [0, 1], 4)
    try:
        with pytest.raises(tgba.TgbaError):
            tgba.tgba_basis_info(b, 2, 4)                 # sector index out of range
        S = torch.empty(8, dtype=torch.float32, device="cuda")
        with pytest.raises(tgba.TgbaError):
            tgba.tgba_dsf(b, 1, 0.1, 0, 1, 8, 0.1, S)      # m = 1 is not k = 0
        with pytest.raises(tgba.TgbaError):
            tgba.tgba_dsf(b, 0, 0.1, 0, 1, 8, -1.0, S)     # eta <= 0
    finally:
        tgba.tgba_basis_free(b)
