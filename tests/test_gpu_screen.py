"""The learned pair screener on the GPU against the MLP oracle: back-propagation (FP32 kernels)
against float64 gradients, tensor-core inference (BF16 layer 2) against the float64 forward
pass, and a small end-to-end training + screened assembly whose eigenvalue error is measured."""
import math

import numpy as np
import pytest
import torch

from oracle import basis as obs
from oracle import mlp
from oracle import modes as md
from paper_2410_04204_gb300 import inputs, tgba
from tests.gpu_helpers import GpuSector

pytestmark = pytest.mark.gpu
H = 256


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_gradient_matches_oracle():
    theta = mlp.init(H, inputs.SEED).astype(np.float32)
    s = tgba.tgba_screen_create(H, theta)
    try:
        assert tgba.tgba_screen_nparams(s) == mlp.n_params(H)
        assert np.array_equal(tgba.tgba_screen_params(s), theta)
        g = inputs.rng(11)
        x = g.uniform(-1, 1, (300, mlp.D_IN)).astype(np.float32)
        t = g.normal(-4, 2, 300).astype(np.float32)
        grad = torch.empty(len(theta), dtype=torch.float32, device="cuda")
        loss = tgba.tgba_screen_grad(s, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), grad)
        lo, go = mlp.loss_and_grad(theta.astype(np.float64), H, x.astype(np.float64), t.astype(np.float64))
        gg = grad.cpu().numpy()
        assert abs(loss - lo) <= 1e-5 * lo
        # FP32 accumulation over a batch of 300 and 256 hidden units: blockwise relative 1e-4
        o = 0
        for shape in mlp.shapes(H):
            n = int(np.prod(shape))
            ref = go[o:o + n]
            assert np.abs(gg[o:o + n] - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-7, shape
            o += n
    finally:
        tgba.tgba_screen_free(s)


def test_inference_matches_oracle_forward():
    L, mq = 12, 6
    theta = mlp.init(H, 5).astype(np.float32)
    theta[-1] = -3.0
    s = tgba.tgba_screen_create(H, theta)
    b = tgba.tgba_build_basis(L, 1.0, [0], mq)
    try:
        g = GpuSector(b, 0, mq)
        pred = torch.empty(g.n_ns * g.n_r, dtype=torch.float32, device="cuda")
        tgba.tgba_screen_predict(s, b, 0, pred)
        P = pred.cpu().numpy().reshape(g.n_ns, g.n_r)
        nn, nr = md.momenta_n(L, md.NS), md.momenta_n(L, md.R)
        ka, kb = g.keys[:g.n_ns], g.keys[g.n_ns:]
        rows = [(a, c) for a in range(g.n_ns) for c in range(g.n_r)]
        x = mlp.features(L, [ka[a][1] for a, _ in rows], [kb[c][1] for _, c in rows], nn, nr)
        y, (z1, h1, z2, h2) = mlp.forward(theta.astype(np.float64), H, x)
        w3 = theta.astype(np.float64)[-H - 1:-1]
        scale = np.abs(h2 * w3).sum(1) + abs(theta[-1])
        got = P[tuple(np.array(rows).T)]
        # two BF16 roundings (h1 and W2, 2^-9 each) feed an FP32 sum: |dy| <= 2^-6 * scale
        assert np.all(np.abs(got - y) <= 2.0 ** -6 * scale), float(np.max(np.abs(got - y) / scale))
    finally:
        tgba.tgba_basis_free(b)
        tgba.tgba_screen_free(s)


def test_train_and_screen_small():
    """Train on all sectors of L = 14 (M <= 6), screen the k = 0 sector of L = 14 and L = 16:
    the lowest 20 eigenvalues stay within 1e-6 relative of the exact assembly."""
    tr = tgba.tgba_build_basis(14, 1.0, list(range(14)), 6)
    try:
        s, stats = tgba.tgba_screen_train([tr], 200000, inputs.SEED, 6)
    finally:
        tgba.tgba_basis_free(tr)
    try:
        assert stats["val_rmse"] < 1.0 and math.isclose(stats["margin"], 3 * stats["val_rmse"])
        for L in (14, 16):
            b = tgba.tgba_build_basis(L, 1.0, [0], 6)
            try:
                g = GpuSector(b, 0, 6)
                n = g.n_ns + g.n_r
                ev = torch.empty(n, dtype=torch.float64, device="cuda")
                tgba.tgba_compute_x(b)
                tgba.tgba_eigvals(b, 0.1, ev)
                exact = ev.cpu().numpy()[:20].copy()
                tgba.tgba_compute_x(b, s, 1e-8, 0.1)
                n_eval, n_scr = tgba.tgba_x_stats(b)
                assert n_eval + n_scr == g.n_ns * g.n_r
                tgba.tgba_eigvals(b, 0.1, ev)
                got = ev.cpu().numpy()[:20]
                assert np.abs(got - exact).max() <= 1e-6 * np.abs(exact).max()
            finally:
                tgba.tgba_basis_free(b)
    finally:
        tgba.tgba_screen_free(s)


def test_screened_stage_keeps_exactly_the_predicted_pairs():
    """The tensor-core scoring compacts the kept pairs into per-size lists: every pair whose
    prediction passes the threshold gets the exact Pfaffian (bit for bit the unscreened value),
    every other pair 0, and the counts of tgba_x_stats agree.  Random weights with a bias that
    drops about half of the pairs; pairs within 1e-4 of the threshold are not judged (the two
    sides may round the comparison differently)."""
    L, mq, hx, tau = 16, 6, 0.1, 1e-8
    theta = mlp.init(H, 7).astype(np.float32)
    s = tgba.tgba_screen_create(H, theta)
    b = tgba.tgba_build_basis(L, 1.0, [0], mq)
    try:
        g = GpuSector(b, 0, mq)
        pred = torch.empty(g.n_ns * g.n_r, dtype=torch.float32, device="cuda")
        tgba.tgba_screen_predict(s, b, 0, pred)
        y = pred.cpu().numpy().reshape(g.n_ns, g.n_r).astype(np.float64)
        n = g.nqp[:g.n_ns, None].astype(np.float64) + g.nqp[None, g.n_ns:]
        margin = 1.0                                       # a created (untrained) screener's margin
        v = y - 0.5 * math.log10(L / 24.0) * n + (math.log10(L * hx) - math.log10(tau) + margin)
        med = float(np.median(v))
        theta[-1] -= med                                   # shift b3 so that about half is dropped
        tgba.tgba_screen_free(s)
        s = tgba.tgba_screen_create(H, theta)
        v = v - med
        tgba.tgba_compute_x(b)
        exact = g.x()
        tgba.tgba_compute_x(b, s, tau, hx)
        scr = g.x()
        n_eval, n_scr = tgba.tgba_x_stats(b)
        keep, drop = v >= 1e-4, v <= -1e-4
        assert drop.sum() > 0.2 * v.size and keep.sum() > 0.2 * v.size
        assert np.array_equal(scr[keep], exact[keep])
        assert np.all(scr[drop] == 0)
        assert n_eval + n_scr == v.size
        assert keep.sum() <= n_eval <= v.size - drop.sum()
    finally:
        tgba.tgba_basis_free(b)
        tgba.tgba_screen_free(s)
