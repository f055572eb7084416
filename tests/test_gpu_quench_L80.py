"""The quench at the size of the L = 80 benchmark workload (M <= 10, h_z0 = 0.5 -> h_z = 1,
2000 times in [0, 100]; Eq. 10, the norm statement of the Quench section, Eq. S6) through the
C ABI.

* Both propagation paths (eigendecomposition, as Eq. 10 writes it, and the batched Chebyshev
  expansion with all variants in one graph) against the oracle's quench on nested cutoffs of
  338, 760 and 1018 states, stored by tests/golden/make_quench_L80.py (direct Pfaffians of the
  whole operator string for X and the overlaps, dense eigenpairs).
* The two paths against each other on the benchmark's own basis (3.8e8 Pfaffian elements) at a
  cutoff keeping more than 4096 states, for the weakest and the strongest field of its grid.
"""
import os

import numpy as np
import pytest
import torch

from paper_2410_04204_gb300 import inputs, tgba

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quench_L80.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def golden():
    cases, cur = {}, None
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#"):
                continue
            if line.startswith("case"):
                _, cut, hx, chi, n2 = line.split()
                cur = (float(cut), float(hx))
                cases[cur] = (int(chi), float(n2), [])
            else:
                cases[cur][2].append(float(line))
    return {k: (c, n, np.array(v)) for k, (c, n, v) in cases.items()}


@pytest.mark.parametrize("method", [1, 2])
def test_quench_L80_against_oracle(method):
    w = inputs.QUENCH_L80
    q = w.quench
    ref = golden()
    keys = sorted(ref)
    b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp, max(c for c, _ in keys))
    try:
        tgba.tgba_compute_x(b)
        n_t = q["n_t"]
        mx = torch.empty(len(keys) * n_t, dtype=torch.float64, device="cuda")
        nrm = torch.empty(len(keys), dtype=torch.float64, device="cuda")
        chi = tgba.tgba_quench(b, 0, q["h_z0"], [hx for _, hx in keys], [c for c, _ in keys], q["t_max"], n_t, mx,
                               nrm, method=method)
        m = mx.cpu().numpy().reshape(len(keys), n_t)
        for i, k in enumerate(keys):
            c_ref, n_ref, m_ref = ref[k]
            assert chi[i] == c_ref, (k, chi[i], c_ref)
            assert abs(nrm[i].item() - n_ref) < 1e-12
            err = np.abs(m[i] - m_ref).max()
            assert err < 1e-9, (k, method, err)
    finally:
        tgba.tgba_basis_free(b)


def test_quench_L80_chebyshev_matches_eigen_above_4096_states():
    w = inputs.QUENCH_L80
    q = w.quench
    b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp, w.e_cut, w.max_per_parity)
    try:
        tgba.tgba_compute_x(b)
        info = tgba.tgba_basis_info(b, 0, w.max_qp)
        E = info["E0"]
        e_vac = E[:info["n_ns"]].min()
        cut = inputs.nested_cutoffs(E - e_vac, [4500])[0]
        hxs = [inputs.QUENCH_L80_HX[0], inputs.QUENCH_L80_HX[-1]]
        n_t = q["n_t"]
        out = {}
        for method in (1, 2):
            mx = torch.empty(len(hxs) * n_t, dtype=torch.float64, device="cuda")
            chi = tgba.tgba_quench(b, 0, q["h_z0"], hxs, [cut] * len(hxs), q["t_max"], n_t, mx, method=method)
            assert np.all(chi > 4096)
            out[method] = mx.cpu().numpy()
        assert np.abs(out[1] - out[2]).max() < 1e-9
    finally:
        tgba.tgba_basis_free(b)
