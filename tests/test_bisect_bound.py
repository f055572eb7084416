"""The numerical premise of the eigenvalue bisection's single-precision phase, checked on the
CPU (no GPU): the Sturm count evaluated in float32 on T scaled to norm below 1 is the exact
count of a matrix within 5u||T||_inf of T (u = 2^-24; Weyl's inequality), so a bracket found
with it and widened by 8u||T||_inf on each side holds the eigenvalue.  Here the float32
recurrence (the three-term determinant form with power-of-two rescaling every 8 rows and the
smallest-normal replacement of a zero term) runs vectorised over all eigenvalue indices, on
the tridiagonal form of a matrix shaped like H_eff (diagonal energies and a weak off-diagonal
NS x R block), and every widened bracket must contain LAPACK's eigenvalue."""
import numpy as np
import scipy.linalg as sla

F32 = np.float32
TINY = F32(np.finfo(np.float32).tiny)


def _count32(d, e2, x):
    """Sturm counts at the float32 points x (vector), float32 arithmetic."""
    n = len(d)
    pm = np.ones_like(x)
    pc = d[0] - x
    pc = np.where(pc == 0, -TINY, pc)
    cnt = (pc < 0).astype(np.int64)
    for i in range(1, n):
        pn = (d[i] - x) * pc - e2[i - 1] * pm
        pn = np.where(pn == 0, np.where(pc > 0, -TINY, TINY), pn).astype(F32)
        cnt += (np.signbit(pn) != np.signbit(pc))
        pm, pc = pc, pn
        if i % 8 == 0:
            big = np.maximum(np.abs(pm), np.abs(pc))
            sc = np.ldexp(F32(1), -np.frexp(np.maximum(big, TINY))[1] + 1).astype(F32)
            pm, pc = pm * sc, pc * sc
    return cnt


def test_float32_bracket_widened_by_8u_norm_holds_the_eigenvalue():
    rng = np.random.default_rng(2410)
    n = 320
    A = np.zeros((n, n))
    A[np.arange(n), np.arange(n)] = np.sort(rng.uniform(-25.0, -13.0, n))
    X = rng.normal(size=(n // 2, n // 2)) * 0.02
    A[:n // 2, n // 2:] = X
    A[n // 2:, :n // 2] = X.T
    H = sla.hessenberg(A)
    d, e = np.diag(H).copy(), np.diag(H, -1).copy()
    lam = np.linalg.eigvalsh(A)
    r = np.abs(np.concatenate([[0.0], e])) + np.abs(np.concatenate([e, [0.0]]))
    lo, hi = (d - r).min(), (d + r).max()
    tnorm = max(abs(lo), abs(hi))
    sig = 2.0 ** -np.frexp(tnorm)[1]
    d32 = (d * sig).astype(F32)
    e32 = (e * e * sig * sig).astype(F32)
    dl = F32(2.0 ** -21) * F32(tnorm * sig)
    k = np.arange(n)
    a = np.full(n, F32(lo * sig) - 2 * dl, dtype=F32)
    b = np.full(n, F32(hi * sig) + 2 * dl, dtype=F32)
    for _ in range(40):
        mid = (F32(0.5) * (a + b)).astype(F32)
        left = _count32(d32, e32, mid) <= k
        a = np.where(left, mid, a)
        b = np.where(left, b, mid)
        if np.all(b - a <= dl):
            break
    A64 = a.astype(np.float64) / sig - float(dl) / sig
    B64 = b.astype(np.float64) / sig + float(dl) / sig
    assert np.all(A64 <= lam) and np.all(lam < B64)
    # and the bracket is narrow: about 3 dl, so the FP64 phase starts 2^-19 ||T|| wide
    assert np.all(B64 - A64 <= 4 * float(dl) / sig)
