"""The adjoint CG's iteration schedule (no GPU).

The persistent CG kernel reorders conjugate gradients so that an iteration
needs two grid-wide synchronisations: the rod pass forms r_k = r_{k-1} -
alpha Ap_{k-1} and p_k = r_k + beta p_{k-1} where it reads them, the
constraint pass applies the same update to its own constraints (lambda, r,
p) and stores Ap_k, and one grid sum gives p.Ap, r.Ap, Ap.Ap and r.r, from
which alpha_k = r.r / p.Ap and beta_k = (r.r - 2 alpha r.Ap + alpha^2
Ap.Ap) / r.r (the expansion of |r_k - alpha_k Ap_k|^2).  This restates that
schedule in numpy and checks that it produces the textbook CG iterates
(Hestenes-Stiefel, Fletcher-Reeves beta) and stops after the same number of
iterations, on seeded symmetric positive definite systems.
"""
import numpy as np
import pytest


def textbook_cg(A, b, tol, maxit):
    lam = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    tol2 = tol * tol * rr
    hist = [lam.copy()]
    it = 0
    while it < maxit and rr > tol2:
        Ap = A @ p
        alpha = rr / (p @ Ap)
        lam = lam + alpha * p
        r = r - alpha * Ap
        rrn = r @ r
        p = r + (rrn / rr) * p
        rr = rrn
        it += 1
        hist.append(lam.copy())
    return lam, it, hist


def two_sync_cg(A, b, tol, maxit):
    """The kernel's schedule: pass k applies update k-1 and computes Ap_k."""
    lam = np.zeros_like(b)
    R = b.copy()
    P = np.zeros_like(b)
    AP = np.zeros_like(b)
    alpha = beta = 0.0
    tol2 = tol * tol * (b @ b)
    hist = []
    it = 0
    while True:
        rk = R - alpha * AP            # rod pass and constraint pass alike
        pk = rk + beta * P
        Ap = A @ pk
        lam = lam + alpha * P          # lambda_k = lambda_{k-1} + alpha_{k-1} p_{k-1}
        R, P, AP = rk, pk, Ap
        hist.append(lam.copy())
        pap, rap, apap, rr = pk @ Ap, rk @ Ap, Ap @ Ap, rk @ rk
        if not rr > tol2 or it >= maxit:
            break
        alpha = rr / pap if pap > 0 else 0.0
        if not alpha > 0:
            break
        rrn = rr - 2.0 * alpha * rap + alpha * alpha * apap
        beta = rrn / rr if rrn > 0 else 0.0
        it += 1
    return lam, it, hist


def spd(rng, n, cond):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (q * ev) @ q.T


@pytest.mark.parametrize("seed,n,cond", [(0, 40, 1e2), (1, 120, 1e4), (2, 200, 10.0)])
def test_two_sync_schedule_gives_the_textbook_iterates(seed, n, cond):
    rng = np.random.default_rng(seed)
    A = spd(rng, n, cond)
    b = rng.standard_normal(n)
    tol = 1e-10
    lam_t, it_t, hist_t = textbook_cg(A, b, tol, 10 * n)
    lam_s, it_s, hist_s = two_sync_cg(A, b, tol, 10 * n)
    # the same iteration count (within 1 % once CG runs past n iterations,
    # where finite precision has spoilt the conjugacy and the rounding of the
    # two schedules' recurrences decides the last iteration)
    assert it_s == it_t if it_t <= n else abs(it_s - it_t) <= max(1, it_t // 100)
    # the same iterates while the recurrences are accurate (the early ones),
    # and the same answer at the end
    for k in range(min(8, it_t)):
        assert np.linalg.norm(hist_s[k] - hist_t[k]) <= 1e-10 * max(np.linalg.norm(hist_t[k]), 1e-300)
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(lam_s - x) <= 1e-7 * np.linalg.norm(x) * cond
    assert np.linalg.norm(A @ lam_s - b) <= 1.01 * tol * np.linalg.norm(b)


def test_two_sync_schedule_respects_max_iter_and_zero_rhs():
    rng = np.random.default_rng(3)
    A = spd(rng, 30, 1e3)
    b = rng.standard_normal(30)
    lam_t, it_t, _ = textbook_cg(A, b, 1e-14, 5)
    lam_s, it_s, _ = two_sync_cg(A, b, 1e-14, 5)
    assert it_s == it_t == 5
    assert np.allclose(lam_s, lam_t, rtol=1e-10, atol=1e-14)
    lam0, it0, _ = two_sync_cg(A, np.zeros(30), 1e-8, 100)
    assert it0 == 0 and not lam0.any()
