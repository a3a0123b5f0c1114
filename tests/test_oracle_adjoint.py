"""The oracle's adjoint of one constrained step against central finite
differences of the oracle's own forward step (h = 1e-6).

Differentiation workload (scaled down): loss = sum of squared post-step
centre displacements from seeded targets; gradient with respect to the
initial centres, orientations (tangent space of the unit quaternion) and
the viscosity (every drag coefficient is proportional to it), plus the
input forces and a loss on the post-step quaternions.  The forward steps of
the finite differences find their own pair lists and solve their own LCPs
(exact active-set enumeration up to 20 constraints, FISTA to 1e-13 above);
the tests assert that neither the pair list nor the active set changes
between them, so the loss is smooth there.  Every closest-point branch
(interior, one parameter clamped, both clamped) occurs among the active
constraints of these systems.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as ADJ
from paper_2109_08206_gb300 import workloads as W

EPS = 1e-6

SYSTEMS = [(1, 20, 9.0, 3.0), (2, 30, 10.0, 3.0), (3, 16, 8.0, 4.0), (4, 12, 7.0, 3.0)]


def make(seed, n, box, L):
    s = W.tiny_system(300 + seed, n, box=box, length=L)
    s.f_nc *= 30.0
    targets = s.x + 0.01 * np.random.default_rng(seed).standard_normal(s.x.shape)
    return s, targets


def tangent_basis(th):
    return np.linalg.svd(th.reshape(1, 4))[2][1:]


def branches(s, fw):
    pb = O.problem_of(s)
    p = O.axis(s.quat)
    xw = O.wrap(s.x, s.box)
    box = np.asarray(s.box)
    hl = 0.5 * s.length
    kinds = set()
    for c in np.nonzero(fw["gamma"] > 0)[0]:
        i, j, code = fw["pairs"][c]
        k = np.array([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1])
        _, sc, tc = O.segment_closest(xw[i] - xw[j] - k * box, p[i], p[j], pb.length)
        kinds.add((abs(sc) < hl) + (abs(tc) < hl))
    return kinds


class Evaluator:
    def __init__(self, s, targets, quat_weights=None):
        self.s, self.T, self.w = s, targets, quat_weights
        self.fw0 = ADJ.forward(s.x, s.quat, s.f_nc, O.problem_of(s))

    def loss(self, x=None, quat=None, eta=None, fnc=None):
        s = self.s
        pb = O.problem_of(s)
        if eta is not None:
            pb.viscosity = eta
        fw = ADJ.forward(s.x if x is None else x, s.quat if quat is None else quat, s.f_nc if fnc is None else fnc,
                         pb)
        assert np.array_equal(fw["pairs"], self.fw0["pairs"])
        assert np.array_equal(fw["gamma"] > 0, self.fw0["gamma"] > 0)
        L = ADJ.centre_loss(fw["x"], self.T)
        if self.w is not None:
            L += float(np.sum(self.w * fw["quat"]))
        return L

    def grad(self):
        s, fw = self.s, self.fw0
        return ADJ.step_adjoint(s.x, s.quat, s.f_nc, O.problem_of(s), 2.0 * (fw["x"] - self.T),
                                None if self.w is None else self.w, fw=fw)


def fd(f, a, da):
    return (f(a + da) - f(a - da)) / (2 * EPS)


def rel_err(got, want):
    got, want = np.asarray(got), np.asarray(want)
    return np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)


@pytest.mark.parametrize("seed,n,box,L", SYSTEMS)
def test_gradient_wrt_centres_and_orientations(seed, n, box, L):
    s, T = make(seed, n, box, L)
    ev = Evaluator(s, T)
    g = ev.grad()
    want_x = np.zeros_like(s.x)
    for i in range(s.n):
        for k in range(3):
            d = np.zeros_like(s.x)
            d[i, k] = EPS
            want_x[i, k] = (ev.loss(x=s.x + d) - ev.loss(x=s.x - d)) / (2 * EPS)
    assert rel_err(g["x"], want_x) < 1e-6
    got_q, want_q = [], []
    for i in range(s.n):
        for v in tangent_basis(s.quat[i]):
            qp, qm = s.quat.copy(), s.quat.copy()
            qp[i] = (s.quat[i] + EPS * v) / np.linalg.norm(s.quat[i] + EPS * v)
            qm[i] = (s.quat[i] - EPS * v) / np.linalg.norm(s.quat[i] - EPS * v)
            want_q.append((ev.loss(quat=qp) - ev.loss(quat=qm)) / (2 * EPS))
            got_q.append(g["quat"][i] @ v)
    assert rel_err(got_q, want_q) < 1e-6
    # the reported orientation gradient lies in the tangent space
    assert np.abs(np.sum(g["quat"] * s.quat, axis=1)).max() < 1e-12 * np.abs(g["quat"]).max()


@pytest.mark.parametrize("seed,n,box,L", SYSTEMS[:2])
def test_gradient_wrt_viscosity_and_forces(seed, n, box, L):
    s, T = make(seed, n, box, L)
    ev = Evaluator(s, T)
    g = ev.grad()
    want = (ev.loss(eta=s.viscosity + EPS) - ev.loss(eta=s.viscosity - EPS)) / (2 * EPS)
    assert g["eta"] == pytest.approx(want, rel=1e-5, abs=1e-9 * abs(ev.loss()))
    # on a fixed active set U is affine in F_nc and the loss quadratic, so a
    # central difference is exact up to rounding for any step: take 1e-2
    rng = np.random.default_rng(seed)
    for _ in range(6):
        i, k = int(rng.integers(s.n)), int(rng.integers(6))
        d = np.zeros_like(s.f_nc)
        d[i, k] = 1e-2
        want = (ev.loss(fnc=s.f_nc + d) - ev.loss(fnc=s.f_nc - d)) / 2e-2
        assert g["fnc"][i, k] == pytest.approx(want, rel=1e-6, abs=1e-6 * np.abs(g["fnc"]).max())


def test_gradient_through_the_quaternion_update():
    s, T = make(2, 30, 10.0, 3.0)
    w = np.random.default_rng(5).standard_normal(s.quat.shape)
    ev = Evaluator(s, T, quat_weights=w)
    g = ev.grad()
    rng = np.random.default_rng(6)
    for _ in range(10):
        i = int(rng.integers(s.n))
        k = int(rng.integers(3))
        d = np.zeros_like(s.x)
        d[i, k] = EPS
        want = (ev.loss(x=s.x + d) - ev.loss(x=s.x - d)) / (2 * EPS)
        assert g["x"][i, k] == pytest.approx(want, rel=1e-6, abs=1e-9 * np.abs(g["x"]).max())
        v = tangent_basis(s.quat[i])[k]
        qp, qm = s.quat.copy(), s.quat.copy()
        qp[i] = (s.quat[i] + EPS * v) / np.linalg.norm(s.quat[i] + EPS * v)
        qm[i] = (s.quat[i] - EPS * v) / np.linalg.norm(s.quat[i] - EPS * v)
        want = (ev.loss(quat=qp) - ev.loss(quat=qm)) / (2 * EPS)
        assert g["quat"][i] @ v == pytest.approx(want, rel=1e-6, abs=1e-9 * np.abs(g["quat"]).max())


def test_every_closest_point_branch_is_exercised():
    kinds = set()
    for sysargs in SYSTEMS:
        s, _ = make(*sysargs)
        kinds |= branches(s, ADJ.forward(s.x, s.quat, s.f_nc, O.problem_of(s)))
    assert kinds == {0, 1, 2}   # free parameters per active constraint: both clamped, one, none


def test_no_contact_gradient_is_free_drift():
    # no pairs: x' = x + h M F, so dL/dx = dL/dx' and dL/deta = -(u . U)/eta
    s = W.tiny_system(11, 3, box=40.0, length=3.0)
    s.x = np.array([[5.0, 5, 5], [20, 20, 20], [33, 8, 25]])
    T = s.x + 0.1
    L, g, fw = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, O.problem_of(s), T)
    assert fw["pairs"].shape[0] == 0
    np.testing.assert_allclose(g["x"], 2.0 * (fw["x"] - T), rtol=0, atol=1e-15)
    U = fw["U"]
    assert g["eta"] == pytest.approx(-np.sum(s.dt * 2.0 * (fw["x"] - T) * U[:, :3]) / s.viscosity, rel=1e-12)


@pytest.mark.parametrize("seed,n,box,L", SYSTEMS)
def test_sparse_form_equals_dense_form(seed, n, box, L):
    """The sparse oracle adjoint (scipy sparse D and M, MINRES on the active
    system) gives the dense one's gradient, whose central differences the
    tests above check: the large-system oracle inherits that pin."""
    s, T = make(seed, n, box, L)
    pb = O.problem_of(s)
    Ld, gd, fwd = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, pb, T)
    Ls, gs, fws = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, pb, T, sparse=True)
    assert np.array_equal(fwd["pairs"], fws["pairs"])
    assert Ls == pytest.approx(Ld, rel=1e-13)
    for k in ("x", "quat", "fnc", "lambda"):
        assert rel_err(gs[k], gd[k]) < 1e-10, k
    assert gs["eta"] == pytest.approx(gd["eta"], rel=1e-10)


def test_sparse_form_against_central_differences():
    """The sparse form on its own against central differences of the
    oracle's forward step, on a system of 120 rods (larger than the dense
    tests' and still quick)."""
    s = W.tiny_system(377, 120, box=18.0, length=4.0)
    s.f_nc *= 30.0
    T = s.x + 0.01 * np.random.default_rng(9).standard_normal(s.x.shape)
    pb = O.problem_of(s)
    L0, g, fw0 = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, pb, T, sparse=True)
    assert (fw0["gamma"] > 0).sum() >= 20

    def loss(x=None, quat=None):
        fw = ADJ.forward(s.x if x is None else x, s.quat if quat is None else quat, s.f_nc, pb, sparse=True)
        assert np.array_equal(fw["pairs"], fw0["pairs"])
        assert np.array_equal(fw["gamma"] > 0, fw0["gamma"] > 0)
        return ADJ.centre_loss(fw["x"], T)

    rng = np.random.default_rng(4)
    rods = rng.choice(np.unique(fw0["pairs"][fw0["gamma"] > 0][:, :2]), size=5, replace=False)
    for i in rods:
        k = int(rng.integers(3))
        d = np.zeros_like(s.x)
        d[i, k] = EPS
        want = (loss(x=s.x + d) - loss(x=s.x - d)) / (2 * EPS)
        assert g["x"][i, k] == pytest.approx(want, rel=1e-5, abs=1e-8 * np.abs(g["x"]).max())
        v = tangent_basis(s.quat[i])[k]
        qp, qm = s.quat.copy(), s.quat.copy()
        qp[i] = (s.quat[i] + EPS * v) / np.linalg.norm(s.quat[i] + EPS * v)
        qm[i] = (s.quat[i] - EPS * v) / np.linalg.norm(s.quat[i] - EPS * v)
        want = (loss(quat=qp) - loss(quat=qm)) / (2 * EPS)
        assert g["quat"][i] @ v == pytest.approx(want, rel=1e-5, abs=1e-8 * np.abs(g["quat"]).max())
