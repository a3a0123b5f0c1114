"""Adjoint of one constrained step (oracle side: dense matrices for small
systems, scipy sparse matrices for large ones, the same formulas).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests use it to
check the CUDA adjoint.  It shares no code with the CUDA path.

The step (Appendix Eq. constrainedeom_euler a-c with the constraint problem
of Eq. suppcqpdef) maps (x, theta, eta, F_nc) to
    U = M(F_nc + D gamma),  x' = x + h U_t,  theta' = normalise(theta + h Psi(theta) Omega),
with gamma = argmin 1/2 g^T A g + q^T g, g >= 0, A = D^T M D, q = Phi/h + D^T M F_nc,
and all drag coefficients proportional to the viscosity eta.  For a scalar
loss L(x', theta') the gradient is taken on the fixed pair list and active
set A = {c : gamma_c > 0} (KKT: (A gamma + q)_A = 0, gamma_I = 0):

    u   = dL/dU                       (through the update),
    b   = D^T M u,  lambda_A solves A_AA lambda_A = b_A (minimum-norm
          solution: dense lstsq, or sparse MINRES from zero; b_A lies in
          the range of A_AA),
    w   = D lambda,  nu = M (u - w),
    dL  = [direct terms of the update] + (u - w)^T dM F_tot
          + nu^T (dD gamma) - (dD lambda)^T U - lambda^T dPhi / h,

with F_tot = F_nc + D gamma.  dPhi = e.(dDx + s dp_P - t dp_Q) (envelope: the
closest-point parameters are stationary or clamped), and the derivative of
the D column (e, y_P x e | -e, -y_Q x e) follows the closest points through
their branch: interior (both parameters from the 2x2 stationarity system),
one parameter clamped (the other from its 1-D condition), or both clamped.
Parallel segments (the midpoint reading) are differentiated with s*, t*
held fixed.  dL/dF_nc = nu; dL/d eta = -(u - w)^T U / eta.

Orientation gradients are reported in the tangent space of the unit
quaternion: g - theta (theta . g), the Euclidean gradient of L through the
axis map p(theta) projected onto the unit sphere's tangent plane.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import assemble, axis, drag, find_pairs, segment_closest, solve_apgd, solve_enum, wrap


def _mobility_blocks(p, zeta):
    """Per-rod 6x6 mobility: M_t = I/zp + (1/zpar - 1/zp) p p^T, M_r likewise."""
    zp, zpar, zr, zs = zeta
    n = p.shape[0]
    Mb = np.zeros((n, 6, 6))
    pp = np.einsum("ni,nj->nij", p, p)
    eye = np.eye(3)
    Mb[:, :3, :3] = eye / zp + (1.0 / zpar - 1.0 / zp) * pp
    Mb[:, 3:, 3:] = eye / zr + (1.0 / zs - 1.0 / zr) * pp
    return Mb


def _dense_D(n, pairs, dgeom):
    m = pairs.shape[0]
    D = np.zeros((6 * n, m))
    for c in range(m):
        i, j = pairs[c, 0], pairs[c, 1]
        e, ap, aq = dgeom[c, 0:3], dgeom[c, 3:6], dgeom[c, 6:9]
        D[6 * i:6 * i + 3, c] += e
        D[6 * i + 3:6 * i + 6, c] += ap
        D[6 * j:6 * j + 3, c] -= e
        D[6 * j + 3:6 * j + 6, c] -= aq
    return D


def _sparse_D(n, pairs, dgeom):
    """D as a scipy sparse [6n, m] matrix: column c is (e, y_P x e) at rod i
    and (-e, -y_Q x e) at rod j (Appendix Eq. blockdef)."""
    m = pairs.shape[0]
    i = pairs[:, 0].astype(np.int64)
    j = pairs[:, 1].astype(np.int64)
    cols = np.arange(m)
    rows, vals, cc = [], [], []
    for k in range(3):
        rows += [6 * i + k, 6 * i + 3 + k, 6 * j + k, 6 * j + 3 + k]
        vals += [dgeom[:, k], dgeom[:, 3 + k], -dgeom[:, k], -dgeom[:, 6 + k]]
        cc += [cols] * 4
    return sps.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cc))), shape=(6 * n, m))


def _sparse_M(Mb):
    """The block-diagonal mobility as a scipy sparse [6n, 6n] matrix."""
    n = Mb.shape[0]
    return sps.bsr_matrix((Mb, np.arange(n), np.arange(n + 1)), shape=(6 * n, 6 * n)).tocsr()


def solve(quat, pb, pairs, dgeom, q, tol=1e-13):
    """Exact (enumeration) for up to 20 constraints, else FISTA to tol."""
    if pairs.shape[0] == 0:
        return np.zeros(0)
    if pairs.shape[0] <= 20:
        g, _ = solve_enum(quat, pb, pairs, dgeom, q)
        return g
    g, _, _ = solve_apgd(quat, pb, pairs, dgeom, q, tol=tol)
    return g


def forward(x, quat, fnc, pb, pairs=None, gamma=None, sparse=False):
    """One step on a given (or found) pair list: U, x' (unwrapped) and theta'.
    sparse=True keeps D as a scipy sparse matrix (large systems)."""
    x = np.asarray(x, dtype=np.float64)
    quat = np.asarray(quat, dtype=np.float64)
    if pairs is None:
        pairs = find_pairs(x, quat, pb)
    asm = assemble(x, quat, fnc, pb, pairs)
    if gamma is None:
        gamma = solve(quat, pb, pairs, asm["dgeom"], asm["q"])
    n = x.shape[0]
    p = axis(quat)
    zeta = drag(pb.viscosity, pb.length, pb.diameter)
    Mb = _mobility_blocks(p, zeta)
    D = _sparse_D(n, pairs, asm["dgeom"]) if sparse else _dense_D(n, pairs, asm["dgeom"])
    F = np.asarray(fnc, dtype=np.float64).reshape(n, 6) + np.asarray(D @ gamma).reshape(n, 6)
    U = np.einsum("nij,nj->ni", Mb, F)
    h = pb.dt
    xn = x + h * U[:, :3]
    s, v, om = quat[:, 0], quat[:, 1:], U[:, 3:]
    phi = np.empty_like(quat)
    phi[:, 0] = s - 0.5 * h * np.einsum("ni,ni->n", v, om)
    phi[:, 1:] = v + 0.5 * h * (s[:, None] * om - np.cross(v, om))
    qn = phi / np.linalg.norm(phi, axis=1, keepdims=True)
    return {"pairs": pairs, "gamma": gamma, "U": U, "x": xn, "quat": qn, "phi_q": phi, "F": F, "p": p,
            "Mb": Mb, "D": D, "asm": asm, "zeta": zeta}


def centre_loss(xn, targets):
    """The loss of the differentiation workload: sum of squared post-step centre displacements."""
    d = xn - targets
    return float(np.sum(d * d))


def _axis_jacobian(quat):
    """dp/dtheta for p = (2(ac + sb), 2(bc - sa), s^2 - a^2 - b^2 + c^2): [n, 3, 4]."""
    s, a, b, c = quat[:, 0], quat[:, 1], quat[:, 2], quat[:, 3]
    J = np.zeros((quat.shape[0], 3, 4))
    J[:, 0] = np.stack([2 * b, 2 * c, 2 * s, 2 * a], axis=1)
    J[:, 1] = np.stack([-2 * a, -2 * s, 2 * c, 2 * b], axis=1)
    J[:, 2] = np.stack([2 * s, -2 * a, -2 * b, 2 * c], axis=1)
    return J


def _active_multiplier_sparse(D, Msp, uf, act):
    """lambda_A of A_AA lambda_A = b_A, A_AA = D_A^T M D_A, b = D^T M u, by
    MINRES (Paige & Saunders 1975) from zero to a relative residual of
    1e-15: on this consistent symmetric system its iterates stay in the
    range of A_AA, so it returns the minimum-norm solution also when A_AA is
    singular.  (A sparse LU of A_AA gives the same multiplier to about 1e-12
    but takes minutes at 4e4 active constraints.)"""
    b = D.T @ (Msp @ uf)
    DA = D[:, np.flatnonzero(act)]
    AAA = (DA.T @ Msp @ DA).tocsr()
    bA = b[act]
    lam, info = spla.minres(AAA, bA, rtol=1e-15, maxiter=100 * AAA.shape[0] + 100)
    if info != 0 or np.linalg.norm(AAA @ lam - bA) > 1e-10 * max(np.linalg.norm(bA), 1e-300):
        lam = spla.lsqr(AAA, bA, atol=1e-15, btol=1e-15, iter_lim=100 * AAA.shape[0])[0]
    return lam


def step_adjoint(x, quat, fnc, pb, dL_dxn, dL_dqn=None, fw=None, active_tol=0.0):
    """Gradient of L(x', theta') for given dL/dx' [n,3] and dL/dtheta' [n,4]
    (nullable).  Returns dict: x [n,3], quat [n,4] (tangent), eta, fnc [n,6],
    and the intermediates lambda, u.  A forward taken with sparse=True is
    differentiated with sparse matrices throughout (the same formulas)."""
    x = np.asarray(x, dtype=np.float64)
    quat = np.asarray(quat, dtype=np.float64)
    if fw is None:
        fw = forward(x, quat, fnc, pb)
    n = x.shape[0]
    h = pb.dt
    pairs, gamma, U, Fo, p, Mb, D = fw["pairs"], fw["gamma"], fw["U"], fw["F"], fw["p"], fw["Mb"], fw["D"]
    zp, zpar, zr, zs = fw["zeta"]
    gx = np.array(dL_dxn, dtype=np.float64).reshape(n, 3).copy()   # x' = x + h U_t: direct identity
    gq = np.zeros((n, 4))
    u = np.zeros((n, 6))
    u[:, :3] = h * gx
    if dL_dqn is not None:
        g_qn = np.asarray(dL_dqn, dtype=np.float64).reshape(n, 4)
        phi = fw["phi_q"]
        nrm = np.linalg.norm(phi, axis=1, keepdims=True)
        qn = phi / nrm
        g = (g_qn - qn * np.sum(qn * g_qn, axis=1, keepdims=True)) / nrm      # dL/dphi
        s, v, om = quat[:, 0], quat[:, 1:], U[:, 3:]
        g0, gv = g[:, 0], g[:, 1:]
        gq[:, 0] += g0 + 0.5 * h * np.einsum("ni,ni->n", gv, om)
        gq[:, 1:] += gv + 0.5 * h * (-g0[:, None] * om - np.cross(om, gv))
        u[:, 3:] += 0.5 * h * (-g0[:, None] * v + s[:, None] * gv - np.cross(gv, v))
    uf = u.reshape(-1)
    sparse = sps.issparse(D)
    m = pairs.shape[0]
    lam = np.zeros(m)
    if sparse:
        if m > 0:
            act = gamma > active_tol
            if act.any():
                lam[act] = _active_multiplier_sparse(D, _sparse_M(Mb), uf, act)
    else:
        Mfull = np.zeros((6 * n, 6 * n))
        for k in range(n):
            Mfull[6 * k:6 * k + 6, 6 * k:6 * k + 6] = Mb[k]
        if m > 0:
            b = D.T @ (Mfull @ uf)
            act = gamma > active_tol
            if act.any():
                DA = D[:, act]
                AAA = DA.T @ Mfull @ DA
                lam[act] = np.linalg.lstsq(AAA, b[act], rcond=1e-13)[0]
    w = np.asarray(D @ lam).reshape(n, 6)
    a = u - w
    nu = np.einsum("nij,nj->ni", Mb, a)
    # mobility: d/dp of a^T M(p) F_tot, and d/d eta
    ct, cr = 1.0 / zpar - 1.0 / zp, 1.0 / zs - 1.0 / zr
    gp = np.zeros((n, 3))
    for blk, cc in ((slice(0, 3), ct), (slice(3, 6), cr)):
        aa, ff = a[:, blk], Fo[:, blk]
        gp += cc * (np.sum(p * ff, axis=1, keepdims=True) * aa + np.sum(aa * p, axis=1, keepdims=True) * ff)
    geta = -float(np.sum(a * U)) / pb.viscosity
    # geometry of every constraint
    box = np.asarray(pb.box, dtype=np.float64)
    xw = wrap(x, box)
    hl = 0.5 * pb.length
    for c in range(m):
        if gamma[c] == 0.0 and lam[c] == 0.0:
            continue   # every term of this constraint carries gamma_c or lambda_c
        i, j, code = int(pairs[c, 0]), int(pairs[c, 1]), int(pairs[c, 2])
        k = np.array([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1], dtype=np.float64)
        dx = xw[i] - xw[j] - k * box
        pa, pb_ = p[i], p[j]
        rho, s, t = segment_closest(dx, pa, pb_, pb.length)
        r = dx + s * pa - t * pb_
        e = fw["asm"]["dgeom"][c, 0:3]
        yP, yQ = s * pa, t * pb_
        gc, lc = gamma[c], lam[c]
        at = gc * (nu[i, :3] - nu[j, :3]) - lc * (U[i, :3] - U[j, :3])
        aP = gc * nu[i, 3:] - lc * U[i, 3:]
        aQ = gc * nu[j, 3:] - lc * U[j, 3:]
        be = at + np.cross(aP, yP) - np.cross(aQ, yQ)
        bP = np.cross(e, aP)
        bQ = -np.cross(e, aQ)
        kap = (be - e * np.dot(e, be)) / rho if rho > 0 else np.zeros(3)
        # terms at fixed (s, t), and the Phi term
        g_dx = kap - (lc / h) * e
        g_pa = s * (kap + bP) - (lc / h) * s * e
        g_pb = t * (bQ - kap) + (lc / h) * t * e
        # the closest-point parameters' own derivatives
        sig_s = np.dot(kap + bP, pa)
        sig_t = np.dot(bQ - kap, pb_)
        A_ = np.dot(pa, pa); B_ = np.dot(pa, pb_); C_ = np.dot(pb_, pb_)
        det = A_ * C_ - B_ * B_
        s_free = abs(s) < hl
        t_free = abs(t) < hl
        parallel = not (det > 1e-12 * A_ * C_)
        # R1 = dDx.pa + dpa.(s pa + r) - dpb.(t pa);  R2 = dDx.pb + dpa.(s pb) + dpb.(r - t pb)
        R1 = (pa, s * pa + r, -t * pa)
        R2 = (pb_, s * pb_, r - t * pb_)
        if not parallel and s_free and t_free:
            J = np.array([[A_, -B_], [B_, -C_]])
            xi = np.linalg.solve(J.T, np.array([sig_s, sig_t]))
            for blk, (v1, v2) in enumerate(zip(R1, R2)):
                contrib = -(xi[0] * v1 + xi[1] * v2)
                if blk == 0: g_dx = g_dx + contrib
                elif blk == 1: g_pa = g_pa + contrib
                else: g_pb = g_pb + contrib
        elif not parallel and s_free and not t_free:
            # t clamped: A ds + R1 = 0
            for blk, v1 in enumerate(R1):
                contrib = -(sig_s / A_) * v1
                if blk == 0: g_dx = g_dx + contrib
                elif blk == 1: g_pa = g_pa + contrib
                else: g_pb = g_pb + contrib
        elif not parallel and t_free and not s_free:
            # s clamped: -C dt + R2 = 0
            for blk, v2 in enumerate(R2):
                contrib = (sig_t / C_) * v2
                if blk == 0: g_dx = g_dx + contrib
                elif blk == 1: g_pa = g_pa + contrib
                else: g_pb = g_pb + contrib
        gx[i] += g_dx
        gx[j] -= g_dx
        gp[i] += g_pa
        gp[j] += g_pb
    gq += np.einsum("nk,nkq->nq", gp, _axis_jacobian(quat))
    gq = gq - quat * np.sum(quat * gq, axis=1, keepdims=True)
    return {"x": gx, "quat": gq, "eta": geta, "fnc": nu, "lambda": lam, "u": u}


def loss_and_grad(x, quat, fnc, pb, targets, sparse=False, tol=1e-13):
    """The differentiation workload's loss and gradient (oracle); sparse=True
    for large systems (the oracle's own pair list, solve to tol and sparse
    adjoint)."""
    if sparse:
        x = np.asarray(x, dtype=np.float64)
        quat = np.asarray(quat, dtype=np.float64)
        pairs = find_pairs(x, quat, pb)
        asm = assemble(x, quat, fnc, pb, pairs)
        gamma = solve(quat, pb, pairs, asm["dgeom"], asm["q"], tol=tol)
        fw = forward(x, quat, fnc, pb, pairs=pairs, gamma=gamma, sparse=True)
        L = centre_loss(fw["x"], targets)
        g = step_adjoint(x, quat, fnc, pb, 2.0 * (fw["x"] - targets), fw=fw)
        return L, g, fw
    fw = forward(x, quat, fnc, pb)
    L = centre_loss(fw["x"], targets)
    g = step_adjoint(x, quat, fnc, pb, 2.0 * (fw["x"] - targets), fw=fw)
    return L, g, fw
