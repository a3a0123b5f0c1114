"""Seeded synthetic rod suspensions (inputs only).

This module draws random inputs for the collision-constraint step: rod
centres, orientations (as unit quaternions) and the non-constraint forces
F_nc = F_B + F_E (Appendix "Filament dynamics", Eq. for U = M F with
F = F_C + F_L + F_B + F_E).  It holds none of the step's arithmetic: no
rod-rod distance, no constraint matrix, no mobility application, no solve
and no update.  Both the CPU oracle tests and the CUDA path draw their inputs
from here, so the two sides see identical data.

Every generator uses numpy's PCG64 (``numpy.random.default_rng(seed)``).
Orientations are drawn as unit axis vectors and turned into the quaternion
of the shortest rotation taking e_z to that axis; the method's own
quaternion-to-axis map lives in the oracle and in the CUDA kernels.

Workloads (the paper gives no dataset; these stand in for the shapes of its
bundle, polarity-sorting and aster runs: rods with L/D = 10, tens to hundreds
of thousands of filaments in periodic boxes, isotropic or nematic):

  ``n1000_box40``    1,000 rods, D=1, L=10, periodic cube of side 40,
                     isotropic, F and T ~ N(0, 1) per component.
  ``n100k_phi010``   100,000 rods, volume fraction 0.10 (box 203.1),
                     isotropic, thermal forces plus 50,000 Hookean
                     crosslinker springs (k=10, rest length 1.5) between
                     random rod pairs with centre distance < L.
  ``n400k_nematic``  400,000 rods, volume fraction 0.25 (box 237.5),
                     axes ~ (0.1 xi1, 0.1 xi2, 1) normalised, thermal forces.
  ``n20k_phi015``    20,000 rods, volume fraction 0.15 (box 103.8),
                     isotropic, thermal forces (the differentiation
                     workload; ``loss_targets`` draws its loss targets).
  ``ensemble256``    256 independent systems, rod counts log-uniform in
                     [500, 20000], lengths log-uniform in [5, 20], volume
                     fraction uniform in [0.05, 0.20], axes nematic about
                     a random director per system (spread 0.1 rad),
                     thermal forces.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "RodSystem", "rod_volume", "box_for_fraction", "unit_axes_isotropic",
    "unit_axes_nematic", "quat_from_axis", "thermal_forces", "spring_forces",
    "random_system", "workload", "WORKLOADS", "tiny_system",
]


@dataclass
class RodSystem:
    """One periodic rod suspension plus the parameters of one step."""
    x: np.ndarray            # [n, 3] float64 centres in [0, box)
    quat: np.ndarray         # [n, 4] float64 unit quaternions (s, v1, v2, v3)
    f_nc: np.ndarray         # [n, 6] float64 force (3) then torque (3), lab frame
    box: tuple               # periodic edge lengths
    diameter: float = 1.0
    length: float = 10.0
    viscosity: float = 1.0
    dt: float = 1e-3
    delta_c: float = 1.0
    tol: float = 1e-8
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def rod_volume(diameter: float, length: float) -> float:
    """Volume of a spherocylinder: cylinder of length L plus two hemispherical caps."""
    return math.pi / 4.0 * diameter ** 2 * length + math.pi / 6.0 * diameter ** 3


def box_for_fraction(n: int, diameter: float, length: float, phi: float) -> float:
    """Edge of the periodic cube that holds n rods at volume fraction phi."""
    return (n * rod_volume(diameter, length) / phi) ** (1.0 / 3.0)


def unit_axes_isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Axes uniform on the unit sphere: normalised standard Gaussian vectors."""
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def unit_axes_nematic(rng: np.random.Generator, n: int, spread: float = 0.1, director=None) -> np.ndarray:
    """Axes about +z with a Gaussian angular spread: (spread*xi1, spread*xi2, 1)
    normalised; then, if a unit ``director`` is given, turned by the rotation
    taking e_z onto it (Rodrigues' formula about e_z x director)."""
    v = np.empty((n, 3))
    v[:, 0:2] = spread * rng.standard_normal((n, 2))
    v[:, 2] = 1.0
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    if director is not None:
        d = np.asarray(director, dtype=np.float64)
        d = d / np.linalg.norm(d)
        k = np.array([-d[1], d[0], 0.0])      # e_z x d
        sn, cs = np.linalg.norm(k), d[2]
        if sn > 1e-12:
            k /= sn
            kv = np.cross(k, v)
            v = v * cs + kv * sn + np.outer(v @ k, k) * (1.0 - cs)
        elif cs < 0:
            v = -v
        v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def quat_from_axis(axis: np.ndarray) -> np.ndarray:
    """Unit quaternion (s, v) of the shortest rotation taking e_z onto each axis.

    The rotation about e_z x a by the angle between e_z and a is
    normalise([1 + a_z, -a_y, a_x, 0]); axes within 1e-12 of -e_z get a half
    turn about e_x, [0, 1, 0, 0].
    """
    a = np.asarray(axis, dtype=np.float64)
    q = np.empty((a.shape[0], 4))
    q[:, 0] = 1.0 + a[:, 2]
    q[:, 1] = -a[:, 1]
    q[:, 2] = a[:, 0]
    q[:, 3] = 0.0
    flip = q[:, 0] < 1e-12
    q[flip] = np.array([0.0, 1.0, 0.0, 0.0])
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _thermal_scales(diameter: float, length: float, viscosity: float, dt: float, kT: float):
    """Standard deviations of the thermal force and torque components.

    The paper names the Brownian force F_B but gives no formula for it.  The
    workload uses an isotropic Gaussian force with variance 2 kT zeta / dt per
    component, zeta being the slender-body drag 4 pi eta L / ln(2L/D) that the
    paper quotes (Section "Filament dynamics"), and a torque with variance
    2 kT zeta L^2/12 / dt.  These only set the size of the random input
    forces.
    """
    zeta = 4.0 * math.pi * viscosity * length / math.log(2.0 * length / diameter)
    sig_f = math.sqrt(2.0 * kT * zeta / dt)
    sig_t = math.sqrt(2.0 * kT * zeta * length ** 2 / 12.0 / dt)
    return sig_f, sig_t


def thermal_forces(rng: np.random.Generator, n: int, diameter: float, length: float,
                   viscosity: float, dt: float, kT: float = 1.0) -> np.ndarray:
    """[n, 6] Gaussian thermal force and torque (see ``_thermal_scales``)."""
    sig_f, sig_t = _thermal_scales(diameter, length, viscosity, dt, kT)
    f = np.empty((n, 6))
    f[:, 0:3] = sig_f * rng.standard_normal((n, 3))
    f[:, 3:6] = sig_t * rng.standard_normal((n, 3))
    return f


def spring_forces(rng: np.random.Generator, x: np.ndarray, axis: np.ndarray, box, length: float,
                  n_springs: int, k: float = 10.0, rest: float = 1.5) -> tuple[np.ndarray, dict]:
    """Explicit Hookean crosslinker forces between random near-neighbour rod pairs.

    Pairs are drawn uniformly from all rod pairs whose centres (minimum image)
    lie closer than L.  Each spring attaches at arclengths uniform in
    [-L/2, L/2] on its two rods; with a and b the attachment points,
    l = |b - a| and u = (b - a)/l, rod i gets force k (l - l0) u and torque
    (s_a axis_i) x that force; rod j gets the opposite force and
    (s_b axis_j) x (-force).  The forces are evaluated once, at the initial
    configuration, and enter the step as part of F_nc.
    """
    from scipy.spatial import cKDTree  # input preparation only

    n = x.shape[0]
    boxa = np.asarray(box, dtype=np.float64)
    tree = cKDTree(x, boxsize=boxa)
    cand = tree.query_pairs(r=length, output_type="ndarray")
    cand = cand[np.lexsort((cand[:, 1], cand[:, 0]))]
    pick = rng.choice(cand.shape[0], size=min(n_springs, cand.shape[0]), replace=False)
    pick.sort()
    ij = cand[pick]
    i, j = ij[:, 0], ij[:, 1]
    sa = rng.uniform(-length / 2, length / 2, size=ij.shape[0])
    sb = rng.uniform(-length / 2, length / 2, size=ij.shape[0])
    dxc = x[j] - x[i]
    dxc -= boxa * np.round(dxc / boxa)
    a = sa[:, None] * axis[i]
    b = dxc + sb[:, None] * axis[j]
    d = b - a
    ell = np.linalg.norm(d, axis=1)
    u = d / ell[:, None]
    fi = (k * (ell - rest))[:, None] * u
    f = np.zeros((n, 6))
    np.add.at(f[:, 0:3], i, fi)
    np.add.at(f[:, 0:3], j, -fi)
    np.add.at(f[:, 3:6], i, np.cross(sa[:, None] * axis[i], fi))
    np.add.at(f[:, 3:6], j, np.cross(sb[:, None] * axis[j], -fi))
    return f, {"springs": int(ij.shape[0]), "spring_candidates": int(cand.shape[0])}


def random_system(seed: int, n: int, box, *, length: float = 10.0, diameter: float = 1.0,
                  nematic_spread: float | None = None, director=None, forces: str = "unit",
                  n_springs: int = 0, viscosity: float = 1.0, dt: float = 1e-3,
                  delta_c: float | None = None, tol: float = 1e-8, name: str = "") -> RodSystem:
    """Uniform centres in [0, box)^3 and isotropic (or nematic) axes.

    ``forces``: "unit" draws F and T ~ N(0, 1) per component, "thermal" uses
    ``thermal_forces``, "none" gives zero forces.  ``n_springs`` > 0 adds
    ``spring_forces``.  Initial overlaps are allowed (no rejection).
    """
    rng = np.random.default_rng(seed)
    boxt = tuple(float(b) for b in (box if np.ndim(box) else (box, box, box)))
    x = rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(boxt)
    x = np.where(x >= np.asarray(boxt), 0.0, x)
    axis = (unit_axes_isotropic(rng, n) if nematic_spread is None
            else unit_axes_nematic(rng, n, nematic_spread, director))
    quat = quat_from_axis(axis)
    if forces == "unit":
        f = rng.standard_normal((n, 6))
    elif forces == "thermal":
        f = thermal_forces(rng, n, diameter, length, viscosity, dt)
    elif forces == "none":
        f = np.zeros((n, 6))
    else:
        raise ValueError(forces)
    meta = {"seed": seed}
    if n_springs > 0:
        fs, m = spring_forces(rng, x, axis, boxt, length, n_springs)
        f = f + fs
        meta.update(m)
    return RodSystem(x=x, quat=quat, f_nc=np.ascontiguousarray(f), box=boxt, diameter=diameter,
                     length=length, viscosity=viscosity, dt=dt,
                     delta_c=diameter if delta_c is None else delta_c, tol=tol, name=name, meta=meta)


def _n1000(seed=1):
    return random_system(seed, 1000, 40.0, forces="unit", tol=1e-8, name="n1000_box40")


def _n100k(seed=2, n=100_000, n_springs=50_000):
    box = box_for_fraction(n, 1.0, 10.0, 0.10)
    return random_system(seed, n, box, forces="thermal", n_springs=n_springs, tol=1e-6,
                         name="n100k_phi010")


def _n400k(seed=3, n=400_000):
    box = box_for_fraction(n, 1.0, 10.0, 0.25)
    return random_system(seed, n, box, forces="thermal", nematic_spread=0.1, tol=1e-5,
                         name="n400k_nematic")


def _n20k(seed=5, n=20_000):
    box = box_for_fraction(n, 1.0, 10.0, 0.15)
    return random_system(seed, n, box, forces="thermal", tol=1e-6, name="n20k_phi015")


WORKLOADS = {
    "n1000_box40": _n1000,
    "n100k_phi010": _n100k,
    "n400k_nematic": _n400k,
    "n20k_phi015": _n20k,
}


def workload(name: str, **kw) -> RodSystem:
    """Build a named workload (see the module docstring)."""
    return WORKLOADS[name](**kw)


ENSEMBLE_SPREAD = 0.1   # angular spread (rad) of every ensemble system about its director


def ensemble_specs(seed: int = 1000, count: int = 256):
    """Per-system (n, length, phi, seed, director) of the batched ensemble."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(math.log(500), math.log(20000), size=count)).astype(np.int64)
    length = np.exp(rng.uniform(math.log(5.0), math.log(20.0), size=count))
    phi = rng.uniform(0.05, 0.20, size=count)
    director = unit_axes_isotropic(rng, count)
    return [(int(n[s]), float(length[s]), float(phi[s]), seed + s, director[s]) for s in range(count)]


def ensemble(seed: int = 1000, count: int = 256, scale: float = 1.0) -> list[RodSystem]:
    """The batched ensemble: independent periodic systems of uneven size,
    each a nematic domain about its own random director (spread
    ENSEMBLE_SPREAD), uniform centres and thermal forces.

    ``scale`` < 1 shrinks every rod count (for quick tests); lengths and
    volume fractions are kept (boxes never below L + 2 D).
    """
    out = []
    for n, length, phi, s, director in ensemble_specs(seed, count):
        n_s = max(2, int(round(n * scale)))
        box = box_for_fraction(n_s, 1.0, length, phi)
        box = max(box, length + 2.0 + 1e-6)
        out.append(random_system(s, n_s, box, length=length, nematic_spread=ENSEMBLE_SPREAD, director=director,
                                 forces="thermal", tol=1e-5, name=f"ensemble_{s}"))
    return out


def spring_set(s: RodSystem, count: int, seed: int = 21, kappa: float = 10.0, rest: float = 1.5) -> dict:
    """Bilateral crosslinker springs for a system: ``count`` rod pairs drawn
    uniformly among the pairs whose centres (minimum image) lie closer than
    L, attachment arclengths uniform in [-L/2, L/2], stiffness ``kappa`` and
    rest length ``rest``.  Returns ends [nb, 2] int32 (i < j), arms [nb, 2],
    kappa [nb], rest [nb]."""
    from scipy.spatial import cKDTree  # input preparation only

    rng = np.random.default_rng(seed)
    boxa = np.asarray(s.box, dtype=np.float64)
    cand = cKDTree(s.x, boxsize=boxa).query_pairs(r=s.length, output_type="ndarray")
    cand = cand[np.lexsort((cand[:, 1], cand[:, 0]))]
    pick = np.sort(rng.choice(cand.shape[0], size=min(count, cand.shape[0]), replace=False))
    ends = np.ascontiguousarray(cand[pick], dtype=np.int32)
    arms = rng.uniform(-s.length / 2, s.length / 2, size=(ends.shape[0], 2))
    nb = ends.shape[0]
    return {"ends": ends, "arms": arms, "kappa": np.full(nb, float(kappa)), "rest": np.full(nb, float(rest))}


def loss_targets(s: RodSystem, seed: int = 11, sigma: float = 0.01) -> np.ndarray:
    """Seeded targets of the differentiation workload's loss: the initial
    centres displaced by N(0, sigma^2) per component."""
    rng = np.random.default_rng(seed)
    return s.x + sigma * rng.standard_normal(s.x.shape)


def batch_arrays(systems: list[RodSystem]):
    """Concatenated inputs of a batch: (rod_offset [S+1], x, quat, f_nc, [(box, length)] * S)."""
    off = np.zeros(len(systems) + 1, dtype=np.int64)
    off[1:] = np.cumsum([s.n for s in systems])
    cat = lambda name, w: (np.concatenate([getattr(s, name) for s in systems]) if off[-1] > 0
                           else np.zeros((0, w)))
    return (off, np.ascontiguousarray(cat("x", 3)), np.ascontiguousarray(cat("quat", 4)),
            np.ascontiguousarray(cat("f_nc", 6)), [(s.box, s.length) for s in systems])


def tiny_system(seed: int, n: int, box: float = 14.0, length: float = 3.0, forces: str = "unit",
                dt: float = 1e-3, nematic_spread: float | None = None) -> RodSystem:
    """A small random system for brute-force and active-set checks."""
    return random_system(seed, n, box, length=length, forces=forces, dt=dt,
                         nematic_spread=nematic_spread, tol=1e-10, name=f"tiny_{seed}_{n}")
