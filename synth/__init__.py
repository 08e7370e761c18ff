"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only workload descriptions (mesh sizes, partitions, physical
parameters from Table 1 of the paper) and the seeded random draws.  It holds
none of the method's arithmetic: no assembly, no ionic model, no solver.  Both
the CPU oracle and the CUDA path receive the arrays it produces as inputs.

Workloads (all Q1 hexahedral slabs, h = element size):

* ``tiny``     2x2x2 elements, one element per subdomain: edge cases.
* ``ragged``   10x9x7 elements, 4^3-element blocks with ragged last blocks.
* ``cube8``    8x8x8 elements of a 0.4 cm cube, 2x2x2 subdomains, H/h = 4,
               vertex primal space (1,458 unknowns).
* ``slab32``   32x32x16 elements of a 1.6x1.6x0.8 cm slab, 4x4x2 subdomains,
               H/h = 8, vertex + edge-average primal space (37,026 unknowns).
* ``opt<k>``   (4k)^3 elements of a 0.8 cm cube, 4x4x4 subdomains, H/h = k.
* ``slab128``  128x128x32 elements of a 3.2x3.2x0.8 cm slab, 16x16x4
               subdomains, H/h = 8 (1,098,306 unknowns).
* ``coarse2k`` 32x32x4 elements of a 0.8x0.8x0.1 cm slab (h = 0.025 cm), 2^3-element
               subdomains (16x16x2 = 512), V+E: 2,310 coarse unknowns on 5,445 nodes, so
               the oracle's direct solve stays cheap.
* ``ell8``     8x8x8 isoparametric elements of the truncated ellipsoid of
               Section 6 (phi in [-pi/2, 0], theta in [-3pi/8, pi/8], the wall
               r in [0, 1]), 2x2x2 subdomains, V+E primal space.
* ``ell10``    10x9x6 elements of the same ellipsoid, 4^3-element blocks with
               ragged last blocks.
* ``ell32``    32x32x16 elements of the same ellipsoid, 4x4x2 subdomains, H/h = 8.
* ``shell_small`` / ``shell``  the uneven batch: the lower half (z <= 0) of an ellipsoidal
               shell (inner semi-axes 2.0, 2.0, 5.0 cm, outer 2.8, 2.8, 5.8 cm) meshed by a
               box grid of Q1 elements of size h with the elements whose centroid lies
               outside the shell masked, split into blocks of s^3 elements whose
               connected pieces are the subdomains (uneven in size).  ``shell``: h =
               0.045 cm, 12^3-element blocks (about 1.2 M unknowns, the uneven-batch
               configuration); ``shell_small``: h = 0.35 cm, 4^3-element blocks, for the
               oracle.  Stimulus: the apex of the wall.
* ``beat_slab`` / ``beat_ell``  the whole-beat runs of Test 4: 192x96x24 elements,
               8x8x2 subdomains (8,450 dofs each), 2,400 / 3,400 steps;
               ``beat_*_half`` halve each mesh direction; ``beat_mini`` is a
               0.2x0.2x0.05 cm slab at h = 0.0125 cm (2,890 unknowns) for a
               whole beat the oracle can follow.

The ellipsoid's axes are not printed in the paper: a1 = b1 = 1.5, a2 = b2 =
2.7, c1 = 4.4, c2 = 5.0 cm (a 1.2 cm wall, an idealised left ventricle) are
taken.  Its stimulus is the endocardial surface r = 0 (Section 6).
"""
from __future__ import annotations

import numpy as np

# Table 1: conductivities (S/cm) along fibre, cross-fibre, sheet normal.
SIGMA_I = (3.0e-3, 3.1525e-4, 3.1525e-5)
SIGMA_E = (2.0e-3, 1.3514e-3, 6.757e-4)
# Table 1: Rogers-McCulloch parameters; chi*Cm in mF/cm^3 (Fig. 1 caption).
IONIC = dict(G=1.2, eta1=4.4, eta2=0.012, vth=13.0, vp=100.0, chi_cm=1.0, v_rest=-85.0)
TAU = 0.05  # ms
# Section 6: 100 mA/cm^3 for 1 ms in a slab corner (here a 0.1 cm corner cube).
STIMULUS = dict(amp=100.0, t_on=0.0, t_off=1.0, box=(0.0, 0.1, 0.0, 0.1, 0.0, 0.1))

# Section 6 (Test 4): the portion of ellipsoid; axes a1, a2, b1, b2, c1, c2 in cm.
ELLIPSOID = dict(axes=(1.5, 2.7, 1.5, 2.7, 4.4, 5.0), phi=(-np.pi / 2, 0.0), theta=(-3 * np.pi / 8, np.pi / 8))
# Section 6: on the ellipsoid the endocardium (r = 0) is stimulated; the box is
# in the parametric coordinates (phi, theta, r).
STIMULUS_ELLIPSOID = dict(amp=100.0, t_on=0.0, t_off=1.0,
                          box=(-np.pi / 2, 0.0, -3 * np.pi / 8, np.pi / 8, 0.0, 0.0))

# the masked shell: inner and outer semi-axes (cm) of the lower half of an ellipsoidal wall
SHELL = dict(inner=(2.0, 2.0, 5.0), outer=(2.8, 2.8, 5.8))
# its stimulus: the apex of the wall (box-grid coordinates; the grid's origin is the
# corner (-2.8, -2.8, -5.8) of the shell's bounding box)
STIMULUS_SHELL = dict(amp=100.0, t_on=0.0, t_off=1.0, box=(2.45, 3.15, 2.45, 3.15, 0.0, 0.35))

WORKLOADS = {
    "tiny": dict(n=(2, 2, 2), l=(0.1, 0.1, 0.1), s=(1, 1, 1), primal="V", steps=1),
    "ragged": dict(n=(10, 9, 7), l=(0.5, 0.45, 0.35), s=(4, 4, 4), primal="VE", steps=2),
    "cube8": dict(n=(8, 8, 8), l=(0.4, 0.4, 0.4), s=(4, 4, 4), primal="V", steps=1),
    "cube8ve": dict(n=(8, 8, 8), l=(0.4, 0.4, 0.4), s=(4, 4, 4), primal="VE", steps=1),
    "cube8vef": dict(n=(8, 8, 8), l=(0.4, 0.4, 0.4), s=(4, 4, 4), primal="VEF", steps=1),
    "slab32": dict(n=(32, 32, 16), l=(1.6, 1.6, 0.8), s=(8, 8, 8), primal="VE", steps=20),
    "slab128": dict(n=(128, 128, 32), l=(3.2, 3.2, 0.8), s=(8, 8, 8), primal="VE", steps=400),
    "coarse2k": dict(n=(32, 32, 4), l=(0.8, 0.8, 0.1), s=(2, 2, 2), primal="VE", steps=2),
}
for _name, _n, _s in (("ell8", (8, 8, 8), (4, 4, 4)), ("ell10", (10, 9, 6), (4, 4, 4)),
                      ("ell32", (32, 32, 16), (8, 8, 8))):
    WORKLOADS[_name] = dict(n=_n, ellipsoid=ELLIPSOID, s=_s, primal="VE", steps=2)
# Section 6, Test 4 (Table 11): a whole beat on 8x8x2 subdomains of a 192x96x24 mesh
# (8,450 dofs per subdomain), the slab for 2,400 steps and the ellipsoid for 3,400;
# the *_half variants halve every mesh direction (1,274 dofs per subdomain).
WORKLOADS["beat_slab"] = dict(n=(192, 96, 24), l=(1.92, 1.92, 0.48), s=(24, 12, 12), primal="VE", steps=2400)
WORKLOADS["beat_ell"] = dict(n=(192, 96, 24), ellipsoid=ELLIPSOID, s=(24, 12, 12), primal="VE", steps=3400)
# a whole beat small enough for the oracle: h = 0.0125 cm (at h = 0.05 cm, as in cube8,
# the front from the corner stimulus does not propagate), 2x2x2 subdomains
WORKLOADS["beat_mini"] = dict(n=(16, 16, 4), l=(0.2, 0.2, 0.05), s=(8, 8, 2), primal="VE", steps=2400)
WORKLOADS["beat_slab_half"] = dict(n=(96, 48, 12), l=(1.92, 1.92, 0.48), s=(12, 6, 6), primal="VE", steps=2400)
WORKLOADS["beat_ell_half"] = dict(n=(96, 48, 12), ellipsoid=ELLIPSOID, s=(12, 6, 6), primal="VE", steps=3400)
for _k in (4, 8, 12, 16, 20):
    WORKLOADS[f"opt{_k}"] = dict(n=(4 * _k,) * 3, l=(0.8, 0.8, 0.8), s=(_k,) * 3,
                                 primal="VE", steps=40)


for _name, _h, _s in (("shell_small", 0.35, 4), ("shell", 0.045, 12)):
    _n = (int(np.ceil(5.6 / _h - 1e-9)), int(np.ceil(5.6 / _h - 1e-9)), int(np.ceil(5.8 / _h - 1e-9)))
    WORKLOADS[_name] = dict(n=_n, l=tuple(_h * v for v in _n), s=(_s, _s, _s), primal="VE", shell=SHELL,
                            steps=50)


def shell_mask(n, l, shell):
    """1 for the elements whose centroid lies in the lower half (z <= 0) of the wall between
    the inner and the outer ellipsoid, in the grid's element order (x fastest); the grid's
    origin is the corner (-a_out, -b_out, -c_out) of the shell's bounding box."""
    (ai, bi, ci), (ao, bo, co) = shell["inner"], shell["outer"]
    h = [l[d] / n[d] for d in range(3)]
    ex, ey, ez = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    x = (ex.ravel(order="F") + 0.5) * h[0] - ao
    y = (ey.ravel(order="F") + 0.5) * h[1] - bo
    z = (ez.ravel(order="F") + 0.5) * h[2] - co
    r_in = (x / ai) ** 2 + (y / bi) ** 2 + (z / ci) ** 2
    r_out = (x / ao) ** 2 + (y / bo) ** 2 + (z / co) ** 2
    return ((z <= 0.0) & (r_in >= 1.0) & (r_out <= 1.0)).astype(np.uint8)


def workload(name: str) -> dict:
    """Return a copy of a named workload description (with its element mask, if any)."""
    w = dict(WORKLOADS[name])
    w["name"] = name
    if "shell" in w:
        w["mask"] = shell_mask(w["n"], w["l"], w["shell"])
    return w


def stimulus(w: dict) -> dict:
    """The stimulus of a workload: a corner box of a slab, the endocardium of the ellipsoid,
    the apex of the masked shell."""
    if "shell" in w:
        return dict(STIMULUS_SHELL)
    return dict(STIMULUS_ELLIPSOID if "ellipsoid" in w else STIMULUS)


def n_nodes(w: dict) -> int:
    nx, ny, nz = w["n"]
    return (nx + 1) * (ny + 1) * (nz + 1)


def initial_state(n: int, seed: int = 0, sigma_mv: float = 1.0):
    """Resting state plus seeded noise: V0 ~ N(0, sigma) mV, u_e = 0, w = 0.

    Returns (u_i, u_e, w) as float64 arrays of length n, with u_i = V0 so that
    the transmembrane potential u_i - u_e equals V0.
    """
    rng = np.random.default_rng(seed)
    v0 = rng.normal(0.0, sigma_mv, size=n)
    return v0.astype(np.float64), np.zeros(n), np.zeros(n)


def random_vector(n: int, seed: int) -> np.ndarray:
    """A seeded N(0,1) float64 vector (right-hand sides for operator tests)."""
    return np.random.default_rng(seed).standard_normal(n)
