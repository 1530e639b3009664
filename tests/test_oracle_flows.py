"""Pins of the oracle's walls: mid-link bounce-back (Sec. II, Eq. lbe-bb) with
the moving-wall term C (Eq. c, lbe-bb-corr), against analytic flows.

* Plane Couette flow between walls moving at -U and +U: the steady profile is
  linear between the mid-link wall positions z = 0.5 and z = N - 1.5
  (reading Q10: wall layers at 0 and N-1).  BGK with half-way bounce-back
  holds the linear profile exactly, so the check is to 1e-9.
* Body-force Poiseuille flow at rest walls: u = g z'(H - z') / (2 nu) with
  nu = (2 tau - 1) / 6 (Sec. II); within 1e-2 at H = 30 and converging at
  second order in H.
* Total mass is conserved to round-off with tangentially moving walls (the
  C terms of the two tangential links of a node cancel); over long runs the
  bound is a few ulp per step.
"""
import numpy as np
import pytest

import oracle
from paper_1005_2594_gb300 import workloads


def _channel(nz, U=0.0, g=0.0, tau=1.0):
    p = workloads.base_params(2, 2, nz, periodic=(1, 1, 0), g=(g, 0.0, 0.0),
                              wall_vel={4: (-U, 0.0, 0.0), 5: (U, 0.0, 0.0)})
    p["tau"] = tau
    return oracle.Oracle(p)


def _profile(o, nz):
    _, u, owner = o.fields()
    u = u.reshape(nz, 2, 2, 3)
    return u[1:nz - 1, 0, 0, :]


def test_couette_linear_profile_exact():
    nz, U = 32, 0.02
    o = _channel(nz, U=U)
    m0, _ = o.totals()
    o.step(16000)
    ux = _profile(o, nz)
    H = nz - 2
    zp = np.arange(1, nz - 1) - 0.5
    exact = -U + 2.0 * U * zp / H
    assert np.max(np.abs(ux[:, 0] - exact)) < 1e-9 * U
    assert np.max(np.abs(ux[:, 1:])) < 1e-12
    m1, _ = o.totals()
    # no systematic change: only round-off, a few ulp per step
    assert abs(m1 - m0) / m0 < 16000 * 4e-16


@pytest.mark.parametrize("tau", [1.0])
def test_poiseuille_second_order(tau):
    g = 1e-5
    errs = []
    for nz in (16, 32):
        o = _channel(nz, g=g, tau=tau)
        H = nz - 2
        nu = (2 * tau - 1) / 6.0
        o.step(int(12 * H * H / (np.pi ** 2 * nu)) + 500)
        ux = _profile(o, nz)[:, 0]
        zp = np.arange(1, nz - 1) - 0.5
        exact = g * zp * (H - zp) / (2 * nu)
        errs.append(np.max(np.abs(ux - exact)) / np.max(exact))
    assert errs[1] < 1e-2, errs
    order = np.log(errs[0] / errs[1]) / np.log(30.0 / 14.0)
    assert order > 1.7, (errs, order)


def test_mass_conserved_with_moving_walls():
    p = workloads.base_params(8, 6, 10, periodic=(1, 1, 0),
                              wall_vel={4: (-0.03, 0.01, 0.0), 5: (0.02, -0.02, 0.0)})
    o = oracle.Oracle(p)
    rng = np.random.default_rng(5)
    pop = o.populations()
    fluid = o.owner() == -1
    base = oracle.equilibrium(1.0, [0.0, 0.0, 0.0])
    pop[fluid] = base * (1.0 + rng.uniform(-0.02, 0.02, (fluid.sum(), 19)))
    o.set_populations(pop)
    m0, _ = o.totals()
    o.step(50)
    m1, _ = o.totals()
    assert abs(m1 - m0) / m0 < 1e-13
