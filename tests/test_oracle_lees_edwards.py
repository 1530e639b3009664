"""The oracle's Lees-Edwards shear (Sec. IV, reading Q25) against what the
mathematics fixes (CPU).

The box is periodic along x, but its images along x slide past each other in
z: the image above moves with velocity offset U and is displaced by U t.  A
population crossing the plane between x = nx-1 and x = 0 comes from the
neighbouring image: from a point a distance U t along z from its periodic
source (linear interpolation between two nodes), with its equilibrium part
moved by -+U.  The pins:

* U = 0 is the plain periodic box, bit for bit;
* start-up Couette flow settles to the exact linear profile of slope U / nx,
  continuous across the plane, and the momentum moved across the plane per
  step, Delta p_LE of Eq. (mu), gives the plasma's viscosity rho nu, at
  tau = 1 (1/6) and tau = 0.8 (1/10);
* a transverse shear wave (Kelvin mode) on that flow, whose phase fronts tilt
  and cross the plane at the image's offset, follows its exact solution --
  with the offset's sign flipped the error is ~45 times larger;
* the interpolation and the Galilean shift conserve mass;
* a cell closer than the reflection distance to the plane and moving toward
  it has its normal velocity negated, and never covers a node next to it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1005_2594_gb300 import workloads


def _eq(u):
    f = np.zeros(19)
    oracle.lib().orc_equilibrium(1.0, oracle._dp(np.asarray(u, dtype=np.float64)), oracle._dp(f))
    return f


def test_zero_offset_is_the_periodic_box():
    p = workloads.base_params(8, 6, 10, periodic=(1, 1, 1), g=(1e-5, 2e-5, 0.0))
    rng = np.random.default_rng(0)
    a, b = oracle.Oracle(p), oracle.Oracle(p)
    pop = a.populations() * (1 + 0.01 * rng.standard_normal((a.N, 19)))
    a.set_populations(pop)
    b.set_populations(pop)
    b.set_lees_edwards(0.0)
    a.step(20)
    b.step(20)
    np.testing.assert_array_equal(a.populations(), b.populations())
    assert b.lees_edwards()["steps"] == 20


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_couette_startup_is_exact_and_gives_the_plasma_viscosity(tau):
    nx, ny, nz, U = 16, 2, 4, 0.01
    p = workloads.base_params(nx, ny, nz, periodic=(1, 1, 1))
    p["tau"] = tau
    o = oracle.Oracle(p)
    o.set_lees_edwards(U)
    m0, _ = o.totals()
    o.step(2000)
    _, u, _ = o.fields()
    uz = u[:, 2].reshape(nz, ny, nx).mean(axis=(0, 1))
    x = np.arange(nx)
    slope, icpt = np.polyfit(x, uz, 1)
    assert abs(slope / (U / nx) - 1) < 1e-9
    assert np.abs(uz - (slope * x + icpt)).max() < 1e-12
    # continuous across the plane: x = nx continues as x = 0 of the image above
    assert abs(uz[-1] + slope - (uz[0] + U)) < 1e-12
    # Eq. (mu): mu_app = -Delta p_LE / (l_y l_z gamma_dot) = rho nu, nu = (tau - 1/2) / 3
    le = o.lees_edwards()
    assert abs(-le["P"] / (ny * nz * slope) - (tau - 0.5) / 3.0) < 1e-9
    m1, _ = o.totals()
    assert abs(m1 - m0) < 1e-12 * m0


def test_kelvin_mode_crosses_the_sheared_plane():
    """u_y is advected by v_z = gd (x - x0) as a passive field (continuity
    holds for any u_y(x, z)): u_y = A(t) sin(k (z - gd (x - x0) t)) with
    A(t) = A exp(-nu k^2 (t + gd^2 t^3 / 3))"""
    nx, ny, nz, U = 32, 2, 32, 0.032
    gd, x0, A, k = U / nx, (nx - 1) / 2.0, 1e-3, 2 * math.pi / nz
    p = workloads.base_params(nx, ny, nz, periodic=(1, 1, 1))
    o = oracle.Oracle(p)
    z, _, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, z = x.reshape(-1), z.reshape(-1)
    o.set_populations(np.array([_eq((0.0, A * math.sin(k * zi), gd * (xi - x0))) for xi, zi in zip(x, z)]))
    o.set_lees_edwards(U)
    T = 150
    o.step(T)
    _, u, _ = o.fields()
    exact = A * np.exp(-(1.0 / 6.0) * k * k * (T + gd * gd * T ** 3 / 3)) * np.sin(k * (z - gd * (x - x0) * T))
    assert np.abs(exact).max() > 0.3 * A  # the wave is still there, tilted by gd T nx / nz = 0.15 periods
    assert np.abs(u[:, 1] - exact).max() < 2e-2 * A


def test_interpolation_and_shift_conserve_mass():
    p = workloads.base_params(12, 4, 9, periodic=(1, 1, 1), g=(0.0, 0.0, 1e-5))
    rng = np.random.default_rng(1)
    o = oracle.Oracle(p)
    o.set_populations(o.populations() * (1 + 0.02 * rng.standard_normal((o.N, 19))))
    o.set_lees_edwards(0.0371)  # the offset passes between nodes every step
    m0, _ = o.totals()
    o.step(200)
    m1, _ = o.totals()
    assert abs(m1 - m0) < 1e-12 * m0
    assert o.lees_edwards()["bad"] == 0


@pytest.mark.parametrize("side", [0, 1])
def test_cell_reflects_at_the_sheared_plane(side):
    nx = 40
    p = workloads.base_params(nx, 20, 20, periodic=(1, 1, 1), R=(3.0, 1.5), sigma=(3.3, 1.6))
    p["rho_p"] = 20.0  # heavy enough to reach the plane through resting fluid
    o = oracle.Oracle(p)
    o.set_lees_edwards(0.01)
    dr = max(p["sig_perp"], max(p["R_perp"], p["R_par"]) + 1.0)
    v = 0.05
    x = dr + 0.5 - 0.5 if side == 0 else nx - 0.5 - dr - 0.5  # half a node outside dr
    o.set_particles([[x, 9.7, 10.2]], [[1.0, 0.0, 0.0, 0.0]], V=[[-v if side == 0 else v, 0.0, 0.0]])
    toward = -1.0 if side == 0 else 1.0
    flipped = None
    for s in range(40):
        X0 = o.particles()["X"][0, 0]
        o.step(1)
        pt = o.particles()
        own = o.owner().reshape(20, 20, nx)
        assert (own[:, :, 0] == -1).all() and (own[:, :, nx - 1] == -1).all()
        if flipped is None and pt["V"][0, 0] * toward < 0:
            flipped = s
            dist = X0 + 0.5 if side == 0 else nx - 0.5 - X0
            assert dr - 0.05 < dist < dr  # at the first step inside
            break
        # outside the distance the fluid only brakes the cell
        assert pt["V"][0, 0] * toward > 0.03
    assert flipped is not None and o.lees_edwards()["reflections"] == 1
    assert o.lees_edwards()["bad"] == 0
