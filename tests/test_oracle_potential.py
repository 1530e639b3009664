"""Pins of the oracle's Berne-Pechukas-scaled Hookean potentials (Sec. III,
Eqs. phi, epsilon, sigma, sigmaw).

* Contact distances in the three orientations of Fig. (potential-force):
  face to face (o_i || o_j || r) 2 sig_par, side by side (o_i || o_j, both
  normal to r) 2 sig_perp, crossed (o_i normal to o_j, r || o_i)
  sigbar / sqrt(1 - chi); for the paper's sig_perp = 6, sig_par = 2 (Sec. IV,
  4 um and 4/3 um at dx = 2/3 um) these are 4, 12 and 12 / sqrt(1.8).
* Strength: eps = epsbar / sqrt(1 - chi^2 (o_i.o_j)^2): aligned cells are
  stiffer by 1 / sqrt(1 - chi^2) (the paper notes the face-to-face case is
  considerably stiffer); crossed cells have eps = epsbar.
* Cell-wall range: sqrt(sig_par^2 + sig_w^2) face on, sqrt(sig_perp^2 +
  sig_w^2) side on (Berne-Pechukas sphere-ellipsoid scaling).
* Forces are minus the gradient of phi (central differences), torques minus
  the derivative of phi with respect to a rotation angle of the cell, and a
  pair's forces and torques balance: F_i + F_j = 0, T_i + T_j + r x F_j = 0.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_1005_2594_gb300 import workloads


def paper_params(mu=0.0):
    p = workloads.base_params(64, 64, 64, R=(5.5, 11.0 / 6.0), sigma=(6.0, 2.0), eps=0.05, mu=mu)
    return p


def onset(params, oi, oj, rhat):
    """smallest r at which the pair energy vanishes, by bisection"""
    lo, hi = 1e-3, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        phi = oracle.pair(params, mid * np.asarray(rhat, float), oi, oj)[0]
        if phi > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


ex, ey, ez = np.eye(3)


def test_contact_distances_paper_numbers():
    p = paper_params()
    assert abs(onset(p, ez, ez, ez) - 4.0) < 1e-9          # face to face: 2 sig_par
    assert abs(onset(p, ez, ez, ex) - 12.0) < 1e-9         # side by side: 2 sig_perp
    assert abs(onset(p, ez, ex, ez) - 12.0 / math.sqrt(1.8)) < 1e-9  # crossed
    # Fig. (potential-force): the onset depends on orientation, side > crossed > face
    assert onset(p, ez, ez, ex) > onset(p, ez, ex, ez) > onset(p, ez, ez, ez)


def test_strength_special_cases():
    p = paper_params()
    chi = (4.0 - 36.0) / (4.0 + 36.0)
    # at half the contact distance phi = eps / 4
    phi_face = oracle.pair(p, 2.0 * ez, ez, ez)[0]
    assert abs(phi_face - 0.05 / math.sqrt(1 - chi * chi) / 4.0) < 1e-15
    s_cross = 12.0 / math.sqrt(1.8)
    phi_cross = oracle.pair(p, 0.5 * s_cross * ez, ez, ex)[0]
    assert abs(phi_cross - 0.05 / 4.0) < 1e-15
    phi_side = oracle.pair(p, 6.0 * ex, ez, ez)[0]
    assert abs(phi_side - 0.05 / math.sqrt(1 - chi * chi) / 4.0) < 1e-15


def test_wall_range_special_cases():
    p = paper_params()
    for o, expect in ((ez, math.sqrt(4.0 + 0.25)), (ex, math.sqrt(36.0 + 0.25))):
        lo, hi = 1e-3, 50.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if oracle.wall(p, mid * ez, o)[0] > 0:
                lo = mid
            else:
                hi = mid
        assert abs(lo - expect) < 1e-9
    phi = oracle.wall(p, 0.5 * math.sqrt(4.25) * ez, ez)[0]
    assert abs(phi - 0.05 / 4.0) < 1e-15


def _random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("mu", [0.0, 2.0])
def test_pair_forces_torques_are_derivatives(mu):
    p = paper_params(mu)
    rng = np.random.default_rng(42 + int(mu))
    h = 1e-6
    checked = 0
    while checked < 30:
        oi, oj = _random_unit(rng), _random_unit(rng)
        rv = _random_unit(rng) * rng.uniform(2.0, 11.0)
        phi, Fi, Fj, Ti, Tj = oracle.pair(p, rv, oi, oj)
        if phi < 1e-5:
            continue
        checked += 1
        scale = max(np.abs(Fi).max(), 1e-12)
        # F_j = -d phi / d X_j = -d phi / d r
        g = np.zeros(3)
        for k in range(3):
            d = np.zeros(3)
            d[k] = h
            g[k] = (oracle.pair(p, rv + d, oi, oj)[0] - oracle.pair(p, rv - d, oi, oj)[0]) / (2 * h)
        np.testing.assert_allclose(Fj, -g, atol=1e-6 * scale + 1e-12)
        np.testing.assert_allclose(Fi, g, atol=1e-6 * scale + 1e-12)
        # torque = -d phi / d theta for a small rotation of the cell about axis k
        tscale = max(np.abs(Ti).max(), np.abs(Tj).max(), 1e-12)
        for k in range(3):
            R = Rotation.from_rotvec(h * np.eye(3)[k]).as_matrix()
            Rm = R.T
            dphi_i = (oracle.pair(p, rv, R @ oi, oj)[0] - oracle.pair(p, rv, Rm @ oi, oj)[0]) / (2 * h)
            dphi_j = (oracle.pair(p, rv, oi, R @ oj)[0] - oracle.pair(p, rv, oi, Rm @ oj)[0]) / (2 * h)
            assert abs(Ti[k] + dphi_i) < 1e-6 * tscale + 1e-12
            assert abs(Tj[k] + dphi_j) < 1e-6 * tscale + 1e-12
        # balance of linear and angular momentum
        np.testing.assert_allclose(Fi + Fj, 0.0, atol=1e-15 * scale)
        np.testing.assert_allclose(Ti + Tj + np.cross(rv, Fj), 0.0, atol=1e-12 * max(tscale, scale))


def test_wall_forces_torques_are_derivatives():
    p = paper_params()
    rng = np.random.default_rng(9)
    h = 1e-6
    checked = 0
    while checked < 30:
        oi = _random_unit(rng)
        rv = _random_unit(rng) * rng.uniform(1.0, 6.0)
        phi, Fi, Ti = oracle.wall(p, rv, oi)
        if phi < 1e-6:
            continue
        checked += 1
        scale = np.abs(Fi).max()
        g = np.zeros(3)
        for k in range(3):
            d = np.zeros(3)
            d[k] = h
            g[k] = (oracle.wall(p, rv + d, oi)[0] - oracle.wall(p, rv - d, oi)[0]) / (2 * h)
        # r = x_wall - X_i: F_i = -d phi / d X_i = +d phi / d r
        np.testing.assert_allclose(Fi, g, atol=1e-6 * scale + 1e-12)
        for k in range(3):
            R = Rotation.from_rotvec(h * np.eye(3)[k]).as_matrix()
            dphi = (oracle.wall(p, rv, R @ oi)[0] - oracle.wall(p, rv, R.T @ oi)[0]) / (2 * h)
            assert abs(Ti[k] + dphi) < 1e-6 * max(np.abs(Ti).max(), 1e-12) + 1e-12


def test_potential_is_compact_and_repulsive():
    p = paper_params()
    rng = np.random.default_rng(1)
    for _ in range(200):
        oi, oj = _random_unit(rng), _random_unit(rng)
        rh = _random_unit(rng)
        s = onset(p, oi, oj, rh)
        assert s <= 12.0 + 1e-9  # never beyond 2 sig_perp
        phi, Fi, Fj, _, _ = oracle.pair(p, 0.9 * s * rh, oi, oj)
        assert phi > 0
        assert np.dot(Fj, rh) > 0  # j is pushed away from i
        assert oracle.pair(p, 1.01 * s * rh, oi, oj)[0] == 0.0
