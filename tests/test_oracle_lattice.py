"""Pins of the oracle's lattice-Boltzmann part (Sec. II, Eqs. col, adv, neq).

Each check is fixed by mathematics or by the paper, not by re-typing the
oracle's formulas:

* the velocity set and weights (Sec. II, weights after Eq. neq) are recovered
  from the equilibrium itself and checked against the D3Q19 isotropy sums;
* Eq. (neq) must equal the third-order Taylor polynomial of the Maxwellian
  weight factor exp(c.u / c_s^2 - u^2 / (2 c_s^2)): the remainder must scale
  as |u|^4;
* its moments: sum n^eq = rho, sum n^eq c = rho u, sum n^eq cc = rho (c_s^2 I + uu);
* BGK (Eq. col) conserves rho and j (Sec. II: both are collision invariants),
  and with tau = 1 relaxes a node to n^eq in one step;
* Guo forcing (reading Q1) adds exactly rho g of momentum per node and step.
"""
import math

import numpy as np

import oracle
from paper_1005_2594_gb300 import workloads

# interface direction order (0, +x, -x, +y, -y, +z, -z, then the twelve
# (+-1,+-1,0)-type vectors each followed by its opposite)
C_IFACE = np.array([
    [0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])


def _weights_and_velocities():
    w = oracle.equilibrium(1.0, [0.0, 0.0, 0.0])
    eps = 1e-3
    c = np.zeros((19, 3))
    for k in range(3):
        u = np.zeros(3)
        u[k] = eps
        fp = oracle.equilibrium(1.0, u)
        fm = oracle.equilibrium(1.0, -u)
        # n^eq(u) - n^eq(-u) = 6 alpha eps c_k exactly for c_k in {-1, 0, 1}
        c[:, k] = (fp - fm) / (6.0 * w * eps)
    return w, c


def test_weights_and_velocity_set():
    w, c = _weights_and_velocities()
    assert np.allclose(c, np.round(c), atol=1e-9)
    c = np.round(c).astype(int)
    np.testing.assert_array_equal(c, C_IFACE)
    c2 = (c * c).sum(axis=1)
    for r in range(19):
        expect = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[c2[r]]
        assert abs(w[r] - expect) < 1e-16
    assert abs(w.sum() - 1.0) < 1e-15
    # isotropy up to fourth order
    np.testing.assert_allclose(np.einsum("r,ri->i", w, c), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("r,ri,rj->ij", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("r,ri,rj,rk->ijk", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("r,ri,rj,rk,rl->ijkl", w, c, c, c, c), iso4, atol=1e-16)


def test_equilibrium_is_third_order_maxwellian_expansion():
    w, c = _weights_and_velocities()
    c = np.round(c)
    rng = np.random.default_rng(7)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        errs = []
        for mag in (0.04, 0.02):
            u = mag * d
            feq = oracle.equilibrium(1.3, u)
            maxw = 1.3 * w * np.exp(3.0 * (c @ u) - 1.5 * (u @ u))
            errs.append(np.max(np.abs(feq - maxw) / w))
        # fourth-order remainder: halving u divides the error by 16
        assert 13.0 < errs[0] / errs[1] < 19.0, errs


def test_equilibrium_moments():
    w, c = _weights_and_velocities()
    c = np.round(c)
    rng = np.random.default_rng(3)
    for _ in range(10):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        f = oracle.equilibrium(rho, u)
        assert abs(f.sum() - rho) < 1e-14
        np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("r,ri,rj->ij", f, c, c), rho * (np.eye(3) / 3.0 + np.outer(u, u)),
                                   atol=1e-15)


def _one_node(tau=1.0, g=(0.0, 0.0, 0.0)):
    p = workloads.base_params(1, 1, 1, periodic=(1, 1, 1), g=g)
    p["tau"] = tau
    return oracle.Oracle(p)


def test_bgk_collision_invariants_and_relaxation():
    rng = np.random.default_rng(11)
    _, c = _weights_and_velocities()
    c = np.round(c)
    for tau in (1.0, 0.7, 1.6):
        o = _one_node(tau)
        f0 = oracle.equilibrium(1.0, [0.02, -0.01, 0.03]) * (1.0 + rng.uniform(-0.05, 0.05, 19))
        o.set_populations(f0[None, :])
        o.step(1)
        f1 = o.populations()[0]
        assert abs(f1.sum() - f0.sum()) < 1e-15
        np.testing.assert_allclose(f1 @ c, f0 @ c, atol=1e-16)
        rho = f0.sum()
        feq = oracle.equilibrium(rho, (f0 @ c) / rho)
        # n* = n - (n - n^eq) / tau, and the 1-node periodic lattice streams onto itself
        np.testing.assert_allclose(f1, f0 - (f0 - feq) / tau, atol=1e-16)


def test_guo_force_adds_rho_g_per_step():
    g = np.array([1e-4, -2e-4, 3e-5])
    _, c = _weights_and_velocities()
    c = np.round(c)
    o = _one_node(1.0, tuple(g))
    f0 = oracle.equilibrium(1.05, [0.01, 0.0, -0.02])
    o.set_populations(f0[None, :])
    j = [f0 @ c]
    rho = f0.sum()
    for _ in range(5):
        o.step(1)
        f = o.populations()[0]
        j.append(f @ c)
        assert abs(f.sum() - rho) < 1e-14
    dj = np.diff(np.array(j), axis=0)
    np.testing.assert_allclose(dj, np.tile(rho * g, (5, 1)), atol=1e-15)
    # reported velocity carries the half-step force: u = (j + rho g / 2) / rho
    r, u, _ = o.fields()
    np.testing.assert_allclose(u[0], (j[-1] + 0.5 * rho * g) / rho, atol=1e-16)
