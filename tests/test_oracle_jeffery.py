"""Jeffery orbits of an ellipsoid in shear (oracle, and the GPU path with -m gpu).

A spheroid with its symmetry axis in the flow-gradient plane of a simple
shear u = gamma z e_x turns that axis at Jeffery's rate
    d alpha / dt = gamma / 2 (1 + lambda cos 2 alpha),
    lambda = (r^2 - 1) / (r^2 + 1),  r = R_par / R_perp,
alpha being the angle of the axis from the gradient direction z; its
angular velocity about the vorticity axis y is that rate.  The run: a
(5,5,2) cell at the centre of a 32 x 24 x 32 shear cell (walls z moving
-/+U), the fluid started on the linear profile, the cell on Jeffery's rate
of its start; the measured rate is compared with the law at the cell's
current orientation every 50 steps after the first 100.  Bars: within 10 %
for the axis along the flow and at 45 degrees; within 35 % for the flat
disc (axis along the gradient, the slowest rate and the thinnest lattice
disc, 4 nodes, which turns like a thicker one); and the rate with the axis
along the flow at least 4 times that of the flat disc (Jeffery: 1 / r^2 =
6.25; a sphere: 1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1005_2594_gb300 import workloads

U = 0.01
DIMS = (32, 24, 32)
R = (5.0, 2.0)


def _params():
    nx, ny, nz = DIMS
    return workloads.base_params(nx, ny, nz, periodic=(1, 1, 0), R=R, wall_vel={4: (-U, 0, 0), 5: (U, 0, 0)})


def _rates():
    nx, ny, nz = DIMS
    gd = 2 * U / (nz - 2)  # walls at z = 0.5 and nz - 1.5
    r = R[1] / R[0]
    lam = (r * r - 1) / (r * r + 1)
    return gd, lam


def _start(alpha0):
    """linear-shear populations, cell state (X, q, V, L)"""
    p = _params()
    nx, ny, nz = DIMS
    gd, lam = _rates()
    z = np.repeat(np.arange(nz), nx * ny)
    ux = -U + 2 * U * (z - 0.5) / (nz - 2)
    pop = np.array([oracle.equilibrium(1.0, [u, 0.0, 0.0]) for u in ux])
    q = np.array([[math.cos(alpha0 / 2), 0.0, math.sin(alpha0 / 2), 0.0]])
    X = np.array([[nx / 2, ny / 2, 0.5 + (nz - 2) / 2]])
    m = p["rho_p"] * 4 / 3 * math.pi * R[0] ** 2 * R[1]
    Iperp = m * (R[1] ** 2 + R[0] ** 2) / 5
    w0 = gd / 2 * (1 + lam * math.cos(2 * alpha0))
    return p, pop, X, q, np.zeros((1, 3)), np.array([[0.0, Iperp * w0, 0.0]])


def _measure(sim, omega_of, steps=400, every=50):
    """(measured, Jeffery) rates at the samples after the first 100 steps"""
    gd, lam = _rates()
    out = []
    for s in range(0, steps, every):
        sim.step(every)
        qc = sim.particles()["q"][0]
        ax = oracle.axis(qc)
        alpha = math.atan2(ax[0], ax[2])
        if s + every > 100:
            out.append((omega_of(sim), gd / 2 * (1 + lam * math.cos(2 * alpha))))
    return np.array(out)


def _check(results):
    fast, diag, flat = (results[a] for a in (math.pi / 2, math.pi / 4, 0.0))
    for name, res, bar in (("along the flow", fast, 0.10), ("45 degrees", diag, 0.10), ("flat", flat, 0.35)):
        ratio = res[:, 0] / res[:, 1]
        assert (res[:, 0] > 0).all(), name
        assert np.abs(ratio - 1).max() < bar, (name, ratio)
    assert fast[:, 0].mean() > 4.0 * flat[:, 0].mean()


def test_oracle_turns_at_jefferys_rate():
    results = {}
    for a in (math.pi / 2, math.pi / 4, 0.0):
        p, pop, X, q, V, L = _start(a)
        o = oracle.Oracle(p)
        own = o.owner()
        pop[own != -1] = 0.0
        o.set_populations(pop)
        o.set_particles(X, q, V, L)
        results[a] = _measure(o, lambda s: s.force_parts()["Om"][0][1])
    _check(results)


@pytest.mark.gpu
def test_gpu_turns_at_jefferys_rate():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1005_2594_gb300 import bloodlb as bl

    results = {}
    for a in (math.pi / 2, math.pi / 4, 0.0):
        p, pop, X, q, V, L = _start(a)
        sim = bl.Simulation(p)
        own = sim.owner()
        pop[own != -1] = 0.0
        sim.set_populations(pop)
        sim.set_particles(X, q, V, L)
        results[a] = _measure(sim, lambda s: s.force_parts()["Om"][0][1])
        sim.close()
    _check(results)
