"""GPU parity with the potentials of Sec. III active in every step.

Two workloads in which contacts last for the whole run (see
``workloads.sediment_stacks`` and ``workloads.tube_contacts``): cells denser
than the plasma rest on a wall under a body force, some stacked on others,
with the paper's potential range sigma = 12/11 R and strength eps = eps_w =
0.05.  The first has the plane walls of a shear cell, the second the curved
staircase wall of a tube given as a wall mask (bl_walls_set against
orc_set_walls).  Both run the Berne-Pechukas form (mu = 0, Eq. epsilon) and
the Gay-Berne variant mu = 2.

In every one of 100 steps the oracle's pair part (Eqs. phi, epsilon, sigma)
and its wall part (Eq. sigmaw) must be non-zero on some cell, and the GPU's
potential force and torque must match the oracle's to 1e-5 of their largest
value, both over all cells and over the cells that touch only the wall (so
that the wall part is checked on its own).  Owner maps are compared every 10
steps (bit-exact), fields, forces and the cell state after the run (1e-5).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    torch.cuda.init()
    yield


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max() if np.size(a) else 0.0
    s = np.abs(np.asarray(b)).max() if np.size(b) else 0.0
    return d / s if s > 0 else d


def _setup(geometry, mu):
    import oracle
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    mask = None
    if geometry == "sediment":
        p, X, q = workloads.sediment_stacks(mu=mu)
    else:
        p, X, q, mask = workloads.tube_contacts(mu=mu)
    orc, sim = oracle.Oracle(p), bl.Simulation(p, wall_mask=mask)
    if mask is not None:
        orc.set_walls(mask)
    orc.set_particles(X, q)
    sim.set_particles(X, q)
    return orc, sim


@pytest.mark.parametrize("mu", [0.0, 2.0])
@pytest.mark.parametrize("geometry", ["sediment", "tube"])
def test_potentials_active_100_steps(geometry, mu):
    orc, sim = _setup(geometry, mu)
    np.testing.assert_array_equal(sim.owner(), orc.owner())
    worst = {"Fp": 0.0, "Tp": 0.0, "Fw": 0.0, "Tw": 0.0}
    diverged = 0
    for s in range(100):
        orc.step(1)
        sim.step(1)
        fo, fg = orc.force_parts(), sim.force_parts()
        Fw, Tw = orc.wall_parts()
        pair_on = np.abs(fo["Fp"] - Fw).max(axis=1) > 0
        wall_on = np.abs(Fw).max(axis=1) > 0
        assert pair_on.any() and wall_on.any(), ("a potential is off at step", s)
        worst["Fp"] = max(worst["Fp"], rel(fg["Fp"], fo["Fp"]))
        worst["Tp"] = max(worst["Tp"], rel(fg["Tp"], fo["Tp"]))
        only_wall = wall_on & ~pair_on
        assert only_wall.any()
        worst["Fw"] = max(worst["Fw"], rel(fg["Fp"][only_wall], Fw[only_wall]))
        worst["Tw"] = max(worst["Tw"], rel(fg["Tp"][only_wall], Tw[only_wall]))
        if s % 10 == 9:
            diverged += int((sim.owner() != orc.owner()).sum())
    sim.sync()
    rho_o, u_o, own = orc.fields()
    rho_g, u_g, _ = sim.fields()
    fl = own == -1
    po, pg = orc.particles(), sim.particles()
    errs = dict(worst)
    errs.update({"u": rel(u_g[fl], u_o[fl]), "rho": rel(rho_g[fl], rho_o[fl])})
    for k in ("F", "T", "X", "q", "V", "L"):
        errs[k] = rel(pg[k], po[k])
    print("%s mu=%g, 100 steps: %s" % (geometry, mu, {k: "%.2e" % v for k, v in errs.items()}))
    assert diverged == 0, "owner-map divergence: %d node-steps" % diverged
    for k, v in errs.items():
        assert v < 1e-5, (k, v)


def test_arteriole_matches_oracle():
    """Sec. IV's arteriole as the bench runs it (radius 46.5 nodes, 786 cells
    sigma = (6, 2) at 42 % of the lumen overlapping one another and, edge-on,
    the wall on their fcc start, cell stiffness 0.05 and cell-wall stiffness
    0.005, body force on plasma and cells): 10 steps against the oracle, owner maps bit-exact every step,
    then fields, forces and the cell state to 1e-5"""
    import oracle
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import rheology

    p, X, q, mask = rheology.arteriole_case(start="close")
    orc, sim = oracle.Oracle(p), bl.Simulation(p, wall_mask=mask)
    orc.set_walls(mask)
    orc.set_particles(X, q)
    sim.set_particles(X, q)
    np.testing.assert_array_equal(sim.owner(), orc.owner())
    for _ in range(10):
        orc.step(1)
        sim.step(1)
        np.testing.assert_array_equal(sim.owner(), orc.owner())
    rho_o, u_o, own = orc.fields()
    rho_g, u_g, _ = sim.fields()
    fl = own == -1
    po, pg = orc.particles(), sim.particles()
    errs = {"u": rel(u_g[fl], u_o[fl]), "rho": rel(rho_g[fl], rho_o[fl])}
    for k in ("F", "T", "X", "q", "V", "L"):
        errs[k] = rel(pg[k], po[k])
    print("arteriole, 10 steps: %s" % {k: "%.2e" % v for k, v in errs.items()})
    for k, v in errs.items():
        assert v < 1e-5, (k, v)
