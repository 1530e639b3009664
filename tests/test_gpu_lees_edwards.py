"""GPU parity of the Lees-Edwards shear (Sec. IV, reading Q25) with the FP64
oracle.

The oracle pins the method itself (tests/test_oracle_lees_edwards.py: the
periodic limit, exact start-up Couette flow and mu_app = 1/6, a Kelvin mode
across the plane, mass, the reflection rule).  Here the GPU's two passes
after each sweep -- the gather of the shifted crossing populations with the
moments the sweep leaves beside the plane, and the interpolating scatter --
and the reflection in the cell update are compared with it:

* plasma under a body force with random initial populations, so that the
  flow varies along z and the interpolation matters; the offset passes
  between nodes every step; under every sweep mapping; the momentum moved
  across the plane (Delta p_LE of Eq. mu) every step;
* the same replayed as CUDA graphs of many steps (the offset comes from a
  device-side step counter);
* cells driven into the plane from both sides, reflected there, in a
  sheared suspension: owner maps bit-exact every step, fields, forces and
  cell state within 1e-5.
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


def _plasma(seed=3):
    import oracle
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    p = workloads.base_params(24, 12, 16, periodic=(1, 1, 1), g=(0.0, 2e-5, 1e-5))
    orc = oracle.Oracle(p)
    rng = np.random.default_rng(seed)
    pop = orc.populations() * (1 + 0.01 * rng.standard_normal((orc.N, 19)))
    return p, pop, orc, bl


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_plasma_shear_per_step(variant):
    p, pop, orc, bl = _plasma()
    sim = bl.Simulation(p)
    sim.sweep_variant(variant)
    orc.set_populations(pop)
    sim.set_populations(pop)
    U = 0.0137
    orc.set_lees_edwards(U)
    sim.lees_edwards(U)
    worst_P = 0.0
    for s in range(60):
        orc.step(1)
        sim.step(1)
        P_g, n_g = sim.lees_edwards_momentum()
        le = orc.lees_edwards()
        assert n_g == le["steps"] == s + 1
        worst_P = max(worst_P, abs(P_g - le["P_sum"]) / max(abs(le["P_sum"]), 1e-12))
    rho_o, u_o, _ = orc.fields()
    rho_g, u_g, _ = sim.fields()
    errs = {"u": rel(u_g, u_o), "rho": rel(rho_g - p["rho0"], rho_o - p["rho0"]), "P": worst_P}
    print("variant %d, 60 steps: %s" % (variant, {k: "%.2e" % v for k, v in errs.items()}))
    assert errs["u"] < 1e-5 and errs["rho"] < 1e-4 and errs["P"] < 1e-5, errs
    sim.close()


def test_plasma_shear_graph_replay():
    p, pop, orc, bl = _plasma(seed=4)
    sim = bl.Simulation(p)
    orc.set_populations(pop)
    sim.set_populations(pop)
    U = -0.0211
    orc.set_lees_edwards(U)
    sim.lees_edwards(U)
    orc.step(101)
    sim.step(100)  # pairs of steps as graph replays
    sim.step(1)    # and a lone step
    P_g, n_g = sim.lees_edwards_momentum()
    le = orc.lees_edwards()
    _, u_o, _ = orc.fields()
    _, u_g, _ = sim.fields()
    print("graph replay, 101 steps: u %.2e, P %.2e" % (rel(u_g, u_o), abs(P_g - le["P_sum"]) / abs(le["P_sum"])))
    assert n_g == 101
    assert rel(u_g, u_o) < 1e-5
    assert abs(P_g - le["P_sum"]) < 1e-5 * abs(le["P_sum"])
    sim.close()


def test_cells_reflected_at_the_plane():
    import oracle
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    nx, ny, nz = 40, 24, 24
    p = workloads.base_params(nx, ny, nz, periodic=(1, 1, 1), R=(3.0, 1.5), sigma=(3.3, 1.6), eps=0.05)
    p["rho_p"] = 20.0  # heavy enough to reach the plane through the fluid
    dr = max(p["sig_perp"], max(p["R_perp"], p["R_par"]) + 1.0)
    X = np.array([[dr + 0.1, 6.3, 7.1], [dr + 0.3, 17.6, 15.2], [nx - 1 - dr - 0.1, 6.8, 17.4],
                  [nx - 1 - dr - 0.4, 16.9, 6.6], [nx / 2, 12.2, 11.8], [nx / 2 + 7.5, 12.4, 12.1]])
    rng = np.random.default_rng(7)
    q = rng.standard_normal((len(X), 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    V = np.array([[-0.05, 0.0, 0.002], [-0.04, 0.001, 0.0], [0.05, 0.0, -0.002], [0.045, 0.0, 0.001],
                  [0.0, 0.0, 0.01], [-0.01, 0.0, 0.0]])
    orc, sim = oracle.Oracle(p), bl.Simulation(p)
    U = 0.02
    orc.set_lees_edwards(U)
    sim.lees_edwards(U)
    orc.set_particles(X, q, V=V)
    sim.set_particles(X, q, V=V)
    for _ in range(60):
        orc.step(1)
        sim.step(1)
        np.testing.assert_array_equal(sim.owner(), orc.owner())
    le = orc.lees_edwards()
    assert le["reflections"] >= 4 and le["bad"] == 0, le
    sim.sync()
    rho_o, u_o, own = orc.fields()
    rho_g, u_g, _ = sim.fields()
    fl = own == -1
    po, pg = orc.particles(), sim.particles()
    errs = {"u": rel(u_g[fl], u_o[fl])}
    for k in ("F", "T", "X", "q", "V", "L"):
        errs[k] = rel(pg[k], po[k])
    P_g, _ = sim.lees_edwards_momentum()
    errs["P"] = abs(P_g - le["P_sum"]) / abs(le["P_sum"])
    print("cells at the plane, 60 steps, %d reflections: %s" % (le["reflections"],
                                                               {k: "%.2e" % v for k, v in errs.items()}))
    for k, v in errs.items():
        assert v < 1e-5, (k, v)
    sim.close()


def test_rejects_walls():
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    p = workloads.base_params(16, 12, 12, periodic=(1, 1, 0))
    sim = bl.Simulation(p)
    with pytest.raises(bl.BloodLBError):
        sim.lees_edwards(0.01)
    sim.close()
