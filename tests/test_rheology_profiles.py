"""Radial profiles of tube flow and the two-layer fit of Sec. IV (CPU).

Sec. IV fits the arteriole's radial velocity profile with a modified
axial-train model: a cell-depleted layer of width delta next to the wall,
with the plasma viscosity, around a core of viscosity mu_c.  These tests pin
the profile function, the fit and the binning of lattice fields.
"""
import math

import numpy as np

from paper_1005_2594_gb300 import rheology, workloads

F, MU = 2e-6, 1.0 / 6.0


def test_two_layer_profile_limits_and_continuity():
    r = np.linspace(0.0, 30.0, 301)
    R = 30.0
    # no layer: the core's Poiseuille profile; equal viscosities: the plasma's
    np.testing.assert_allclose(rheology.axial_train(r, R, 0.0, 2.5, F, MU), rheology.poiseuille(r, R, F, 2.5 * MU),
                               rtol=1e-12, atol=0)
    np.testing.assert_allclose(rheology.axial_train(r, R, 7.0, 1.0, F, MU), rheology.poiseuille(r, R, F, MU),
                               rtol=1e-12, atol=0)
    # continuous at the core radius, and the stress f r / 2 on both sides
    Rc = R - 4.0
    lo, hi = rheology.axial_train([Rc - 1e-7, Rc + 1e-7], R, 4.0, 3.0, F, MU)
    assert abs(lo - hi) < 1e-6 * abs(lo)  # the slope alone moves it by ~5e-8 of its value
    eps = 1e-4
    d_in = (rheology.axial_train(Rc - eps, R, 4.0, 3.0, F, MU) - rheology.axial_train(Rc - 2 * eps, R, 4.0, 3.0, F, MU)) / eps
    d_out = (rheology.axial_train(Rc + 2 * eps, R, 4.0, 3.0, F, MU) - rheology.axial_train(Rc + eps, R, 4.0, 3.0, F, MU)) / eps
    assert abs(3.0 * MU * d_in + F * Rc / 2) < 1e-3 * F * Rc
    assert abs(MU * d_out + F * Rc / 2) < 1e-3 * F * Rc


def test_fit_recovers_layer_width_and_viscosity_ratio():
    R = 30.0
    r = np.arange(30) + 0.5
    for delta, ratio in ((2.0, 2.43), (4.5, 1.8), (1.0, 3.5)):
        u = rheology.axial_train(r, R, delta, ratio, F, MU)
        d, m = rheology.fit_axial_train(r, u, R, F, MU)
        assert abs(d - delta) < 1e-3 and abs(m - ratio) < 1e-3 * ratio, (d, m, delta, ratio)
    # the effective radius of a plasma-only profile
    u = rheology.poiseuille(r, 29.6, F, MU)
    assert abs(rheology.fit_poiseuille_radius(r, u, F, MU) - 29.6) < 1e-6


def test_radial_binning_of_lattice_fields():
    """a synthetic tube: Poiseuille velocity on the fluid nodes, cell nodes
    inside radius 8; the bins give the profile at their nodes' mean radius
    and a cell fraction of 1 inside, 0 outside"""
    p = workloads.base_params(16, 40, 40, periodic=(1, 1, 1))
    radius = 18.0
    mask = workloads.tube_mask(p, radius, axis=0)
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = (ny - 1) / 2.0
    r = np.hypot(y - c, z - c).reshape(-1)
    owner = np.where(mask > 0, -2 - 6, -1).astype(np.int32)
    owner[(r < 8.0) & (mask == 0)] = 0
    u = np.zeros((nx * ny * nz, 3))
    u[:, 0] = np.where(owner == -1, rheology.poiseuille(r, radius, F, MU), 0.0)
    centres, um, H, n = rheology.radial_profiles(u, owner, p, radius)
    assert len(centres) == math.ceil(radius)
    for k in range(len(centres)):
        sel = (r >= k) & (r < k + 1) & (r < radius) & (owner == -1)
        if sel.any():
            assert abs(um[k] - u[sel, 0].mean()) < 1e-15
            assert n[k] == sel.sum()
    assert np.all(H[:8] == 1.0) and np.all(H[9:] == 0.0)


def test_arteriole_case_in_lattice_units():
    """Sec. IV's units and arteriole: dt from tau = 1 and the plasma's
    kinematic viscosity 1.09e-6 m^2/s at dx = 2/3 um; the cell stiffness
    1.47e-15 J is 0.05 lattice units; radius 31 um, sigma = (4, 4/3) um,
    R = 11/12 sigma and 42 % of the lumen in cells, all inside the tube"""
    dx = rheology.DX_UM * 1e-6
    assert abs((2 * 1.0 - 1) / 6 * dx * dx / rheology.DT_S - 1.09e-6) < 1e-3 * 1.09e-6
    p, X, q, mask = rheology.arteriole_case()
    assert abs(p["eps"] - 0.05) < 5e-4 and abs(p["eps_w"] - 0.005) < 5e-5
    assert (p["sig_perp"], p["sig_par"]) == (6.0, 2.0)
    assert abs(p["R_perp"] - 5.5) < 1e-12 and abs(p["R_par"] - 11.0 / 6.0) < 1e-12
    radius = 31.0 / rheology.DX_UM
    lumen = math.pi * radius ** 2 * p["nx"]
    assert abs(len(X) * workloads.cell_volume(p) / lumen - 0.42) < 2e-3
    c = (p["ny"] - 1) / 2.0
    assert np.all(np.hypot(X[:, 1] - c, X[:, 2] - c) + p["R_perp"] < radius)
    assert mask.reshape(p["nz"], p["ny"], p["nx"])[int(c), int(c), :].max() == 0  # the axis is open
    # the pseudo-shear rate Q / (2 pi R^3) of Poiseuille flow is u_max / (4 R)
    u_max = rheology.poiseuille(0.0, radius, 1e-6, 1 / 6.0)
    Q = math.pi * radius ** 2 * u_max / 2
    assert abs(rheology.pseudo_shear_rate(Q, radius) * rheology.DT_S - u_max / (4 * radius)) < 1e-15


def test_shear_cell_analysis_and_case():
    """Sec. IV's shear cell: the profile v_z(x) averages the fluid nodes of
    each plane, the shear rate comes from its central half only (a profile
    with steeper layers beside the sheared plane keeps the central slope), and
    the case has the paper's number density with every cell beyond the
    reflection distance"""
    p = workloads.base_params(16, 3, 4, periodic=(1, 1, 1))
    N = 16 * 3 * 4
    x = np.arange(N) % 16
    u = np.zeros((N, 3))
    u[:, 2] = 2e-4 * (x - 7.5)
    owner = np.full(N, -1)
    owner[::7] = 0  # cell nodes carry no fluid velocity
    u[owner == 0, 2] = 99.0
    prof = rheology.x_profile(u, owner, p)
    np.testing.assert_allclose(prof, 2e-4 * (np.arange(16) - 7.5), rtol=0, atol=1e-15)
    bent = prof + np.where(np.arange(16) < 4, -3e-4 * (4 - np.arange(16)), 0.0)
    bent = bent + np.where(np.arange(16) >= 12, 3e-4 * (np.arange(16) - 11), 0.0)
    assert abs(rheology.central_shear_rate(bent, 16) - 2e-4) < 1e-15
    p, X, q = rheology.le_shear_case()
    vol_m3 = p["nx"] * p["ny"] * p["nz"] * (rheology.DX_UM * 1e-6) ** 3
    assert len(X) == round(6.4e15 * vol_m3)
    dr = rheology.le_reflect_distance(p)
    assert dr == max(p["sig_perp"], p["R_perp"] + 1.0) == 6.5
    assert (X[:, 0] + 0.5 > dr).all() and (p["nx"] - 0.5 - X[:, 0] > dr).all()
    sig_vol = len(X) * 4.0 / 3.0 * math.pi * p["sig_perp"] ** 2 * p["sig_par"] / (p["nx"] * p["ny"] * p["nz"])
    assert abs(sig_vol - 0.56) < 0.02  # the paper's hematocrit of 56 %
