"""Apparent viscosity of the suspension in tube flow.

Sec. IV characterises the model by the apparent viscosity of a suspension
driven through a tube by a body force: the viscosity a Newtonian fluid would
need to carry the same volume flux Q, mu_app = pi R^4 rho_bar g / (8 Q),
relative to the plasma's rho_bar nu.  On the lattice the walls sit midway
between a staircase of nodes, so the radius that the Poiseuille formula
needs is not R exactly; the relative viscosity is therefore taken as the
ratio of fluxes under the same driving, plasma alone over suspension:
mu_rel = Q_plasma / Q.

Q is the volume flux along the tube axis (x): the axial velocity of the
fluid nodes summed over the lattice and divided by the tube length, plus the
cells' share, V_x times the cell volume over the length.

The refined case (``tube_case(k)``) is the same physical system on a lattice
k times finer under diffusive scaling at fixed tau: box, tube radius, cells
and positions x k, body force / k^3 (an acceleration in lattice units), and
the contact strength x k so that potential forces, like lattice forces, stay
the same in lattice units.
"""
import math

import numpy as np

from . import bloodlb as bl
from . import workloads


def tube_case(k=1, radius=30.0, length=128, hct=0.35, g=2e-6, R=(7.0, 3.0), seed=1007, cells=True):
    """params, X, q, wall mask of the tube refined k times (X, q empty
    without cells).  The coarse cross-section is 2 radius + 8 nodes wide."""
    n = int(2 * radius + 8)
    p = workloads.base_params(length * k, n * k, n * k, periodic=(1, 1, 1), R=(R[0] * k, R[1] * k), eps=float(k),
                              g=(g / k ** 3, 0.0, 0.0), body_force_on_cells=1)
    mask = workloads.tube_mask(p, radius * k, axis=0)
    if not cells:
        return p, np.zeros((0, 3)), np.zeros((0, 4)), mask
    pc = workloads.base_params(length, n, n, periodic=(1, 1, 1), R=R)
    n_cells = int(round(hct * math.pi * radius ** 2 * length / workloads.cell_volume(pc)))
    c = (n - 1) / 2.0
    rmax = max(R)

    def inside(x):
        return np.hypot(x[:, 1] - c, x[:, 2] - c) + rmax + 1.0 < radius

    X, q = workloads.fcc_cells(pc, n_cells, seed, inside)
    # the same places on the finer lattice: the axis moves from (n - 1) / 2
    # to (k n - 1) / 2
    Xk = X * k
    Xk[:, 1:] += (k - 1) / 2.0
    return p, Xk, q, mask


# Sec. IV's units: dx = 2/3 um, dt = 6.80e-8 s (tau = 1 with the plasma's
# kinematic viscosity), dm = 3.05e-16 kg, so that one lattice energy unit is
# dm dx^2 / dt^2 = 2.93e-14 J
DX_UM, DT_S = 2.0 / 3.0, 6.80e-8
E_UNIT_J = 3.05e-16 * (DX_UM * 1e-6) ** 2 / DT_S ** 2


def arteriole_case(cells=True, g=8e-6, hct=0.42, eps_w_J=1.47e-16, seed=1010, start="wide"):
    """Sec. IV's arteriole in lattice units: radius 31 um (46.5 nodes), closed
    periodically at 43 um (64 nodes); cells of the potential's half-axes
    sigma_perp = 4 um, sigma_par = 4/3 um (6 and 2 nodes) with coupling
    half-axes R = 11/12 sigma, cell stiffness 1.47e-15 J, cell-wall stiffness
    eps_w_J (1.47e-16 J in the paper), cells at hct of the lumen (42 %) on a
    jittered fcc start; the body force g drives plasma and cells.  The start
    keeps each centre R_perp + 1 from the wall ("wide": no orientation
    reaches it) or R_par + 1 ("close": cells lying edge-on to the wall reach
    into it, and the wall potential pushes them out).  Returns params, X, q,
    wall mask (X, q empty without cells)."""
    radius, length = 31.0 / DX_UM, 64
    n = int(2 * radius + 8)
    sig = (4.0 / DX_UM, (4.0 / 3.0) / DX_UM)
    R = (sig[0] * 11.0 / 12.0, sig[1] * 11.0 / 12.0)
    p = workloads.base_params(length, n, n, periodic=(1, 1, 1), R=R, sigma=sig, eps=1.47e-15 / E_UNIT_J,
                              eps_w=eps_w_J / E_UNIT_J, g=(g, 0.0, 0.0), body_force_on_cells=1)
    mask = workloads.tube_mask(p, radius, axis=0)
    if not cells:
        return p, np.zeros((0, 3)), np.zeros((0, 4)), mask
    n_cells = int(round(hct * math.pi * radius ** 2 * length / workloads.cell_volume(p)))
    c = (n - 1) / 2.0
    margin = {"wide": R[0], "close": R[1]}[start] + 1.0

    def inside(x):
        return np.hypot(x[:, 1] - c, x[:, 2] - c) + margin < radius

    X, q = workloads.fcc_cells(p, n_cells, seed, inside)
    return p, X, q, mask


def pseudo_shear_rate(Q, radius):
    """Sec. IV's pseudo-shear rate Q / (2 pi R^3), in 1/s"""
    return Q / (2.0 * math.pi * radius ** 3) / DT_S


def flux(sim, p):
    """volume flux along x (lattice units)"""
    import torch

    N = p["nx"] * p["ny"] * p["nz"]
    rho = torch.empty(N, dtype=torch.float64, device="cuda")
    u = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    bl.bl_fields_get(sim.ctx, N, rho, u, None, on_device=True)
    torch.cuda.synchronize()
    q_fluid = float(u[:, 0].sum()) / p["nx"]
    if sim.n == 0:
        return q_fluid
    V = sim.particles()["V"]
    vol = 4.0 / 3.0 * math.pi * p["R_perp"] ** 2 * p["R_par"]
    return q_fluid + float(V[:, 0].sum()) * vol / p["nx"]


def radial_profiles(u, owner, p, radius, axis=0):
    """Radial profiles about the tube axis (through the box centre): bins of
    unit width from the axis to `radius`; per bin the mean axial velocity of
    its fluid nodes and the cell fraction, cell nodes over cell and fluid
    nodes (Sec. IV, the arteriole's velocity and concentration profiles).
    u: N x 3 (or N axial values), owner: N, node n = x + nx (y + ny z).
    Returns (bin centres, mean axial velocity, cell fraction, fluid nodes per
    bin)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [x.reshape(-1), y.reshape(-1), z.reshape(-1)]
    c = [(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0]
    others = [k for k in range(3) if k != axis]
    r = np.sqrt(sum((coords[k] - c[k]) ** 2 for k in others))
    ua = np.asarray(u)
    ua = ua[:, axis] if ua.ndim == 2 else ua
    own = np.asarray(owner)
    nb = int(math.ceil(radius))
    b = np.minimum((r).astype(np.int64), nb)
    inside = (r < radius) & (own > -2)
    fl = inside & (own == -1)
    cell = inside & (own >= 0)
    n_fl = np.bincount(b[fl], minlength=nb + 1)[:nb]
    n_cell = np.bincount(b[cell], minlength=nb + 1)[:nb]
    u_sum = np.bincount(b[fl], weights=ua[fl], minlength=nb + 1)[:nb]
    centres = np.arange(nb) + 0.5
    with np.errstate(invalid="ignore", divide="ignore"):
        u_mean = np.where(n_fl > 0, u_sum / np.maximum(n_fl, 1), np.nan)
        H = np.where(n_fl + n_cell > 0, n_cell / np.maximum(n_fl + n_cell, 1), np.nan)
    return centres, u_mean, H, n_fl


def poiseuille(r, R, f, mu):
    """Hagen-Poiseuille profile of a tube of radius R under force density f"""
    return f / (4.0 * mu) * (R * R - np.asarray(r) ** 2)


def axial_train(r, R, delta, mu_ratio, f, mu_b):
    """The two-layer (modified axial-train) profile that Sec. IV fits to the
    arteriole: a cell-depleted layer of width delta next to the wall with the
    plasma viscosity mu_b, and a core of viscosity mu_c = mu_ratio mu_b; the
    shear stress f r / 2 is continuous at the core radius R - delta."""
    r = np.asarray(r, dtype=np.float64)
    Rc = R - delta
    outer = f / (4.0 * mu_b) * (R * R - r * r)
    core = f / (4.0 * mu_b) * (R * R - Rc * Rc) + f / (4.0 * mu_b * mu_ratio) * (Rc * Rc - r * r)
    return np.where(r >= Rc, outer, core)


def fit_poiseuille_radius(r, u, f, mu, weights=None):
    """effective wall radius of a plasma-only profile (the staircase wall's
    position is uncertain by about half a node)"""
    from scipy.optimize import curve_fit

    ok = np.isfinite(u)
    sig = None if weights is None else 1.0 / np.sqrt(np.maximum(weights[ok], 1))
    (R,), _ = curve_fit(lambda rr, R: poiseuille(rr, R, f, mu), r[ok], u[ok], p0=[r[ok].max() + 0.5], sigma=sig)
    return float(R)


def fit_axial_train(r, u, R, f, mu_b, weights=None):
    """(delta, mu_c / mu_b) of the two-layer profile closest to u(r), the wall
    radius R and the boundary viscosity mu_b (the plasma's) given"""
    from scipy.optimize import curve_fit

    ok = np.isfinite(u)
    sig = None if weights is None else 1.0 / np.sqrt(np.maximum(weights[ok], 1))
    (delta, ratio), _ = curve_fit(lambda rr, d, m: axial_train(rr, R, d, m, f, mu_b), r[ok], u[ok], p0=[0.1 * R, 2.0],
                                  bounds=([0.0, 1.0], [R, 100.0]), sigma=sig)
    return float(delta), float(ratio)


def run(p, X, q, mask, steps, samples=20, model=None, gap_range=None, stream=None, profile_radius=None):
    """steps of the tube from rest (with `model` attached over gap_range =
    (gap_lo, gap_hi[, speed_lo, speed_hi])); the flux sampled at `samples` even
    intervals over the second half.  Returns (mean flux, flux samples,
    milliseconds of stepping, CUDA events on the stream, read-outs excluded)."""
    import torch

    st = torch.cuda.current_stream() if stream is None else stream
    prof = []
    sim = bl.Simulation(p, stream=st.cuda_stream, wall_mask=mask)
    if len(X):
        sim.set_particles(X, q)
        if model is not None:
            bl.bl_mlp_attach_range(sim.ctx, model, *gap_range)
    half = steps // 2
    every = max(2, (steps - half) // samples) // 2 * 2
    ms = 0.0

    def advance(k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sim.step(k)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    out = []
    try:
        ms += advance(half)
        done = half
        while done + every <= steps:
            ms += advance(every)
            done += every
            out.append(flux(sim, p))
            if profile_radius is not None:
                _, u, own = sim.fields()
                prof.append(radial_profiles(u, own, p, profile_radius))
        sim.sync()
    finally:
        sim.close()
    if profile_radius is None:
        return float(np.mean(out)), out, ms
    centres = prof[0][0]
    u_mean = np.nanmean(np.array([pr[1] for pr in prof]), axis=0)
    H = np.nanmean(np.array([pr[2] for pr in prof]), axis=0)
    n_fl = np.sum(np.array([pr[3] for pr in prof]), axis=0)
    return float(np.mean(out)), out, ms, (centres, u_mean, H, n_fl)


# ---------------------------------------------------------------------------
# Lees-Edwards shear cell (Sec. IV): plane Couette flow of a homogeneous
# suspension, the velocity gradient along x, the flow along z


def le_reflect_distance(p):
    """Sec. IV's reflection distance sigma_perp, raised to max(R) + 1 so that
    no cell covers a node beside the sheared plane (the library's default)"""
    return max(p["sig_perp"], max(p["R_perp"], p["R_par"]) + 1.0)


def le_shear_case(cells=True, nx=128, ny=40, nz=40, number_density_m3=6.4e15, seed=1011):
    """Sec. IV's shear cell in lattice units: 128 x 40 x 40 (85 x 27 x 27
    um^3), periodic, sheared across the x plane; cells with sigma = (4, 4/3)
    um = (6, 2) nodes and R = 11/12 sigma at the paper's number density
    6.4e15 / m^3 (its hematocrit of 56 %), stiffness 1.47e-15 J, on a jittered
    fcc start with centres kept half a node beyond the reflection distance.
    Returns params, X, q (empty without cells)."""
    sig = (4.0 / DX_UM, (4.0 / 3.0) / DX_UM)
    R = (sig[0] * 11.0 / 12.0, sig[1] * 11.0 / 12.0)
    p = workloads.base_params(nx, ny, nz, periodic=(1, 1, 1), R=R, sigma=sig, eps=1.47e-15 / E_UNIT_J)
    if not cells:
        return p, np.zeros((0, 3)), np.zeros((0, 4))
    n_cells = int(round(number_density_m3 * nx * ny * nz * (DX_UM * 1e-6) ** 3))
    dr = le_reflect_distance(p)

    def inside(x):
        return (x[:, 0] + 0.5 > dr + 0.5) & (nx - 0.5 - x[:, 0] > dr + 0.5)

    X, q = workloads.fcc_cells(p, n_cells, seed, inside)
    return p, X, q


def x_profile(u, owner, p, axis_flow=2):
    """mean flow velocity of the fluid nodes in each plane x = const"""
    nx = p["nx"]
    x = np.arange(len(owner)) % nx
    fl = np.asarray(owner) == -1
    s = np.bincount(x[fl], weights=np.asarray(u)[fl, axis_flow], minlength=nx)
    c = np.bincount(x[fl], minlength=nx)
    return s / np.maximum(c, 1)


def central_shear_rate(prof, nx):
    """Sec. IV: the shear rate from a linear fit of v_z(x) over the central
    half of the box, away from the sheared plane"""
    x = np.arange(nx)
    sel = (x >= nx // 4) & (x < nx - nx // 4)
    return float(np.polyfit(x[sel], prof[sel], 1)[0])


def run_le(p, X, q, U, steps, samples=20, stream=None):
    """steps of the shear cell from rest under the offset U; over the second
    half, Delta p_LE and the v_z(x) profile sampled `samples` times.
    Returns dict(mu_rel = mu_app / mu of Eq. (mu), gamma_dot per step and in
    1/s, the mean profile, the momentum transfer per step, ms of stepping)."""
    import torch

    st = torch.cuda.current_stream() if stream is None else stream
    sim = bl.Simulation(p, stream=st.cuda_stream)
    sim.lees_edwards(U)
    if len(X):
        sim.set_particles(X, q)
    half = steps // 2
    every = max(2, (steps - half) // samples) // 2 * 2
    ms = 0.0

    def advance(k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sim.step(k)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    prof = []
    try:
        ms += advance(half)
        P0, n0 = sim.lees_edwards_momentum()
        done = half
        while done + every <= steps:
            ms += advance(every)
            done += every
            _, u, own = sim.fields()
            prof.append(x_profile(u, own, p))
        P1, n1 = sim.lees_edwards_momentum()
        sim.sync()
    finally:
        sim.close()
    v = np.mean(prof, axis=0)
    gd = central_shear_rate(v, p["nx"])
    P = (P1 - P0) / (n1 - n0)
    mu = p["rho0"] * (p["tau"] - 0.5) / 3.0
    return {"mu_rel": -P / (p["ny"] * p["nz"] * gd) / mu, "gamma_dot": gd, "gamma_dot_per_s": gd / DT_S,
            "profile": v, "P_per_step": P, "ms": ms, "steps": done}
