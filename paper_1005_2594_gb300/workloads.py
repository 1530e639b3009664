"""Seeded synthetic workloads shaped like the paper's microvessel suspensions.

This module only generates inputs: lattice parameters, wall masks and cell
states drawn from seeded random numbers.  It holds none of the method's
arithmetic (no equilibrium, no potential, no inside test) and is the one
module that both the CUDA tests and the oracle tests use to make their inputs.

Conventions of the produced parameter dict (shared vocabulary of the library
and of the oracle):

* lattice ``nx, ny, nz``; ``periodic`` per axis; a non-periodic axis carries
  solid wall layers at index 0 and N-1, faces numbered x-,x+,y-,y+,z-,z+ =
  0..5; ``wall_vel`` is an 8 x 3 table of wall velocities (ids 6, 7 are for
  extra walls given by a mask);
* ``tau`` = 1 and ``rho0`` = 1 as in the paper; ``g`` body force (acceleration);
* cell half-axes ``R_par, R_perp`` (fluid coupling) and ``sig_par, sig_perp``
  (potential), strengths ``eps, eps_w``, wall sphere ``sig_w`` = 1/2,
  Gay-Berne exponents ``mu, nu`` with ``chi_prime``, neighbour radius
  ``r_cut``, cell density ``rho_p``.

Cell states: centres from random sequential addition, symmetry axes uniform
on the sphere with a uniform spin about them.  Two cells are accepted as
disjoint by the Perram-Wertheim contact function of two spheroids (a
textbook geometric test, evaluated on a grid of its parameter; cells may
touch but not overlap).  Above the jamming limit of random sequential addition the rest
of the cells go on a jittered lattice and may overlap, as in a dense fcc
start; the pair potential then pushes them apart.
"""
import math

import numpy as np

# ---------------------------------------------------------------------------
# parameters


def base_params(nx, ny, nz, periodic=(1, 1, 1), R=(7.0, 3.0), sigma=None, eps=1.0, eps_w=None,
                mu=0.0, nu=1.0, chi_prime=None, g=(0.0, 0.0, 0.0), body_force_on_cells=0,
                wall_vel=None, r_cut=None):
    """Parameter dict.  R = (R_perp, R_par).  sigma = (sig_perp, sig_par)
    defaults to R.  r_cut defaults to max(2.5 sigma0, 2 sig_perp), sigma0 =
    2 sig_par being the disc thickness."""
    R_perp, R_par = float(R[0]), float(R[1])
    if sigma is None:
        sigma = (R_perp, R_par)
    sig_perp, sig_par = float(sigma[0]), float(sigma[1])
    if r_cut is None:
        r_cut = max(2.5 * 2.0 * sig_par, 2.0 * sig_perp)
    if chi_prime is None:
        chi_prime = (sig_par ** 2 - sig_perp ** 2) / (sig_par ** 2 + sig_perp ** 2)
    wv = np.zeros((8, 3))
    if wall_vel is not None:
        for k, v in wall_vel.items():
            wv[k] = v
    return {
        "nx": int(nx), "ny": int(ny), "nz": int(nz), "periodic": tuple(int(p) for p in periodic),
        "wall_vel": wv, "tau": 1.0, "rho0": 1.0, "g": tuple(float(x) for x in g),
        "body_force_on_cells": int(body_force_on_cells),
        "R_par": R_par, "R_perp": R_perp, "sig_par": sig_par, "sig_perp": sig_perp,
        "eps": float(eps), "eps_w": float(eps if eps_w is None else eps_w), "sig_w": 0.5,
        "mu": float(mu), "nu": float(nu), "chi_prime": float(chi_prime), "r_cut": float(r_cut),
        "rho_p": 1.0, "move_particles": 1,
    }


def cell_volume(params):
    return 4.0 / 3.0 * math.pi * params["R_perp"] ** 2 * params["R_par"]


# ---------------------------------------------------------------------------
# orientations


def random_axes_and_quaternions(rng, n):
    """Symmetry axis uniform on S^2 and a uniform spin about it.  Returns the
    axes (n x 3) and the quaternions (w, x, y, z) that turn e_z into them."""
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    axes = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    psi = rng.uniform(0.0, 2.0 * math.pi, n)
    q = np.zeros((n, 4))
    for i in range(n):
        o = axes[i]
        # rotation taking e_z to o: about e_z x o by the angle between them
        ax = np.array([-o[1], o[0], 0.0])
        sa = np.linalg.norm(ax)
        ang = math.atan2(sa, o[2])
        if sa < 1e-300:
            ax = np.array([1.0, 0.0, 0.0])
            ang = 0.0 if o[2] > 0 else math.pi
        else:
            ax = ax / sa
        qa = np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)])
        qs = np.array([math.cos(psi[i] / 2), 0.0, 0.0, math.sin(psi[i] / 2)])
        q[i] = _qmul(qa, qs)
    return axes, q


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


# ---------------------------------------------------------------------------
# packing


def _support(Rp, Ra, axes, n):
    """support half-width of spheroids (equatorial Rp, polar Ra) along unit n"""
    c = np.sum(axes * n, axis=-1)
    return np.sqrt(Rp * Rp * (1.0 - c * c) + Ra * Ra * c * c)


_LAM = np.linspace(0.0, 1.0, 25)[1:-1]


def _contact_scale2(Rp, Ra, o, O, d):
    """Squared scale factor at which a spheroid with axis o at the origin and
    spheroids with axes O at displacements d would touch (Perram-Wertheim
    contact function, maximised over a grid of its parameter).  Values above
    1 mean the two spheroids are disjoint."""
    k = d.shape[0]
    eye = np.eye(3)
    Mi = Rp * Rp * eye + (Ra * Ra - Rp * Rp) * np.outer(o, o)
    Mj = Rp * Rp * eye[None] + (Ra * Ra - Rp * Rp) * np.einsum("ki,kj->kij", O, O)
    lam = _LAM[None, :, None, None]
    M = (1.0 - lam) * Mi[None, None] + lam * Mj[:, None]
    rhs = np.broadcast_to(d[:, None, :, None], (k, _LAM.size, 3, 1))
    sol = np.linalg.solve(M, rhs)[..., 0]
    F = _LAM[None, :] * (1.0 - _LAM[None, :]) * np.einsum("kli,ki->kl", sol, d)
    return F.max(axis=1)


def pack_cells(params, n, seed, lumen=None, clearance=1.0, max_fail=1500, refresh_every=1):
    """Seeded cell states (X n x 3, q n x 4) by random sequential addition.
    ``lumen`` is an optional callable (X, half_widths_xyz, radius) -> bool
    telling whether a cell fits inside the fluid region; walled axes keep the
    cell between the wall layers.  A candidate is accepted when every
    neighbour is disjoint from it after scaling both by ``clearance``.  After
    ``max_fail`` rejections in a row the addition stops and the remaining
    cells go on a jittered lattice.  The pool of free voxels is listed anew
    after every ``refresh_every`` placements (and every 64 rejections); large
    lattices use a coarser interval.  Returns X, q and the number placed
    without overlap."""
    rng = np.random.default_rng(seed)
    L = np.array([params["nx"], params["ny"], params["nz"]], dtype=np.float64)
    per = params["periodic"]
    Rp, Ra = params["R_perp"], params["R_par"]
    dmax = 2.0 * clearance * max(Rp, Ra)
    nb = np.maximum(1, np.floor(L / dmax).astype(int))
    bw = L / nb
    cap = 64
    bucket = -np.ones((nb[0], nb[1], nb[2], cap), dtype=np.int64)
    bcount = np.zeros((nb[0], nb[1], nb[2]), dtype=np.int64)
    X = np.zeros((n, 3))
    axes_all, q_all = random_axes_and_quaternions(rng, n)
    offs = np.array([[dx, dy, dz] for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    eye = np.eye(3)
    # candidate centres are drawn from unit voxels not yet known to be blocked:
    # a voxel is blocked once it lies inside a placed spheroid grown by
    # 0.9 R_par, where no new centre can fit
    shape = tuple(int(v) for v in L)
    blocked = np.zeros(shape, dtype=bool)
    for k in range(3):
        if not per[k]:
            idx = [slice(None)] * 3
            idx[k] = slice(0, int(math.ceil(1.0 + Ra + 0.5)))
            blocked[tuple(idx)] = True
            idx[k] = slice(int(math.floor(L[k] - 2.0 - Ra - 0.5)), None)
            blocked[tuple(idx)] = True
    gp, ga = Rp + 0.9 * Ra, 1.9 * Ra
    ext = int(math.ceil(gp)) + 1
    loc = np.arange(-ext, ext + 1)
    LZ, LY, LX = np.meshgrid(loc, loc, loc, indexing="ij")
    free = None
    placed = 0
    fails = 0
    since = 0  # placements since the pool was listed
    while placed < n and fails < max_fail:
        fails += 1
        if free is None or (fails % 64 == 1 and (fails > 1 or since >= refresh_every)):
            since = 0
            free = np.flatnonzero(~blocked.reshape(-1))
            if free.size == 0:
                break
        v = free[rng.integers(free.size)]
        if blocked.reshape(-1)[v]:
            continue
        if fails % 8 == 0:
            # a fresh orientation for this cell after repeated rejections
            a1, q1 = random_axes_and_quaternions(rng, 1)
            axes_all[placed], q_all[placed] = a1[0], q1[0]
        vi = np.array(np.unravel_index(v, shape), dtype=np.float64)
        x = vi + rng.uniform(0.0, 1.0, 3)
        o = axes_all[placed]
        hw = _support(Rp, Ra, o[None, :], eye)  # half-widths along x, y, z
        inside_box = True
        for k in range(3):
            if not per[k] and (x[k] < 1.0 + hw[k] + 0.5 or x[k] > L[k] - 2.0 - hw[k] - 0.5):
                inside_box = False
        if not inside_box:
            continue
        if lumen is not None and not lumen(x, hw, max(Rp, Ra)):
            continue
        b = np.floor(x / bw).astype(int) % nb
        nbk = (b[None, :] + offs) % nb[None, :]
        cand = bucket[nbk[:, 0], nbk[:, 1], nbk[:, 2]].reshape(-1)
        cand = np.unique(cand[cand >= 0])
        ok = True
        if cand.size:
            d = X[cand] - x
            for k in range(3):
                if per[k]:
                    d[:, k] -= L[k] * np.round(d[:, k] / L[k])
            near = np.einsum("ki,ki->k", d, d) < dmax * dmax
            if np.any(near):
                ok = bool(np.all(_contact_scale2(Rp, Ra, o, axes_all[cand[near]], d[near]) > clearance ** 2))
        if ok:
            X[placed] = x
            c = bcount[b[0], b[1], b[2]]
            if c >= cap:
                raise ValueError("bucket overflow")
            bucket[b[0], b[1], b[2], c] = placed
            bcount[b[0], b[1], b[2]] = c + 1
            # block the voxels of the grown spheroid around the new centre
            base = np.floor(x).astype(int)
            gx, gy, gz = base[0] + LX, base[1] + LY, base[2] + LZ
            dxv, dyv, dzv = gx + 0.5 - x[0], gy + 0.5 - x[1], gz + 0.5 - x[2]
            dpar = dxv * o[0] + dyv * o[1] + dzv * o[2]
            dd = dxv * dxv + dyv * dyv + dzv * dzv
            hit = dpar * dpar / (ga * ga) + (dd - dpar * dpar) / (gp * gp) <= 1.0
            gx, gy, gz = gx[hit] % shape[0], gy[hit] % shape[1], gz[hit] % shape[2]
            blocked[gx, gy, gz] = True
            placed += 1
            since += 1
            fails = 0
    n_free = placed
    if placed < n:
        # dense remainder: jittered lattice sites, overlaps allowed
        m = int(math.ceil((n - placed) ** (1.0 / 3.0))) + 1
        sites = []
        for k in range(3):
            lo = 1.0 + Rp + 0.5 if not per[k] else 0.0
            hi = L[k] - 2.0 - Rp - 0.5 if not per[k] else L[k]
            sites.append(np.linspace(lo, hi, m, endpoint=per[k] == 0))
        grid = np.stack(np.meshgrid(*sites, indexing="ij"), axis=-1).reshape(-1, 3)
        rng.shuffle(grid)
        for s in grid:
            if placed >= n:
                break
            hw = _support(Rp, Ra, axes_all[placed][None, :], eye)
            if lumen is not None and not lumen(s, hw, max(Rp, Ra)):
                continue
            X[placed] = s + rng.uniform(-0.25, 0.25, 3)
            placed += 1
        if placed < n:
            raise ValueError("could not place %d cells" % n)
    for k in range(3):
        if per[k]:
            X[:, k] = np.mod(X[:, k], L[k])
    return X, q_all, n_free


# ---------------------------------------------------------------------------
# named workloads


def small_shear(seed=1001, n_cells=20, mu=0.0):
    """32^3, tau = 1, periodic x,y, walls at z moving -/+0.01 along x; 20
    oblate cells R = (3.5, 3.5, 1.5), sigma0 = 3, eps = 1."""
    p = base_params(32, 32, 32, periodic=(1, 1, 0), R=(3.5, 1.5), eps=1.0, mu=mu, nu=1.0,
                    wall_vel={4: (-0.01, 0.0, 0.0), 5: (0.01, 0.0, 0.0)})
    X, q, _ = pack_cells(p, n_cells, seed)
    return p, X, q


def shear_cell(n=128, phi=0.30, U=0.02, seed=1002, R=(7.0, 3.0), mu=0.0, n_cells=None):
    """n^3 shear cell, walls at z moving -/+U along x, (7,7,3) cells at
    volume fraction phi of the box."""
    p = base_params(n, n, n, periodic=(1, 1, 0), R=R, eps=1.0, mu=mu,
                    wall_vel={4: (-U, 0.0, 0.0), 5: (U, 0.0, 0.0)})
    if n_cells is None:
        n_cells = int(round(phi * n ** 3 / cell_volume(p)))
    X, q, _ = pack_cells(p, n_cells, seed)
    return p, X, q


def duct(n=256, n_cells=8192, g=1e-6, seed=1003, R=(7.0, 3.0)):
    """n^3 duct: periodic x, walls y and z at rest, body force g along x on
    plasma and cells."""
    p = base_params(n, n, n, periodic=(1, 0, 0), R=R, eps=1.0, g=(g, 0.0, 0.0), body_force_on_cells=1)
    X, q, _ = pack_cells(p, n_cells, seed, refresh_every=64)
    return p, X, q


def ensemble(n_boxes=64, seed=1004, R=(7.0, 3.0), sizes=(48, 64, 80, 96), hct=(0.10, 0.20, 0.30, 0.40, 0.45),
             U=(0.005, 0.05), max_fail=300):
    """Uneven shear cells for rheology sweeps: cube edges drawn from
    ``sizes``, volume fractions from ``hct``, wall speeds uniform in ``U``
    (walls at z moving -/+U along x); (7,7,3) cells.  Returns a list of
    (params, X, q, description)."""
    rng = np.random.default_rng(seed)
    vol = 4.0 / 3.0 * math.pi * R[0] * R[0] * R[1]
    out = []
    for b in range(n_boxes):
        n = int(rng.choice(sizes))
        phi = float(rng.choice(hct))
        u = float(rng.uniform(U[0], U[1]))
        p = base_params(n, n, n, periodic=(1, 1, 0), R=R, eps=1.0, wall_vel={4: (-u, 0.0, 0.0), 5: (u, 0.0, 0.0)})
        m = max(1, int(round(phi * n ** 3 / vol)))
        X, q, _ = pack_cells(p, m, seed * 1000 + b, refresh_every=16, max_fail=max_fail)
        out.append((p, X, q, "%d^3, %d cells (%.0f %%), U = %.4f" % (n, m, 100 * phi, u)))
    return out


def tube_mask(params, radius, axis=0):
    """uint8 wall mask of a tube of the given radius about the axis through
    the box centre (mask value 7 -> wall id 6, at rest)."""
    nx, ny, nz = params["nx"], params["ny"], params["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = [(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0]
    coords = [x, y, z]
    others = [k for k in range(3) if k != axis]
    r2 = sum((coords[k] - c[k]) ** 2 for k in others)
    return np.where(r2 > radius * radius, 7, 0).astype(np.uint8).reshape(-1)


def fcc_cells(params, n, seed, inside):
    """Dense start for volume fractions where random addition jams: centres
    on a face-centred cubic lattice, jittered by up to 1/4 lattice unit, with
    uniformly random orientations; overlapping neighbours are allowed (the
    pair potential pushes them apart).  ``inside`` maps centres (m x 3) to a
    bool array of admissible ones; the lattice constant is the largest (in
    steps of 1 %) giving at least n admissible sites, of which a seeded
    random choice of n is kept.  Returns X, q."""
    rng = np.random.default_rng(seed)
    L = np.array([params["nx"], params["ny"], params["nz"]], dtype=np.float64)
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    a = (4.0 * float(np.prod(L)) / n) ** (1.0 / 3.0)
    for _ in range(400):
        m = np.floor(L / a).astype(int)
        g = np.stack(np.meshgrid(*(np.arange(k) for k in m), indexing="ij"), axis=-1).reshape(-1, 1, 3)
        sites = ((g + basis[None]) * a).reshape(-1, 3) + 0.25 * a
        sites = sites[inside(sites)]
        if len(sites) >= n:
            break
        a *= 0.99
    else:
        raise ValueError("could not place %d cells" % n)
    sites = sites[rng.permutation(len(sites))[:n]]
    X = sites + rng.uniform(-0.25, 0.25, (n, 3))
    _, q = random_axes_and_quaternions(rng, n)
    return np.mod(X, L), q


def tube(nx=512, ny=256, nz=256, radius=120.0, hct=0.35, g=1e-6, seed=1005, R=(7.0, 3.0), n_cells=None):
    """periodic box with a tube along x of the given radius, body force g
    along x on plasma and cells, cells at hematocrit hct of the lumen volume
    on a jittered fcc start (35 % is beyond where random addition jams).
    Returns params, X, q, wall mask."""
    p = base_params(nx, ny, nz, periodic=(1, 1, 1), R=R, eps=1.0, g=(g, 0.0, 0.0), body_force_on_cells=1)
    if n_cells is None:
        n_cells = int(round(hct * math.pi * radius ** 2 * nx / cell_volume(p)))
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    rmax = max(p["R_perp"], p["R_par"])

    def inside(x):
        return np.hypot(x[:, 1] - cy, x[:, 2] - cz) + rmax + 1.0 < radius

    X, q = fcc_cells(p, n_cells, seed, inside)
    return p, X, q, tube_mask(p, radius, axis=0)


def _axis_quaternion(ax):
    """quaternion (w, x, y, z) turning e_z into the unit vector ax"""
    ax = np.asarray(ax, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    v = np.array([-ax[1], ax[0], 0.0])
    s = np.linalg.norm(v)
    ang = math.atan2(s, ax[2])
    v = v / s if s > 1e-300 else np.array([1.0, 0.0, 0.0])
    return np.array([math.cos(ang / 2), *(math.sin(ang / 2) * v)])


def sediment_stacks(mu=0.0, seed=1011):
    """Contacts that last: the small shear cell (32^3, walls z moving -/+0.01
    along x, cells R = (3.5, 1.5)) with the paper's potential range and
    strength (sigma = 12/11 R, eps = eps_w = 0.05), cells 1.5 times denser than
    the plasma under a body force g = -5e-5 along z on plasma and cells.
    Stacks of nearly face-on cells rest on the lower wall (within the wall
    sphere of Eq. sigmaw, each on the one below within its pair range), two
    side-on cells lie on the wall, and a pair and a single cell float higher
    up, the pair within its range.  Returns params, X, q."""
    R = (3.5, 1.5)
    sig = (R[0] * 12.0 / 11.0, R[1] * 12.0 / 11.0)
    p = base_params(32, 32, 32, periodic=(1, 1, 0), R=R, sigma=sig, eps=0.05, mu=mu,
                    g=(0.0, 0.0, -5e-5), body_force_on_cells=1,
                    wall_vel={4: (-0.01, 0.0, 0.0), 5: (0.01, 0.0, 0.0)})
    p["rho_p"] = 1.5
    rng = np.random.default_rng(seed)

    def tilted(t, a):
        return np.array([math.cos(t / 2), math.sin(t / 2) * math.cos(a), math.sin(t / 2) * math.sin(a), 0.0])

    X, q = [], []
    face = math.sqrt(sig[1] ** 2 + 0.25)  # face-on reach of the wall sphere from the wall node layer z = 0
    for (x, y, h) in ((6.0, 6.0, 2), (20.0, 8.0, 3), (9.0, 22.0, 2), (24.0, 24.0, 1)):
        z = face - 0.12
        for _ in range(h):
            X.append([x + rng.uniform(-0.5, 0.5), y + rng.uniform(-0.5, 0.5), z])
            q.append(tilted(rng.uniform(0.0, 0.15), rng.uniform(0.0, 2 * math.pi)))
            z += 2 * sig[1] - 0.10
    side = math.sqrt(sig[0] ** 2 + 0.25)
    for (x, y) in ((15.0, 16.0), (28.0, 14.0)):
        X.append([x, y, side - 0.10])
        a = rng.uniform(0.0, 2 * math.pi)
        q.append(np.array([math.cos(math.pi / 4), math.sin(math.pi / 4) * math.cos(a),
                           math.sin(math.pi / 4) * math.sin(a), 0.0]))
    for (x, y, z) in ((16.0, 4.0, 18.0), (16.0 + 2 * sig[0] - 0.2, 4.3, 18.2), (5.0, 14.0, 22.0)):
        X.append([x, y, z])
        q.append(tilted(rng.uniform(0.0, 0.5), rng.uniform(0.0, 2 * math.pi)))
    q = np.array(q)
    return p, np.array(X), q / np.linalg.norm(q, axis=1)[:, None]


def tube_contacts(mu=0.0, seed=1013, radius=11.0):
    """Cells resting on the wall of a tube given as a wall mask: 40 x 28 x 28
    periodic box, tube of the given radius along x, body force (2e-5, 0, -5e-5)
    on plasma and cells, cells 1.5 times denser than the plasma, sigma =
    12/11 R, eps = eps_w = 0.05.  Four cells lie nearly face-on on the lower
    part of the tube wall (within the wall sphere of its surface nodes), two
    of them with a second cell resting on top.  Returns params, X, q, mask."""
    R = (3.5, 1.5)
    sig = (R[0] * 12.0 / 11.0, R[1] * 12.0 / 11.0)
    nx, ny, nz = 40, 28, 28
    p = base_params(nx, ny, nz, periodic=(1, 1, 1), R=R, sigma=sig, eps=0.05, mu=mu,
                    g=(2e-5, 0.0, -5e-5), body_force_on_cells=1)
    p["rho_p"] = 1.5
    mask = tube_mask(p, radius, axis=0)
    rng = np.random.default_rng(seed)
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    face = math.sqrt(sig[1] ** 2 + 0.25)
    X, q = [], []
    for k, x in enumerate((5.0, 14.0, 23.0, 32.0)):
        th = rng.uniform(-0.4, 0.4)
        d = radius + 0.5 - face + 0.05
        nvec = np.array([0.0, math.sin(th), -math.cos(th)])  # outward wall normal at the cell
        X.append([x, cy + d * nvec[1], cz + d * nvec[2]])
        qa = _axis_quaternion(nvec + rng.uniform(-0.1, 0.1, 3))
        q.append(qa)
        if k % 2 == 0:
            X.append([x + 0.3, X[-1][1] - (2 * sig[1] - 0.1) * nvec[1], X[-1][2] - (2 * sig[1] - 0.1) * nvec[2]])
            q.append(qa)
    return p, np.array(X), np.array(q), mask


def vessel_loop(nx=1024, ny=256, nz=64, r0=16.0, h=64.0, wall_id=6):
    """uint8 wall mask of a synthetic vessel network for the indexed lattice:
    a parent vessel of radius r0 along x through the box centre (periodic in
    x) that splits into two daughters of radius r0 2^(-1/3) (Murray's law,
    the parent's cube equal to the sum of the daughters'), offset by -+h in
    y, which run parallel and rejoin -- the bifurcation and confluence of a
    microvascular loop.  Each vessel is the union of capsules (segments with
    round ends) along its centre line; nodes outside every capsule are wall
    (mask value wall_id + 1).  Returns the mask (N bytes) and the lumen's
    centre-line segments ((x0, y0), (x1, y1), radius) in the z = (nz-1)/2
    plane."""
    rd = r0 * 2.0 ** (-1.0 / 3.0)
    yc, zc = (ny - 1) / 2.0, (nz - 1) / 2.0
    xa, xb, xc, xd = 0.125 * nx, 0.375 * nx, 0.625 * nx, 0.875 * nx
    segs = [((-r0, yc), (xa, yc), r0), ((xd, yc), (nx + r0, yc), r0)]
    for s in (-1.0, 1.0):
        segs += [((xa, yc), (xb, yc + s * h), rd), ((xb, yc + s * h), (xc, yc + s * h), rd),
                 ((xc, yc + s * h), (xd, yc), rd)]
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    # squared in-plane distance to each centre line, then one z slice at a time
    d2xy = []
    for (x0, y0), (x1, y1), r in segs:
        dx, dy = x1 - x0, y1 - y0
        t = np.clip(((x - x0) * dx + (y - y0) * dy) / (dx * dx + dy * dy), 0.0, 1.0)
        d2xy.append(((x - (x0 + t * dx)) ** 2 + (y - (y0 + t * dy)) ** 2, r))
    mask = np.empty((nz, ny, nx), dtype=np.uint8)
    for k in range(nz):
        inside = np.zeros((ny, nx), dtype=bool)
        for d2, r in d2xy:
            inside |= d2 + (k - zc) ** 2 < r * r
        mask[k] = np.where(inside, 0, wall_id + 1)
    return mask.reshape(-1), segs
