"""FP64 CPU oracle of the coupled LB / rigid-ellipsoid step (arXiv:1005.2594).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: the arithmetic lives in ``bloodlb_oracle.c`` (plain C,
double precision, compiled with ``-ffp-contract=off``) and this module only
marshals arguments through ctypes.

Parameters are passed as the plain dict produced by the seeded workload
generators (keys: nx, ny, nz, periodic, wall_vel, tau, rho0, g,
body_force_on_cells, R_par, R_perp, sig_par, sig_perp, eps, eps_w, sig_w, mu,
nu, chi_prime, r_cut, rho_p, move_particles).

Parity unpinned: nothing.  Every function here is pinned by a test under
``tests/test_oracle_*.py``; see the module docstrings there for the pins.
"""
import ctypes
import os

import numpy as np

from .build import build as _build

NQ = 19
FLUID = -1

_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("wall_vel", (ctypes.c_double * 3) * 8),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("body_force_on_cells", ctypes.c_int),
        ("R_par", ctypes.c_double), ("R_perp", ctypes.c_double),
        ("sig_par", ctypes.c_double), ("sig_perp", ctypes.c_double),
        ("eps", ctypes.c_double), ("eps_w", ctypes.c_double), ("sig_w", ctypes.c_double),
        ("mu", ctypes.c_double), ("nu", ctypes.c_double), ("chi_prime", ctypes.c_double),
        ("r_cut", ctypes.c_double), ("rho_p", ctypes.c_double),
        ("move_particles", ctypes.c_int),
    ]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        P = ctypes.POINTER(_Params)
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int32)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [P]
        L.orc_destroy.argtypes = [vp]
        L.orc_set_walls.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
        L.orc_set_particles.argtypes = [vp, ctypes.c_int, D, D, D, D]
        L.orc_step.argtypes = [vp, ctypes.c_int]
        L.orc_get_fields.argtypes = [vp, D, D, I]
        L.orc_get_populations.argtypes = [vp, D]
        L.orc_set_populations.argtypes = [vp, D]
        L.orc_get_particles.argtypes = [vp, D, D, D, D, D, D]
        L.orc_get_force_parts.argtypes = [vp, D, D, D, D, D, D, D]
        L.orc_get_pending.argtypes = [vp, D, D]
        L.orc_get_wall_parts.argtypes = [vp, D, D]
        L.orc_get_counters.argtypes = [vp, D, D]
        L.orc_boundary_links.restype = ctypes.c_long
        L.orc_boundary_links.argtypes = [vp, I, ctypes.c_long]
        L.orc_contact_links.restype = ctypes.c_long
        L.orc_contact_links.argtypes = [vp, I, ctypes.c_long]
        L.orc_cell_list.restype = ctypes.c_long
        L.orc_cell_list.argtypes = [vp, I, I, I]
        L.orc_totals.argtypes = [vp, D, D]
        L.orc_num_nodes.restype = ctypes.c_long
        L.orc_num_nodes.argtypes = [vp]
        L.orc_get_owner.argtypes = [vp, I]
        L.orc_equilibrium.argtypes = [ctypes.c_double, D, D]
        L.orc_axis.argtypes = [D, D]
        L.orc_pair.restype = ctypes.c_double
        L.orc_pair.argtypes = [P, D, D, D, D, D, D, D]
        L.orc_wall.restype = ctypes.c_double
        L.orc_wall.argtypes = [P, D, D, D, D]
        L.orc_integrate_one.argtypes = [P, D, D, D, D, D, D, D]
        L.orc_set_lees_edwards.restype = ctypes.c_int
        L.orc_set_lees_edwards.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        L.orc_get_lees_edwards.argtypes = [vp, D]
        _lib = L
    return _lib


def make_params(d: dict) -> _Params:
    p = _Params()
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
    for k in range(3):
        p.periodic[k] = int(d["periodic"][k])
        p.g[k] = float(d.get("g", (0.0, 0.0, 0.0))[k])
    wv = np.zeros((8, 3))
    given = np.asarray(d.get("wall_vel", np.zeros((8, 3))), dtype=np.float64)
    wv[: given.shape[0]] = given
    for w in range(8):
        for k in range(3):
            p.wall_vel[w][k] = float(wv[w, k])
    p.tau = float(d.get("tau", 1.0))
    p.rho0 = float(d.get("rho0", 1.0))
    p.body_force_on_cells = int(d.get("body_force_on_cells", 0))
    for key in ("R_par", "R_perp", "sig_par", "sig_perp", "eps", "eps_w", "sig_w", "mu", "nu",
                "chi_prime", "r_cut", "rho_p"):
        setattr(p, key, float(d.get(key, 0.0)))
    p.move_particles = int(d.get("move_particles", 1))
    return p


def equilibrium(rho, u):
    out = np.zeros(NQ)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_equilibrium(float(rho), _dp(uu), _dp(out))
    return out


def axis(q):
    qq = np.ascontiguousarray(q, dtype=np.float64)
    o = np.zeros(3)
    lib().orc_axis(_dp(qq), _dp(o))
    return o


def pair(params: dict, rvec, oi, oj):
    """phi, F_i, F_j, tau_i, tau_j of one cell pair; rvec = X_j - X_i."""
    p = make_params(params)
    r = np.ascontiguousarray(rvec, dtype=np.float64)
    a = np.ascontiguousarray(oi, dtype=np.float64)
    b = np.ascontiguousarray(oj, dtype=np.float64)
    Fi, Fj, Ti, Tj = (np.zeros(3) for _ in range(4))
    phi = lib().orc_pair(ctypes.byref(p), _dp(r), _dp(a), _dp(b), _dp(Fi), _dp(Fj), _dp(Ti), _dp(Tj))
    return phi, Fi, Fj, Ti, Tj


def wall(params: dict, rvec, oi):
    """phi, F_i, tau_i of a cell and one surface wall node; rvec = x_wall - X_i."""
    p = make_params(params)
    r = np.ascontiguousarray(rvec, dtype=np.float64)
    a = np.ascontiguousarray(oi, dtype=np.float64)
    Fi, Ti = np.zeros(3), np.zeros(3)
    phi = lib().orc_wall(ctypes.byref(p), _dp(r), _dp(a), _dp(Fi), _dp(Ti))
    return phi, Fi, Ti


def integrate_one(params: dict, X, q, V, L, F, T):
    """One leap-frog step of a single cell; returns new X, q, V, L, Omega."""
    p = make_params(params)
    X, q, V, L = (np.array(a, dtype=np.float64) for a in (X, q, V, L))
    F, T = np.ascontiguousarray(F, dtype=np.float64), np.ascontiguousarray(T, dtype=np.float64)
    Om = np.zeros(3)
    lib().orc_integrate_one(ctypes.byref(p), _dp(X), _dp(q), _dp(V), _dp(L), _dp(Om), _dp(F), _dp(T))
    return X, q, V, L, Om


class Oracle:
    """One lattice with its cells, stepped on the CPU in FP64."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._p = make_params(params)
        self._h = lib().orc_create(ctypes.byref(self._p))
        self.N = int(lib().orc_num_nodes(self._h))
        self.shape = (int(params["nz"]), int(params["ny"]), int(params["nx"]))
        self.np = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def set_walls(self, mask):
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        assert m.size == self.N
        lib().orc_set_walls(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))

    def set_particles(self, X, q, V=None, L=None):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        n = X.shape[0]
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(n, 4)
        V = np.zeros((n, 3)) if V is None else np.ascontiguousarray(V, dtype=np.float64).reshape(n, 3)
        L = np.zeros((n, 3)) if L is None else np.ascontiguousarray(L, dtype=np.float64).reshape(n, 3)
        lib().orc_set_particles(self._h, n, _dp(X), _dp(q), _dp(V), _dp(L))
        self.np = n

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros((self.N, 3))
        owner = np.zeros(self.N, dtype=np.int32)
        lib().orc_get_fields(self._h, _dp(rho), _dp(u), _ip(owner))
        return rho, u, owner

    def owner(self):
        o = np.zeros(self.N, dtype=np.int32)
        lib().orc_get_owner(self._h, _ip(o))
        return o

    def populations(self):
        pop = np.zeros((self.N, NQ))
        lib().orc_get_populations(self._h, _dp(pop))
        return pop

    def set_populations(self, pop):
        pop = np.ascontiguousarray(pop, dtype=np.float64).reshape(self.N, NQ)
        lib().orc_set_populations(self._h, _dp(pop))

    def particles(self):
        n = self.np
        out = {k: np.zeros((n, 3)) for k in ("F", "T", "X", "V", "L")}
        out["q"] = np.zeros((n, 4))
        lib().orc_get_particles(self._h, _dp(out["F"]), _dp(out["T"]), _dp(out["X"]), _dp(out["q"]),
                                _dp(out["V"]), _dp(out["L"]))
        return out

    def force_parts(self):
        n = self.np
        out = {k: np.zeros((n, 3)) for k in ("Fh", "Th", "Fc", "Tc", "Fp", "Tp", "Om")}
        lib().orc_get_force_parts(self._h, *(_dp(out[k]) for k in ("Fh", "Th", "Fc", "Tc", "Fp", "Tp", "Om")))
        return out

    def wall_parts(self):
        """wall-potential part (Eq. sigmaw) of the last step's Fp, Tp"""
        Fw, Tw = np.zeros((self.np, 3)), np.zeros((self.np, 3))
        lib().orc_get_wall_parts(self._h, _dp(Fw), _dp(Tw))
        return Fw, Tw

    def pending(self):
        PF, PT = np.zeros((self.np, 3)), np.zeros((self.np, 3))
        lib().orc_get_pending(self._h, _dp(PF), _dp(PT))
        return PF, PT

    def counters(self):
        c = np.zeros(7)
        wm = np.zeros((8, 3))
        lib().orc_get_counters(self._h, _dp(c), _dp(wm))
        return {"sumC": c[0], "mass_created": c[1], "mass_deleted": c[2], "n_covered": int(c[3]),
                "n_uncovered": int(c[4]), "n_switched": int(c[5]), "t": int(c[6]), "wallmom": wm}

    def set_lees_edwards(self, U, d_reflect=None):
        """Sec. IV's sheared plane between x = nx-1 and x = 0 (reading Q25):
        the image above slides along z with velocity offset U; cells reflect
        within d_reflect of the plane, by default max(sigma_perp, max(R) + 1),
        so that they never cover a node next to it.  Every axis periodic, no
        wall node."""
        p = self.params
        if d_reflect is None:
            d_reflect = max(p["sig_perp"], max(p["R_perp"], p["R_par"]) + 1.0)
        if lib().orc_set_lees_edwards(self._h, float(U), float(d_reflect)) != 0:
            raise ValueError("Lees-Edwards needs every axis periodic and no wall node")

    def lees_edwards(self):
        """z-momentum moved along +x across the sheared plane in the last step
        and summed since it was set, the steps summed, the cell reflections,
        and the crossings whose source was not fluid"""
        o = np.zeros(5)
        lib().orc_get_lees_edwards(self._h, _dp(o))
        return {"P": o[0], "P_sum": o[1], "steps": int(o[2]), "reflections": int(o[3]), "bad": int(o[4])}

    def boundary_links(self):
        n = lib().orc_boundary_links(self._h, None, 0)
        out = np.zeros((max(n, 1), 3), dtype=np.int32)
        lib().orc_boundary_links(self._h, _ip(out), n)
        return out[:n]

    def contact_links(self):
        n = lib().orc_contact_links(self._h, None, 0)
        out = np.zeros((max(n, 1), 3), dtype=np.int32)
        lib().orc_contact_links(self._h, _ip(out), n)
        return out[:n]

    def cell_list(self):
        nb = np.zeros(3, dtype=np.int32)
        nbins = lib().orc_cell_list(self._h, _ip(nb), None, None)
        start = np.zeros(nbins + 1, dtype=np.int32)
        ids = np.zeros(max(self.np, 1), dtype=np.int32)
        lib().orc_cell_list(self._h, _ip(nb), _ip(start), _ip(ids))
        return nb, start, ids[: self.np]

    def totals(self):
        m = ctypes.c_double(0.0)
        j = np.zeros(3)
        lib().orc_totals(self._h, ctypes.byref(m), _dp(j))
        return m.value, j
