"""Python binding of the CUDA library ``libbloodlb.so`` (C ABI in
``include/bloodlb.h``): argument marshalling only.  Every step of the coupled
time step runs in the library's kernels; there is no CPU fallback, and
loading fails loudly if the library has not been built.

The functions carry the C names.  Arrays are numpy arrays (host) or CUDA
tensors (``on_device`` read-outs).  Parameters come as the plain dict of
``paper_1005_2594_gb300.workloads``.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbloodlb.so")

BL_OK = 0
BL_EINVAL = -1
BL_ENOMEM = -2
BL_EUNSTABLE = -3
BL_EOVERFLOW = -4
BL_EBARRIER = -5
BL_ECUDA = -6
BL_ESTATE = -7

BL_STORE_F32 = 0
BL_STORE_BF16 = 1
BL_STORE_F16 = 2

TIMING_GROUPS = ("lattice_sweep", "cell_list", "potentials", "leapfrog_claims", "resolve_fill")

ABI_FUNCTIONS = (
    "bl_lb_init", "bl_walls_set", "bl_particles_set", "bl_step", "bl_fields_get", "bl_forces_get",
    "bl_force_parts_get", "bl_wall_momentum_get", "bl_lees_edwards_set", "bl_lees_edwards_get",
    "bl_populations_get", "bl_populations_set",
    "bl_boundary_links_get", "bl_contact_links_get", "bl_cell_links_get", "bl_cell_list_get", "bl_cell_list_build_static",
    "bl_sweep_variant", "bl_autotune", "bl_ensemble_create", "bl_ensemble_step", "bl_ensemble_sync",
    "bl_ensemble_destroy", "bl_mlp_create", "bl_mlp_params_set", "bl_mlp_params_get", "bl_mlp_forward",
    "bl_mlp_grad", "bl_mlp_adam", "bl_mlp_sync", "bl_mlp_destroy", "bl_mlp_attach", "bl_mlp_attach_range", "bl_pair_features",
    "bl_timing_enable",
    "bl_timing_read", "bl_launch_count", "bl_sync", "bl_last_error", "bl_destroy",
    "bl_sparse_index_build", "bl_sparse_init", "bl_sparse_step", "bl_sparse_fields_get", "bl_sparse_populations_get",
    "bl_sparse_populations_set", "bl_sparse_wall_momentum_get", "bl_sparse_sync", "bl_sparse_nodes",
    "bl_sparse_launch_count", "bl_sparse_last_error", "bl_sparse_destroy",
)


class BloodLBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bloodlb error %d: %s" % (code, msg))
        self.code = code


class bl_lb_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("wall_vel", (ctypes.c_double * 3) * 8),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("store_dtype", ctypes.c_int),
        ("body_force_on_cells", ctypes.c_int),
    ]


class bl_particle_params(ctypes.Structure):
    _fields_ = [
        ("R_par", ctypes.c_double), ("R_perp", ctypes.c_double),
        ("sig_par", ctypes.c_double), ("sig_perp", ctypes.c_double),
        ("eps", ctypes.c_double), ("eps_w", ctypes.c_double), ("sig_w", ctypes.c_double),
        ("mu", ctypes.c_double), ("nu", ctypes.c_double), ("chi_prime", ctypes.c_double),
        ("r_cut", ctypes.c_double), ("rho_p", ctypes.c_double),
        ("move_particles", ctypes.c_int), ("reserved", ctypes.c_int),
    ]


_lib = None


def lib():
    """Load the CUDA library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library %s is not built; run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, D, I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    F = ctypes.POINTER(ctypes.c_float)
    i64 = ctypes.c_int64
    sig = {
        "bl_lb_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(bl_lb_params), vp]),
        "bl_walls_set": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_uint8)]),
        "bl_particles_set": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(bl_particle_params), D, D, D, D]),
        "bl_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "bl_fields_get": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
        "bl_forces_get": (ctypes.c_int, [vp, D, D, D, D, D, D]),
        "bl_force_parts_get": (ctypes.c_int, [vp, D, D, D, D, D, D, D]),
        "bl_wall_momentum_get": (ctypes.c_int, [vp, D]),
        "bl_lees_edwards_set": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double]),
        "bl_lees_edwards_get": (ctypes.c_int, [vp, D, ctypes.POINTER(i64)]),
        "bl_populations_get": (ctypes.c_int, [vp, D]),
        "bl_populations_set": (ctypes.c_int, [vp, D]),
        "bl_boundary_links_get": (ctypes.c_int, [vp, I, i64, ctypes.POINTER(i64)]),
        "bl_contact_links_get": (ctypes.c_int, [vp, I, i64, ctypes.POINTER(i64)]),
        "bl_cell_links_get": (ctypes.c_int, [vp, I, i64, ctypes.POINTER(i64)]),
        "bl_cell_list_get": (ctypes.c_int, [vp, I, I, I]),
        "bl_cell_list_build_static": (ctypes.c_int, [vp, ctypes.c_int, I, ctypes.c_double, I, vp, vp, vp]),
        "bl_sweep_variant": (ctypes.c_int, [vp, ctypes.c_int]),
        "bl_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "bl_ensemble_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, vp]),
        "bl_ensemble_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "bl_ensemble_sync": (ctypes.c_int, [vp]),
        "bl_ensemble_destroy": (None, [vp]),
        "bl_mlp_create": (ctypes.c_int, [ctypes.POINTER(vp), vp]),
        "bl_mlp_params_set": (ctypes.c_int, [vp, F, F]),
        "bl_mlp_params_get": (ctypes.c_int, [vp, F, F]),
        "bl_mlp_forward": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        "bl_mlp_grad": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, F, F]),
        "bl_mlp_adam": (ctypes.c_int, [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "bl_mlp_sync": (ctypes.c_int, [vp]),
        "bl_mlp_destroy": (None, [vp]),
        "bl_mlp_attach": (ctypes.c_int, [vp, vp, ctypes.c_double]),
        "bl_mlp_attach_range": (ctypes.c_int, [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double]),
        "bl_pair_features": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        "bl_timing_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "bl_timing_read": (ctypes.c_int, [vp, D, ctypes.POINTER(i64), ctypes.c_int]),
        "bl_launch_count": (i64, [vp]),
        "bl_sync": (ctypes.c_int, [vp]),
        "bl_last_error": (ctypes.c_char_p, [vp]),
        "bl_destroy": (None, [vp]),
        "bl_sparse_index_build": (ctypes.c_int, [ctypes.POINTER(bl_lb_params), ctypes.POINTER(ctypes.c_uint8),
                                                 ctypes.POINTER(i64), I, I]),
        "bl_sparse_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(bl_lb_params),
                                          ctypes.POINTER(ctypes.c_uint8), vp]),
        "bl_sparse_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "bl_sparse_fields_get": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "bl_sparse_populations_get": (ctypes.c_int, [vp, D]),
        "bl_sparse_populations_set": (ctypes.c_int, [vp, D]),
        "bl_sparse_wall_momentum_get": (ctypes.c_int, [vp, D]),
        "bl_sparse_sync": (ctypes.c_int, [vp]),
        "bl_sparse_nodes": (i64, [vp]),
        "bl_sparse_launch_count": (i64, [vp]),
        "bl_sparse_last_error": (ctypes.c_char_p, [vp]),
        "bl_sparse_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def lb_params(d: dict, store_dtype=BL_STORE_F32) -> bl_lb_params:
    p = bl_lb_params()
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
    wv = np.zeros((8, 3))
    given = np.asarray(d.get("wall_vel", np.zeros((8, 3))), dtype=np.float64)
    wv[: given.shape[0]] = given
    for k in range(3):
        p.periodic[k] = int(d["periodic"][k])
        p.g[k] = float(d.get("g", (0.0, 0.0, 0.0))[k])
    for w in range(8):
        for k in range(3):
            p.wall_vel[w][k] = float(wv[w, k])
    p.tau = float(d.get("tau", 1.0))
    p.rho0 = float(d.get("rho0", 1.0))
    p.store_dtype = int(store_dtype)
    p.body_force_on_cells = int(d.get("body_force_on_cells", 0))
    return p


def particle_params(d: dict) -> bl_particle_params:
    p = bl_particle_params()
    for key in ("R_par", "R_perp", "sig_par", "sig_perp", "eps", "eps_w", "sig_w", "mu", "nu", "chi_prime",
                "r_cut", "rho_p"):
        setattr(p, key, float(d.get(key, 0.0)))
    p.move_particles = int(d.get("move_particles", 1))
    return p


def _check(ctx, rc):
    if rc != BL_OK:
        msg = lib().bl_last_error(ctx)
        raise BloodLBError(rc, msg.decode() if msg else "")
    return rc


# --- the C functions, one to one -------------------------------------------


def bl_lb_init(params: dict, stream=None, store_dtype=BL_STORE_F32):
    ctx = ctypes.c_void_p()
    p = lb_params(params, store_dtype)
    rc = lib().bl_lb_init(ctypes.byref(ctx), ctypes.byref(p), ctypes.c_void_p(stream or 0))
    if rc != BL_OK:
        raise BloodLBError(rc, "bl_lb_init")
    return ctx


def bl_walls_set(ctx, mask):
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    return _check(ctx, lib().bl_walls_set(ctx, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))


def bl_particles_set(ctx, params: dict, X, q, V=None, L=None):
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    n = X.shape[0]
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(n, 4)
    V = np.zeros((n, 3)) if V is None else np.ascontiguousarray(V, dtype=np.float64).reshape(n, 3)
    L = np.zeros((n, 3)) if L is None else np.ascontiguousarray(L, dtype=np.float64).reshape(n, 3)
    pp = particle_params(params)
    return _check(ctx, lib().bl_particles_set(ctx, n, ctypes.byref(pp), _dp(X), _dp(q), _dp(V), _dp(L)))


def bl_step(ctx, nsteps=1):
    return _check(ctx, lib().bl_step(ctx, int(nsteps)))


def bl_sync(ctx):
    return _check(ctx, lib().bl_sync(ctx))


def bl_sweep_variant(ctx, variant):
    return _check(ctx, lib().bl_sweep_variant(ctx, int(variant)))


def bl_autotune(ctx, trial_steps=20):
    """Times the sweep variants on this context (it advances by the trial
    steps), keeps the fastest and returns its number."""
    choice = ctypes.c_int(-1)
    _check(ctx, lib().bl_autotune(ctx, int(trial_steps), ctypes.byref(choice)))
    return choice.value


def bl_ensemble_create(ctxs, stream=None):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    ens = ctypes.c_void_p()
    rc = lib().bl_ensemble_create(ctypes.byref(ens), arr, len(ctxs), ctypes.c_void_p(stream or 0))
    if rc != BL_OK:
        raise BloodLBError(rc, "bl_ensemble_create")
    return ens


def bl_ensemble_step(ens, nsteps=1):
    rc = lib().bl_ensemble_step(ens, int(nsteps))
    if rc != BL_OK:
        raise BloodLBError(rc, "bl_ensemble_step")
    return rc


def bl_ensemble_sync(ens):
    rc = lib().bl_ensemble_sync(ens)
    if rc != BL_OK:
        raise BloodLBError(rc, "bl_ensemble_sync")
    return rc


def bl_ensemble_destroy(ens):
    if ens:
        lib().bl_ensemble_destroy(ens)


MLP_NPAR = 5510


def _fp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _mcheck(rc, what):
    if rc != BL_OK:
        raise BloodLBError(rc, what)
    return rc


def bl_mlp_create(stream=None):
    m = ctypes.c_void_p()
    _mcheck(lib().bl_mlp_create(ctypes.byref(m), ctypes.c_void_p(stream or 0)), "bl_mlp_create")
    return m


def bl_mlp_params_set(m, theta=None, norm=None):
    t = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32).reshape(MLP_NPAR)
    n = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32).reshape(40)
    return _mcheck(lib().bl_mlp_params_set(m, _fp(t), _fp(n)), "bl_mlp_params_set")


def bl_mlp_params_get(m):
    t, n = np.zeros(MLP_NPAR, dtype=np.float32), np.zeros(40, dtype=np.float32)
    _mcheck(lib().bl_mlp_params_get(m, _fp(t), _fp(n)), "bl_mlp_params_get")
    return t, n


def bl_mlp_forward(m, x, y):
    """x, y: CUDA float32 tensors (B x 14, B x 6)"""
    return _mcheck(lib().bl_mlp_forward(m, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                        ctypes.c_void_p(y.data_ptr())), "bl_mlp_forward")


def bl_mlp_grad(m, x, y, want_grad=False):
    """x, y: CUDA float32 tensors; returns (loss, grad or None)"""
    loss = np.zeros(1, dtype=np.float32)
    g = np.zeros(MLP_NPAR, dtype=np.float32) if want_grad else None
    _mcheck(lib().bl_mlp_grad(m, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), int(x.shape[0]),
                              _fp(loss), _fp(g)), "bl_mlp_grad")
    return float(loss[0]), g


def bl_mlp_adam(m, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    return _mcheck(lib().bl_mlp_adam(m, float(lr), float(beta1), float(beta2), float(eps)), "bl_mlp_adam")


def bl_mlp_sync(m):
    return _mcheck(lib().bl_mlp_sync(m), "bl_mlp_sync")


def bl_mlp_destroy(m):
    if m:
        lib().bl_mlp_destroy(m)


def bl_mlp_attach(ctx, m, gap_cut):
    return _check(ctx, lib().bl_mlp_attach(ctx, m, float(gap_cut)))


def bl_mlp_attach_range(ctx, m, gap_lo, gap_hi, speed_lo=0.0, speed_hi=float("inf")):
    return _check(ctx, lib().bl_mlp_attach_range(ctx, m, float(gap_lo), float(gap_hi), float(speed_lo),
                                                  float(min(speed_hi, 1e300))))


def bl_pair_features(ctx, pairs, out):
    """pairs: CUDA int32 tensor (n x 2); out: CUDA float32 tensor (n x 14)"""
    return _check(ctx, lib().bl_pair_features(ctx, ctypes.c_void_p(pairs.data_ptr()), int(pairs.shape[0]),
                                              ctypes.c_void_p(out.data_ptr())))


def bl_fields_get(ctx, N, rho=None, u=None, owner=None, on_device=False):
    """Host: returns (rho, u, owner) numpy arrays.  Device: pass CUDA tensors
    (float64 N, float64 N x 3, int32 N) and they are written on the stream."""
    if on_device:
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)
        _check(ctx, lib().bl_fields_get(ctx, ptr(rho), ptr(u), ptr(owner), 1))
        return rho, u, owner
    rho = np.zeros(N)
    u = np.zeros((N, 3))
    owner = np.zeros(N, dtype=np.int32)
    _check(ctx, lib().bl_fields_get(ctx, ctypes.c_void_p(rho.ctypes.data), ctypes.c_void_p(u.ctypes.data),
                                    ctypes.c_void_p(owner.ctypes.data), 0))
    return rho, u, owner


def bl_forces_get(ctx, n):
    out = {k: np.zeros((n, 3)) for k in ("F", "T", "X", "V", "L")}
    out["q"] = np.zeros((n, 4))
    _check(ctx, lib().bl_forces_get(ctx, _dp(out["F"]), _dp(out["T"]), _dp(out["X"]), _dp(out["q"]),
                                    _dp(out["V"]), _dp(out["L"])))
    return out


def bl_force_parts_get(ctx, n):
    keys = ("Fh", "Th", "Fp", "Tp", "Om", "PF", "PT")
    out = {k: np.zeros((n, 3)) for k in keys}
    _check(ctx, lib().bl_force_parts_get(ctx, *(_dp(out[k]) for k in keys)))
    return out


def bl_wall_momentum_get(ctx):
    out = np.zeros((8, 3))
    _check(ctx, lib().bl_wall_momentum_get(ctx, _dp(out)))
    return out


def bl_lees_edwards_set(ctx, U, d_reflect=0.0):
    _check(ctx, lib().bl_lees_edwards_set(ctx, float(U), float(d_reflect)))


def bl_lees_edwards_get(ctx):
    P = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(ctx, lib().bl_lees_edwards_get(ctx, ctypes.byref(P), ctypes.byref(n)))
    return P.value, int(n.value)


def bl_populations_get(ctx, N):
    pop = np.zeros((N, 19))
    _check(ctx, lib().bl_populations_get(ctx, _dp(pop)))
    return pop


def bl_populations_set(ctx, pop):
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    return _check(ctx, lib().bl_populations_set(ctx, _dp(pop)))


def _links(fn, ctx):
    cnt = ctypes.c_int64(0)
    _check(ctx, fn(ctx, None, 0, ctypes.byref(cnt)))
    out = np.zeros((max(cnt.value, 1), 3), dtype=np.int32)
    _check(ctx, fn(ctx, _ip(out), cnt.value, ctypes.byref(cnt)))
    return out[: cnt.value]


def bl_boundary_links_get(ctx):
    return _links(lib().bl_boundary_links_get, ctx)


def bl_contact_links_get(ctx):
    return _links(lib().bl_contact_links_get, ctx)


def bl_cell_links_get(ctx):
    return _links(lib().bl_cell_links_get, ctx)


def bl_cell_list_get(ctx, n):
    nb = np.zeros(3, dtype=np.int32)
    _check(ctx, lib().bl_cell_list_get(ctx, _ip(nb), None, None))
    start = np.zeros(int(np.prod(nb)) + 1, dtype=np.int32)
    ids = np.zeros(max(n, 1), dtype=np.int32)
    _check(ctx, lib().bl_cell_list_get(ctx, _ip(nb), _ip(start), _ip(ids)))
    return nb, start, ids[:n]


def bl_cell_list_build_static(X_dev, n, dims, r_cut, start_dev, ids_dev, stream=None):
    """Cell list into device arrays without any device allocation (see the
    header): X_dev, start_dev, ids_dev are CUDA tensors (float64 n x 3,
    int32 nbins + 1, int32 n).  Returns (status, nb)."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    nb = np.zeros(3, dtype=np.int32)
    rc = lib().bl_cell_list_build_static(ctypes.c_void_p(X_dev.data_ptr() if n else 0), int(n), _ip(d),
                                         float(r_cut), _ip(nb), ctypes.c_void_p(start_dev.data_ptr()),
                                         ctypes.c_void_p(ids_dev.data_ptr() if n else 0),
                                         ctypes.c_void_p(stream or 0))
    return rc, nb


def bl_timing_enable(ctx, enable=True):
    return _check(ctx, lib().bl_timing_enable(ctx, 1 if enable else 0))


def bl_timing_read(ctx):
    n = len(TIMING_GROUPS)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().bl_timing_read(ctx, _dp(ms), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n))
    return {g: (ms[i], int(cnt[i])) for i, g in enumerate(TIMING_GROUPS)}


def bl_launch_count(ctx):
    return int(lib().bl_launch_count(ctx))


def bl_last_error(ctx):
    m = lib().bl_last_error(ctx)
    return m.decode() if m else ""


def bl_destroy(ctx):
    if ctx:
        lib().bl_destroy(ctx)


# --- convenience wrapper ------------------------------------------------------


class Simulation:
    """One lattice with its cells on the GPU (owns one library context)."""

    def __init__(self, params: dict, store_dtype=BL_STORE_F32, stream=None, wall_mask=None):
        self.params = dict(params)
        self.N = int(params["nx"]) * int(params["ny"]) * int(params["nz"])
        self.ctx = bl_lb_init(params, stream=stream, store_dtype=store_dtype)
        self.n = 0
        if wall_mask is not None:
            bl_walls_set(self.ctx, wall_mask)

    def close(self):
        if getattr(self, "ctx", None):
            bl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, X, q, V=None, L=None):
        bl_particles_set(self.ctx, self.params, X, q, V, L)
        self.n = np.asarray(X).reshape(-1, 3).shape[0]

    def step(self, n=1):
        bl_step(self.ctx, n)

    def sync(self):
        bl_sync(self.ctx)

    def fields(self):
        return bl_fields_get(self.ctx, self.N)

    def owner(self):
        return self.fields()[2]

    def particles(self):
        return bl_forces_get(self.ctx, self.n)

    def force_parts(self):
        return bl_force_parts_get(self.ctx, self.n)

    def populations(self):
        return bl_populations_get(self.ctx, self.N)

    def set_populations(self, pop):
        bl_populations_set(self.ctx, pop)

    def boundary_links(self):
        return bl_boundary_links_get(self.ctx)

    def contact_links(self):
        return bl_contact_links_get(self.ctx)

    def cell_links(self):
        """the step's own per-cell bounce-link lists, (node, r, cell) sorted"""
        return bl_cell_links_get(self.ctx)

    def cell_list(self):
        return bl_cell_list_get(self.ctx, self.n)

    def wall_momentum(self):
        return bl_wall_momentum_get(self.ctx)

    def lees_edwards(self, U, d_reflect=0.0):
        """shear the box across the plane between x = nx-1 and x = 0 with
        velocity offset U along z (Sec. IV); d_reflect <= 0: the default
        reflection distance"""
        bl_lees_edwards_set(self.ctx, U, d_reflect)

    def lees_edwards_momentum(self):
        """(z-momentum moved along +x across the plane, summed; steps summed)"""
        return bl_lees_edwards_get(self.ctx)

    def autotune(self, trial_steps=20):
        return bl_autotune(self.ctx, trial_steps)

    def sweep_variant(self, variant):
        bl_sweep_variant(self.ctx, variant)


class Ensemble:
    """Independent simulations advanced together (bl_ensemble_*); the
    members must outlive the ensemble."""

    def __init__(self, sims, stream=None):
        self.sims = list(sims)
        self.ens = bl_ensemble_create([s.ctx for s in self.sims], stream)

    def step(self, n=1):
        bl_ensemble_step(self.ens, n)

    def sync(self):
        bl_ensemble_sync(self.ens)

    def close(self):
        if getattr(self, "ens", None):
            bl_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- the indexed lattice of vessel networks ---------------------------------


def _sparse_check(h, rc):
    if rc != BL_OK:
        msg = lib().bl_sparse_last_error(h) if h else b""
        raise BloodLBError(rc, msg.decode() if msg else "")
    return rc


def _mask_ptr(mask, N):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    if m.size != N:
        raise ValueError("mask has %d entries, the lattice %d nodes" % (m.size, N))
    return m, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def bl_sparse_index_build(params: dict, mask=None):
    """host-only index of a lattice: (dense index of each fluid node, the
    18 x n_fluid neighbour table, fluid index or -1 - wall id)"""
    p = lb_params(params)
    N = int(params["nx"]) * int(params["ny"]) * int(params["nz"])
    m, mp = _mask_ptr(mask, N)
    n = ctypes.c_int64(0)
    _sparse_check(None, lib().bl_sparse_index_build(ctypes.byref(p), mp, ctypes.byref(n), None, None))
    dense = np.zeros(max(n.value, 1), dtype=np.int32)
    nbr = np.zeros((18, max(n.value, 1)), dtype=np.int32)
    _sparse_check(None, lib().bl_sparse_index_build(ctypes.byref(p), mp, ctypes.byref(n), _ip(dense), _ip(nbr)))
    return dense[: n.value], nbr[:, : n.value]


def bl_sparse_init(params: dict, wall_mask=None, store_dtype=BL_STORE_F32, stream=None):
    N = int(params["nx"]) * int(params["ny"]) * int(params["nz"])
    p = lb_params(params, store_dtype=store_dtype)
    m, mp = _mask_ptr(wall_mask, N)
    h = ctypes.c_void_p(None)
    _sparse_check(None, lib().bl_sparse_init(ctypes.byref(h), ctypes.byref(p), mp, ctypes.c_void_p(stream or 0)))
    return h.value


def bl_sparse_step(h, n):
    _sparse_check(h, lib().bl_sparse_step(h, int(n)))


def bl_sparse_sync(h):
    _sparse_check(h, lib().bl_sparse_sync(h))


def bl_sparse_fields_get(h, N, rho=None, u=None, on_device=False):
    """host: returns (rho, u) on the dense grid; on_device: fills the given
    float64 tensors (N, N x 3)"""
    if on_device:
        _sparse_check(h, lib().bl_sparse_fields_get(h, rho.data_ptr() if rho is not None else None,
                                                     u.data_ptr() if u is not None else None, 1))
        return rho, u
    rho = np.zeros(N)
    u = np.zeros((N, 3))
    _sparse_check(h, lib().bl_sparse_fields_get(h, rho.ctypes.data, u.ctypes.data, 0))
    return rho, u


def bl_sparse_populations_get(h, N):
    pop = np.zeros((N, 19))
    _sparse_check(h, lib().bl_sparse_populations_get(h, _dp(pop)))
    return pop


def bl_sparse_populations_set(h, N, pop):
    pop = np.ascontiguousarray(pop, dtype=np.float64).reshape(N, 19)
    _sparse_check(h, lib().bl_sparse_populations_set(h, _dp(pop)))


def bl_sparse_wall_momentum_get(h):
    out = np.zeros((8, 3))
    _sparse_check(h, lib().bl_sparse_wall_momentum_get(h, _dp(out)))
    return out


def bl_sparse_nodes(h):
    return int(lib().bl_sparse_nodes(h))


def bl_sparse_launch_count(h):
    return int(lib().bl_sparse_launch_count(h))


def bl_sparse_last_error(h):
    msg = lib().bl_sparse_last_error(h)
    return msg.decode() if msg else ""


def bl_sparse_destroy(h):
    lib().bl_sparse_destroy(h)


class SparseLattice:
    """The indexed lattice (only fluid nodes stored) of a geometry given by
    face walls and a wall mask; plasma only."""

    def __init__(self, params: dict, wall_mask=None, store_dtype=BL_STORE_F32, stream=None):
        self.params = dict(params)
        self.N = int(params["nx"]) * int(params["ny"]) * int(params["nz"])
        self.h = bl_sparse_init(params, wall_mask, store_dtype, stream)
        self.n_fluid = bl_sparse_nodes(self.h)

    def close(self):
        if getattr(self, "h", None):
            bl_sparse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        bl_sparse_step(self.h, n)

    def sync(self):
        bl_sparse_sync(self.h)

    def fields(self):
        return bl_sparse_fields_get(self.h, self.N)

    def populations(self):
        return bl_sparse_populations_get(self.h, self.N)

    def set_populations(self, pop):
        bl_sparse_populations_set(self.h, self.N, pop)

    def wall_momentum(self):
        return bl_sparse_wall_momentum_get(self.h)

    def launch_count(self):
        return bl_sparse_launch_count(self.h)
