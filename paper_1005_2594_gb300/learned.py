"""Training pipeline of the learned near-contact correction.

The paper explains what is missing at short range: once no fluid node lies
between two cells, the lattice carries no lubrication force, and the paper
adds no analytic one (Sec. II).  This module generates what the method itself
computes at a finer resolution, trains the network on the difference, and
measures what the network gains (all on the GPU, through the library):

* approach runs: two cells move towards each other with prescribed velocities
  (``move_particles = 2``) through resting plasma, once at the coarse
  resolution and once refined k times.  Under the diffusive scaling of the
  lattice units (dx / k, dt / k^2, tau fixed) the fine run has cells and box
  k times larger, lattice velocities / k and angular velocities / k^2; its
  lattice forces are then directly comparable with the coarse ones and its
  lattice torques are divided by k;
* samples: at windows of the coarse run, the features of the ordered pair
  (``bl_pair_features``) and the difference fine - coarse of the hydrodynamic
  force and torque on the first cell (total minus potential, averaged over
  the window), in its body frame;
* augmentation: both cells are bodies of revolution with a mirror plane, so
  spinning either about its own axis, flipping either axis, and reflecting the
  whole pair through the equatorial plane of the first cell give the same
  pair again (or its mirror image); each sample is repeated under random
  draws of these symmetries (``symmetry_transform``), which is what lets a
  few hundred runs cover the 14 inputs;
* training: Adam on the standardised mean squared error (``bl_mlp_*``), runs
  split into training and validation sets, the parameters of the lowest
  validation loss kept.
"""
import math

import numpy as np

from . import bloodlb as bl
from . import workloads


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _contact(Rpar, Rperp, oi, oj, n):
    chi = (Rpar ** 2 - Rperp ** 2) / (Rpar ** 2 + Rperp ** 2)
    a, b, c = n @ oi, n @ oj, oi @ oj
    S = 1.0 - 0.5 * chi * ((a + b) ** 2 / (1.0 + chi * c) + (a - b) ** 2 / (1.0 - chi * c))
    return 2.0 * Rperp / math.sqrt(S)


def approach_setup(rng, L=48, R=(7.0, 3.0), gap0=4.5, speed=(0.01, 0.03), spin=0.001):
    """one coarse approach: cell states (X, q, V, W) for a box L^3 and the
    number of coarse steps until the gap would reach about 0.2"""
    _, q = workloads.random_axes_and_quaternions(rng, 2)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    oi, oj = _rot(q[0])[:, 2], _rot(q[1])[:, 2]
    d0 = _contact(R[1], R[0], oi, oj, n) + gap0
    c = np.full(3, L / 2.0)
    X = np.array([c - 0.5 * d0 * n, c + 0.5 * d0 * n])
    v = rng.uniform(*speed)
    tang = rng.normal(size=3)
    tang -= (tang @ n) * n
    tang *= 0.2 * v / max(np.linalg.norm(tang), 1e-12)
    V = np.array([0.5 * v * n + 0.5 * tang, -0.5 * v * n - 0.5 * tang])
    W = rng.uniform(-spin, spin, (2, 3))
    steps = int((gap0 - 0.2) / v)
    return X, q, V, W, steps


def _sim(L, R, X, q, V, W, k, stream=None):
    """a prescribed-motion simulation refined k times (box, cells and
    positions x k, velocities / k, angular velocities / k^2)"""
    Rk = (R[0] * k, R[1] * k)
    p = workloads.base_params(L * k, L * k, L * k, periodic=(1, 1, 1), R=Rk)
    p["move_particles"] = 2
    s = bl.Simulation(p, stream=stream)
    m = p["rho_p"] * 4.0 / 3.0 * math.pi * Rk[0] ** 2 * Rk[1]
    Ip, Ia = m * (Rk[1] ** 2 + Rk[0] ** 2) / 5.0, 2.0 * m * Rk[0] ** 2 / 5.0
    Lang = []
    for i in range(2):
        Rm = _rot(q[i])
        I = Rm @ np.diag([Ip, Ip, Ia]) @ Rm.T
        Lang.append(I @ (W[i] / k ** 2))
    s.set_particles(X * k, q, V / k, np.array(Lang))
    return s


def _hydro(s):
    """hydrodynamic force and torque of the last step"""
    pp = s.force_parts()
    return pp["Fh"], pp["Th"]


def approach_samples(n_runs, seed, k=2, L=48, R=(7.0, 3.0), window=6, gap_max=3.0, gap_stop=0.3, **setup):
    """features (n x 14), targets (n x 6: fine - coarse force and torque on
    the first cell of each ordered pair, body frame), the coarse force and
    torque in the same frame, and the run index of each sample"""
    import torch

    rng = np.random.default_rng(seed)
    feats, targ, coarse, runs = [], [], [], []
    pairs = torch.tensor([[0, 1], [1, 0]], dtype=torch.int32, device="cuda")
    fout = torch.zeros((2, 14), dtype=torch.float32, device="cuda")
    for run in range(n_runs):
        X, q, V, W, steps = approach_setup(rng, L=L, R=R, **setup)
        sc, sf = _sim(L, R, X, q, V, W, 1), _sim(L, R, X, q, V, W, k)
        for t0 in range(0, steps - window + 1, window):
            bl.bl_pair_features(sc.ctx, pairs, fout)
            f = fout.cpu().numpy().astype(np.float64)
            if min(f[0, 7], f[1, 7]) < gap_stop:
                break  # the approach ends short of contact
            qc = sc.particles()["q"]
            Fc, Tc, Ff, Tf = np.zeros((2, 3)), np.zeros((2, 3)), np.zeros((2, 3)), np.zeros((2, 3))
            for _ in range(window):
                sc.step(1)
                a, b = _hydro(sc)
                Fc += a / window
                Tc += b / window
            for _ in range(window * k * k):
                sf.step(1)
                a, b = _hydro(sf)
                Ff += a / (window * k * k)
                Tf += b / (window * k * k * k)
            if f[0, 7] > gap_max:
                continue
            for i in range(2):
                Rt = _rot(qc[i]).T
                feats.append(f[i])
                targ.append(np.concatenate([Rt @ (Ff[i] - Fc[i]), Rt @ (Tf[i] - Tc[i])]))
                coarse.append(np.concatenate([Rt @ Fc[i], Rt @ Tc[i]]))
                runs.append(run)
        sc.close()
        sf.close()
    return (np.array(feats).reshape(-1, 14), np.array(targ).reshape(-1, 6), np.array(coarse).reshape(-1, 6),
            np.array(runs, dtype=np.int64))


def _qmul(a, b):
    w1, x1, y1, z1 = a.T
    w2, x2, y2, z2 = b.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)


def symmetry_transform(X, Y, phi, psi, flip_i, flip_j, mirror):
    """Features and targets of the same pair after, in this order:
    the body frame of i turned by phi about its axis (q_i -> q_i qz(phi)),
    j described by q_j qz(psi), the axis of i flipped (q_i -> q_i qx(pi))
    where flip_i, that of j where flip_j, and the whole pair reflected through
    the plane through X_i normal to the axis of i where mirror.  In the body
    frame of i the reflection is P = diag(1, 1, -1): polar vectors (position,
    velocity, force) go to P v, axial ones (angular velocity, torque) to
    -P v, and q_rel = (w, x, y, z) to (w, -x, -y, z).  All arguments are
    per-sample arrays."""
    X = np.array(X, dtype=np.float64)
    Y = np.array(Y, dtype=np.float64)
    n = X.shape[0]
    p, q, dv, dw = X[:, 0:3], X[:, 3:7], X[:, 8:11], X[:, 11:14]
    F, T = Y[:, 0:3], Y[:, 3:6]
    c, s = np.cos(phi), np.sin(phi)
    for v in (p, dv, dw, F, T):  # R_z(phi)^T v
        x, y = v[:, 0].copy(), v[:, 1].copy()
        v[:, 0], v[:, 1] = c * x + s * y, -s * x + c * y
    zero = np.zeros(n)
    q = _qmul(np.stack([np.cos(0.5 * phi), zero, zero, -np.sin(0.5 * phi)], axis=1), q)
    q = _qmul(q, np.stack([np.cos(0.5 * psi), zero, zero, np.sin(0.5 * psi)], axis=1))
    fi, fj, mi = (np.asarray(a, dtype=bool) for a in (flip_i, flip_j, mirror))
    for v in (p, dv, dw, F, T):  # R_x(pi)^T v
        v[fi, 1:] *= -1.0
    qx = np.tile([0.0, 1.0, 0.0, 0.0], (n, 1))
    q[fi] = _qmul(qx[fi] * [1.0, -1.0, -1.0, -1.0], q[fi])
    q[fj] = _qmul(q[fj], qx[fj])
    for v in (p, dv, F):
        v[mi, 2] *= -1.0
    for v in (dw, T):
        v[mi, :2] *= -1.0
    q[mi, 1:3] *= -1.0
    q[q[:, 0] < 0] *= -1.0
    X[:, 3:7] = q
    return X, Y


def augment(X, Y, rng, copies):
    """the samples followed by `copies` images under random symmetries"""
    Xs, Ys = [np.asarray(X, dtype=np.float64)], [np.asarray(Y, dtype=np.float64)]
    n = X.shape[0]
    for _ in range(copies):
        a, b = symmetry_transform(X, Y, rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n),
                                  rng.random(n) < 0.5, rng.random(n) < 0.5, rng.random(n) < 0.5)
        Xs.append(a)
        Ys.append(b)
    return np.vstack(Xs), np.vstack(Ys)


def norm_of(X, Y):
    """standardisation (means and scales) of features and targets"""
    sx = X.std(axis=0)
    sy = Y.std(axis=0)
    return np.concatenate([X.mean(axis=0), np.where(sx > 1e-12, sx, 1.0), Y.mean(axis=0),
                           np.where(sy > 1e-12, sy, 1.0)])


def train(X, Y, epochs=2000, lr=2e-3, seed=0, model=None, Xv=None, Yv=None, check_every=25):
    """full-batch Adam on the GPU; with a validation set (Xv, Yv) the
    parameters of the lowest validation loss are kept (early stopping).
    Returns (model handle, training-loss history, validation-loss history)"""
    import torch

    rng = np.random.default_rng(seed)
    m = model or bl.bl_mlp_create()
    theta = np.zeros(bl.MLP_NPAR)
    k = 0
    for rows, cols in ((64, 14), (64, 1), (64, 64), (64, 1), (6, 64), (6, 1)):
        size = rows * cols
        if cols > 1:
            lim = 1.0 / math.sqrt(cols)
            theta[k:k + size] = rng.uniform(-lim, lim, size)
        k += size
    bl.bl_mlp_params_set(m, theta, norm_of(X, Y))
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(Y, dtype=torch.float32, device="cuda")
    val = Xv is not None
    if val:
        xv = torch.tensor(Xv, dtype=torch.float32, device="cuda")
        yv = torch.tensor(Yv, dtype=torch.float32, device="cuda")
    hist, vhist = [], []
    best, best_theta = float("inf"), None
    for it in range(epochs):
        if val and it % check_every == 0:
            vl, _ = bl.bl_mlp_grad(m, xv, yv)
            vhist.append(vl)
            if vl < best:
                best, best_theta = vl, bl.bl_mlp_params_get(m)[0]
        loss, _ = bl.bl_mlp_grad(m, xd, yd)
        hist.append(loss)
        bl.bl_mlp_adam(m, lr=lr)
    if val:
        vl, _ = bl.bl_mlp_grad(m, xv, yv)
        if vl >= best and best_theta is not None:
            bl.bl_mlp_params_set(m, best_theta, None)
    return m, hist, vhist


def fit(X, Y, runs, seed=0, copies=16, clip=4.0, val_frac=0.2, epochs=2000, lr=1e-3, model=None):
    """the training recipe: whole runs split into training and validation
    sets, the training samples augmented by the pair's symmetries and their
    targets clipped at `clip` standard deviations, then `train` with early
    stopping.  Returns (model handle, dict of losses, sizes and the ranges of
    gap and relative speed of the training samples, outside which the network
    is not to be used)."""
    rng = np.random.default_rng(seed)
    ids = np.unique(runs)
    rng.shuffle(ids)
    val = np.isin(runs, ids[:max(1, int(round(len(ids) * val_frac)))])
    Xt, Yt = augment(X[~val], Y[~val], rng, copies)
    mu, sd = Yt.mean(axis=0), Yt.std(axis=0)
    Yt = np.clip(Yt, mu - clip * sd, mu + clip * sd)
    m, hist, vhist = train(Xt, Yt, epochs=epochs, lr=lr, seed=seed, model=model, Xv=X[val], Yv=Y[val])
    return m, {"train_samples": Xt.shape[0], "val_samples": int(val.sum()), "loss_first": hist[0],
               "loss_last": hist[-1], "val_best": min(vhist), "val_best_epoch": 25 * int(np.argmin(vhist)),
               "gap_min": float(X[:, 7].min()), "gap_max": float(X[:, 7].max()),
               "speed_min": float(np.linalg.norm(X[:, 8:11], axis=1).min()),
               "speed_max": float(np.linalg.norm(X[:, 8:11], axis=1).max())}


def errors(m, X, Y, scale):
    """mean over samples of the squared error summed over the six outputs,
    each output divided by `scale`: without the correction (the coarse
    method alone) and with it"""
    P = predict(m, X)
    e0 = float((((Y) / scale) ** 2).sum(axis=1).mean())
    e1 = float((((Y - P) / scale) ** 2).sum(axis=1).mean())
    return e0, e1


def predict(m, X):
    import torch

    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.zeros((X.shape[0], 6), dtype=torch.float32, device="cuda")
    bl.bl_mlp_forward(m, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)
