"""FP64 oracle of the learned near-contact correction (test infrastructure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only tests, the smoke
check and the CPU leg of the benchmark use it; it shares no code with the
CUDA path.

The paper motivates the correction and leaves it open: below the resolution of
the lattice, no fluid node lies between two cells and the lubrication force
is missing (Sec. II, discussion of the coupling), and the paper deliberately
adds no analytic lubrication term.  The correction here is a small network
trained on what the method itself gives at a finer resolution:

  features x (14) of an ordered pair (i, j), all in the body frame of i:
    p      = R_i^T r,            r = X_j - X_i (minimum image)          (3)
    q_rel  = q_i^* (x) q_j, sign fixed so that w >= 0                   (4)
    gap    = |r| - sigma_R(o_i, o_j, r^)                                 (1)
    dv     = R_i^T (V_j - V_i)                                           (3)
    dw     = R_i^T (W_j - W_i)                                           (3)
  sigma_R is the Berne-Pechukas contact distance of Sec. III (Eq. sigma)
  built from the fluid-coupling half-axes: sigma_bar = 2 R_perp,
  chi = (R_par^2 - R_perp^2) / (R_par^2 + R_perp^2).

  network (inputs and outputs standardised with stored means and scales):
    h1 = tanh(W1 x~ + b1)    64
    h2 = tanh(W2 h1 + b2)    64
    y~ = W3 h2 + b3          6     y = (dF, dT) on i in the body frame of i

Pins (tests/test_oracle_mlp.py): the backward pass against central
differences; the features against rigid rotations of the whole pair, the
quaternion sign and the closed-form contact distances.
"""
import numpy as np

N_IN, N_HID, N_OUT = 14, 64, 6
SHAPES = (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    """flat parameter vector (order W1, b1, W2, b2, W3, b3; row-major) -> dict"""
    out, k = {}, 0
    for name, shape in SHAPES:
        m = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + m], dtype=np.float64).reshape(shape)
        k += m
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(theta, x):
    """standardised inputs x (B x 14) -> standardised outputs (B x 6), cache"""
    p = unflatten(theta)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, h1, h2)


def backward(theta, cache, dy):
    """gradient of sum(dy * y) with respect to the flat parameters"""
    p = unflatten(theta)
    x, h1, h2 = cache
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    d2 = (dy @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return flatten(g)


def loss_and_grad(theta, x, y_target):
    """mean over the batch of the squared error summed over the 6 outputs"""
    y, cache = forward(theta, x)
    r = y - y_target
    B = x.shape[0]
    loss = float((r * r).sum() / B)
    return loss, backward(theta, cache, 2.0 * r / B)


def init_params(seed):
    """uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases"""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = 1.0 / np.sqrt(shape[1])
            p[name] = rng.uniform(-lim, lim, shape)
        else:
            p[name] = np.zeros(shape)
    return flatten(p)


# ---------------------------------------------------------------------------
# features of an ordered pair


def rotmat(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def contact_distance(R_par, R_perp, oi, oj, rhat):
    """Berne-Pechukas contact distance (Eq. sigma) with the fluid-coupling half-axes"""
    chi = (R_par ** 2 - R_perp ** 2) / (R_par ** 2 + R_perp ** 2)
    a, b, c = rhat @ oi, rhat @ oj, oi @ oj
    S = 1.0 - 0.5 * chi * ((a + b) ** 2 / (1.0 + chi * c) + (a - b) ** 2 / (1.0 - chi * c))
    return 2.0 * R_perp / np.sqrt(S)


def pair_features(R_par, R_perp, dims, periodic, Xi, qi, Vi, Wi, Xj, qj, Vj, Wj):
    r = np.asarray(Xj, dtype=np.float64) - np.asarray(Xi, dtype=np.float64)
    for k in range(3):
        if periodic[k]:
            if r[k] > 0.5 * dims[k]:
                r[k] -= dims[k]
            elif r[k] < -0.5 * dims[k]:
                r[k] += dims[k]
    Ri = rotmat(qi)
    oi, oj = Ri[:, 2], rotmat(qj)[:, 2]
    rl = np.sqrt(r @ r)
    gap = rl - contact_distance(R_par, R_perp, oi, oj, r / rl)
    qc = np.array([qi[0], -qi[1], -qi[2], -qi[3]])
    qr = qmul(qc, qj)
    if qr[0] < 0:
        qr = -qr
    return np.concatenate([Ri.T @ r, qr, [gap], Ri.T @ (np.asarray(Vj) - np.asarray(Vi)),
                           Ri.T @ (np.asarray(Wj) - np.asarray(Wi))])
