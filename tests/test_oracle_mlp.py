"""Pins of the FP64 oracle of the learned near-contact correction.

* backward pass: every parameter gradient against central differences of the
  loss (h = 1e-6), relative error below 1e-6;
* features: unchanged under a rigid rotation of the whole pair (positions,
  axes, velocities), unchanged under q -> -q of either cell; the gap of the
  closed-form contact distances of Sec. III with the fluid-coupling axes:
  face to face 2 R_par, side by side 2 R_perp, crossed with one axis along
  the line of centres 2 R_perp / sqrt(1 - chi);
* a network with zero weights returns its output bias.
"""
import numpy as np

from oracle import mlp


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init_params(5) + rng.normal(0, 0.05, mlp.N_PARAMS)
    x = rng.normal(0, 1, (7, mlp.N_IN))
    y = rng.normal(0, 1, (7, mlp.N_OUT))
    _, g = mlp.loss_and_grad(theta, x, y)
    idx = rng.choice(mlp.N_PARAMS, 200, replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, x, y)[0] - mlp.loss_and_grad(tm, x, y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_zero_network_returns_output_bias():
    p = mlp.unflatten(np.zeros(mlp.N_PARAMS))
    p["b3"] = np.arange(6.0)
    y, _ = mlp.forward(mlp.flatten(p), np.ones((3, mlp.N_IN)))
    np.testing.assert_array_equal(y, np.tile(np.arange(6.0), (3, 1)))


def _random_q(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def test_features_are_frame_invariant_and_sign_free():
    rng = np.random.default_rng(11)
    Rpar, Rperp = 3.0, 7.0
    dims, per = (200, 200, 200), (0, 0, 0)
    Xi, Xj = np.array([100.0, 100, 100]), np.array([103.0, 108, 97])
    qi, qj = _random_q(rng), _random_q(rng)
    Vi, Vj, Wi, Wj = (rng.normal(0, 0.01, 3) for _ in range(4))
    f0 = mlp.pair_features(Rpar, Rperp, dims, per, Xi, qi, Vi, Wi, Xj, qj, Vj, Wj)
    g = _random_q(rng)
    G = mlp.rotmat(g)
    c = np.array([100.0, 100, 100])
    f1 = mlp.pair_features(Rpar, Rperp, dims, per, c + G @ (Xi - c), mlp.qmul(g, qi), G @ Vi, G @ Wi,
                           c + G @ (Xj - c), mlp.qmul(g, qj), G @ Vj, G @ Wj)
    np.testing.assert_allclose(f1, f0, atol=1e-12)
    f2 = mlp.pair_features(Rpar, Rperp, dims, per, Xi, -qi, Vi, Wi, Xj, -qj, Vj, Wj)
    np.testing.assert_allclose(f2, f0, atol=1e-12)


def test_gap_of_closed_form_contact_distances():
    Rpar, Rperp = 3.0, 7.0
    chi = (Rpar ** 2 - Rperp ** 2) / (Rpar ** 2 + Rperp ** 2)
    dims, per, z = (100, 100, 100), (0, 0, 0), np.zeros(3)
    qz = np.array([1.0, 0, 0, 0])                      # axis along z
    qx = np.array([np.cos(np.pi / 4), 0, np.sin(np.pi / 4), 0])  # axis along x
    X0 = np.array([50.0, 50, 50])
    # face to face along the common axis: contact at 2 R_par
    f = mlp.pair_features(Rpar, Rperp, dims, per, X0, qz, z, z, X0 + [0, 0, 10.0], qz, z, z)
    assert abs(f[7] - (10.0 - 2 * Rpar)) < 1e-12
    # side by side, axes parallel, perpendicular to the line of centres: 2 R_perp
    f = mlp.pair_features(Rpar, Rperp, dims, per, X0, qz, z, z, X0 + [20.0, 0, 0], qz, z, z)
    assert abs(f[7] - (20.0 - 2 * Rperp)) < 1e-12
    # crossed axes, one of them along the line of centres (x)
    f = mlp.pair_features(Rpar, Rperp, dims, per, X0, qz, z, z, X0 + [20.0, 0, 0], qx, z, z)
    assert abs(f[7] - (20.0 - 2 * Rperp / np.sqrt(1 - chi))) < 1e-12
    # crossed axes, both perpendicular to the line of centres: side on, 2 R_perp
    f = mlp.pair_features(Rpar, Rperp, dims, per, X0, qz, z, z, X0 + [0, 20.0, 0], qx, z, z)
    assert abs(f[7] - (20.0 - 2 * Rperp)) < 1e-12
