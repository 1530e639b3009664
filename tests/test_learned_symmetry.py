"""Pin of the symmetry augmentation of the learned correction's training data.

Each symmetry is applied to the physical pair (positions, orientations,
velocities) and the features and body-frame targets are recomputed from
scratch with the oracle: the features by ``oracle.mlp.pair_features``, the
targets as the oracle's pair-potential force and torque on the first cell
(Sec. III), which, like the hydrodynamic ones, are a polar and an axial
vector.  ``learned.symmetry_transform`` must reproduce both from the
untransformed sample alone.  The reflected orientation is built as a rotation
matrix and converted to a quaternion here (Shepperd's method), independently
of the transform's quaternion algebra.
"""
import numpy as np

import oracle
from oracle import mlp


def _unit(v):
    return v / np.linalg.norm(v)


def _quat_of_matrix(R):
    """unit quaternion (w, x, y, z) of a proper rotation matrix, w >= 0"""
    tr = np.trace(R)
    cand = [1.0 + tr, 1.0 + R[0, 0] - R[1, 1] - R[2, 2], 1.0 - R[0, 0] + R[1, 1] - R[2, 2],
            1.0 - R[0, 0] - R[1, 1] + R[2, 2]]
    k = int(np.argmax(cand))
    s = 2.0 * np.sqrt(cand[k])
    if k == 0:
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif k == 1:
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif k == 2:
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    return q if q[0] >= 0 else -q


def _sample(p, dims, Xi, qi, Vi, Wi, Xj, qj, Vj, Wj):
    f = mlp.pair_features(p["R_par"], p["R_perp"], dims, (0, 0, 0), Xi, qi, Vi, Wi, Xj, qj, Vj, Wj)
    _, Fi, _, Ti, _ = oracle.pair(p, Xj - Xi, mlp.rotmat(qi)[:, 2], mlp.rotmat(qj)[:, 2])
    Ri = mlp.rotmat(qi)
    return f, np.concatenate([Ri.T @ Fi, Ri.T @ Ti])


def test_symmetry_transform_matches_the_transformed_pair():
    from paper_1005_2594_gb300 import learned, workloads

    p = workloads.base_params(64, 64, 64, periodic=(0, 0, 0), R=(7.0, 3.0))
    dims = (64, 64, 64)
    rng = np.random.default_rng(8)
    qz = lambda a: np.array([np.cos(0.5 * a), 0.0, 0.0, np.sin(0.5 * a)])
    qx = np.array([0.0, 1.0, 0.0, 0.0])
    Pb = np.diag([1.0, 1.0, -1.0])
    n_force = 0
    for trial in range(64):
        qi, qj = _unit(rng.normal(size=4)), _unit(rng.normal(size=4))
        Xi = np.array([32.0, 32.0, 32.0])
        Xj = Xi + _unit(rng.normal(size=3)) * rng.uniform(7.0, 15.0)
        Vi, Vj, Wi, Wj = (rng.normal(0, 0.01, 3) for _ in range(4))
        f0, y0 = _sample(p, dims, Xi, qi, Vi, Wi, Xj, qj, Vj, Wj)
        phi, psi = rng.uniform(0, 2 * np.pi, 2)
        fi, fj, mi = trial % 2 == 1, (trial // 2) % 2 == 1, (trial // 4) % 2 == 1
        # the same pair described differently
        qi2 = mlp.qmul(qi, qz(phi))
        qj2 = mlp.qmul(qj, qz(psi))
        if fi:
            qi2 = mlp.qmul(qi2, qx)
        if fj:
            qj2 = mlp.qmul(qj2, qx)
        Xj2, Vi2, Vj2, Wi2, Wj2 = Xj, Vi, Vj, Wi, Wj
        if mi:  # reflection through the plane through X_i normal to the axis of i
            oi = mlp.rotmat(qi2)[:, 2]
            Pw = np.eye(3) - 2.0 * np.outer(oi, oi)
            Xj2 = Xi + Pw @ (Xj - Xi)
            Vi2, Vj2, Wi2, Wj2 = Pw @ Vi, Pw @ Vj, -Pw @ Wi, -Pw @ Wj
            qj2 = _quat_of_matrix(Pw @ mlp.rotmat(qj2) @ Pb)
        f1, y1 = _sample(p, dims, Xi, qi2, Vi2, Wi2, Xj2, qj2, Vj2, Wj2)
        xa, ya = learned.symmetry_transform(f0[None], y0[None], np.array([phi]), np.array([psi]), [fi], [fj], [mi])
        np.testing.assert_allclose(xa[0], f1, atol=1e-10, err_msg=f"features, trial {trial}")
        scale = max(np.abs(y1).max(), 1e-300)
        np.testing.assert_allclose(ya[0] / scale, y1 / scale, atol=1e-10, err_msg=f"targets, trial {trial}")
        n_force += np.abs(y1).max() > 1e-6
    assert n_force >= 16  # enough pairs inside the potential's range to test the targets


def test_augment_keeps_the_originals_and_unit_quaternions():
    from paper_1005_2594_gb300 import learned

    rng = np.random.default_rng(2)
    X = rng.normal(size=(10, 14))
    X[:, 3:7] /= np.linalg.norm(X[:, 3:7], axis=1, keepdims=True)
    X[:, 3:7] *= np.sign(X[:, 3:4])
    Y = rng.normal(size=(10, 6))
    Xa, Ya = learned.augment(X, Y, rng, 3)
    assert Xa.shape == (40, 14) and Ya.shape == (40, 6)
    np.testing.assert_array_equal(Xa[:10], X)
    np.testing.assert_allclose(np.linalg.norm(Xa[:, 3:7], axis=1), 1.0, atol=1e-12)
    assert (Xa[:, 3] >= 0).all()
    np.testing.assert_array_equal(np.tile(X[:, 7], 4), Xa[:, 7])  # the gap is invariant
    # lengths of the polar and axial vectors are invariant
    for a, b in ((0, 3), (8, 11), (11, 14)):
        np.testing.assert_allclose(np.linalg.norm(Xa[:, a:b], axis=1), np.tile(np.linalg.norm(X[:, a:b], axis=1), 4))


def test_approach_runs_start_at_the_stated_gap():
    """The training runs' set-up: two cells gap0 apart (the oracle's contact
    distance with the fluid-coupling half-axes), moving towards each other
    along the line of centres with equal and opposite velocities."""
    from paper_1005_2594_gb300 import learned

    rng = np.random.default_rng(4)
    R = (7.0, 3.0)
    for _ in range(20):
        X, q, V, W, steps = learned.approach_setup(rng, L=48, R=R, gap0=4.5)
        r = X[1] - X[0]
        n = r / np.linalg.norm(r)
        oi, oj = mlp.rotmat(q[0])[:, 2], mlp.rotmat(q[1])[:, 2]
        gap = np.linalg.norm(r) - mlp.contact_distance(R[1], R[0], oi, oj, n)
        assert abs(gap - 4.5) < 1e-9
        np.testing.assert_allclose(V[0], -V[1], atol=1e-15)
        assert V[0] @ n > 0 and V[1] @ n < 0  # approaching
        assert steps * 2 * (V[0] @ n) <= 4.5 - 0.2 + 1e-9  # stops short of contact
