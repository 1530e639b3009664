"""Seeded input generators (no method arithmetic): sizes, counts, and the
constraints each recipe states."""
import math

import numpy as np

from paper_1005_2594_gb300 import workloads


def test_fcc_start_fills_the_lumen_with_the_requested_cells():
    p = workloads.base_params(64, 48, 48, periodic=(1, 1, 1), R=(7.0, 3.0))
    c = np.array([23.5, 23.5])

    def inside(x):
        return np.hypot(x[:, 1] - c[0], x[:, 2] - c[1]) + 8.0 < 22.0

    X, q = workloads.fcc_cells(p, 40, 3, inside)
    assert X.shape == (40, 3) and q.shape == (40, 4)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)
    # jitter of at most 1/4 node around admissible sites
    assert (np.hypot(X[:, 1] - c[0], X[:, 2] - c[1]) + 8.0 < 22.0 + 0.25 * math.sqrt(2) + 1e-9).all()
    assert ((X >= 0) & (X < np.array([64, 48, 48]))).all()
    X2, q2 = workloads.fcc_cells(p, 40, 3, inside)
    np.testing.assert_array_equal(X, X2)  # seeded


def test_tube_workload_has_the_lumen_hematocrit():
    p, X, q, mask = workloads.tube()
    assert (p["nx"], p["ny"], p["nz"]) == (512, 256, 256)
    n = int(round(0.35 * math.pi * 120.0 ** 2 * 512 / workloads.cell_volume(p)))
    assert len(X) == n == 13166
    r = np.hypot(X[:, 1] - 127.5, X[:, 2] - 127.5)
    assert r.max() + 7.0 < 120.0
    m = mask.reshape(256, 256, 512)  # z, y, x
    assert m[127, 127, 0] == 0 and m[0, 0, 0] == 7  # lumen on the axis, wall in the corner


def test_ensemble_members_are_uneven_and_seeded():
    boxes = workloads.ensemble(n_boxes=6, seed=1004, sizes=(48, 64), max_fail=50)
    sizes = {b[0]["nx"] for b in boxes}
    assert sizes <= {48, 64}
    for p, X, q, desc in boxes:
        assert p["periodic"] == (1, 1, 0) and len(X) > 0
        assert np.abs(p["wall_vel"][5, 0]) > 0


def test_refined_tube_is_the_same_system_under_diffusive_scaling():
    """rheology.tube_case(k): lengths x k (box, radius, cells, positions about
    the axis), body force / k^3, contact strength x k; the same cells."""
    from paper_1005_2594_gb300 import rheology

    p1, X1, q1, m1 = rheology.tube_case(1)
    p2, X2, q2, m2 = rheology.tube_case(2)
    assert (p2["nx"], p2["ny"], p2["nz"]) == (2 * p1["nx"], 2 * p1["ny"], 2 * p1["nz"])
    assert p2["R_perp"] == 2 * p1["R_perp"] and p2["R_par"] == 2 * p1["R_par"]
    assert abs(p2["g"][0] * 8 - p1["g"][0]) < 1e-18 and p2["eps"] == 2 * p1["eps"]
    np.testing.assert_array_equal(q2, q1)
    c1, c2 = (p1["ny"] - 1) / 2.0, (p2["ny"] - 1) / 2.0
    np.testing.assert_allclose(X2[:, 0], 2 * X1[:, 0])
    np.testing.assert_allclose(X2[:, 1:] - c2, 2 * (X1[:, 1:] - c1))  # same place relative to the axis
    # the lumen doubles in radius: 4x the wall-free cross-section, 8x the volume up to the staircase
    ratio = (m2 == 0).sum() / (m1 == 0).sum()
    assert 7.8 < ratio < 8.2
