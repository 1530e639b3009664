"""The indexed lattice's host-side index and its vessel geometry (CPU).

bl_sparse_index_build numbers the fluid nodes in dense order and tabulates
each one's 18 neighbours (fluid index, or -1 - wall id); it runs on the host
and is checked here against a brute force over the dense grid with numpy, for
face walls, masks of every wall id and periodic axes.  The synthetic vessel
loop is checked for the properties its docstring states.
"""
import ctypes

import numpy as np
import pytest

from paper_1005_2594_gb300 import bloodlb as bl
from paper_1005_2594_gb300 import workloads

C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0], [-1, -1, 0],
              [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1],
              [0, 1, -1], [0, -1, 1]])


def _brute(p, mask):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wall = np.full((nz, ny, nx), -1)
    # the first walled axis in x, y, z order names the face (ids 0..5); a
    # mask value k in 1..8 overrides with id k - 1
    for k, (c, n) in reversed(list(enumerate(((x, nx), (y, ny), (z, nz))))):
        if p["periodic"][k]:
            continue
        wall[c == 0] = 2 * k
        wall[c == n - 1] = 2 * k + 1
    m = mask.reshape(nz, ny, nx).astype(int)
    wall = np.where(m > 0, m - 1, wall)
    fluid = wall < 0
    ids = np.full((nz, ny, nx), 0)
    ids[fluid] = np.arange(fluid.sum())
    code = np.where(fluid, ids, -1 - wall)
    nbr = np.stack([np.roll(code, (-C[r, 2], -C[r, 1], -C[r, 0]), axis=(0, 1, 2))[fluid] for r in range(1, 19)])
    dense = (x + nx * (y + ny * z))[fluid]
    return dense, nbr


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 0, 1), (0, 0, 0), (0, 1, 0)])
def test_index_matches_brute_force(periodic):
    p = workloads.base_params(11, 9, 7, periodic=periodic)
    rng = np.random.default_rng(sum(periodic))
    mask = np.where(rng.random(11 * 9 * 7) < 0.25, rng.integers(1, 9, 11 * 9 * 7), 0).astype(np.uint8)
    dense, nbr = bl.bl_sparse_index_build(p, mask)
    d_ref, n_ref = _brute(p, mask)
    np.testing.assert_array_equal(dense, d_ref)
    np.testing.assert_array_equal(nbr, n_ref)
    # every fluid neighbour is the node one lattice vector away (periodic)
    assert (nbr < len(dense)).all()


def test_capacity_too_small_is_refused():
    p = workloads.base_params(6, 5, 4, periodic=(1, 0, 1))
    dense, _ = bl.bl_sparse_index_build(p)
    n = ctypes.c_int64(len(dense) - 1)
    buf = np.zeros(len(dense), dtype=np.int32)
    rc = bl.lib().bl_sparse_index_build(ctypes.byref(bl.lb_params(p)), None, ctypes.byref(n), bl._ip(buf), None)
    assert rc == bl.BL_EINVAL


def test_vessel_loop_geometry():
    nx, ny, nz, r0, h = 96, 48, 24, 6.0, 12.0
    mask, segs = workloads.vessel_loop(nx, ny, nz, r0, h)
    m = mask.reshape(nz, ny, nx)
    yc, zc = (ny - 1) / 2.0, (nz - 1) / 2.0
    # Murray's law: parent radius cubed = sum of the two daughters'
    rd = {r for (_, _, r) in segs} - {r0}
    assert len(rd) == 1 and abs(2 * rd.pop() ** 3 - r0 ** 3) < 1e-9
    # mirror symmetric in y and z about the centre; open across the periodic x end
    np.testing.assert_array_equal(m, m[:, ::-1, :])
    np.testing.assert_array_equal(m, m[::-1, :, :])
    assert m[int(zc), int(yc), 0] == 0 and m[int(zc), int(yc), nx - 1] == 0
    # the daughters' centre lines are open, the box corners are wall
    assert m[int(zc), int(round(yc + h)), nx // 2] == 0 and m[int(zc), int(round(yc - h)), nx // 2] == 0
    assert m[0, 0, 0] == 7 and m[-1, -1, -1] == 7
    # the lumen at the loop's middle cross-section is two discs of radius rd
    sec = (m[:, :, nx // 2] == 0).sum()
    assert abs(sec - 2 * np.pi * (r0 * 2 ** (-1 / 3)) ** 2) < 0.1 * sec
