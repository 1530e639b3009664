"""The cell-list build that allocates nothing (bl_cell_list_build_static) must
give the same list as the allocating read-out (bl_cell_list_get).

It exists for callers that cannot call cudaMalloc when they need the list
(device memory already held by their own pool allocator, or a time loop that
must avoid the synchronisation an allocation can cause): its scratch is a
fixed array reserved on every GPU that loads the library.  Two calls in a
row, on different workloads, must both match (the shared array keeps the
previous call's contents).  The file is named so that pytest collects it
last; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    torch.cuda.init()
    yield


def _reference_list(p, X, q):
    from paper_1005_2594_gb300 import bloodlb as bl

    sim = bl.Simulation(p)
    sim.set_particles(X, q)
    nb, start, ids = sim.cell_list()
    sim.close()
    return nb, start, ids


def test_static_cell_list_matches_allocating_entry_point():
    import torch

    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    stream = torch.cuda.current_stream()
    cases = [workloads.small_shear(), workloads.shear_cell(n=64, phi=0.30)]
    for p, X, q in cases:  # two calls in a row on the same reserved scratch
        nb_ref, start_ref, ids_ref = _reference_list(p, X, q)
        dims = (p["nx"], p["ny"], p["nz"])
        n = X.shape[0]
        Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
        start_d = torch.full((int(np.prod(nb_ref)) + 1,), -7, dtype=torch.int32, device="cuda")
        ids_d = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        rc, nb = bl.bl_cell_list_build_static(Xd, n, dims, p["r_cut"], start_d, ids_d, stream.cuda_stream)
        assert rc == bl.BL_OK
        stream.synchronize()
        np.testing.assert_array_equal(nb, nb_ref)
        np.testing.assert_array_equal(start_d.cpu().numpy(), start_ref)
        np.testing.assert_array_equal(ids_d.cpu().numpy(), ids_ref)


def test_static_cell_list_rejects_oversize_requests():
    import torch

    from paper_1005_2594_gb300 import bloodlb as bl

    Xd = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc, _ = bl.bl_cell_list_build_static(Xd, 70000, (64, 64, 64), 7.5, out, out)
    assert rc == bl.BL_EINVAL
    rc, _ = bl.bl_cell_list_build_static(Xd, 1, (4096, 4096, 64), 1.0, out, out)
    assert rc == bl.BL_EINVAL
    # a tiny r_cut: bin counts far beyond INT_MAX are rejected, not converted
    rc, nb = bl.bl_cell_list_build_static(Xd, 1, (64, 64, 64), 1e-12, out, out)
    assert rc == bl.BL_EINVAL
    assert (nb == 0).all()  # a rejected request leaves nb untouched
