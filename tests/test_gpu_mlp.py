"""The learned near-contact correction's tensor-core kernels against the FP64
oracle (oracle/mlp.py), through the C ABI.

Bars: forward outputs and the loss within 2e-2 relative, the gradient within
3e-2 relative to its largest component: weights and activations are rounded
to BF16 (8 significant bits, relative step 2^-8 = 3.9e-3) before every
product, and a product of 64 terms accumulated in FP32 keeps that order of
error.  Training: Adam on the GPU cuts the loss of a teacher-student fit by
more than 20 times.
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


def _data(seed, B):
    from oracle import mlp

    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed) + rng.normal(0, 0.05, mlp.N_PARAMS)
    mx, sx = rng.normal(0, 1, 14), rng.uniform(0.5, 2.0, 14)
    my, sy = rng.normal(0, 1, 6), rng.uniform(0.5, 2.0, 6)
    x = mx + sx * rng.normal(0, 1, (B, 14))
    y = my + sy * rng.normal(0, 1, (B, 6))
    norm = np.concatenate([mx, sx, my, sy])
    return theta, norm, x, y


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def test_forward_loss_and_gradient_match_oracle():
    import torch

    from oracle import mlp
    from paper_1005_2594_gb300 import bloodlb as bl

    theta, norm, x, y = _data(21, 333)  # a ragged last tile
    m = bl.bl_mlp_create()
    bl.bl_mlp_params_set(m, theta, norm)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    out = torch.zeros((x.shape[0], 6), dtype=torch.float32, device="cuda")
    bl.bl_mlp_forward(m, xd, out)
    torch.cuda.synchronize()
    xs = (x - norm[:14]) / norm[14:28]
    ys = (y - norm[28:34]) / norm[34:40]
    yo, _ = mlp.forward(theta, xs)
    y_raw = yo * norm[34:40] + norm[28:34]
    assert rel(out.cpu().numpy(), y_raw) < 2e-2
    loss_o, g_o = mlp.loss_and_grad(theta, xs, ys)
    loss_g, g_g = bl.bl_mlp_grad(m, xd, yd, want_grad=True)
    print("loss gpu %.6f oracle %.6f, grad rel err %.3e" % (loss_g, loss_o, rel(g_g, g_o)))
    assert abs(loss_g - loss_o) < 2e-2 * loss_o
    assert rel(g_g, g_o) < 3e-2
    # the same data give the same gradient (fixed reduction order)
    _, g_again = bl.bl_mlp_grad(m, xd, yd, want_grad=True)
    assert rel(g_again, g_g) < 1e-5
    bl.bl_mlp_destroy(m)


def test_adam_training_fits_a_teacher():
    import torch

    from oracle import mlp
    from paper_1005_2594_gb300 import bloodlb as bl

    rng = np.random.default_rng(5)
    teacher = mlp.init_params(99) * 2.0
    x = rng.normal(0, 1, (4096, 14))
    y, _ = mlp.forward(teacher, x)
    norm = np.concatenate([np.zeros(14), np.ones(14), np.zeros(6), np.ones(6)])
    m = bl.bl_mlp_create()
    bl.bl_mlp_params_set(m, mlp.init_params(7), norm)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    first = None
    for it in range(600):
        loss, _ = bl.bl_mlp_grad(m, xd, yd)
        if it == 0:
            first = loss
        bl.bl_mlp_adam(m, lr=3e-3)
    last, _ = bl.bl_mlp_grad(m, xd, yd)
    print("teacher fit: loss %.4e -> %.4e" % (first, last))
    assert last < first / 20
    bl.bl_mlp_destroy(m)


def _overlap_state(seed=17, n=10):
    from paper_1005_2594_gb300 import workloads

    p = workloads.base_params(30, 26, 22, periodic=(1, 1, 0), R=(5.0, 2.5))
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(0, 30, n), rng.uniform(0, 26, n), rng.uniform(6.5, 15.5, n)])
    _, q = workloads.random_axes_and_quaternions(rng, n)
    V = rng.uniform(-0.02, 0.02, (n, 3))
    L = rng.uniform(-5.0, 5.0, (n, 3))
    return p, X, q, V, L


def test_pair_features_match_oracle():
    import torch

    import oracle
    from oracle import mlp
    from paper_1005_2594_gb300 import bloodlb as bl

    p, X, q, V, L = _overlap_state()
    orc, sim = oracle.Oracle(p), bl.Simulation(p)
    orc.set_particles(X, q, V, L)
    sim.set_particles(X, q, V, L)
    Om = orc.force_parts()["Om"]
    n = X.shape[0]
    pairs = np.array([(i, j) for i in range(n) for j in range(n) if i != j], dtype=np.int32)
    pd = torch.tensor(pairs, device="cuda")
    out = torch.zeros((len(pairs), 14), dtype=torch.float32, device="cuda")
    bl.bl_pair_features(sim.ctx, pd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    dims = (p["nx"], p["ny"], p["nz"])
    ref = np.array([mlp.pair_features(p["R_par"], p["R_perp"], dims, p["periodic"], X[i], q[i], V[i], Om[i],
                                      X[j], q[j], V[j], Om[j]) for i, j in pairs])
    scale = np.abs(ref).max(axis=0)
    err = (np.abs(got - ref) / scale).max()
    print("pair features: max error relative to each feature's range %.2e" % err)
    assert err < 1e-5


def test_prescribed_motion_matches_oracle():
    import oracle
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    p = workloads.base_params(32, 32, 32, periodic=(1, 1, 1), R=(3.5, 1.5))
    p["move_particles"] = 2
    X = np.array([[10.2, 16.1, 15.7], [19.4, 15.8, 16.3]])
    q = np.array([[1.0, 0, 0, 0], [np.cos(0.3), np.sin(0.3), 0, 0]])
    V = np.array([[0.02, 0.0, 0.0], [-0.02, 0.0, 0.0]])
    L = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, -0.5]])
    orc, sim = oracle.Oracle(p), bl.Simulation(p)
    orc.set_particles(X, q, V, L)
    sim.set_particles(X, q, V, L)
    for _ in range(20):
        orc.step(1)
        sim.step(1)
        np.testing.assert_array_equal(sim.owner(), orc.owner())
    po, pg = orc.particles(), sim.particles()
    for k in ("X", "q", "F", "T"):
        assert rel(pg[k], po[k]) < 1e-5, k
    np.testing.assert_array_equal(pg["V"], V)


@pytest.mark.parametrize("lo,speed", [(None, None), (0.5, None), (0.5, (0.01, 0.03))])
def test_attached_network_adds_rotated_correction_to_close_pairs(lo, speed):
    """A network whose output is its bias b3 adds R_i b3 once per close pair
    (gap below the cut-off, not below lo and relative speed within the
    window when those are given, from the oracle's features) to the
    potential part of the force and torque; the other pairs keep the plain
    method."""
    import oracle
    from oracle import mlp
    from paper_1005_2594_gb300 import bloodlb as bl

    p, X, q, V, L = _overlap_state(seed=23, n=12)
    cut = 2.0
    theta = np.zeros(mlp.N_PARAMS)
    b3 = np.array([0.1, -0.2, 0.3, 0.01, 0.02, -0.03])
    theta[-6:] = b3
    norm = np.concatenate([np.zeros(14), np.ones(14), np.zeros(6), np.ones(6)])
    m = bl.bl_mlp_create()
    bl.bl_mlp_params_set(m, theta, norm)
    a, b = bl.Simulation(p), bl.Simulation(p)
    if lo is None:
        bl.bl_mlp_attach(b.ctx, m, cut)
    elif speed is None:
        bl.bl_mlp_attach_range(b.ctx, m, lo, cut)
    else:
        bl.bl_mlp_attach_range(b.ctx, m, lo, cut, speed[0], speed[1])

    def selected(f):
        sp = np.linalg.norm(f[8:11])
        return f[7] < cut and (lo is None or f[7] >= lo) and (speed is None or speed[0] <= sp <= speed[1])

    for s in (a, b):
        s.set_particles(X, q, V, L)
        s.step(1)
        s.sync()
    dF = b.force_parts()["Fp"] - a.force_parts()["Fp"]
    dT = b.force_parts()["Tp"] - a.force_parts()["Tp"]
    orc = oracle.Oracle(p)
    orc.set_particles(X, q, V, L)
    Om = orc.force_parts()["Om"]
    dims = (p["nx"], p["ny"], p["nz"])
    n = X.shape[0]
    eF, eT = np.zeros((n, 3)), np.zeros((n, 3))
    npairs = 0
    for i in range(n):
        R = mlp.rotmat(q[i])
        for j in range(n):
            if i == j:
                continue
            f = mlp.pair_features(p["R_par"], p["R_perp"], dims, p["periodic"], X[i], q[i], V[i], Om[i], X[j],
                                  q[j], V[j], Om[j])
            if selected(f):
                eF[i] += R @ b3[:3]
                eT[i] += R @ b3[3:]
                npairs += 1
    assert npairs > 0
    if lo is not None:  # the range leaves out some close pairs
        n_close = sum(mlp.pair_features(p["R_par"], p["R_perp"], dims, p["periodic"], X[i], q[i], V[i], Om[i], X[j],
                                        q[j], V[j], Om[j])[7] < cut for i in range(n) for j in range(n) if i != j)
        assert n_close > npairs
    np.testing.assert_allclose(dF, eF, atol=1e-5)
    np.testing.assert_allclose(dT, eT, atol=1e-5)
    a.close()
    b.close()
    bl.bl_mlp_destroy(m)


def test_tube_flux_of_plasma_is_poiseuille():
    """The tube observables: plasma alone, driven by g in a tube of radius R,
    carries the Poiseuille flux pi R_eff^4 g / (8 nu) once developed, with the
    staircase's effective radius within half a node of R; its radial profile
    is the parabola g (R_eff^2 - r^2) / (4 nu) of a radius that agrees with
    the flux's, and the cell fraction is zero in every bin."""
    import math

    from paper_1005_2594_gb300 import rheology

    R = 10.0
    p, X, q, mask = rheology.tube_case(1, radius=R, length=16, cells=False, g=1e-5)
    Q, samples, _, (r, u, H, n) = rheology.run(p, X, q, mask, 6000, samples=4, profile_radius=R)
    nu = (p["tau"] - 0.5) / 3.0
    g = p["g"][0]
    R_eff = (8.0 * Q * nu / (math.pi * g)) ** 0.25
    R_prof = rheology.fit_poiseuille_radius(r, u, g, nu, n)
    dev = np.abs(u - rheology.poiseuille(r, R_prof, g, nu))[r < R - 2].max() / np.nanmax(u)
    print("tube radius %.1f: effective radius %.3f (flux), %.3f (profile), profile deviation %.1e, "
          "flux spread %.1e" % (R, R_eff, R_prof, dev, np.std(samples) / Q))
    assert abs(R_eff - R) < 0.5
    assert np.std(samples) / Q < 1e-3  # developed
    assert abs(R_prof - R_eff) < 0.25 and dev < 2e-2
    assert np.all(H[n > 0] == 0.0)
