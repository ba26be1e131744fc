"""Hand-written adjoint of the FP64 subcycle: gradient of the kinetic energy
after n subcycles with respect to the per-element P* field and the nodal wind
stress, checked by central finite differences of the GPU forward (per-element
and nodal directions) and of the CPU oracle (nodal and uniform-P* directions),
independent of the checkpoint interval, and through torch.autograd."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_00466_gb300 import mevp  # noqa: E402
from paper_2402_00466_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mevp.load()


def setup(case, pstar=None, tau=None, params=None):
    st = mevp.State(case["nx"], case["ny"], case["n_s"], vertex_xy=case["xy"],
                    params=params or case["params"])
    reset(st, case, pstar, tau)
    return st


def reset(st, case, pstar=None, tau=None):
    st.set_ice(case["H"], case["A"])
    st.set_forcing(case["tau"] if tau is None else tau)
    st.set_strength_field(pstar)
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    st.begin_step()


def J_gpu(st, case, n, pstar, tau):
    reset(st, case, pstar, tau)
    st.run_subcycles(n)
    v = st.velocity()
    m = st.read("NODAL_MASS")
    return 0.5 * float(np.sum(m * (v[0] ** 2 + v[1] ** 2)))


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_adjoint_matches_gpu_finite_differences(n_s):
    case = W.small_case(12, 10, n_s, seed=81)
    n = 30
    ne, nn, _ = W.sizes(12, 10)
    P0 = np.full(ne, case["params"]["Pstar"])
    st = setup(case, P0)
    J, gP, gT = st.adjoint_kinetic_energy(n, checkpoint_every=7)
    assert abs(J - J_gpu(st, case, n, P0, case["tau"])) <= 1e-12 * abs(J)
    rng = np.random.default_rng(3)
    for _ in range(4):
        dP = rng.standard_normal(ne)
        dT = rng.standard_normal((2, nn))
        for dirP, dirT in ((dP, 0 * dT), (0 * dP, dT)):
            eP = 1e-6 * P0.mean() / np.abs(dirP).max() if np.any(dirP) else 0.0
            eT = 1e-6 * np.abs(case["tau"]).max() / np.abs(dirT).max() if np.any(dirT) else 0.0
            Jp = J_gpu(st, case, n, P0 + eP * dirP, case["tau"] + eT * dirT)
            Jm = J_gpu(st, case, n, P0 - eP * dirP, case["tau"] - eT * dirT)
            fd = (Jp - Jm) / 2.0
            ad = eP * float(gP @ dirP) + eT * float(np.sum(gT * dirT))
            assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-14 * abs(J), (fd, ad)
    st.close()


@pytest.mark.parametrize("n_a", [3, 6])
@pytest.mark.parametrize("n_s", [3, 6])
def test_adjoint_with_dg_ice_matches_gpu_finite_differences(n_a, n_s):
    """DG1/DG2 H and A: the strength varies over the element (P_g at the Gauss
    points, the -P/2 term projected per point); per-element P* and nodal
    wind-stress directions against central differences of the GPU forward."""
    nx, ny = 11, 9
    case = W.small_case(nx, ny, n_s, seed=91 + n_a)
    ne, nn, _ = W.sizes(nx, ny)
    rng = np.random.default_rng(92 + n_a)
    H = np.vstack([rng.uniform(0.6, 1.6, ne)] + [rng.uniform(-0.2, 0.2, ne)] * (n_a - 1))
    A = np.vstack([rng.uniform(0.8, 0.95, ne)] + [rng.uniform(-0.04, 0.04, ne)] * (n_a - 1))
    case = dict(case, H=H, A=A)
    n = 25
    P0 = case["params"]["Pstar"] * rng.uniform(0.8, 1.2, ne)
    st = mevp.State(nx, ny, n_s, vertex_xy=case["xy"], n_adv=n_a, params=case["params"])
    reset(st, case, P0)
    J, gP, gT = st.adjoint_kinetic_energy(n, checkpoint_every=6)
    assert abs(J - J_gpu(st, case, n, P0, case["tau"])) <= 1e-12 * abs(J)
    for _ in range(3):
        dP = rng.standard_normal(ne)
        dT = rng.standard_normal((2, nn))
        for dirP, dirT in ((dP, 0 * dT), (0 * dP, dT)):
            eP = 1e-6 * P0.mean() / np.abs(dirP).max() if np.any(dirP) else 0.0
            eT = 1e-6 * np.abs(case["tau"]).max() / np.abs(dirT).max() if np.any(dirT) else 0.0
            Jp = J_gpu(st, case, n, P0 + eP * dirP, case["tau"] + eT * dirT)
            Jm = J_gpu(st, case, n, P0 - eP * dirP, case["tau"] - eT * dirT)
            fd = (Jp - Jm) / 2.0
            ad = eP * float(gP @ dirP) + eT * float(np.sum(gT * dirT))
            assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-14 * abs(J), (fd, ad)
    st.close()


@pytest.mark.parametrize("n_a", [1, 3])
@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", ["perturbed", "wavy", "curved"])
def test_adjoint_general_mesh_matches_gpu_finite_differences(geometry, n_s, n_a):
    """Bilinear and curved elements (the Gauss-point reverse mode with the
    stored mass factors and Jacobians): per-element P* and nodal wind-stress
    directions against central differences of the GPU forward."""
    nx, ny = 10, 8
    case = W.small_case(nx, ny, n_s, seed=111 + n_s + n_a, geometry=geometry)
    ne, nn, _ = W.sizes(nx, ny)
    rng = np.random.default_rng(112 + n_s)
    if n_a > 1:
        H = np.vstack([rng.uniform(0.6, 1.6, ne)] + [rng.uniform(-0.2, 0.2, ne)] * (n_a - 1))
        A = np.vstack([rng.uniform(0.8, 0.95, ne)] + [rng.uniform(-0.04, 0.04, ne)] * (n_a - 1))
        case = dict(case, H=H, A=A)
    n = 20
    P0 = case["params"]["Pstar"] * rng.uniform(0.8, 1.2, ne)
    st = mevp.State(nx, ny, n_s, vertex_xy=case["xy"], n_adv=n_a, params=case["params"])
    reset(st, case, P0)
    J, gP, gT = st.adjoint_kinetic_energy(n, checkpoint_every=6)
    assert abs(J - J_gpu(st, case, n, P0, case["tau"])) <= 1e-12 * abs(J)
    for _ in range(3):
        dP = rng.standard_normal(ne)
        dT = rng.standard_normal((2, nn))
        for dirP, dirT in ((dP, 0 * dT), (0 * dP, dT)):
            eP = 1e-6 * P0.mean() / np.abs(dirP).max() if np.any(dirP) else 0.0
            eT = 1e-6 * np.abs(case["tau"]).max() / np.abs(dirT).max() if np.any(dirT) else 0.0
            Jp = J_gpu(st, case, n, P0 + eP * dirP, case["tau"] + eT * dirT)
            Jm = J_gpu(st, case, n, P0 - eP * dirP, case["tau"] - eT * dirT)
            fd = (Jp - Jm) / 2.0
            ad = eP * float(gP @ dirP) + eT * float(np.sum(gT * dirT))
            assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-14 * abs(J), (fd, ad)
    st.close()


def test_adjoint_general_mesh_matches_oracle_finite_differences():
    """Curved mesh: wind-stress directions and a uniform P* direction against
    central differences of the FP64 oracle."""
    nx, ny = 8, 7
    case = W.small_case(nx, ny, 6, seed=121, geometry="curved")
    n = 15
    ne, nn, _ = W.sizes(nx, ny)
    st = setup(case)
    J, gP, gT = st.adjoint_kinetic_energy(n, checkpoint_every=4)
    st.close()
    m, _ = oracle.lumped(nx, ny, case["xy"], 6, 1, case["params"], case["H"])

    def J_orc(params, tau):
        v, _ = oracle.subcycles(nx, ny, case["xy"], 6, 1, params, case["H"], case["A"], tau,
                                case["vel0"], case["S0"], n)
        return 0.5 * float(np.sum(m * (v[0] ** 2 + v[1] ** 2)))

    p0 = case["params"]
    assert abs(J_orc(p0, case["tau"]) - J) <= 1e-10 * abs(J)
    eps = 1e-6 * p0["Pstar"]
    fd = (J_orc(dict(p0, Pstar=p0["Pstar"] + eps), case["tau"]) -
          J_orc(dict(p0, Pstar=p0["Pstar"] - eps), case["tau"])) / (2 * eps)
    assert abs(fd - gP.sum()) <= 1e-5 * abs(fd), (fd, gP.sum())
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = rng.standard_normal((2, nn))
        # a larger step than elsewhere: a direction whose derivative is small
        # against the terms it sums (cancellation) needs the rounding of the
        # two oracle runs divided by less
        e = 1e-5 * np.abs(case["tau"]).max() / np.abs(d).max()
        fd = (J_orc(p0, case["tau"] + e * d) - J_orc(p0, case["tau"] - e * d)) / (2 * e)
        ad = float(np.sum(gT * d))
        scale = float(np.sum(np.abs(gT * d)))
        assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-8 * scale, (fd, ad, scale)


def test_adjoint_matches_oracle_finite_differences():
    """Directional derivatives against central differences of the FP64 oracle:
    nodal wind-stress directions and a uniform P* direction (the oracle takes
    P* as a scalar parameter)."""
    case = W.small_case(8, 7, 6, seed=83)
    n = 20
    ne, nn, _ = W.sizes(8, 7)
    st = setup(case)
    J, gP, gT = st.adjoint_kinetic_energy(n, checkpoint_every=6)
    st.close()
    m, _ = oracle.lumped(8, 7, case["xy"], 6, 1, case["params"], case["H"])

    def J_orc(params, tau):
        v, _ = oracle.subcycles(8, 7, case["xy"], 6, 1, params, case["H"], case["A"], tau,
                                case["vel0"], case["S0"], n)
        return 0.5 * float(np.sum(m * (v[0] ** 2 + v[1] ** 2)))

    p0 = case["params"]
    assert abs(J_orc(p0, case["tau"]) - J) <= 1e-10 * abs(J)
    eps = 1e-6 * p0["Pstar"]
    fd = (J_orc(dict(p0, Pstar=p0["Pstar"] + eps), case["tau"]) -
          J_orc(dict(p0, Pstar=p0["Pstar"] - eps), case["tau"])) / (2 * eps)
    assert abs(fd - gP.sum()) <= 1e-5 * abs(fd), (fd, gP.sum())
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = rng.standard_normal((2, nn))
        e = 1e-6 * np.abs(case["tau"]).max() / np.abs(d).max()
        fd = (J_orc(p0, case["tau"] + e * d) - J_orc(p0, case["tau"] - e * d)) / (2 * e)
        ad = float(np.sum(gT * d))
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


def test_checkpoint_interval_does_not_change_the_gradient():
    """Bitwise the same gradient for every checkpoint interval, including
    k >= n (every velocity recorded by the forward sweep, no recomputation)."""
    case = W.small_case(9, 9, 6, seed=85)
    out = []
    for k in (1, 4, 13, 24, 25, 1000):
        st = setup(case)
        out.append(st.adjoint_kinetic_energy(25, checkpoint_every=k))
        v_after = st.velocity()
        st.close()
        st2 = setup(case)
        st2.run_subcycles(25)
        assert np.array_equal(v_after, st2.velocity())  # the state ends after the n subcycles
        st2.close()
    for J, gP, gT in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(gP, out[0][1]) and np.array_equal(gT, out[0][2])


def test_autograd_function():
    case = W.small_case(10, 8, 3, seed=87)
    ne, nn, _ = W.sizes(10, 8)
    st = setup(case)
    p = torch.full((ne,), case["params"]["Pstar"], dtype=torch.float64, device="cuda",
                   requires_grad=True)
    t = torch.tensor(case["tau"], dtype=torch.float64, device="cuda", requires_grad=True)
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    J = mevp.kinetic_energy(st, p, t, 15, checkpoint_every=5)
    (3.0 * J).backward()
    reset(st, case, p.detach().cpu().numpy(), case["tau"])
    J2, gP, gT = st.adjoint_kinetic_energy(15, checkpoint_every=5)
    assert abs(float(J.detach()) - J2) <= 1e-14 * abs(J2)
    assert np.allclose(p.grad.cpu().numpy(), 3.0 * gP, rtol=1e-14, atol=0)
    assert np.allclose(t.grad.cpu().numpy(), 3.0 * gT, rtol=1e-14, atol=0)
    st.close()


def test_adjoint_mesh256_dg1_configuration():
    """256x256 DG1 FP64, 100 subcycles, checkpoints every 10: 20 seeded
    directions (10 per-element P*, 10 nodal wind stress), central differences
    with a step of 1e-6 relative.  At the stability-bound alpha = beta = 2000
    of this 2 km mesh: at alpha = beta = 300 the iteration amplifies any
    perturbation about 20-fold per subcycle until it saturates, so J is not
    differentiable on the scale of the difference step there."""
    case = W.make_case("mesh256_dg1")
    case["params"] = dict(case["params"], alpha=2000.0, beta=2000.0)
    n = 100
    ne, nn, _ = W.sizes(256, 256)
    P0 = np.full(ne, case["params"]["Pstar"])
    st = setup(case, P0)
    J, gP, gT = st.adjoint_kinetic_energy(n, checkpoint_every=10)
    rng = np.random.default_rng(7)
    worst = 0.0
    for i in range(20):
        if i % 2 == 0:
            d = rng.standard_normal(ne)
            e = 1e-6 * P0.mean() / np.abs(d).max()
            fd = (J_gpu(st, case, n, P0 + e * d, case["tau"]) -
                  J_gpu(st, case, n, P0 - e * d, case["tau"])) / 2
            ad = e * float(gP @ d)
        else:
            d = rng.standard_normal((2, nn))
            e = 1e-6 * np.abs(case["tau"]).max() / np.abs(d).max()
            fd = (J_gpu(st, case, n, P0, case["tau"] + e * d) -
                  J_gpu(st, case, n, P0, case["tau"] - e * d)) / 2
            ad = e * float(np.sum(gT * d))
        worst = max(worst, abs(fd - ad) / abs(ad))
    st.close()
    print(f"mesh256_dg1 adjoint vs central differences: worst relative error {worst:.2e}")
    assert worst <= 1e-4, worst


@pytest.mark.parametrize("n_s,n_a,geometry", [(6, 1, "uniform"), (3, 3, "uniform"),
                                              (6, 1, "curved"), (8, 3, "perturbed")])
def test_adjoint_per_element_pstar_matches_oracle_finite_differences(n_s, n_a, geometry):
    """dJ/dP*_K against central differences of the FP64 oracle run with a
    per-element P* field: the five elements with the largest gradient one by
    one, and five random directions over all elements (relative steps 1e-4
    and 5e-5, Richardson-combined); rectilinear, curved (isoparametric) and
    perturbed (bilinear) meshes."""
    nx, ny = 8, 7
    case = W.small_case(nx, ny, n_s, seed=85 + n_s, geometry=geometry)
    ne, nn, _ = W.sizes(nx, ny)
    n = 20
    p0 = case["params"]
    rng = np.random.default_rng(11 + n_a)
    H, A = case["H"], case["A"]
    if n_a > 1:
        H = np.concatenate([H, rng.uniform(-0.2, 0.2, (n_a - 1, ne))])
        A = np.concatenate([A * 0.95, rng.uniform(-0.03, 0.03, (n_a - 1, ne))])
    field = p0["Pstar"] * rng.uniform(0.7, 1.3, ne)
    st = mevp.State(nx, ny, n_s, vertex_xy=case["xy"], n_adv=n_a, params=p0)
    st.set_ice(H, A)
    st.set_forcing(case["tau"])
    st.set_strength_field(field)
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    st.begin_step()
    J, gP, _ = st.adjoint_kinetic_energy(n, checkpoint_every=6)
    st.close()
    m, _ = oracle.lumped(nx, ny, case["xy"], n_s, n_a, p0, H)

    def J_orc(pk):
        v, _ = oracle.subcycles(nx, ny, case["xy"], n_s, n_a, p0, H, A, case["tau"],
                                case["vel0"], case["S0"], n, Pstar_K=pk)
        return 0.5 * float(np.sum(m * (v[0] ** 2 + v[1] ** 2)))

    assert abs(J_orc(field) - J) <= 1e-10 * abs(J)
    dirs = [np.eye(ne)[K] for K in np.argsort(-np.abs(gP))[:5]]
    dirs += [rng.standard_normal(ne) for _ in range(5)]
    for d in dirs:
        # central differences at steps e and e/2, Richardson-combined so that
        # their O(e^2) truncation error cancels; steps large enough that the
        # rounding noise of the two oracle runs, which the iteration amplifies,
        # stays far below the tolerance
        e = 1e-4 * field.mean() / np.abs(d).max()
        fd1 = (J_orc(field + e * d) - J_orc(field - e * d)) / (2 * e)
        fd2 = (J_orc(field + 0.5 * e * d) - J_orc(field - 0.5 * e * d)) / e
        fd = (4.0 * fd2 - fd1) / 3.0
        ad = float(gP @ d)
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, fd1, fd2, ad)
