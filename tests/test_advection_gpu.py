"""Parity of the CUDA advection of H and A (DG upwind, SSP Runge-Kutta) and of
the momentum subcycle with DG1/DG2 ice fields against the FP64 oracle, and a
loop of whole outer steps (advect, begin_step, subcycles)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_00466_gb300 import mevp  # noqa: E402
from paper_2402_00466_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

L2_TOL = 1e-11
INF_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mevp.load()


def assert_close(x, ref, what, l2_tol=L2_TOL, inf_tol=INF_TOL):
    x, ref = np.asarray(x), np.asarray(ref)
    n2, ninf = np.linalg.norm(ref), np.abs(ref).max()
    l2 = np.linalg.norm(x - ref) / (n2 if n2 > 0 else 1.0)
    linf = np.abs(x - ref).max() / (ninf if ninf > 0 else 1.0)
    assert l2 <= l2_tol and linf <= inf_tol, f"{what}: rel L2 {l2:.3e}, rel Linf {linf:.3e}"


def dg_ice(ne, n_a, seed):
    """DG coefficients (n_a, N_e) of H and A: mean plus small slopes/curvatures."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = np.zeros((n_a, ne)); A = np.zeros((n_a, ne))
    H[0] = rng.uniform(0.5, 1.8, ne)
    A[0] = rng.uniform(0.75, 0.97, ne)
    if n_a > 1:
        H[1:] = rng.uniform(-0.3, 0.3, (n_a - 1, ne))
        A[1:] = rng.uniform(-0.08, 0.08, (n_a - 1, ne))
    return H, A


def make_state(case, n_a, H, A, params=None, precision="fp64"):
    st = mevp.State(case["nx"], case["ny"], case["n_s"], vertex_xy=case["xy"], n_adv=n_a,
                    params=params or case["params"], precision=precision)
    st.set_ice(H, A)
    st.set_forcing(case["tau"], case.get("vo"))
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    return st


SHAPES = [(1, 1), (3, 2), (37, 23), (130, 5)]


@pytest.mark.parametrize("n_a", [1, 3, 6])
@pytest.mark.parametrize("geometry", ["uniform", "perturbed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_advect_parity(n_a, geometry, shape):
    """5 advection steps with the velocity held fixed (zero on the boundary)."""
    nx, ny = shape
    case = W.small_case(nx, ny, 6, seed=210 + nx, geometry=geometry)
    ne = nx * ny
    H, A = dg_ice(ne, n_a, 211 + ny)
    vel = 3.0 * case["vel0"]  # up to 0.3 m/s
    case["vel0"] = vel
    with make_state(case, n_a, H, A) as st:
        st.advect(5)
        Hg, Ag = st.read("H"), st.read("A")
    Ho, Ao = oracle.advect(nx, ny, case["xy"], n_a, vel, case["params"]["dt"], 5, H, A)
    assert np.abs(Ho - H).max() > 1e-8 or ne == 1  # something moved
    assert_close(Hg.reshape(n_a, ne), Ho, "H")
    assert_close(Ag.reshape(n_a, ne), Ao, "A")


@pytest.mark.parametrize("n_a", [1, 3, 6])
def test_advect_with_boundary_inflow(n_a):
    """A velocity that crosses the domain boundary: inflow edges take the
    element's own trace on both sides."""
    nx, ny = 9, 7
    case = W.small_case(nx, ny, 3, seed=220, geometry="perturbed")
    ne, nn = nx * ny, (2 * nx + 1) * (2 * ny + 1)
    nc = W.node_coords(nx, ny, case["xy"])
    L = case["L"]
    vel = np.stack([0.3 + 0.1 * np.sin(3 * nc[1] / L), -0.2 + 0.1 * np.cos(2 * nc[0] / L)])
    case["vel0"] = vel
    H, A = dg_ice(ne, n_a, 221)
    with make_state(case, n_a, H, A) as st:
        st.advect(3)
        Hg, Ag = st.read("H"), st.read("A")
    Ho, Ao = oracle.advect(nx, ny, case["xy"], n_a, vel, case["params"]["dt"], 3, H, A)
    assert_close(Hg.reshape(n_a, ne), Ho, "H")
    assert_close(Ag.reshape(n_a, ne), Ao, "A")


@pytest.mark.parametrize("n_a", [1, 3, 6])
def test_advect_conserves_mass(n_a):
    """v = 0 on the boundary: sum_K int_K H is conserved on the GPU over 50
    steps (uniform mesh: int_K H = area * H_0)."""
    nx, ny = 40, 30
    case = W.small_case(nx, ny, 6, seed=230)
    ne = nx * ny
    H, A = dg_ice(ne, n_a, 231)
    case["vel0"] = 4.0 * case["vel0"]
    with make_state(case, n_a, H, A) as st:
        st.advect(50)
        Hg = st.read("H").reshape(n_a, ne)
    assert abs(Hg[0].sum() - H[0].sum()) <= 1e-13 * H[0].sum()
    assert np.abs(Hg - H).max() > 1e-4


@pytest.mark.parametrize("n_a", [3, 6])
@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", ["uniform", "perturbed"])
def test_subcycles_with_dg_ice(n_a, n_s, geometry):
    """Momentum subcycles with DG1/DG2 H, A: the ice strength and the lumped
    mass vary inside the element (Listing 1 evaluates H, A at the Gauss
    points)."""
    nx, ny = 23, 17
    case = W.small_case(nx, ny, n_s, seed=240 + n_a + n_s, geometry=geometry)
    ne = nx * ny
    H, A = dg_ice(ne, n_a, 241 + n_s)
    H[0, :7] = 0.05  # thin ice with slopes: max(0, H) clips inside elements
    with make_state(case, n_a, H, A) as st:
        st.begin_step()
        m = st.read("NODAL_MASS")
        st.run_subcycles(7)
        vg, Sg = st.velocity(), st.stress()
    mo, _ = oracle.lumped(nx, ny, case["xy"], n_s, n_a, case["params"], H)
    assert_close(m, mo, "mass", 1e-13, 1e-13)
    vo, So = oracle.subcycles(nx, ny, case["xy"], n_s, n_a, case["params"], H, A, case["tau"],
                              case["vel0"], case["S0"], 7)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


@pytest.mark.parametrize("n_a", [1, 3])
@pytest.mark.parametrize("geometry", ["uniform", "perturbed"])
def test_outer_steps(n_a, geometry):
    """Three outer steps of the solution procedure of Sec. 2 (advect with the
    current velocity, then the momentum subcycles), 16 km mesh from rest."""
    nx = ny = 32
    case = W.small_case(nx, ny, 6, seed=250, geometry=geometry, moving=False)
    ne = nx * ny
    H, A = dg_ice(ne, n_a, 251)
    p = case["params"]
    vel, S = case["vel0"].copy(), case["S0"].copy()
    Ho, Ao = H.copy(), A.copy()
    for _ in range(3):
        Ho, Ao = oracle.advect(nx, ny, case["xy"], n_a, vel, p["dt"], 1, Ho, Ao)
        vel, S = oracle.subcycles(nx, ny, case["xy"], 6, n_a, p, Ho, Ao, case["tau"], vel, S, 40)
    with make_state(case, n_a, H, A) as st:
        for _ in range(3):
            st.advect(1)
            st.begin_step()
            st.run_subcycles(40)
        vg, Sg = st.velocity(), st.stress()
        Hg = st.read("H").reshape(n_a, ne)
    assert np.abs(vel).max() > 1e-3
    assert_close(Hg, Ho, "H")
    assert_close(vg, vel, "velocity")
    assert_close(Sg, S, "stress")


def test_mixed_state_advects_with_its_velocity():
    """The mixed path advects DG0 ice with its (compensated) velocity."""
    nx, ny = 20, 16
    case = W.small_case(nx, ny, 6, seed=260)
    ne = nx * ny
    H, A = dg_ice(ne, 1, 261)
    with make_state(case, 1, H, A, precision="mixed") as st:
        st.begin_step()
        st.run_subcycles(5)
        v = st.velocity()
        st.advect(2)
        Hg = st.read("H")
    Ho, _ = oracle.advect(nx, ny, case["xy"], 1, v, case["params"]["dt"], 2, H, A)
    assert_close(Hg.reshape(1, ne), Ho, "H")


@pytest.mark.parametrize("n_a", [3, 6])
@pytest.mark.parametrize("n_s", [3, 6])
def test_mixed_subcycles_with_dg_ice(n_a, n_s):
    """The mixed path with DG1/DG2 H, A (FP32 strength per Gauss point),
    fused and two-kernel launches, against the FP64 oracle at the mixed
    path's stated tolerances (velocity 5e-6 / 3e-5, stress 5e-5 / 2e-4)."""
    nx, ny = 37, 23
    case = W.small_case(nx, ny, n_s, seed=280 + n_a + n_s)
    H, A = dg_ice(nx * ny, n_a, 281 + n_s)
    H[0, :9] = 0.05
    vo, So = oracle.subcycles(nx, ny, case["xy"], n_s, n_a, case["params"], H, A, case["tau"],
                              case["vel0"], case["S0"], 7)
    got = []
    for fused in (1, 0):
        with make_state(case, n_a, H, A, precision="mixed") as st:
            st.set_option(mevp.MEVP_OPT_FUSED, fused)
            st.begin_step()
            st.run_subcycles(7)
            got.append((st.velocity(), st.stress()))
    for vg, Sg in got:
        assert_close(vg, vo, "velocity", 5e-6, 3e-5)
        assert_close(Sg, So, "stress", 5e-5, 2e-4)
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])


def test_mixed_outer_steps_with_dg2_ice():
    """Three outer steps (advect DG2 H, A; begin_step; 40 mixed subcycles)
    against the oracle's."""
    nx = ny = 32
    case = W.small_case(nx, ny, 6, seed=290, moving=False)
    H, A = dg_ice(nx * ny, 6, 291)
    p = case["params"]
    vel, S = case["vel0"].copy(), case["S0"].copy()
    Ho, Ao = H.copy(), A.copy()
    for _ in range(3):
        Ho, Ao = oracle.advect(nx, ny, case["xy"], 6, vel, p["dt"], 1, Ho, Ao)
        vel, S = oracle.subcycles(nx, ny, case["xy"], 6, 6, p, Ho, Ao, case["tau"], vel, S, 40)
    with make_state(case, 6, H, A, precision="mixed") as st:
        for _ in range(3):
            st.advect(1)
            st.begin_step()
            st.run_subcycles(40)
        vg, Sg = st.velocity(), st.stress()
        Hg = st.read("H").reshape(6, nx * ny)
    assert_close(Hg, Ho, "H", 1e-6, 1e-5)
    assert_close(vg, vel, "velocity", 5e-6, 3e-5)
    assert_close(Sg, S, "stress", 5e-5, 2e-4)


def test_dg_ice_refusals():
    case = W.small_case(6, 5, 6, seed=270)
    H, A = dg_ice(30, 3, 271)
    with make_state(case, 3, H, A) as st:
        st.begin_step()
        with pytest.raises(mevp.MevpError) as e:
            st.advect(-1)
        assert e.value.code == -1
