"""Parity of the CUDA path with the FP64 oracle on general (non-affine)
quadrilateral meshes and with the 8-dof stress space of App. A.

The oracle builds each element's map, Jacobian and iMJwPSI matrix from the
four vertices (Gauss-Jordan inverse of the local mass matrix); the CUDA path
evaluates the bilinear map on the fly and factors the mass matrix from its
exact affine determinant.  Same bar as the rectilinear path: relative L2
<= 1e-11 and relative max <= 1e-10 per field.
"""
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


def errors(x, ref):
    x, ref = np.asarray(x), np.asarray(ref)
    n2 = np.linalg.norm(ref)
    ninf = np.abs(ref).max()
    return (np.linalg.norm(x - ref) / (n2 if n2 > 0 else 1.0),
            np.abs(x - ref).max() / (ninf if ninf > 0 else 1.0))


def assert_close(x, ref, what, l2_tol=L2_TOL, inf_tol=INF_TOL):
    l2, linf = errors(x, ref)
    assert l2 <= l2_tol and linf <= inf_tol, f"{what}: rel L2 {l2:.3e}, rel Linf {linf:.3e}"


def make_state(case, params=None):
    st = mevp.State(case["nx"], case["ny"], case["n_s"], vertex_xy=case["xy"],
                    params=params or case["params"])
    st.set_ice(case["H"], case["A"])
    st.set_forcing(case["tau"], case.get("vo"))
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    return st


def gpu_run(case, n_sub, params=None):
    with make_state(case, params) as st:
        st.begin_step()
        st.run_subcycles(n_sub)
        st.sync()
        return st.velocity(), st.stress()


def oracle_run(case, n_sub, params=None, openmp=False):
    return oracle.subcycles(case["nx"], case["ny"], case["xy"], case["n_s"], 1,
                            params or case["params"], case["H"], case["A"], case["tau"],
                            case["vel0"], case["S0"], n_sub, vo=case.get("vo"), openmp=openmp)


SHAPES = [(1, 1), (3, 2), (37, 23), (130, 5)]
GEOMS = ["perturbed", "wavy"]


# ---------------------------------------------------------------- stages
@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", GEOMS + ["uniform"])
@pytest.mark.parametrize("shape", SHAPES)
def test_strain_stage(n_s, geometry, shape):
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=140 + nx, geometry=geometry)
    rng = np.random.default_rng(nx * 11 + ny)
    vel = case["vel0"] + rng.normal(0, 1e-3, case["vel0"].shape)
    with make_state(case) as st:
        st.set_velocity(vel)
        E = st.strain()
    assert_close(E, oracle.strain(nx, ny, case["xy"], n_s, vel), "strain")


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", GEOMS + ["uniform"])
@pytest.mark.parametrize("shape", SHAPES)
def test_divergence_stage(n_s, geometry, shape):
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=150 + nx, geometry=geometry)
    with make_state(case) as st:
        F = st.force()
    Fo = oracle.divergence(nx, ny, case["xy"], n_s, case["S0"])
    # interior nodal forces are differences of O(sigma h) contributions
    l2, _ = errors(F, Fo)
    scale = np.abs(case["S0"]).max() * (case["L"] / nx)
    assert np.abs(F - Fo).max() <= 1e-13 * scale and l2 <= 1e-11


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("shape", SHAPES)
def test_lumped_mass(geometry, shape):
    nx, ny = shape
    case = W.small_case(nx, ny, 6, seed=160, geometry=geometry)
    case["H"] = case["H"] - 0.5  # some H < 0: the mass uses max(0, H)
    with make_state(case) as st:
        st.begin_step()
        m = st.read("NODAL_MASS")
    mo, _ = oracle.lumped(nx, ny, case["xy"], 6, 1, case["params"], case["H"])
    assert_close(m, mo, "mass", 1e-13, 1e-13)


# ---------------------------------------------------------------- subcycles
@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n_sub", [1, 7])
def test_subcycles_general(n_s, geometry, shape, n_sub):
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=170 + nx + ny, geometry=geometry)
    vg, Sg = gpu_run(case, n_sub)
    vo, So = oracle_run(case, n_sub)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n_sub", [1, 7])
def test_subcycles_dg8_rectilinear(shape, n_sub):
    nx, ny = shape
    case = W.small_case(nx, ny, 8, seed=180 + nx + ny)
    vg, Sg = gpu_run(case, n_sub)
    vo, So = oracle_run(case, n_sub)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


def test_dg8_mixed_precision_against_oracle():
    """The mixed path also takes the 8-dof stress (stated field error of the
    mixed path: velocity 5e-6 / 3e-5, stress 5e-5 / 2e-4)."""
    case = W.small_case(24, 18, 8, seed=181)
    with mevp.State(24, 18, 8, vertex_xy=case["xy"], params=case["params"],
                    precision="mixed") as st:
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"])
        st.set_velocity(case["vel0"])
        st.set_stress(case["S0"])
        st.begin_step()
        st.run_subcycles(7)
        vg, Sg = st.velocity(), st.stress()
    vo, So = oracle_run(case, 7)
    assert_close(vg, vo, "velocity", 5e-6, 3e-5)
    assert_close(Sg, So, "stress", 5e-5, 2e-4)


def test_perturbed_mesh_100_subcycles_from_rest():
    """64 x 64 perturbed mesh (8 km elements), DG2, 100 subcycles from rest
    under the cyclone: the whole subcycle loop on a general mesh."""
    nx = ny = 64
    case = W.small_case(nx, ny, 6, seed=191, geometry="perturbed", moving=False)
    vg, Sg = gpu_run(case, 100)
    vo, So = oracle_run(case, 100, openmp=True)
    assert np.abs(vo).max() > 1e-3
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


def test_wavy_mesh_256_short_horizon():
    """256 x 256 smoothly curvilinear mesh, DG2: 3 subcycles, every output."""
    nx = ny = 256
    case = W.small_case(nx, ny, 6, seed=193, geometry="wavy")
    vg, Sg = gpu_run(case, 3)
    vo, So = oracle_run(case, 3, openmp=True)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


def test_rotated_mesh_matches_rectilinear_result():
    """A rigidly rotated uniform mesh (affine elements, run by the general
    kernels) with rotated wind, velocity and stress gives the rotated
    velocity of the unrotated run on the rectilinear kernels (frame
    invariance of the method), and matches the oracle."""
    nx, ny = 9, 7
    case = W.small_case(nx, ny, 6, seed=195)
    # rotate the mesh, the wind, the velocity and the stress by theta
    th = 0.37
    c, s = np.cos(th), np.sin(th)
    R = np.array([[c, -s], [s, c]])
    rot = dict(case)
    rot["xy"] = case["xy"] @ R.T
    rot["tau"] = R @ case["tau"]
    rot["vel0"] = R @ case["vel0"]
    S = case["S0"]
    # sigma' = R sigma R^T, componentwise on the DG coefficients
    s11, s12, s22 = S[0], S[1], S[2]
    rot["S0"] = np.stack([c * c * s11 - 2 * c * s * s12 + s * s * s22,
                          c * s * (s11 - s22) + (c * c - s * s) * s12,
                          s * s * s11 + 2 * c * s * s12 + c * c * s22])
    vr, _ = gpu_run(rot, 5)
    vu, _ = gpu_run(case, 5)
    assert_close(vr, R @ vu, "rotated velocity", 1e-11, 1e-10)
    vo, So = oracle_run(rot, 5)
    vg, Sg = gpu_run(rot, 5)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("shape", [(1, 1), (37, 23), (130, 5)])
def test_mixed_general_mesh(n_s, geometry, shape):
    """The mixed path on general quads (FP32 map records, per-element FP32
    mass factorisation): fused and two-kernel launches bitwise equal, and
    within the mixed path's stated tolerances of the FP64 oracle (velocity
    5e-6 / 3e-5, stress 5e-5 / 2e-4)."""
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=400 + n_s + nx, geometry=geometry)
    got = []
    for fused in (1, 0):
        with mevp.State(nx, ny, n_s, vertex_xy=case["xy"], params=case["params"],
                        precision="mixed") as st:
            st.set_option(mevp.MEVP_OPT_FUSED, fused)
            st.set_ice(case["H"], case["A"])
            st.set_forcing(case["tau"])
            st.set_velocity(case["vel0"])
            st.set_stress(case["S0"])
            st.begin_step()
            st.run_subcycles(7)
            got.append((st.velocity(), st.stress()))
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])
    vo, So = oracle_run(case, 7)
    assert_close(got[0][0], vo, "velocity", 5e-6, 3e-5)
    assert_close(got[0][1], So, "stress", 5e-5, 2e-4)


def test_mixed_wavy_mesh_100_subcycles_from_rest():
    """64 x 64 curvilinear mesh, DG2, mixed path, 100 subcycles from rest."""
    nx = ny = 64
    case = W.small_case(nx, ny, 6, seed=411, geometry="wavy", moving=False)
    with mevp.State(nx, ny, 6, vertex_xy=case["xy"], params=case["params"],
                    precision="mixed") as st:
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"])
        st.begin_step()
        st.run_subcycles(100)
        vg, Sg = st.velocity(), st.stress()
    vo, So = oracle_run(case, 100, openmp=True)
    assert np.abs(vo).max() > 1e-3
    assert_close(vg, vo, "velocity", 5e-6, 3e-5)
    assert_close(Sg, So, "stress", 5e-5, 2e-4)


@pytest.mark.parametrize("geometry", ["perturbed", "curved"])
def test_mixed_adjoint_refusal(geometry):
    """The adjoint differentiates the FP64 path only."""
    case = W.small_case(6, 5, 6, seed=197, geometry=geometry)
    with mevp.State(6, 5, 6, vertex_xy=case["xy"], params=case["params"],
                    precision="mixed") as st:
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"])
        st.begin_step()
        with pytest.raises(mevp.MevpError) as e:
            st.adjoint_kinetic_energy(2, 1)
        assert e.value.code == -7


# ---------------------------------------------------------------- isoparametric
ISO_GEOMS = ["wavy_iso", "curved"]


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", ISO_GEOMS)
@pytest.mark.parametrize("shape", SHAPES)
def test_iso_stages(n_s, geometry, shape):
    """Curved (isoparametric Q2) elements: strain, forces and lumped mass
    against the oracle."""
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=500 + nx, geometry=geometry)
    rng = np.random.default_rng(nx * 13 + ny)
    vel = case["vel0"] + rng.normal(0, 1e-3, case["vel0"].shape)
    with make_state(case) as st:
        st.set_velocity(vel)
        E = st.strain()
        st.set_velocity(case["vel0"])
        F = st.force()
        st.begin_step()
        m = st.read("NODAL_MASS")
    assert_close(E, oracle.strain(nx, ny, case["xy"], n_s, vel), "strain")
    Fo = oracle.divergence(nx, ny, case["xy"], n_s, case["S0"])
    scale = np.abs(case["S0"]).max() * (case["L"] / nx)
    assert np.abs(F - Fo).max() <= 1e-13 * scale and errors(F, Fo)[0] <= 1e-11
    mo, _ = oracle.lumped(nx, ny, case["xy"], n_s, 1, case["params"], case["H"])
    assert_close(m, mo, "mass", 1e-13, 1e-13)


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", ISO_GEOMS)
@pytest.mark.parametrize("shape", SHAPES)
def test_iso_subcycles(n_s, geometry, shape):
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=520 + nx + ny, geometry=geometry)
    vg, Sg = gpu_run(case, 7)
    vo, So = oracle_run(case, 7)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


def test_iso_mesh_100_subcycles_from_rest():
    """64 x 64 randomly curved isoparametric mesh, DG2, 100 subcycles."""
    nx = ny = 64
    case = W.small_case(nx, ny, 6, seed=531, geometry="curved", moving=False)
    vg, Sg = gpu_run(case, 100)
    vo, So = oracle_run(case, 100, openmp=True)
    assert np.abs(vo).max() > 1e-3
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")


def test_iso_with_bilinear_nodes_matches_the_vertex_mesh():
    """Node positions that are the bilinear images of the vertices describe
    the same elements as the vertex mesh: the two GPU paths agree."""
    nx, ny = 17, 11
    case = W.small_case(nx, ny, 6, seed=533, geometry="perturbed")
    iso = dict(case, xy=W.node_coords(nx, ny, case["xy"]).T.copy())
    va, Sa = gpu_run(case, 9)
    vb, Sb = gpu_run(iso, 9)
    assert_close(vb, va, "velocity", 1e-12, 1e-11)
    assert_close(Sb, Sa, "stress", 1e-12, 1e-11)


@pytest.mark.parametrize("n_a", [1, 3, 6])
def test_iso_advection(n_a):
    nx, ny = 19, 13
    case = W.small_case(nx, ny, 6, seed=540 + n_a, geometry="curved")
    ne = nx * ny
    rng = np.random.default_rng(n_a)
    H = np.vstack([rng.uniform(0.5, 1.5, ne)] + [rng.uniform(-0.2, 0.2, ne)] * (n_a - 1))
    A = np.vstack([rng.uniform(0.8, 0.95, ne)] + [rng.uniform(-0.05, 0.05, ne)] * (n_a - 1))
    vel = 3.0 * case["vel0"]
    with mevp.State(nx, ny, 6, vertex_xy=case["xy"], n_adv=n_a, params=case["params"]) as st:
        st.set_ice(H, A)
        st.set_forcing(case["tau"])
        st.set_velocity(vel)
        st.advect(4)
        Hg, Ag = st.read("H").reshape(n_a, ne), st.read("A").reshape(n_a, ne)
    Ho, Ao = oracle.advect(nx, ny, case["xy"], n_a, vel, case["params"]["dt"], 4, H, A)
    assert_close(Hg, Ho, "H")
    assert_close(Ag, Ao, "A")


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("geometry", ISO_GEOMS)
@pytest.mark.parametrize("shape", [(1, 1), (37, 23), (130, 5)])
def test_mixed_iso_mesh(n_s, geometry, shape):
    """The mixed path on curved (isoparametric) meshes: FP32 node offsets from
    the centre node, Jacobians at the Gauss points in shared memory; fused
    and two-kernel launches bitwise equal, and within the mixed path's stated
    tolerances of the FP64 oracle (velocity 5e-6 / 3e-5, stress 5e-5 / 2e-4)."""
    nx, ny = shape
    case = W.small_case(nx, ny, n_s, seed=560 + n_s + nx, geometry=geometry)
    got = []
    for fused in (1, 0):
        with mevp.State(nx, ny, n_s, vertex_xy=case["xy"], params=case["params"],
                        precision="mixed") as st:
            st.set_option(mevp.MEVP_OPT_FUSED, fused)
            st.set_ice(case["H"], case["A"])
            st.set_forcing(case["tau"])
            st.set_velocity(case["vel0"])
            st.set_stress(case["S0"])
            st.begin_step()
            st.run_subcycles(7)
            got.append((st.velocity(), st.stress()))
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])
    vo, So = oracle_run(case, 7)
    assert_close(got[0][0], vo, "velocity", 5e-6, 3e-5)
    assert_close(got[0][1], So, "stress", 5e-5, 2e-4)


@pytest.mark.parametrize("n_a", [3, 6])
def test_mixed_iso_with_dg_ice(n_a):
    """Mixed path, curved mesh, DG1/DG2 H and A (FP32 strength per Gauss
    point)."""
    nx, ny = 23, 17
    case = W.small_case(nx, ny, 6, seed=570 + n_a, geometry="curved")
    ne = nx * ny
    rng = np.random.default_rng(571 + n_a)
    H = np.vstack([rng.uniform(0.5, 1.8, ne)] + [rng.uniform(-0.3, 0.3, ne)] * (n_a - 1))
    A = np.vstack([rng.uniform(0.75, 0.97, ne)] + [rng.uniform(-0.08, 0.08, ne)] * (n_a - 1))
    with mevp.State(nx, ny, 6, vertex_xy=case["xy"], n_adv=n_a, params=case["params"],
                    precision="mixed") as st:
        st.set_ice(H, A)
        st.set_forcing(case["tau"])
        st.set_velocity(case["vel0"])
        st.set_stress(case["S0"])
        st.begin_step()
        st.run_subcycles(7)
        vg, Sg = st.velocity(), st.stress()
    vo, So = oracle.subcycles(nx, ny, case["xy"], 6, n_a, case["params"], H, A, case["tau"],
                              case["vel0"], case["S0"], 7)
    assert_close(vg, vo, "velocity", 5e-6, 3e-5)
    assert_close(Sg, So, "stress", 5e-5, 2e-4)


def test_mixed_iso_mesh_100_subcycles_from_rest():
    """64 x 64 curved mesh, DG2, mixed path, 100 subcycles from rest."""
    nx = ny = 64
    case = W.small_case(nx, ny, 6, seed=575, geometry="wavy_iso", moving=False)
    with mevp.State(nx, ny, 6, vertex_xy=case["xy"], params=case["params"],
                    precision="mixed") as st:
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"])
        st.begin_step()
        st.run_subcycles(100)
        vg, Sg = st.velocity(), st.stress()
    vo, So = oracle_run(case, 100, openmp=True)
    assert np.abs(vo).max() > 1e-3
    assert_close(vg, vo, "velocity", 5e-6, 3e-5)
    assert_close(Sg, So, "stress", 5e-5, 2e-4)


@pytest.mark.parametrize("workload", ["mesh1024_dg2_wavy", "mesh1024_dg2_iso"])
def test_curvilinear_1024_max_size(workload):
    """The 1024x1024 curvilinear workloads (1M elements, 4.2M nodes) in the
    benchmark's launch configuration: 2 FP64 subcycles from a moving state at
    the stability-bound alpha = beta, every output against the oracle, and
    the mixed path at its stated tolerances."""
    case = W.make_case(workload)
    p = dict(case["params"], alpha=8000.0, beta=8000.0)
    case["vel0"] = W.smooth_velocity(1024, 1024, 5, amp=0.05)
    vg, Sg = gpu_run(case, 2, params=p)
    vo, So = oracle_run(case, 2, params=p, openmp=True)
    assert_close(vg, vo, "velocity")
    assert_close(Sg, So, "stress")
    with mevp.State(1024, 1024, 6, vertex_xy=case["xy"], params=p, precision="mixed") as st:
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"])
        st.set_velocity(case["vel0"])
        st.set_stress(case["S0"])
        st.begin_step()
        st.run_subcycles(2)
        vm, Sm = st.velocity(), st.stress()
    assert_close(vm, vo, "velocity (mixed)", 5e-6, 3e-5)
    assert_close(Sm, So, "stress (mixed)", 5e-5, 2e-4)
