"""Ensembles of uneven domains advanced together (one persistent launch per
subcycle in the mixed precision, element + node launches in FP64): bitwise the
results of stepping each member alone, for every work decomposition, with and
without CUDA graph replay; the autotuner leaves no trace in the results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_00466_gb300 import mevp  # noqa: E402
from paper_2402_00466_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MEMBERS = [(40, 33, 6, 1), (17, 9, 3, 2), (64, 20, 6, 3), (5, 70, 3, 4), (1, 1, 6, 5)]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mevp.load()


def make_members(precision):
    states, cases = [], []
    for nx, ny, ns, seed in MEMBERS:
        case = W.small_case(nx, ny, ns, seed=500 + seed)
        p = dict(case["params"], alpha=300.0 + 50 * seed, coriolis_f=1.46e-4 * (1 - 0.3 * seed))
        st = mevp.State(nx, ny, ns, vertex_xy=case["xy"], precision=precision, params=p)
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"], case["vel0"] * 0.1 if seed == 3 else None)
        st.set_velocity(case["vel0"])
        st.set_stress(case["S0"])
        states.append(st)
        cases.append(case)
    return states, cases


def results(states):
    return [(st.velocity(), st.stress()) for st in states]


def step_alone(precision, counts):
    states, _ = make_members(precision)
    for st in states:
        st.begin_step()
        for n in counts:
            st.run_subcycles(n)
    out = results(states)
    for st in states:
        st.close()
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_ensemble_bitwise_equals_members_alone(precision):
    counts = (3, 70, 1)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ref = step_alone(precision, counts)
        shapes = mevp.mevp_ensemble_shapes(precision)
        assert len(shapes) >= 2
        for shape in range(len(shapes)):
            for graphs in (1, 0):
                states, _ = make_members(precision)
                with mevp.Ensemble(states) as ens:
                    ens.set_shape(shape)
                    ens.set_graphs(graphs)
                    ens.begin_step()
                    for n in counts:
                        ens.run_subcycles(n)
                    got = results(states)
                for st in states:
                    st.close()
                for m, ((va, Sa), (vb, Sb)) in enumerate(zip(got, ref)):
                    assert np.array_equal(va, vb), (shape, graphs, m, "velocity")
                    assert np.array_equal(Sa, Sb), (shape, graphs, m, "stress")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_leaves_no_trace(precision):
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ref = step_alone(precision, (9,))
        states, _ = make_members(precision)
        with mevp.Ensemble(states) as ens:
            ens.begin_step()
            best = ens.autotune(4)
            assert 0 <= best < len(mevp.mevp_ensemble_shapes(precision))
            ens.run_subcycles(9)
            got = results(states)
        for st in states:
            st.close()
    for (va, Sa), (vb, Sb) in zip(got, ref):
        assert np.array_equal(va, vb) and np.array_equal(Sa, Sb)


def test_members_stay_usable_and_mixing_is_rejected():
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        a, _ = make_members("mixed")
        b, _ = make_members("fp64")
        with pytest.raises(mevp.MevpError) as e:
            mevp.Ensemble([a[0], b[0]])
        assert e.value.code == -1
        with pytest.raises(mevp.MevpError):
            mevp.Ensemble([a[0], a[0]])
        # a member stepped on its own between ensemble runs stays consistent
        ref = step_alone("mixed", (5, 3, 4))
        with mevp.Ensemble(a) as ens:
            ens.begin_step()
            ens.run_subcycles(5)
            for st in a:
                st.run_subcycles(3)
            ens.run_subcycles(4)
            got = results(a)
        for (va, Sa), (vb, Sb) in zip(got, ref):
            assert np.array_equal(va, vb) and np.array_equal(Sa, Sb)
        for st in a + b:
            st.close()


# members of every kind: stress dofs, DG0/DG1/DG2 ice, rectilinear, bilinear
# and curved meshes (nx, ny, n_s, n_a, geometry, seed)
KINDS = [(40, 33, 6, 1, "uniform", 11), (23, 17, 8, 1, "uniform", 12),
         (19, 26, 6, 6, "uniform", 13), (31, 12, 3, 3, "perturbed", 14),
         (17, 21, 8, 6, "wavy", 15), (14, 11, 6, 1, "curved", 16), (9, 13, 3, 3, "wavy_iso", 17),
         (12, 9, 3, 1, "uniform", 18)]


def make_kinds(precision):
    states = []
    for nx, ny, ns, na, geo, seed in KINDS:
        case = W.small_case(nx, ny, ns, seed=600 + seed, geometry=geo)
        rng = np.random.default_rng(seed)
        ne = nx * ny
        H = np.vstack([rng.uniform(0.5, 1.8, ne)] + [rng.uniform(-0.2, 0.2, ne)] * (na - 1))
        A = np.vstack([rng.uniform(0.75, 0.97, ne)] + [rng.uniform(-0.05, 0.05, ne)] * (na - 1))
        p = dict(case["params"], alpha=300.0 + 40 * seed)
        st = mevp.State(nx, ny, ns, vertex_xy=case["xy"], n_adv=na, precision=precision, params=p)
        st.set_ice(H, A)
        st.set_forcing(case["tau"])
        st.set_velocity(case["vel0"])
        st.set_stress(case["S0"])
        states.append(st)
    return states


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_ensemble_of_every_member_kind(precision):
    """Members that are not batched (8 stress dofs, DG1/DG2 ice, general and
    curved meshes) run their single-state launches inside the ensemble's
    stream and graphs: still bitwise the results of stepping each alone, for
    every shape, with and without graphs, and after autotuning."""
    counts = (3, 9, 1)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        alone = make_kinds(precision)
        for st in alone:
            st.begin_step()
            for n in counts:
                st.run_subcycles(n)
        ref = results(alone)
        for st in alone:
            st.close()
        for shape in range(len(mevp.mevp_ensemble_shapes(precision))):
            for graphs in (1, 0):
                states = make_kinds(precision)
                with mevp.Ensemble(states) as ens:
                    ens.set_shape(shape)
                    ens.set_graphs(graphs)
                    ens.begin_step()
                    if shape == 0 and graphs:
                        ens.autotune(3)
                    for n in counts:
                        ens.run_subcycles(n)
                    got = results(states)
                for st in states:
                    st.close()
                for m, ((va, Sa), (vb, Sb)) in enumerate(zip(got, ref)):
                    assert np.array_equal(va, vb), (shape, graphs, m, "velocity")
                    assert np.array_equal(Sa, Sb), (shape, graphs, m, "stress")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble8_matches_the_oracle(precision):
    """The 8-member ensemble (uneven sides 16..64, DG1/DG2 members), captured
    as CUDA graphs, after autotuning, against the FP64 oracle member by member:
    the FP64 parity bar (rel L2 1e-11, rel max 1e-10), or the mixed path's
    stated per-field errors (velocity 5e-6 / 3e-5, stress 5e-5 / 2e-4)."""
    import oracle
    tol = ({"velocity": (1e-11, 1e-10), "stress": (1e-11, 1e-10)} if precision == "fp64"
           else {"velocity": (5e-6, 3e-5), "stress": (5e-5, 2e-4)})
    cases = W.make_ensemble("ensemble8")
    n_sub = cases[0]["n_sub"]
    side = torch.cuda.Stream()  # a non-default stream: graph replay is on
    with torch.cuda.stream(side):
        states = []
        for c in cases:
            st = mevp.State(c["nx"], c["ny"], c["n_s"], vertex_xy=c["xy"], precision=precision,
                            params=c["params"])
            st.set_ice(c["H"], c["A"])
            st.set_forcing(c["tau"])
            st.set_velocity(c["vel0"])
            st.set_stress(c["S0"])
            states.append(st)
        with mevp.Ensemble(states) as ens:
            ens.begin_step()
            ens.autotune(4)
            ens.run_subcycles(n_sub)
            got = results(states)
        for st in states:
            st.close()
    assert len({c["n_s"] for c in cases}) == 2  # DG1 and DG2 members both present
    for m, (c, (v, S)) in enumerate(zip(cases, got)):
        vo, So = oracle.subcycles(c["nx"], c["ny"], c["xy"], c["n_s"], 1, c["params"], c["H"],
                                  c["A"], c["tau"], c["vel0"], c["S0"], n_sub, openmp=True)
        for name, x, ref in (("velocity", v, vo), ("stress", S, So)):
            l2 = np.linalg.norm(x - ref) / np.linalg.norm(ref)
            linf = np.abs(x - ref).max() / np.abs(ref).max()
            assert l2 <= tol[name][0] and linf <= tol[name][1], (m, name, l2, linf)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble64_matches_the_oracle_over_two_subcycles(precision):
    """The full 64-member ensemble workload (sides 64..512, 4.1 M elements, DG1
    and DG2) in the configuration the benchmark times -- batched persistent
    launches, CUDA graphs, autotuned shape -- against the oracle member by
    member after 2 subcycles (the workload's alpha = 300 amplifies any
    rounding difference on its finer members over longer horizons)."""
    import oracle
    tol = ({"velocity": (1e-11, 1e-10), "stress": (1e-11, 1e-10)} if precision == "fp64"
           else {"velocity": (5e-6, 3e-5), "stress": (5e-5, 2e-4)})
    cases = W.make_ensemble("ensemble64")
    n_sub = 2
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        states = []
        for c in cases:
            st = mevp.State(c["nx"], c["ny"], c["n_s"], vertex_xy=c["xy"], precision=precision,
                            params=c["params"])
            st.set_ice(c["H"], c["A"])
            st.set_forcing(c["tau"])
            st.set_velocity(c["vel0"])
            st.set_stress(c["S0"])
            states.append(st)
        with mevp.Ensemble(states) as ens:
            ens.begin_step()
            ens.autotune(2)
            ens.run_subcycles(n_sub)
            got = results(states)
        for st in states:
            st.close()
    for m, (c, (v, S)) in enumerate(zip(cases, got)):
        vo, So = oracle.subcycles(c["nx"], c["ny"], c["xy"], c["n_s"], 1, c["params"], c["H"],
                                  c["A"], c["tau"], c["vel0"], c["S0"], n_sub, openmp=True)
        for name, x, ref in (("velocity", v, vo), ("stress", S, So)):
            l2 = np.linalg.norm(x - ref) / np.linalg.norm(ref)
            linf = np.abs(x - ref).max() / np.abs(ref).max()
            assert l2 <= tol[name][0] and linf <= tol[name][1], (m, name, l2, linf)
