"""GPU test of mevp_run_subcycles_noalloc, the entry point for callers that
cannot allocate device memory (their memory belongs to a host model or
coupler, or they must not risk cudaMalloc's device-wide synchronisation).

It runs two outer steps in a row through the C ABI on caller-owned device
arrays and checks each against the state-based entry points
(mevp_begin_step + mevp_run_subcycles) at the FP64 parity tolerance.  The
file sorts last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_00466_gb300 import mevp  # noqa: E402
from paper_2402_00466_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

L2_TOL = 1e-11
INF_TOL = 1e-10


def _close(x, ref, what):
    n2 = np.linalg.norm(ref)
    ninf = np.abs(ref).max()
    l2 = np.linalg.norm(x - ref) / (n2 if n2 > 0 else 1.0)
    linf = np.abs(x - ref).max() / (ninf if ninf > 0 else 1.0)
    assert l2 <= L2_TOL and linf <= INF_TOL, f"{what}: rel L2 {l2:.3e}, rel Linf {linf:.3e}"


@pytest.mark.parametrize("n_s,ocean,side_stream", [(3, False, False), (6, False, False),
                                                    (8, False, False), (6, True, False),
                                                    (3, True, True)])
def test_noalloc_matches_state_api_on_two_calls(n_s, ocean, side_stream):
    """Two calls in a row against the state API; with an ocean current (the
    node kernel reading the caller's v_ocean) and on a non-default stream."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny = 48, 40
    case = W.small_case(nx, ny, n_s, seed=77 + 3 * ocean)
    p = case["params"]
    vo = W.smooth_velocity(nx, ny, 79, amp=0.15, L=case["L"]) if ocean else None
    steps = (7, 6)  # an odd count exercises the copy back from the scratch buffer

    ref = []
    with mevp.State(nx, ny, n_s, vertex_xy=case["xy"], params=p) as st:
        st.set_ice(case["H"], case["A"])
        st.set_forcing(case["tau"], vo)
        st.set_velocity(case["vel0"])
        st.set_stress(case["S0"])
        for n in steps:
            st.begin_step()
            st.run_subcycles(n)
            ref.append((st.velocity(), st.stress()))

    xy = case["xy"].reshape(ny + 1, nx + 1, 2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    xline, yline = dev(xy[0, :, 0]), dev(xy[:, 0, 1])
    H, A, tau = dev(case["H"][0]), dev(case["A"][0]), dev(case["tau"])
    vel, S = dev(case["vel0"]), dev(case["S0"])
    v_ocean = dev(vo) if ocean else None
    stream = torch.cuda.Stream() if side_stream else None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())  # the uploads above
    for (n, (v_ref, S_ref)) in zip(steps, ref):
        if stream is None:
            mevp.mevp_run_subcycles_noalloc(nx, ny, n_s, p, xline, yline, H, A, tau, v_ocean,
                                            vel, S, n)
            torch.cuda.synchronize()
        else:
            mevp.mevp_run_subcycles_noalloc(nx, ny, n_s, p, xline, yline, H, A, tau, v_ocean,
                                            vel, S, n, stream=stream.cuda_stream)
            stream.synchronize()
        _close(vel.cpu().numpy(), v_ref, "velocity")
        _close(S.cpu().numpy(), S_ref, "stress")


def test_noalloc_rejects_lines_that_do_not_increase():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny = 6, 5
    ne, nn, _ = W.sizes(nx, ny)
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")  # noqa: E731
    xline = torch.linspace(0.0, 6e3, nx + 1, dtype=torch.float64, device="cuda")
    yline = torch.linspace(0.0, 5e3, ny + 1, dtype=torch.float64, device="cuda")
    for bad in (xline.flip(0).contiguous(), torch.cat([xline[:3], xline[2:3], xline[4:]])):
        with pytest.raises(mevp.MevpError) as e:
            mevp.mevp_run_subcycles_noalloc(nx, ny, 3, W.DEFAULT_PARAMS, bad, yline, z(ne),
                                            z(ne), z(2, nn), None, z(2, nn), z(3, 3, ne), 2)
        assert e.value.code == -1 and "increase" in str(e.value)
    # the scratch keeps no trace of the refusal: a valid call still succeeds
    mevp.mevp_run_subcycles_noalloc(nx, ny, 3, W.DEFAULT_PARAMS, xline, yline, z(ne) + 1.0,
                                    z(ne) + 0.9, z(2, nn), None, z(2, nn), z(3, 3, ne), 2)
    torch.cuda.synchronize()


def test_noalloc_rejects_meshes_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx = ny = 256
    ne, nn, _ = W.sizes(nx, ny)
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")  # noqa: E731
    with pytest.raises(mevp.MevpError) as e:
        mevp.mevp_run_subcycles_noalloc(nx, ny, 6, W.DEFAULT_PARAMS, z(nx + 1), z(ny + 1), z(ne),
                                        z(ne), z(2, nn), None, z(2, nn), z(3, 6, ne), 1)
    assert e.value.code == -1 and "scratch" in str(e.value)
