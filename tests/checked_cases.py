"""Small cases through every kernel family, for the bounds-checked build.

Run as a script with the library to test in MEVP_LIBRARY; writes every output
array to the .npz path given as the only argument.  Every state is synced
after its run, so an out-of-bounds access raises MevpError(MEVP_ERR_BOUNDS)
in the checked build."""
import sys

import numpy as np
import torch

from paper_2402_00466_gb300 import mevp
from paper_2402_00466_gb300 import workloads as W


def state(case, precision="fp64", n_a=1, H=None, A=None):
    st = mevp.State(case["nx"], case["ny"], case["n_s"], vertex_xy=case["xy"], n_adv=n_a,
                    precision=precision, params=case["params"])
    st.set_ice(case["H"] if H is None else H, case["A"] if A is None else A)
    st.set_forcing(case["tau"])
    st.set_velocity(case["vel0"])
    st.set_stress(case["S0"])
    return st


def run_all():
    out = {}
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for n_s in (3, 6, 8):
            for shape in ((1, 1), (37, 23)):
                for geo in ("uniform", "perturbed"):
                    case = W.small_case(*shape, n_s, seed=300 + n_s, geometry=geo)
                    with state(case) as st:
                        st.begin_step()
                        st.run_subcycles(9)  # graph chunks and direct launches
                        st.sync()
                        key = f"fp64_{n_s}_{shape[0]}_{geo}"
                        out[key + "_v"], out[key + "_S"] = st.velocity(), st.stress()
                        out[key + "_E"], out[key + "_F"] = st.strain(), st.force()
        for n_s in (3, 6):
            case = W.small_case(33, 19, n_s, seed=310 + n_s)
            for fused in (1, 0):
                with state(case, "mixed") as st:
                    st.set_option(mevp.MEVP_OPT_FUSED, fused)
                    st.begin_step()
                    st.run_subcycles(9)
                    st.sync()
                    out[f"mixed_{n_s}_{fused}_v"], out[f"mixed_{n_s}_{fused}_S"] = (
                        st.velocity(), st.stress())
        for n_s in (3, 6, 8):  # curved meshes, FP64 and mixed (fused and two-kernel)
            case = W.small_case(37, 23, n_s, seed=350 + n_s, geometry="curved")
            for prec, fused in (("fp64", 1), ("mixed", 1), ("mixed", 0)):
                with state(case, prec) as st:
                    st.set_option(mevp.MEVP_OPT_FUSED, fused)
                    st.begin_step()
                    st.run_subcycles(5)
                    st.sync()
                    key = f"iso_{prec}_{n_s}_{fused}"
                    out[key + "_v"], out[key + "_S"] = st.velocity(), st.stress()
                    out[key + "_E"], out[key + "_F"] = st.strain(), st.force()
        for n_s in (3, 6, 8):  # bilinear general meshes, mixed
            case = W.small_case(37, 23, n_s, seed=355 + n_s, geometry="wavy")
            for fused in (1, 0):
                with state(case, "mixed") as st:
                    st.set_option(mevp.MEVP_OPT_FUSED, fused)
                    st.begin_step()
                    st.run_subcycles(5)
                    st.sync()
                    out[f"gen_mixed_{n_s}_{fused}_v"] = st.velocity()
        for n_a in (1, 3, 6):
            case = W.small_case(21, 13, 6, seed=320 + n_a, geometry="perturbed")
            ne = 21 * 13
            rng = np.random.default_rng(n_a)
            H = np.vstack([rng.uniform(0.5, 1.5, ne)] + [rng.uniform(-0.1, 0.1, ne)] * (n_a - 1))
            A = np.vstack([rng.uniform(0.8, 0.95, ne)] + [rng.uniform(-0.02, 0.02, ne)] * (n_a - 1))
            case["vel0"] = 3.0 * case["vel0"]
            with state(case, n_a=n_a, H=H, A=A) as st:
                st.advect(2)
                st.begin_step()
                st.run_subcycles(5)
                st.sync()
                out[f"adv_{n_a}_H"], out[f"adv_{n_a}_v"] = st.read("H"), st.velocity()
        case = W.small_case(24, 20, 3, seed=330)
        with state(case) as st:
            st.begin_step()
            J, gP, gT = st.adjoint_kinetic_energy(12, 5)
            st.sync()
            out["adj_gP"], out["adj_gT"] = gP, gT
        for geo, ns in (("curved", 6), ("perturbed", 8)):  # general-mesh adjoint, DG1 ice
            case = W.small_case(13, 11, ns, seed=335 + ns, geometry=geo)
            ne = 13 * 11
            rng = np.random.default_rng(ns)
            H = np.vstack([rng.uniform(0.6, 1.5, ne)] + [rng.uniform(-0.1, 0.1, ne)] * 2)
            A = np.vstack([rng.uniform(0.8, 0.95, ne)] + [rng.uniform(-0.02, 0.02, ne)] * 2)
            with state(case, n_a=3, H=H, A=A) as st:
                st.begin_step()
                J, gP, gT = st.adjoint_kinetic_energy(8, 3)
                st.sync()
                out[f"adj_{geo}_gP"], out[f"adj_{geo}_gT"] = gP, gT
        members = [W.small_case(n, n + 3, 3 + 3 * (n % 2), seed=340 + n) for n in (9, 14, 20)]
        members.append(W.small_case(11, 9, 8, seed=345, geometry="curved"))
        members.append(W.small_case(10, 12, 6, seed=346, geometry="wavy"))
        for prec in ("mixed", "fp64"):
            sts = [state(c, prec) for c in members]
            ens = mevp.Ensemble(sts)
            ens.begin_step()
            ens.run_subcycles(7)
            for i, s_ in enumerate(sts):
                s_.sync()
                out[f"ens_{prec}_{i}_v"] = s_.velocity()
            ens.close()
            for s_ in sts:
                s_.close()
        for n_s, ocean in ((3, False), (8, True)):  # the no-alloc entry point
            nx, ny = 17, 12
            case = W.small_case(nx, ny, n_s, seed=360 + n_s)
            xy = case["xy"].reshape(ny + 1, nx + 1, 2)
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
            vo = dev(W.smooth_velocity(nx, ny, 361, amp=0.1, L=case["L"])) if ocean else None
            vel, S = dev(case["vel0"]), dev(case["S0"])
            mevp.mevp_run_subcycles_noalloc(nx, ny, n_s, case["params"], dev(xy[0, :, 0]),
                                            dev(xy[:, 0, 1]), dev(case["H"][0]),
                                            dev(case["A"][0]), dev(case["tau"]), vo, vel, S, 5)
            torch.cuda.synchronize()
            out[f"noalloc_{n_s}_v"], out[f"noalloc_{n_s}_S"] = vel.cpu().numpy(), S.cpu().numpy()
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_all())
