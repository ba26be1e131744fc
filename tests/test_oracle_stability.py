"""The mEVP iteration's sensitivity to rounding at the workload's alpha = beta
(no GPU).

Eq. 3 is a pseudo-time iteration.  Where the ice is rigid (Delta at Delta_min)
its stress relaxation acts like an explicit step of stiffness
gamma = zeta_max dt / (rho H h^2), zeta_max = P / (2 Delta_min), and the
iteration is stable only when alpha * beta is large enough against gamma;
on fine meshes (small h) the workload's alpha = beta = 300 is not.  Then two
runs whose inputs differ by one unit in the last place -- a stand-in for two
correct FP64 implementations that round differently -- separate
exponentially until the difference saturates, so no element-wise comparison
of two implementations over the full 500 subcycles can hold at that alpha.
With alpha h at about 4e6 m the same difference stays at rounding level.

This is what lets the GPU parity tests compare at alpha = beta = 300 over a
short horizon only, and over the full horizon at the stability-bound alpha.
The runs use the 2 km spacing of the 256 x 256 workload (a 32 x 32 patch of
64 km) and the 0.5 km spacing of the 1024 x 1024 workload, DG2 stress, the
workload's ice recipe and a cyclone's wind, from rest.
"""
import numpy as np
import pytest

import oracle
from paper_2402_00466_gb300 import workloads as W

N_SUB = 500
CHUNK = 25


def _separation(h, ab, n_s=6, nx=32, seed=3):
    """Relative L2 difference of velocity and stress, after every CHUNK
    subcycles, between a run and the same run with the ice height of one
    element (at the centre) moved by one ulp."""
    L = nx * h
    ne, nn, _ = W.sizes(nx, nx)
    xy = W.uniform_vertices(nx, nx, L, L)
    H, A = W.ice_grf(nx, nx, (seed, seed + 1), L=L)
    tau = W.cyclone_wind_stress(W.node_coords(nx, nx, xy), W.cyclone_params(seed + 2000, L))
    H2 = H.copy()
    K = (nx // 2) * nx + nx // 2  # an element at the centre
    H2[0, K] = np.nextafter(H2[0, K], np.inf)
    p = dict(W.DEFAULT_PARAMS, alpha=ab, beta=ab)
    rest = np.zeros((2, nn))
    runs = [[rest.copy(), np.zeros((3, n_s, ne)), h] for h in (H, H2)]
    dv, ds = [], []
    for _ in range(N_SUB // CHUNK):
        for r in runs:
            r[0], r[1] = oracle.subcycles(nx, nx, xy, n_s, 1, p, r[2], A, tau, r[0], r[1], CHUNK,
                                          vn=rest, openmp=True)
        (v1, S1, _), (v2, S2, _) = runs
        dv.append(np.linalg.norm(v1 - v2) / np.linalg.norm(v1))
        ds.append(np.linalg.norm(S1 - S2) / np.linalg.norm(S1))
    return np.array(dv), np.array(ds)


@pytest.mark.parametrize("h", [2e3, 0.5e3])
def test_workload_alpha_amplifies_rounding_until_it_saturates(h):
    dv, ds = _separation(h, 300.0)
    k = lambda p: p // CHUNK - 1  # noqa: E731  (index of subcycle p)
    assert dv[k(25)] < 1e-13                      # starts near rounding level
    growth = (dv[k(200)] / dv[k(100)]) ** (1 / 100)
    assert growth > 1.03                          # exponential separation per subcycle
    assert dv[-1] > 1e-4 and ds[-1] > 1e-3        # far above rounding after 500 subcycles
    assert dv.max() < 0.5                         # bounded: the difference saturates
    late = (dv[-1] / dv[k(400)]) ** (1 / 100)
    assert late < growth                          # and its growth has slowed down


@pytest.mark.parametrize("h,ab", [(2e3, 2000.0), (0.5e3, 8000.0)])
def test_stability_bound_alpha_keeps_rounding_level(h, ab):
    assert 3.9e6 <= ab * h <= 4.1e6  # alpha h at about 4e6 m
    dv, ds = _separation(h, ab)
    assert dv.max() < 1e-13 and ds.max() < 1e-12
