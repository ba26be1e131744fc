"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics (no GPU).  Each test names what pins it: printed constants,
closed forms, invariants, textbook quadrature, or the independent brute-force
restatement in ``bruteforce.py``."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2402_00466_gb300 import workloads as W
from tests import bruteforce as BF

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
P0 = dict(W.DEFAULT_PARAMS)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def perturbed_vertices(nx, ny, L, seed, amp=0.2):
    """Non-affine quads: interior vertices moved by up to amp*h."""
    xy = W.uniform_vertices(nx, ny, L, L).reshape(ny + 1, nx + 1, 2)
    rng = np.random.Generator(np.random.PCG64(seed))
    h = L / nx
    xy[1:-1, 1:-1] += rng.uniform(-amp * h, amp * h, xy[1:-1, 1:-1].shape)
    return xy.reshape(-1, 2).copy()


# --------------------------------------------------------------------------
# Quadrature (App. A: NGP = 2 for 3 stress dofs, 3 for 6 or 8)
# --------------------------------------------------------------------------
def test_ngp_rule_matches_paper():
    for k, v in GOLD["ngp"].items():
        if k.startswith("_"):
            continue
        assert oracle.ngp(int(k)) == v
    for bad in (0, 1, 2, 4, 5, 7, 9):
        assert oracle.ngp(bad) == -1


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gauss_textbook(n):
    x, w = oracle.gauss(n)
    xr, wr = BF.gauss01(n)  # numpy's Golub-Welsch based rule
    assert np.allclose(x, xr, rtol=0, atol=1e-15) and np.allclose(w, wr, rtol=0, atol=1e-15)
    closed = {2: ([0.5 - 0.5 / math.sqrt(3), 0.5 + 0.5 / math.sqrt(3)], [0.5, 0.5]),
              3: ([0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)],
                  [5 / 18, 8 / 18, 5 / 18])}
    if n in closed:
        assert np.allclose(x, closed[n][0], atol=1e-15) and np.allclose(w, closed[n][1], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3])
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = oracle.gauss(n)
    for a in range(2 * n):
        for b in range(2 * n):
            q = np.sum(np.outer(w, w) * np.outer(x ** b, x ** a))
            assert abs(q - 1.0 / ((a + 1) * (b + 1))) < 1e-15
    # and not beyond: degree 2n is integrated inexactly
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-6


# --------------------------------------------------------------------------
# Bases
# --------------------------------------------------------------------------
def test_dg_basis_orthogonal_closed_form_mass():
    x, w = BF.gauss01(6)
    XI, ET = np.meshgrid(x, x)
    Wt = np.outer(w, w)
    phi = np.array([[oracle.dg_basis(8, a, b) for a, b in zip(r1, r2)] for r1, r2 in zip(XI, ET)])
    M = np.einsum("ij,ijs,ijt->st", Wt, phi, phi)
    expect = np.diag([1, 1 / 12, 1 / 12, 1 / 180, 1 / 144, 1 / 180, 1 / 2160, 1 / 2160])
    assert np.allclose(M, expect, atol=1e-15)


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_dg_basis_spans_total_degree(n_s):
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 1, (30, 2))
    mine = np.array([oracle.dg_basis(n_s, a, b) for a, b in pts])
    other = np.array([BF.dg_bf(n_s, np.array(a), np.array(b)) for a, b in pts])
    # same span: least-squares fit of one by the other is exact
    coef = np.linalg.lstsq(mine, other, rcond=None)[0]
    assert np.allclose(mine @ coef, other, atol=1e-13)
    assert np.linalg.matrix_rank(mine) == n_s


def test_q2_lagrange_partition_and_gradients():
    nodes = [0.0, 0.5, 1.0]
    for b in range(3):
        for a in range(3):
            phi, _, _ = oracle.q2_basis(nodes[a], nodes[b])
            e = np.zeros(9); e[a + 3 * b] = 1.0
            assert np.allclose(phi, e, atol=1e-15)
    rng = np.random.default_rng(1)
    for xi, eta in rng.uniform(0, 1, (20, 2)):
        phi, dx, de = oracle.q2_basis(xi, eta)
        assert abs(phi.sum() - 1) < 1e-14 and abs(dx.sum()) < 1e-13 and abs(de.sum()) < 1e-13
        # reproduces the biquadratic p = xi^2 eta^2 + 3 xi eta and its gradient
        nv = np.array([(nodes[j % 3], nodes[j // 3]) for j in range(9)])
        pv = nv[:, 0] ** 2 * nv[:, 1] ** 2 + 3 * nv[:, 0] * nv[:, 1]
        assert abs(phi @ pv - (xi ** 2 * eta ** 2 + 3 * xi * eta)) < 1e-14
        assert abs(dx @ pv - (2 * xi * eta ** 2 + 3 * eta)) < 1e-13
        assert abs(de @ pv - (2 * xi ** 2 * eta + 3 * xi)) < 1e-13


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("affine", [True, False])
def test_projection_matrix_is_left_inverse(n_s, affine):
    """iMJwPSI applied to the Gauss values of a DG function returns its coefficients."""
    nx = ny = 3
    L = 3e3
    xy = W.uniform_vertices(nx, ny, L, L) if affine else perturbed_vertices(nx, ny, L, 5)
    g = oracle.ngp(n_s)
    x, _ = oracle.gauss(g)
    XI, ET = np.meshgrid(x, x)
    psi = np.array([oracle.dg_basis(n_s, a, b) for a, b in zip(XI.ravel(), ET.ravel())])  # (ng, ns)
    for K in range(nx * ny):
        det, m = oracle.element_map(nx, ny, xy, n_s, K)
        assert np.allclose(m @ psi, np.eye(n_s), atol=1e-12)
        if affine:
            assert np.allclose(det, (L / nx) ** 2, rtol=1e-14)


# --------------------------------------------------------------------------
# Strain (stage 1)
# --------------------------------------------------------------------------
def _node_xy(nx, ny, xy):
    """CG2 node coordinates through the bilinear map (test-side)."""
    V = np.asarray(xy).reshape(ny + 1, nx + 1, 2)
    nw = 2 * nx + 1
    out = np.zeros((2, (2 * nx + 1) * (2 * ny + 1)))
    for iy in range(2 * ny + 1):
        for ix in range(nw):
            kx, ky = min(ix // 2, nx - 1), min(iy // 2, ny - 1)
            xi, eta = ix / 2 - kx, iy / 2 - ky
            p = ((1 - xi) * (1 - eta) * V[ky, kx] + xi * (1 - eta) * V[ky, kx + 1]
                 + (1 - xi) * eta * V[ky + 1, kx] + xi * eta * V[ky + 1, kx + 1])
            out[:, iy * nw + ix] = p
    return out


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("affine", [True, False])
def test_strain_linear_field_exact(n_s, affine):
    nx, ny, L = 4, 3, 8e3
    xy = W.uniform_vertices(nx, ny, L, L) if affine else perturbed_vertices(nx, ny, L, 7)
    nxy = _node_xy(nx, ny, xy)
    a, b, c, d = 1.3e-6, -0.7e-6, 2.1e-6, -0.4e-6
    vel = np.stack([a * nxy[0] + b * nxy[1], c * nxy[0] + d * nxy[1]])
    E = oracle.strain(nx, ny, xy, n_s, vel)
    const = np.array([a, (b + c) / 2, d])
    assert np.allclose(E[:, 0, :], const[:, None], rtol=1e-11, atol=0)
    assert np.abs(E[:, 1:, :]).max() < 1e-11 * abs(a)


def test_strain_rigid_rotation_zero():
    nx, ny, L = 3, 3, 3e3
    xy = perturbed_vertices(nx, ny, L, 9)
    nxy = _node_xy(nx, ny, xy)
    w = 1e-5
    vel = np.stack([-w * nxy[1], w * nxy[0]])
    E = oracle.strain(nx, ny, xy, 6, vel)
    assert np.abs(E).max() < 1e-15


# --------------------------------------------------------------------------
# Stress (stage 2): paper constants, clamps, closed forms
# --------------------------------------------------------------------------
def _one_element_stress(n_s, E0, H, A, S0, params):
    """1x1 mesh with a constant strain: the Gauss values all equal E0."""
    L = 1e3
    xy = W.uniform_vertices(1, 1, L, L)
    E = np.zeros((3, n_s, 1)); E[:, 0, 0] = E0
    S = np.zeros((3, n_s, 1)); S[:, 0, 0] = S0
    return oracle.stress(1, 1, xy, n_s, 1, params, E, np.array([[H]]), np.array([[A]]), S)


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_stress_single_point_matches_printed_constants(n_s):
    d, s, st = GOLD["delta"], GOLD["stress"], GOLD["strength"]
    p = dict(P0, Pstar=st["Pstar"], C=st["C"], e=2.0)
    e11, e12, e22 = 3e-7, -1.1e-7, -2e-7
    H, A = 1.4, 0.93
    S0 = np.array([-1200.0, 300.0, -800.0])
    out = _one_element_stress(n_s, [e11, e12, e22], H, A, S0, p)
    P = st["Pstar"] * H * math.exp(-st["C"] * (1 - A))
    D = math.sqrt(p["DeltaMin"] ** 2 + d["sq"] * (e11 ** 2 + e22 ** 2) + d["mix"] * e11 * e22
                  + d["shear"] * e12 ** 2)
    ai = 1 / p["alpha"]
    expect = np.array([
        (1 - ai) * S0[0] + ai * (P / D * (s["a"] * e11 + s["b"] * e22) - s["p"] * P),
        (1 - ai) * S0[1] + ai * (P / D * s["c"] * e12),
        (1 - ai) * S0[2] + ai * (P / D * (s["a"] * e22 + s["b"] * e11) - s["p"] * P)])
    assert np.allclose(out[:, 0, 0], expect, rtol=1e-13)
    assert np.abs(out[:, 1:, 0]).max() < 1e-9  # higher coefficients stay zero


def test_stress_general_ellipse_is_hibler_law():
    p = dict(P0, e=1.7)
    e11, e12, e22 = 2e-7, 1.5e-7, -3e-7
    out = _one_element_stress(3, [e11, e12, e22], 1.0, 1.0, np.zeros(3), p)
    P = p["Pstar"]
    ecc = p["e"]
    D = math.sqrt(p["DeltaMin"] ** 2 + (e11 ** 2 + e22 ** 2) * (1 + ecc ** -2)
                  + 4 * ecc ** -2 * e12 ** 2 + 2 * (1 - ecc ** -2) * e11 * e22)
    zeta = P / (2 * D)
    eta = zeta / ecc ** 2
    tr = e11 + e22
    svp = np.array([2 * eta * e11 + (zeta - eta) * tr - P / 2, 2 * eta * e12,
                    2 * eta * e22 + (zeta - eta) * tr - P / 2])
    assert np.allclose(out[:, 0, 0], svp / p["alpha"], rtol=1e-13)


def test_stress_clamps():
    p = dict(P0)
    # negative H -> h = 0 -> no strength, the stress only decays
    out = _one_element_stress(3, [1e-7, 0, 0], -0.5, 0.9, np.array([100.0, 50, -20]), p)
    assert np.allclose(out[:, 0, 0], np.array([100.0, 50, -20]) * (1 - 1 / p["alpha"]), rtol=1e-14)
    # A > 1 clamps to 1 (exp(0) = 1), A < 0 clamps to 0
    hi = _one_element_stress(3, [0, 0, 0], 1.0, 1.7, np.zeros(3), p)
    one = _one_element_stress(3, [0, 0, 0], 1.0, 1.0, np.zeros(3), p)
    assert np.array_equal(hi, one)
    lo = _one_element_stress(3, [0, 0, 0], 1.0, -0.3, np.zeros(3), p)
    zero = _one_element_stress(3, [0, 0, 0], 1.0, 0.0, np.zeros(3), p)
    assert np.array_equal(lo, zero)


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_stress_relaxation_closed_form(n_s):
    """E = 0, uniform H, A: S11_0^p = S22_0^p = -(P/2)(1 - (1-1/alpha)^p), S12 = 0."""
    p = dict(P0)
    nx = ny = 2
    xy = W.uniform_vertices(nx, ny, 4e3, 4e3)
    H = np.full((1, 4), 1.2); A = np.full((1, 4), 0.95)
    S = np.zeros((3, n_s, 4)); E = np.zeros((3, n_s, 4))
    P = p["Pstar"] * 1.2 * math.exp(-p["C"] * 0.05)
    for k in range(1, 41):
        S = oracle.stress(nx, ny, xy, n_s, 1, p, E, H, A, S)
        ref = -(P / 2) * (1 - (1 - 1 / p["alpha"]) ** k)
        assert np.allclose(S[0, 0], ref, rtol=1e-12) and np.allclose(S[2, 0], ref, rtol=1e-12)
        assert np.abs(S[1]).max() == 0 and np.abs(S[:, 1:]).max() < 1e-9


# --------------------------------------------------------------------------
# Divergence (stage 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_divergence_constant_stress(n_s):
    """Constant sigma: interior nodes feel nothing; boundary nodes feel -sigma.n
    times the 1-D Q2 edge weights (h/6, 4h/6, h/6); the total is zero."""
    nx, ny = 3, 2
    hx, hy = 2e3, 3e3
    xy = W.uniform_vertices(nx, ny, nx * hx, ny * hy)
    s11, s12, s22 = -1500.0, 400.0, -900.0
    S = np.zeros((3, n_s, nx * ny))
    S[0, 0], S[1, 0], S[2, 0] = s11, s12, s22
    F = oracle.divergence(nx, ny, xy, n_s, S)
    nw, nh = 2 * nx + 1, 2 * ny + 1
    Fx = F[0].reshape(nh, nw); Fy = F[1].reshape(nh, nw)
    scale = 1500.0 * 3e3
    assert np.abs(Fx[1:-1, 1:-1]).max() < 1e-12 * scale
    assert np.abs(Fy[1:-1, 1:-1]).max() < 1e-12 * scale

    def edge_w(n, h):
        w = np.zeros(2 * n + 1)
        for k in range(n):
            w[2 * k] += h / 6; w[2 * k + 1] += 4 * h / 6; w[2 * k + 2] += h / 6
        return w
    wy, wx = edge_w(ny, hy), edge_w(nx, hx)
    # left edge, outward normal (-1, 0): force = -sigma.n * weight = (s11, s12) w
    assert np.allclose(Fx[:, 0], s11 * wy + np.r_[s12 * hx / 6, np.zeros(nh - 2), -s12 * hx / 6],
                       atol=1e-9 * scale)
    assert np.allclose(F.sum(axis=1), 0, atol=1e-9 * scale)


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("affine", [True, False])
def test_divergence_matches_bruteforce(n_s, affine):
    nx, ny, L = 3, 2, 6e3
    xy = W.uniform_vertices(nx, ny, L, L) if affine else perturbed_vertices(nx, ny, L, 3)
    rng = np.random.default_rng(4)
    S = rng.uniform(-1e3, 1e3, (3, n_s, nx * ny))
    F = oracle.divergence(nx, ny, xy, n_s, S)
    M = BF.Mesh(nx, ny, xy, n_s)
    Fb = M.divergence(M.from_documented(S))
    assert rel(F, Fb) < 1e-13


# --------------------------------------------------------------------------
# Lumped mass
# --------------------------------------------------------------------------
def test_lumped_closed_form():
    nx, ny, h = 3, 3, 1e3
    xy = W.uniform_vertices(nx, ny, nx * h, ny * h)
    H = np.full((1, 9), 1.5)
    m, l = oracle.lumped(nx, ny, xy, 3, 1, P0, H)
    nw = 2 * nx + 1
    L2 = l.reshape(nw, nw)
    assert abs(l.sum() - 9 * h * h) < 1e-6
    assert abs(L2[2, 2] - 4 * h * h / 36) < 1e-9          # interior vertex: 4 x 1/36
    assert abs(L2[1, 2] - 2 * h * h * 4 / 36) < 1e-9      # edge midpoint: 2 x 4/36
    assert abs(L2[1, 1] - h * h * 16 / 36) < 1e-9         # element centre: 16/36
    assert np.allclose(m, P0["rho_ice"] * 1.5 * l, rtol=1e-14)


# --------------------------------------------------------------------------
# Velocity (stage 4) and the whole subcycle
# --------------------------------------------------------------------------
def _free_drift_case(nx=4, ny=4, n_sub=1, dt=120.0, f=1.46e-4, H0=1.3, tau0=(0.21, -0.13)):
    p = dict(P0, Pstar=0.0, dt=dt, coriolis_f=f)
    L = nx * 2e3
    xy = W.uniform_vertices(nx, ny, L, L)
    ne, nn, _ = W.sizes(nx, ny)
    H = np.full((1, ne), H0); A = np.full((1, ne), 0.9)
    tau = np.stack([np.full(nn, tau0[0]), np.full(nn, tau0[1])])
    return p, xy, H, A, tau


def test_rest_stays_at_rest():
    """Zero forcing, zero velocity and stress, uniform H and A: v stays 0 and the
    stress relaxes to -P/2 I.  On a 16 km mesh, where the mEVP iteration is
    stable at alpha = beta = 300 (on a 2 km mesh it amplifies rounding)."""
    nx = ny = 4
    ne, nn, _ = W.sizes(nx, ny)
    xy = W.uniform_vertices(nx, ny, 64e3, 64e3)
    H = np.full((1, ne), 1.1); A = np.full((1, ne), 0.97)
    vel, S = oracle.subcycles(nx, ny, xy, 6, 1, P0, H, A, np.zeros((2, nn)), np.zeros((2, nn)),
                              np.zeros((3, 6, ne)), 50)
    assert np.abs(vel).max() < 1e-16
    P = P0["Pstar"] * 1.1 * math.exp(-P0["C"] * 0.03)
    assert np.allclose(S[0, 0], -(P / 2) * (1 - (1 - 1 / P0["alpha"]) ** 50), rtol=1e-12)


def test_free_drift_recurrence():
    """P* = 0: sigma = 0; uniform H and tau make every interior node follow the
    same complex recurrence (m/l = rho H at every node)."""
    p, xy, H, A, tau = _free_drift_case()
    nx = ny = 4
    ne, nn, _ = W.sizes(nx, ny)
    n_sub = 30
    vel, _ = oracle.subcycles(nx, ny, xy, 3, 1, p, H, A, tau, np.zeros((2, nn)),
                              np.zeros((3, 3, ne)), n_sub)
    rhoH = p["rho_ice"] * 1.3
    z, zn = 0j, 0j
    t = complex(0.21, -0.13)
    for _ in range(n_sub):
        c = p["Cw"] * p["rho_water"] * abs(z)
        z = (rhoH / p["dt"] * (p["beta"] * z + zn) + t) / (rhoH * (1 + p["beta"]) / p["dt"] + c
                                                            + 1j * rhoH * p["coriolis_f"])
    nw = 2 * nx + 1
    grid = vel.reshape(2, nw, nw)[:, 1:-1, 1:-1]
    assert np.allclose(grid[0], z.real, rtol=1e-13) and np.allclose(grid[1], z.imag, rtol=1e-13)
    assert np.all(vel.reshape(2, nw, nw)[:, 0, :] == 0)


def test_converged_subcycle_is_implicit_euler():
    """Many subcycles converge to the implicit Euler step of free drift:
    (rho H/dt + Cw rho_w s + i rho H f) v = tau, s = |v| (solved by bisection)."""
    p, xy, H, A, tau = _free_drift_case(nx=2, ny=2)
    ne, nn, _ = W.sizes(2, 2)
    vel, _ = oracle.subcycles(2, 2, xy, 3, 1, p, H, A, tau, np.zeros((2, nn)),
                              np.zeros((3, 3, ne)), 20000)
    rhoH = p["rho_ice"] * 1.3
    t = complex(0.21, -0.13)
    k = p["Cw"] * p["rho_water"]

    def g(s):
        return abs(t) / abs(rhoH / p["dt"] + k * s + 1j * rhoH * p["coriolis_f"]) - s
    lo, hi = 0.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if g(mid) > 0 else (lo, mid)
    s = 0.5 * (lo + hi)
    v = t / (rhoH / p["dt"] + k * s + 1j * rhoH * p["coriolis_f"])
    centre = vel[:, 2 * 5 + 2]
    assert abs(centre[0] - v.real) < 1e-12 and abs(centre[1] - v.imag) < 1e-12


@pytest.mark.parametrize("n_s", [3, 6, 8])
@pytest.mark.parametrize("affine", [True, False])
def test_whole_subcycle_matches_bruteforce(n_s, affine):
    nx, ny = 2, 2
    case = W.small_case(nx, ny, n_s, seed=21)
    L = case["L"]
    xy = case["xy"] if affine else perturbed_vertices(nx, ny, L, 31, amp=0.15)
    p = case["params"]
    n_sub = 6
    vel, S, E, F, fel = oracle.subcycles(nx, ny, xy, n_s, 1, p, case["H"], case["A"], case["tau"],
                                         case["vel0"], case["S0"], n_sub, want_last=True)
    M = BF.Mesh(nx, ny, xy, n_s)
    vb, Sb, Eb = M.subcycles(case["vel0"], case["S0"], case["H"], case["A"], case["tau"], p, n_sub)
    assert rel(vel, vb) < 1e-12
    assert rel(M.values_documented(S), M.values(Sb)) < 1e-12
    assert rel(M.values_documented(E), M.values(Eb)) < 1e-12


def test_mirror_symmetry():
    """Mirroring the inputs in x (f = 0) mirrors the outputs: u -> -u, s12 -> -s12,
    and DG coefficients odd in xi - 1/2 change sign."""
    nx, ny, n_s = 4, 3, 6
    case = W.small_case(nx, ny, n_s, seed=5)
    p = dict(case["params"], coriolis_f=0.0)
    ne, nn, _ = W.sizes(nx, ny)
    nw, nh = 2 * nx + 1, 2 * ny + 1

    def mnode(a):
        return a.reshape(-1, nh, nw)[:, :, ::-1].reshape(a.shape)

    def melem(a):
        return a.reshape(a.shape[:-1] + (ny, nx))[..., ::-1].reshape(a.shape)
    odd = np.array([1, -1, 1, 1, -1, 1])[:n_s]
    comp_sign = np.array([1, -1, 1])
    vel0, S0, tau = case["vel0"], case["S0"], case["tau"]
    vel0m = mnode(vel0) * np.array([-1, 1])[:, None]
    taum = mnode(tau) * np.array([-1, 1])[:, None]
    S0m = melem(S0) * comp_sign[:, None, None] * odd[None, :, None]
    args = (nx, ny, case["xy"], n_s, 1, p)
    v1, S1 = oracle.subcycles(*args, case["H"], case["A"], tau, vel0, S0, 8)
    v2, S2 = oracle.subcycles(*args, melem(case["H"]), melem(case["A"]), taum, vel0m, S0m, 8)
    assert rel(mnode(v2) * np.array([-1, 1])[:, None], v1) < 1e-12
    assert rel(melem(S2) * comp_sign[:, None, None] * odd[None, :, None], S1) < 1e-12


def test_deterministic_and_openmp_identical():
    case = W.small_case(6, 5, 6, seed=8)
    args = (case["nx"], case["ny"], case["xy"], 6, 1, case["params"], case["H"], case["A"],
            case["tau"], case["vel0"], case["S0"], 5)
    a = oracle.subcycles(*args)
    b = oracle.subcycles(*args)
    c = oracle.subcycles(*args, openmp=True)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_bad_arguments_rejected():
    xy = W.uniform_vertices(2, 2, 1e3, 1e3)
    with pytest.raises(ValueError):
        oracle.strain(2, 2, xy, 1, np.zeros((2, 25)))  # DG0 stress unsupported
    bad = xy.copy().reshape(3, 3, 2)
    bad[1, 1] = bad[2, 2] + 10.0  # folded element: det J <= 0
    with pytest.raises(ValueError):
        oracle.strain(2, 2, bad.reshape(-1, 2), 3, np.zeros((2, 25)))


# --------------------------------------------------------------------------
# Isoparametric (Q2) element maps: the geometry given by the CG2 node
# positions (Sec. 2.1: the element map comes from the velocity's space)
# --------------------------------------------------------------------------
def curved(nx, ny, seed, L=3e3):
    return W.curved_nodes(nx, ny, seed, amp=0.08, L=L)


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_iso_with_bilinear_nodes_reproduces_bilinear_maps(n_s):
    """Node positions that are the bilinear images of the vertices make the
    Q2 map equal the Q1 map: every stage agrees with the vertex geometry."""
    nx, ny, L = 5, 4, 4e3
    xy = perturbed_vertices(nx, ny, L, 7)
    nodes = W.node_coords(nx, ny, xy).T.copy()
    case = W.small_case(nx, ny, n_s, seed=3, L=L)
    args = (case["params"], case["H"], case["A"], case["tau"], case["vel0"], case["S0"], 3)
    va, Sa = oracle.subcycles(nx, ny, xy, n_s, 1, *args)
    vb, Sb = oracle.subcycles(nx, ny, nodes, n_s, 1, *args)
    assert rel(vb, va) < 1e-14 and rel(Sb, Sa) < 1e-14
    ma, _ = oracle.lumped(nx, ny, xy, n_s, 1, case["params"], case["H"])
    mb, _ = oracle.lumped(nx, ny, nodes, n_s, 1, case["params"], case["H"])
    assert rel(mb, ma) < 1e-14


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_iso_strain_of_a_linear_field_is_exact(n_s):
    """On curved elements a physical linear velocity lies in the isoparametric
    space, so its projected strain is the exact constant (higher DG
    coefficients zero)."""
    nx, ny = 4, 3
    nodes = curved(nx, ny, 11)
    a, b, c, d = 2e-6, -1e-6, 3e-6, 0.5e-6
    vel = np.stack([a * nodes[:, 0] + b * nodes[:, 1], c * nodes[:, 0] + d * nodes[:, 1]])
    E = oracle.strain(nx, ny, nodes, n_s, vel)
    for comp, val in ((0, a), (1, 0.5 * (b + c)), (2, d)):
        assert np.allclose(E[comp, 0], val, rtol=1e-12, atol=0)
        assert np.abs(E[comp, 1:]).max() < 1e-12 * abs(val)


def test_iso_rigid_rotation_has_no_strain():
    nx, ny = 4, 4
    nodes = curved(nx, ny, 13)
    w = 1e-5
    vel = np.stack([-w * nodes[:, 1], w * nodes[:, 0]])
    E = oracle.strain(nx, ny, nodes, 6, vel)
    assert np.abs(E).max() < 1e-12 * w


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_iso_forces_sum_to_zero(n_s):
    """sum_j phi_j = 1 gives sum_j grad phi_j = 0 at every quadrature point,
    so the nodal forces of any stress sum to zero on curved elements too."""
    nx, ny = 4, 3
    nodes = curved(nx, ny, 17)
    S = np.random.default_rng(2).uniform(-5e3, 5e3, (3, n_s, nx * ny))
    F = oracle.divergence(nx, ny, nodes, n_s, S)
    scale = np.abs(S).max() * 3e3 / nx
    assert np.abs(F.sum(axis=1)).max() < 1e-12 * scale * nx * ny


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_iso_matches_bruteforce(n_s):
    """Curved elements against the independent numpy restatement (global
    assembly, shifted-Legendre basis) with the method's Gauss rule."""
    nx, ny = 3, 3
    L = 3e3
    nodes = curved(nx, ny, 19, L=L)
    case = W.small_case(nx, ny, n_s, seed=5, L=L)
    bf = BF.Mesh(nx, ny, nodes, n_s)
    vel = case["vel0"]
    E = oracle.strain(nx, ny, nodes, n_s, vel)
    Ebf = bf.strain(vel)
    assert rel(bf.values_documented(E), bf.values(Ebf)) < 1e-12
    F = oracle.divergence(nx, ny, nodes, n_s, case["S0"])
    Fbf = bf.divergence(bf.from_documented(case["S0"]))
    assert rel(F, Fbf) < 1e-12
    vo, So = oracle.subcycles(nx, ny, nodes, n_s, 1, case["params"], case["H"], case["A"],
                              case["tau"], vel, case["S0"], 3)
    vb, Sb, _ = bf.subcycles(vel, case["S0"], case["H"], case["A"], case["tau"], case["params"], 3)
    assert rel(vo, vb) < 1e-11
    assert rel(bf.values_documented(So), bf.values(Sb)) < 1e-11


@pytest.mark.parametrize("n_s", [3, 6, 8])
def test_iso_lumped_area_tiles_the_square(n_s):
    """Curved elements whose boundary nodes stay on the square's sides tile
    the square: sum_j l_j = L^2 (det J of a Q2 map has degree <= 3 in each
    reference variable, which both Gauss rules integrate exactly), and,
    since x is itself the Q2 interpolant of the node positions,
    sum_j l_j x_j = int x dA = L^3 / 2 wherever the rule integrates
    x det J (degree <= 5: the 3-point rule of the 6- and 8-dof spaces)."""
    nx, ny, L = 6, 5, 3e3
    nodes = curved(nx, ny, 11, L=L)
    H = np.full((1, nx * ny), 1.0)
    _, l = oracle.lumped(nx, ny, nodes, n_s, 1, P0, H)
    assert abs(l.sum() - L * L) <= 1e-12 * L * L
    if n_s != 3:
        assert abs(np.dot(l, nodes[:, 0]) - L ** 3 / 2) <= 1e-12 * L ** 3
        assert abs(np.dot(l, nodes[:, 1]) - L ** 3 / 2) <= 1e-12 * L ** 3


# --------------------------------------------------------------------------
# Ocean current (Eq. 2's water drag with v_o != 0, reading 7: c = l Cw rho_w
# |v_o - v^{p-1}|, drag implicit in v^p and explicit in v_o)
# --------------------------------------------------------------------------
def test_free_drift_with_ocean_current_recurrence():
    """P* = 0 (sigma = 0), uniform H, tau and ocean current z_o: every interior
    node follows the complex recurrence (divided by l, m/l = rho H)
      (rho H (1+beta)/dt + c + i rho H f) z^p
          = (rho H/dt)(beta z^{p-1} + z^n) + tau + c z_o,
      c = Cw rho_w |z_o - z^{p-1}|,
    iterated here in scalar complex arithmetic."""
    p, xy, H, A, tau = _free_drift_case()
    nx = ny = 4
    ne, nn, _ = W.sizes(nx, ny)
    zo = complex(0.23, -0.41)  # distinct components: a swapped x/y shows
    vo = np.stack([np.full(nn, zo.real), np.full(nn, zo.imag)])
    z0 = complex(0.05, 0.02)
    vel0 = np.stack([np.full(nn, z0.real), np.full(nn, z0.imag)])
    n_sub = 40
    vel, _ = oracle.subcycles(nx, ny, xy, 3, 1, p, H, A, tau, vel0, np.zeros((3, 3, ne)), n_sub,
                              vn=np.zeros((2, nn)), vo=vo)
    rhoH = p["rho_ice"] * 1.3
    k = p["Cw"] * p["rho_water"]
    t = complex(0.21, -0.13)
    z = z0
    for _ in range(n_sub):
        c = k * abs(zo - z)
        z = (rhoH / p["dt"] * p["beta"] * z + t + c * zo) / (
            rhoH * (1 + p["beta"]) / p["dt"] + c + 1j * rhoH * p["coriolis_f"])
    nw = 2 * nx + 1
    grid = vel.reshape(2, nw, nw)[:, 1:-1, 1:-1]
    assert np.allclose(grid[0], z.real, rtol=1e-13) and np.allclose(grid[1], z.imag, rtol=1e-13)
    assert np.all(vel.reshape(2, nw, nw)[:, :, 0] == 0)


def test_ice_at_rest_in_still_air_is_dragged_to_the_ocean_velocity():
    """No wind, no Coriolis, P* = 0 and a uniform ocean current: the converged
    subcycle of an outer step from v^n = z_o is v = z_o exactly (no drag at
    zero relative velocity, the momentum balance is already satisfied), and
    from rest the iterates approach z_o monotonically along its direction."""
    p, xy, H, A, tau = _free_drift_case(f=0.0)
    nx = ny = 4
    ne, nn, _ = W.sizes(nx, ny)
    zo = complex(-0.31, 0.17)
    vo = np.stack([np.full(nn, zo.real), np.full(nn, zo.imag)])
    still = np.zeros((2, nn))
    nw = 2 * nx + 1
    inner = (slice(None), slice(1, -1), slice(1, -1))
    # from v = v^n = z_o nothing changes
    vel, _ = oracle.subcycles(nx, ny, xy, 3, 1, p, H, A, still, vo, np.zeros((3, 3, ne)), 25,
                              vo=vo)
    g = vel.reshape(2, nw, nw)[inner]
    assert np.allclose(g[0], zo.real, rtol=1e-15) and np.allclose(g[1], zo.imag, rtol=1e-15)
    # from rest (v^n = 0): the direction is that of z_o and |v| grows towards |z_o|
    last = 0.0
    vel = still.copy()
    S = np.zeros((3, 3, ne))
    for _ in range(5):
        vel, S = oracle.subcycles(nx, ny, xy, 3, 1, p, H, A, still, vel, S, 1, vn=still, vo=vo)
        g = vel.reshape(2, nw, nw)[inner]
        zz = complex(g[0].mean(), g[1].mean())
        assert abs(zz.imag * zo.real - zz.real * zo.imag) < 1e-15  # parallel to z_o
        assert last < abs(zz) < abs(zo)
        last = abs(zz)


# --------------------------------------------------------------------------
# DG1/DG2 ice (n_A = 3 or 6): Listing 1 evaluates H and A at every Gauss
# point (H.row(i) times the ice basis there) and clamps the values there;
# the lumped mass integrates the clamped height (reading 8)
# --------------------------------------------------------------------------
def dg_ice(ne, n_a, seed):
    """DG coefficients (n_a, N_e) of H and A: a mean plus slopes/curvatures
    (H stays positive everywhere; A exceeds 1 at some points, so its clamp acts)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = np.zeros((n_a, ne)); A = np.zeros((n_a, ne))
    H[0] = rng.uniform(0.5, 1.8, ne)
    A[0] = rng.uniform(0.75, 0.97, ne)
    H[1:] = rng.uniform(-0.3, 0.3, (n_a - 1, ne))
    A[1:] = rng.uniform(-0.08, 0.08, (n_a - 1, ne))
    return H, A


def _documented_basis(n, xi, eta):
    """The documented DG basis, written out as scalars."""
    xh, eh = xi - 0.5, eta - 0.5
    return [1.0, xh, eh, xh * xh - 1.0 / 12.0, xh * eh, eh * eh - 1.0 / 12.0,
            (xh * xh - 1.0 / 12.0) * eh, xh * (eh * eh - 1.0 / 12.0)][:n]


@pytest.mark.parametrize("n_s,n_a", [(3, 3), (3, 6), (6, 3), (6, 6), (8, 3), (8, 6)])
def test_stress_with_dg_ice_evaluates_strength_at_each_gauss_point(n_s, n_a):
    """E = 0 and S = 0: one update gives S_11 = S_22 = -(1/alpha) Proj(P_g / 2) and
    S_12 = 0.  P_g is computed here point by point in scalar code (h = max(0,
    sum_t H_t psi_t(x_g)), a = clamp(sum_t A_t psi_t(x_g), 0, 1), P = P* h
    exp(-C(1-a))) at numpy's Gauss points, and projected with the documented
    basis, which is orthogonal on rectangles (M_K diagonal, det J cancels)."""
    nx, ny = 3, 2
    ne = nx * ny
    xy = W.uniform_vertices(nx, ny, 3 * 2.5e3, 2 * 1.5e3)  # rectangles, hx != hy
    H, A = dg_ice(ne, n_a, 40 + n_s + n_a)
    A[0, ::2] = 0.995  # some Gauss-point values above 1: the clamp of A acts
    A[1:3, ::2] = 0.08
    p = dict(P0)
    out = oracle.stress(nx, ny, xy, n_s, n_a, p, np.zeros((3, n_s, ne)), H, A,
                        np.zeros((3, n_s, ne)))
    ngp = {3: 2, 6: 3, 8: 3}[n_s]
    x, w = np.polynomial.legendre.leggauss(ngp)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    clamped = 0
    for K in range(ne):
        num = [0.0] * n_s
        den = [0.0] * n_s
        for gy in range(ngp):
            for gx in range(ngp):
                psi_a = _documented_basis(n_a, x[gx], x[gy])
                psi_s = _documented_basis(n_s, x[gx], x[gy])
                hv = sum(H[t, K] * psi_a[t] for t in range(n_a))
                av = sum(A[t, K] * psi_a[t] for t in range(n_a))
                clamped += av > 1.0
                P = p["Pstar"] * max(0.0, hv) * math.exp(-p["C"] * (1.0 - min(1.0, max(0.0, av))))
                wg = w[gx] * w[gy]
                for s in range(n_s):
                    num[s] += wg * psi_s[s] * (-0.5 * P)
                    den[s] += wg * psi_s[s] * psi_s[s]
        expect = np.array([num[s] / den[s] for s in range(n_s)]) / p["alpha"]
        assert np.allclose(out[0, :, K], expect, rtol=1e-12, atol=1e-12 * abs(expect[0]))
        assert np.allclose(out[2, :, K], expect, rtol=1e-12, atol=1e-12 * abs(expect[0]))
        assert np.abs(out[1, :, K]).max() == 0.0
    assert clamped > 0  # the clamp of A was exercised


@pytest.mark.parametrize("n_s,n_a,affine", [(3, 3, True), (6, 3, False), (6, 6, False),
                                            (8, 6, False)])
def test_lumped_mass_with_dg_ice_matches_bruteforce(n_s, n_a, affine):
    """m_j = rho sum_K int_K max(0, H) phi_j with DG1/DG2 H (positive, so the
    clamp is inactive): for these degrees the method's NGP rule is exact (H phi_j
    det J has degree <= 2 NGP - 1 per variable), so the oracle equals the brute
    force's 10x10 rule."""
    nx, ny, L = 3, 2, 6e3
    xy = W.uniform_vertices(nx, ny, L, L) if affine else perturbed_vertices(nx, ny, L, 5)
    H, _ = dg_ice(nx * ny, n_a, 60 + n_s + n_a)
    m, l = oracle.lumped(nx, ny, xy, n_s, n_a, P0, H)
    mb, lb = BF.Mesh(nx, ny, xy, n_s).lumped(H, P0["rho_ice"], "exact")
    assert rel(m, mb) < 1e-14 and rel(l, lb) < 1e-14


def test_lumped_mass_with_dg2_ice_on_the_dg1_rule():
    """DG2 ice with 3 stress dofs: the 2x2 rule is not exact for H phi_j, and the
    reading integrates with the stress space's rule all the same; the brute
    force with that rule agrees, and the exact integral differs."""
    nx, ny, L = 3, 2, 6e3
    xy = W.uniform_vertices(nx, ny, L, L)
    H, _ = dg_ice(nx * ny, 6, 71)
    m, _ = oracle.lumped(nx, ny, xy, 3, 6, P0, H)
    M = BF.Mesh(nx, ny, xy, 3)
    assert rel(m, M.lumped(H, P0["rho_ice"], "method")[0]) < 1e-14
    assert rel(m, M.lumped(H, P0["rho_ice"], "exact")[0]) > 1e-6


# --------------------------------------------------------------------------
# Per-element P* field (the ice strength parameter as a field, the input the
# adjoint differentiates against): a plain substitution of P*_K for P* in
# Listing 1's P = P* h exp(-C(1-A))
# --------------------------------------------------------------------------
def test_uniform_strength_field_equals_scalar_bitwise():
    case = W.small_case(5, 4, 6, seed=12)
    ne = 20
    args = (case["nx"], case["ny"], case["xy"], 6, 1, case["params"], case["H"], case["A"],
            case["tau"], case["vel0"], case["S0"], 7)
    a = oracle.subcycles(*args)
    b = oracle.subcycles(*args, Pstar_K=np.full(ne, case["params"]["Pstar"]))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n_s,n_a", [(3, 1), (6, 3), (8, 6)])
def test_strength_field_acts_element_by_element(n_s, n_a):
    """The stress update is element-local: with a P* field, element K's result
    equals the result of the scalar P* = P*_K, bitwise, for every K."""
    nx, ny = 4, 3
    ne = nx * ny
    xy = perturbed_vertices(nx, ny, 8e3, 9)
    rng = np.random.Generator(np.random.PCG64(90 + n_s))
    H, A = dg_ice(ne, n_a, 91) if n_a > 1 else (rng.uniform(0.3, 2, (1, ne)),
                                                rng.uniform(0.8, 1, (1, ne)))
    E = rng.uniform(-2e-7, 2e-7, (3, n_s, ne))
    S = rng.uniform(-5e3, 5e3, (3, n_s, ne))
    field = P0["Pstar"] * rng.uniform(0.5, 1.5, ne)
    out = oracle.stress(nx, ny, xy, n_s, n_a, P0, E, H, A, S, Pstar_K=field)
    for K in range(ne):
        one = oracle.stress(nx, ny, xy, n_s, n_a, dict(P0, Pstar=field[K]), E, H, A, S)
        assert np.array_equal(out[:, :, K], one[:, :, K])


# --------------------------------------------------------------------------
# The whole subcycle with DG ice, an ocean current and a P* field against the
# brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n_s,n_a", [(3, 3), (3, 6), (6, 3), (6, 6)])
@pytest.mark.parametrize("affine", [True, False])
def test_whole_subcycle_with_dg_ice_ocean_and_strength_field_matches_bruteforce(n_s, n_a,
                                                                                 affine):
    nx, ny = 2, 2
    case = W.small_case(nx, ny, n_s, seed=23)
    L = case["L"]
    ne, nn, _ = W.sizes(nx, ny)
    xy = case["xy"] if affine else perturbed_vertices(nx, ny, L, 33, amp=0.15)
    p = case["params"]
    H, A = dg_ice(ne, n_a, 80 + n_s + n_a)
    vo = W.smooth_velocity(nx, ny, 81, amp=0.2, L=L)
    vo[:, 0] += 0.05  # a current at the boundary nodes too (they stay Dirichlet)
    field = p["Pstar"] * np.random.Generator(np.random.PCG64(82)).uniform(0.5, 1.5, ne)
    n_sub = 6
    vel, S, E, F, fel = oracle.subcycles(nx, ny, xy, n_s, n_a, p, H, A, case["tau"],
                                         case["vel0"], case["S0"], n_sub, vo=vo,
                                         want_last=True, Pstar_K=field)
    M = BF.Mesh(nx, ny, xy, n_s)
    vb, Sb, Eb = M.subcycles(case["vel0"], case["S0"], H, A, case["tau"], p, n_sub, vo=vo,
                             Pstar_K=field)
    assert rel(vel, vb) < 1e-12
    assert rel(M.values_documented(S), M.values(Sb)) < 1e-12
    assert rel(M.values_documented(E), M.values(Eb)) < 1e-12
    # the ocean term moved the ice: without it the result differs
    v0, _ = oracle.subcycles(nx, ny, xy, n_s, n_a, p, H, A, case["tau"], case["vel0"],
                             case["S0"], n_sub, Pstar_K=field)
    assert rel(vel, v0) > 1e-3


def test_delta_at_gauss_points_matches_printed_constants():
    """Delta of Listing 1 with the printed 5/4, 3/2, 1 at every Gauss point of a
    constant strain, and Delta = Delta_min exactly where the strain vanishes."""
    d = GOLD["delta"]
    for n_s in (3, 6, 8):
        E = np.zeros((3, n_s, 2))
        e11, e12, e22 = 3e-7, -1.1e-7, -2e-7
        E[:, 0, 0] = (e11, e12, e22)  # element 0 strained, element 1 rigid
        out = oracle.delta(2, 1, n_s, P0, E)
        D = math.sqrt(P0["DeltaMin"] ** 2 + d["sq"] * (e11 ** 2 + e22 ** 2)
                      + d["mix"] * e11 * e22 + d["shear"] * e12 ** 2)
        assert np.allclose(out[0], D, rtol=1e-14)
        assert np.all(out[1] == P0["DeltaMin"])


def test_velocity_node_without_mass_or_drag_stays_at_rest():
    """A node with no ice (m = 0) moving with the ocean (c = 0): the 2x2 system of
    the velocity update is singular (a = b = 0) and the reading sets v = 0 there;
    where the ice moves relative to the ocean, c > 0 and (with m = 0) the update
    is the pure drag balance c (v - v_o) = F + l tau, v = v_o + (F + l tau) / c."""
    nx = ny = 3
    ne, nn, _ = W.sizes(nx, ny)
    rng = np.random.default_rng(17)
    p = dict(P0)
    m = np.zeros(nn)
    l = rng.uniform(1e5, 2e5, nn)
    vo = rng.uniform(-0.2, 0.2, (2, nn))
    vprev = vo.copy()
    moving = rng.random(nn) < 0.5
    vprev[:, moving] += rng.uniform(-0.1, 0.1, (2, int(moving.sum())))
    F = rng.uniform(-50, 50, (2, nn))
    tau = rng.uniform(-0.3, 0.3, (2, nn))
    out = oracle.velocity(nx, ny, p, F, vprev, np.zeros((2, nn)), tau, vo, m, l)
    nw = 2 * nx + 1
    ix, iy = np.arange(nn) % nw, np.arange(nn) // nw
    interior = (ix > 0) & (iy > 0) & (ix < nw - 1) & (iy < nw - 1)
    rest = interior & ~moving
    assert rest.any() and (interior & moving).any()
    assert np.all(out[:, rest] == 0.0)
    mv = interior & moving
    c = l[mv] * p["Cw"] * p["rho_water"] * np.hypot(*(vo[:, mv] - vprev[:, mv]))
    expect = vo[:, mv] + (F[:, mv] + l[mv] * tau[:, mv]) / c
    assert np.allclose(out[:, mv], expect, rtol=1e-13)
    assert np.all(out[:, ~interior] == 0.0)
