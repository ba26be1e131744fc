"""Pins of the oracle's DG upwind advection of H and A (transport equations
of Sec. 2, discretised as Sec. 2.1 states: DG, upwind flux, explicit
Runge-Kutta) against facts fixed by the mathematics (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_2402_00466_gb300 import workloads as W
from tests import bruteforce as BF

L = 4e3


def mesh(nx, ny, geometry, seed=5):
    if geometry == "uniform":
        return W.uniform_vertices(nx, ny, L, 0.75 * L)
    return W.perturbed_vertices(nx, ny, seed, L=L)


def drift_velocity(nx, ny, xy):
    """A smooth velocity whose normal component keeps one sign on every edge
    (so every integrand is a polynomial on each edge)."""
    nc = W.node_coords(nx, ny, xy)
    return np.stack([0.3 + 0.05 * np.sin(3 * nc[0] / L), 0.25 + 0.05 * np.cos(2 * nc[1] / L)])


def coeffs_of(fn, nx, ny, xy, n_a):
    """DG coefficients (n_a, N_e) of a function that lies in the DG space of
    every element (interpolated at sample points, least squares)."""
    xs = np.array([0.1, 0.35, 0.6, 0.9])
    XI, ET = np.meshgrid(xs, xs)
    xi, eta = XI.ravel(), ET.ravel()
    psi = np.array([oracle.dg_basis(n_a, a, b) for a, b in zip(xi, eta)])
    out = np.zeros((n_a, nx * ny))
    bf = BF.Advection(nx, ny, xy, n_a)
    for K in range(nx * ny):
        P = bf.xmap(K, xi, eta)
        out[:, K] = np.linalg.lstsq(psi, fn(P[:, 0], P[:, 1]), rcond=None)[0]
    return out


@pytest.mark.parametrize("n_a", [1, 3, 6])
@pytest.mark.parametrize("geometry", ["uniform", "perturbed"])
def test_operator_matches_bruteforce(n_a, geometry):
    """Semi-discrete operator against the independent global brute force
    (physical normals, 10-point rules): agrees only if the oracle's
    quadrature is exact and its metric terms, signs and upwinding right."""
    nx, ny = 4, 3
    xy = mesh(nx, ny, geometry)
    vel = drift_velocity(nx, ny, xy)
    rng = np.random.default_rng(1 + n_a)
    H = rng.uniform(0.5, 1.5, (n_a, nx * ny))
    A = rng.uniform(0.2, 0.9, (n_a, nx * ny))
    LH, LA = oracle.advect_operator(nx, ny, xy, n_a, vel, H, A)
    bf = BF.Advection(nx, ny, xy, n_a)
    for got, F in ((LH, H), (LA, A)):
        ref = bf.operator(vel, F)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n_a", [1, 3, 6])
def test_operator_bruteforce_with_reversing_flow(n_a):
    """A rotating velocity (the normal component changes sign along some
    edges): the pointwise upwind choice on both sides still agrees with the
    brute force at the quadrature points the oracle uses."""
    nx, ny = 4, 4
    xy = mesh(nx, ny, "perturbed", seed=11)
    nc = W.node_coords(nx, ny, xy)
    vel = np.stack([-(nc[1] - 0.37 * L), nc[0] - 0.52 * L]) * 1e-4
    rng = np.random.default_rng(7)
    H = rng.uniform(0.5, 1.5, (n_a, nx * ny))
    LH, _ = oracle.advect_operator(nx, ny, xy, n_a, vel, H, H)
    # the brute force with the oracle's own rule (same points, same upwind
    # decisions), since with a sign change no rule is exact
    bf = BF.Advection(nx, ny, xy, n_a, nq={1: 3, 3: 3, 6: 4}[n_a])
    ref = bf.operator(vel, H)
    assert np.abs(LH - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("n_a", [1, 3, 6])
@pytest.mark.parametrize("geometry", ["uniform", "perturbed"])
def test_constant_state_preserved_by_divergence_free_flow(n_a, geometry):
    """H = const under a rigid rotation (div v = 0): the volume and edge terms
    cancel exactly (integration by parts), so L(H) = 0 to rounding.  A wrong
    sign on one edge or a transposed metric term breaks it."""
    nx, ny = 5, 4
    xy = mesh(nx, ny, geometry)
    nc = W.node_coords(nx, ny, xy)
    vel = np.stack([-(nc[1] - 0.4 * L), nc[0] - 0.55 * L]) * 1e-4
    H = coeffs_of(lambda x, y: 1.3 + 0 * x, nx, ny, xy, n_a)
    LH, LA = oracle.advect_operator(nx, ny, xy, n_a, vel, H, 0.5 * H)
    # the scale of the individual terms is H |v| / h; a wrong term is O(1) of it
    assert np.abs(LH).max() <= 1e-12 * 1.3 * np.abs(vel).max() / (L / nx)


@pytest.mark.parametrize("n_a,deg", [(1, 0), (3, 1), (6, 2)])
@pytest.mark.parametrize("geometry", ["uniform", "affine"])
def test_translation_of_polynomials_is_exact(n_a, deg, geometry):
    """Uniform velocity U on an affine mesh (where a global polynomial of the
    space's degree lies in every element's DG space): it is transported
    exactly (continuous data, so upwinding picks the exact trace; the time
    scheme of order deg+1 integrates the polynomial-in-time exact solution
    exactly): H(x, t) = H0(x - U t)."""
    nx, ny = 5, 4
    xy = mesh(nx, ny, "uniform")
    if geometry == "affine":  # parallelograms: a sheared, stretched mesh
        xy = xy @ np.array([[1.0, 0.3], [-0.2, 1.1]]).T
    ne, nn = oracle.sizes(nx, ny)
    U = np.array([0.4, -0.15])
    vel = np.stack([np.full(nn, U[0]), np.full(nn, U[1])])
    c = np.array([1.1, 0.3, -0.2, 0.05, 0.08, -0.04])
    def H0(x, y):
        x, y = x / L, y / L
        terms = [np.ones_like(x), x, y, x * x, x * y, y * y]
        k = {0: 1, 1: 3, 2: 6}[deg]
        return sum(ci * t for ci, t in zip(c[:k], terms[:k]))
    dt, n = 120.0, 7
    H = coeffs_of(H0, nx, ny, xy, n_a)
    A0 = lambda x, y: 0.9 - 0.5 * H0(y, x)  # noqa: E731  (a second field, moved alike)
    A = coeffs_of(A0, nx, ny, xy, n_a)
    H1, A1 = oracle.advect(nx, ny, xy, n_a, vel, dt, n, H, A)
    exact = coeffs_of(lambda x, y: H0(x - U[0] * n * dt, y - U[1] * n * dt), nx, ny, xy, n_a)
    exactA = coeffs_of(lambda x, y: A0(x - U[0] * n * dt, y - U[1] * n * dt), nx, ny, xy, n_a)
    assert np.abs(H1 - exact).max() <= 1e-12
    assert np.abs(A1 - exactA).max() <= 1e-12


@pytest.mark.parametrize("n_a", [1, 3, 6])
def test_mass_conserved_with_no_boundary_flow(n_a):
    """v = 0 on the domain boundary (the Dirichlet velocity of the momentum
    problem): sum_K int_K H is conserved over many steps to rounding."""
    nx, ny = 6, 5
    xy = mesh(nx, ny, "perturbed", seed=13)
    vel = W.smooth_velocity(nx, ny, 3, amp=0.4, L=L)
    rng = np.random.default_rng(3)
    H = rng.uniform(0.3, 2.0, (n_a, nx * ny))
    A = rng.uniform(0.5, 1.0, (n_a, nx * ny))
    bf = BF.Advection(nx, ny, xy, n_a)
    m0, a0 = bf.integral(H), bf.integral(A)
    H1, A1 = oracle.advect(nx, ny, xy, n_a, vel, 120.0, 20, H, A)
    assert abs(bf.integral(H1) - m0) <= 1e-13 * abs(m0)
    assert abs(bf.integral(A1) - a0) <= 1e-13 * abs(a0)
    assert np.abs(H1 - H).max() > 1e-6 and np.abs(A1 - A).max() > 1e-6  # the ice did move


@pytest.mark.parametrize("n_a,order", [(1, 1), (3, 2), (6, 3)])
def test_runge_kutta_step_is_taylor_polynomial(n_a, order):
    """With fixed upwind directions the semi-discrete operator is linear,
    L(H) = Lm H; one SSP-RK step of order p is then exactly
    sum_{k<=p} (dt Lm)^k / k! applied to H (Lm assembled column by column
    from the brute force)."""
    nx, ny = 3, 3
    xy = mesh(nx, ny, "perturbed", seed=17)
    vel = drift_velocity(nx, ny, xy)
    ne = nx * ny
    bf = BF.Advection(nx, ny, xy, n_a)
    N = n_a * ne
    Lm = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N); e[k] = 1.0
        Lm[:, k] = bf.operator(vel, e.reshape(n_a, ne)).ravel()
    dt = 600.0
    rng = np.random.default_rng(19)
    H = rng.uniform(0.5, 1.5, (n_a, ne))
    A = rng.uniform(0.6, 1.0, (n_a, ne))
    step = np.eye(N)
    term = np.eye(N)
    for k in range(1, order + 1):
        term = term @ (dt * Lm) / k
        step = step + term
    ref = (step @ H.ravel()).reshape(n_a, ne)
    refA = (step @ A.ravel()).reshape(n_a, ne)
    H1, A1 = oracle.advect(nx, ny, xy, n_a, vel, dt, 1, H, A)
    assert np.abs(H1 - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(A1 - refA).max() <= 1e-12 * np.abs(refA).max()


def test_first_order_upwind_closed_form():
    """DG0 with a uniform x velocity on a uniform mesh is the textbook
    first-order upwind scheme H_k <- H_k - (U dt/h)(H_k - H_{k-1})."""
    nx, ny = 6, 4
    xy = W.uniform_vertices(nx, ny, 6e3, 4e3)
    ne, nn = oracle.sizes(nx, ny)
    vel = np.zeros((2, nn)); vel[0] = 0.5
    H = np.random.default_rng(0).uniform(0.5, 1.5, (1, ne))
    A = np.random.default_rng(1).uniform(0.5, 1.0, (1, ne))
    H1, A1 = oracle.advect(nx, ny, xy, 1, vel, 120.0, 1, H, A)
    c = 0.5 * 120.0 / 1e3
    for F, F1 in ((H, H1), (A, A1)):
        g = F.reshape(ny, nx)
        exp = g.copy()
        exp[:, 1:] = g[:, 1:] - c * (g[:, 1:] - g[:, :-1])
        assert np.abs(F1.reshape(ny, nx) - exp).max() < 1e-15


def test_first_order_upwind_on_a_one_element_wide_column():
    """A mesh one element wide (nx = 1) with a uniform y velocity: the same
    first-order upwind scheme along the column."""
    nx, ny = 1, 6
    xy = W.uniform_vertices(nx, ny, 1e3, 6e3)
    ne, nn = oracle.sizes(nx, ny)
    vel = np.zeros((2, nn)); vel[1] = -0.4  # flowing south: the upwind side is north
    H = np.random.default_rng(2).uniform(0.5, 1.5, (1, ne))
    H1, A1 = oracle.advect(nx, ny, xy, 1, vel, 120.0, 1, H, 2.0 * H)
    c = 0.4 * 120.0 / 1e3
    exp = H[0].copy()
    exp[:-1] = H[0, :-1] - c * (H[0, :-1] - H[0, 1:])
    assert np.abs(H1[0] - exp).max() < 1e-15 and np.abs(A1[0] - 2.0 * exp).max() < 1e-15
    xy2 = W.uniform_vertices(ny, nx, 6e3, 1e3)  # and a row one element high (ny = 1)
    ne2, nn2 = oracle.sizes(ny, nx)
    vel2 = np.zeros((2, nn2)); vel2[0] = 0.4
    H2, _ = oracle.advect(ny, nx, xy2, 1, vel2, 120.0, 1, H, H)
    exp2 = H[0].copy()
    exp2[1:] = H[0, 1:] - c * (H[0, 1:] - H[0, :-1])
    assert np.abs(H2[0] - exp2).max() < 1e-15


def test_advect_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.advect(2, 2, W.uniform_vertices(2, 2), 2, np.zeros((2, 25)), 1.0, 1,
                      np.zeros((2, 4)), np.zeros((2, 4)))


@pytest.mark.parametrize("n_a", [1, 3, 6])
def test_iso_advection_preserves_a_constant_and_matches_bruteforce(n_a):
    """Curved (isoparametric) elements: a constant under a rigid rotation stays
    put, and the operator agrees with the brute force at the method's rule."""
    nx, ny, L = 4, 4, 3e3
    nodes = W.curved_nodes(nx, ny, 23, amp=0.08, L=L)
    vel = np.stack([-(nodes[:, 1] - 0.4 * L), nodes[:, 0] - 0.55 * L]) * 1e-4
    ne = nx * ny
    H = np.zeros((n_a, ne)); H[0] = 1.3
    LH, _ = oracle.advect_operator(nx, ny, nodes, n_a, vel, H, H)
    assert np.abs(LH).max() <= 1e-12 * 1.3 * np.abs(vel).max() / (L / nx)
    rng = np.random.default_rng(29)
    H = rng.uniform(0.5, 1.5, (n_a, ne))
    LH, _ = oracle.advect_operator(nx, ny, nodes, n_a, vel, H, H)
    ref = BF.Advection(nx, ny, nodes, n_a).operator(vel, H)
    assert np.abs(LH - ref).max() <= 1e-11 * np.abs(ref).max()
