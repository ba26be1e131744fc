"""Seeded synthetic inputs for the mEVP momentum subcycle.

This module only builds inputs: mesh vertices, ice height/concentration
fields, the nodal wind stress of a moving cyclone, and the parameter set.  It
holds none of the method's arithmetic (no strain, stress, divergence, mass or
velocity update), so both the CUDA path and the CPU oracle can take their
inputs from it.

The paper validates on the moving-cyclone benchmark over a 512 km square
(Sec. 4); its definition is not reproduced here.  These are our own seeded
constructions with the same domain, resolution range and magnitudes.
"""
from __future__ import annotations

import math

import numpy as np

# Parameter set (P*, C, e, Delta_min from the paper's stress update, Sec. 3 /
# App. A; alpha = beta = 300, dt = 120 s = 1 h / 30 advection steps, Sec. 4;
# the remaining constants are typical literature values).
DEFAULT_PARAMS = dict(
    Pstar=27500.0, C=20.0, e=2.0, DeltaMin=2e-9, alpha=300.0, beta=300.0, dt=120.0,
    rho_ice=900.0, rho_water=1026.0, Cw=5.5e-3, coriolis_f=1.46e-4)
RHO_AIR = 1.3
C_AIR = 1.2e-3
DOMAIN_M = 512e3

# Workloads: mesh size, DG stress dofs, subcycles per outer step, ice recipe.
CONFIGS = {
    # 32x32 quads, DG1 stress, iid H ~ U[0.3,2], A ~ U[0.8,1], 100 subcycles
    "mesh32_dg1": dict(nx=32, ny=32, n_s=3, n_a=1, n_sub=100, ice="iid", seeds=(1,),
                       wind_seed=11),
    # 256x256 quads, DG2 stress, Gaussian-random H/A with 5 km correlation, 500 subcycles
    "mesh256_dg2": dict(nx=256, ny=256, n_s=6, n_a=1, n_sub=500, ice="grf", seeds=(2, 3),
                        wind_seed=12),
    # 1024x1024 quads, DG2 stress, same recipe, 500 subcycles
    "mesh1024_dg2": dict(nx=1024, ny=1024, n_s=6, n_a=1, n_sub=500, ice="grf", seeds=(4, 5),
                         wind_seed=13),
    # 256x256 quads, DG1 stress, 100 subcycles
    "mesh256_dg1": dict(nx=256, ny=256, n_s=3, n_a=1, n_sub=100, ice="grf", seeds=(7, 8),
                        wind_seed=14),
    # 256x256 smoothly curvilinear quads (general bilinear elements), DG2, 500 subcycles
    "mesh256_dg2_wavy": dict(nx=256, ny=256, n_s=6, n_a=1, n_sub=500, ice="grf", seeds=(2, 3),
                             wind_seed=12, geometry="wavy"),
    # gradient of the final kinetic energy w.r.t. the P* field and the wind
    # stress after 100 subcycles on the 256x256 DG1 mesh, checkpoint every 10
    "adjoint256_dg1": dict(nx=256, ny=256, n_s=3, n_a=1, n_sub=100, ice="grf", seeds=(7, 8),
                           wind_seed=14, adjoint_every=10, vel_seed=16),
    # the same curvilinear map at every CG2 node: 256x256 curved
    # (isoparametric Q2) elements, DG2, 500 subcycles
    "mesh256_dg2_iso": dict(nx=256, ny=256, n_s=6, n_a=1, n_sub=500, ice="grf", seeds=(2, 3),
                            wind_seed=12, geometry="wavy_iso"),
    # the curvilinear meshes at 1024x1024 (the mixed path's HBM-bound size)
    "mesh1024_dg2_wavy": dict(nx=1024, ny=1024, n_s=6, n_a=1, n_sub=500, ice="grf",
                              seeds=(4, 5), wind_seed=13, geometry="wavy"),
    "mesh1024_dg2_iso": dict(nx=1024, ny=1024, n_s=6, n_a=1, n_sub=500, ice="grf",
                             seeds=(4, 5), wind_seed=13, geometry="wavy_iso"),
    # transport of DG2 H and A on 1024x1024 quads with a smooth velocity held
    # fixed (the step before the subcycles); one advection step per bench step
    "advect1024_dg2": dict(nx=1024, ny=1024, n_s=6, n_a=6, n_sub=0, ice="grf", seeds=(4, 5),
                           wind_seed=13, vel_seed=15),
}

# Ensemble of independent square domains on the 512 km square: sides drawn
# log-uniformly in [64, 512] elements, DG1 or DG2 stress at random, Gaussian-
# random ice and a cyclone of its own per member, 200 subcycles per step.
ENSEMBLES = {
    "ensemble64": dict(n_members=64, side_lo=64, side_hi=512, n_sub=200, seed=6),
    "ensemble8": dict(n_members=8, side_lo=16, side_hi=64, n_sub=20, seed=9),
}


def sizes(nx: int, ny: int):
    """(elements, CG2 nodes, vertices)."""
    return nx * ny, (2 * nx + 1) * (2 * ny + 1), (nx + 1) * (ny + 1)


def uniform_vertices(nx: int, ny: int, Lx: float = DOMAIN_M, Ly: float = DOMAIN_M):
    """Vertices (N_v, 2), vertex id = jy*(nx+1) + jx, of a uniform quad mesh."""
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    return np.stack([X.ravel(), Y.ravel()], axis=1).copy()


def node_coords_uniform(nx: int, ny: int, Lx: float = DOMAIN_M, Ly: float = DOMAIN_M):
    """Coordinates (2, N_n) of the CG2 nodes of a uniform mesh (node = iy*(2nx+1)+ix)."""
    xs = np.linspace(0.0, Lx, 2 * nx + 1)
    ys = np.linspace(0.0, Ly, 2 * ny + 1)
    X, Y = np.meshgrid(xs, ys)
    return np.stack([X.ravel(), Y.ravel()])


def ice_iid(nx: int, ny: int, seed: int):
    """DG0 H ~ U[0.3, 2] m and A ~ U[0.8, 1], iid per element; shapes (1, N_e)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = nx * ny
    H = rng.uniform(0.3, 2.0, ne)
    A = rng.uniform(0.8, 1.0, ne)
    return H[None, :].copy(), A[None, :].copy()


def gaussian_random_field(nx: int, ny: int, h_m: float, corr_m: float, seed: int):
    """Unit-variance field on the element grid: white noise filtered in Fourier
    space by a Gaussian kernel of standard deviation corr_m (periodic)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((ny, nx))
    kx = np.fft.fftfreq(nx, d=h_m) * 2.0 * math.pi
    ky = np.fft.fftfreq(ny, d=h_m) * 2.0 * math.pi
    KX, KY = np.meshgrid(kx, ky)
    filt = np.exp(-0.5 * (KX ** 2 + KY ** 2) * corr_m ** 2)
    g = np.fft.ifft2(np.fft.fft2(w) * filt).real
    s = g.std()
    return (g - g.mean()) / (s if s > 0 else 1.0)


def ice_grf(nx: int, ny: int, seeds, L: float = DOMAIN_M, corr_m: float = 5e3):
    """DG0 H = clip(1.15 + 0.3 g1, 0.3, 2), A = clip(0.9 + 0.05 g2, 0.8, 1)."""
    h = L / nx
    g1 = gaussian_random_field(nx, ny, h, corr_m, seeds[0]).ravel()
    g2 = gaussian_random_field(nx, ny, h, corr_m, seeds[1]).ravel()
    H = np.clip(1.15 + 0.3 * g1, 0.3, 2.0)
    A = np.clip(0.9 + 0.05 * g2, 0.8, 1.0)
    return H[None, :].copy(), A[None, :].copy()


def cyclone_params(seed: int, L: float = DOMAIN_M):
    """Moving cyclone: centre uniform in the middle half of the domain, heading
    uniform, translation speed U[5,10] m/s, radius U[60,120] km."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c0 = rng.uniform(0.25 * L, 0.75 * L, 2)
    heading = rng.uniform(0.0, 2.0 * math.pi)
    speed = rng.uniform(5.0, 10.0)
    R = rng.uniform(60e3, 120e3)
    return dict(c0=c0, u=speed * np.array([math.cos(heading), math.sin(heading)]), R=R,
                umax=15.0)


def cyclone_wind_stress(node_xy, cyc, t: float = 0.0):
    """Nodal wind stress (2, N_n) = rho_air C_air |u_a| u_a of the cyclone at time t.

    Tangential, counter-clockwise wind |u_a| = umax (r/R) exp((1 - r^2/R^2)/2),
    maximal (umax) at r = R."""
    c = cyc["c0"] + cyc["u"] * t
    dx = node_xy[0] - c[0]
    dy = node_xy[1] - c[1]
    r = np.sqrt(dx * dx + dy * dy)
    R = cyc["R"]
    speed = cyc["umax"] * (r / R) * np.exp(0.5 * (1.0 - (r / R) ** 2))
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(r > 0, -dy / r, 0.0) * speed
        uy = np.where(r > 0, dx / r, 0.0) * speed
    mag = np.sqrt(ux * ux + uy * uy)
    return np.stack([RHO_AIR * C_AIR * mag * ux, RHO_AIR * C_AIR * mag * uy])


def smooth_velocity(nx: int, ny: int, seed: int, amp: float = 0.1, L: float = DOMAIN_M):
    """A smooth seeded velocity field (2, N_n), zero on the boundary, for tests
    that start from a moving state: sum of a few random sine modes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xy = node_coords_uniform(nx, ny, L, L)
    X, Y = xy[0] / L, xy[1] / L
    out = np.zeros_like(xy)
    for c in range(2):
        for _ in range(4):
            kx, ky = rng.integers(1, 5, 2)
            out[c] += rng.uniform(-1, 1) * np.sin(math.pi * kx * X) * np.sin(math.pi * ky * Y)
    out = amp * out / max(np.abs(out).max(), 1e-30)
    nw, nh = 2 * nx + 1, 2 * ny + 1
    grid = out.reshape(2, nh, nw)
    grid[:, 0, :] = 0.0
    grid[:, -1, :] = 0.0
    grid[:, :, 0] = 0.0
    grid[:, :, -1] = 0.0
    return out


def make_case(name: str, L: float = DOMAIN_M, params: dict | None = None):
    """Inputs of a named workload: dict with nx, ny, n_s, n_a, n_sub, xy, H, A,
    tau, vel0 (zeros), S0 (zeros), params."""
    cfg = dict(CONFIGS[name])
    nx, ny = cfg["nx"], cfg["ny"]
    ne, nn, nv = sizes(nx, ny)
    if cfg["ice"] == "iid":
        H, A = ice_iid(nx, ny, cfg["seeds"][0])
    else:
        H, A = ice_grf(nx, ny, cfg["seeds"], L)
    geometry = cfg.get("geometry", "uniform")
    if geometry == "wavy":
        xy = wavy_vertices(nx, ny, L=L)
    elif geometry == "wavy_iso":
        xy = wavy_nodes(nx, ny, L=L)  # the CG2 node positions
    else:
        xy = uniform_vertices(nx, ny, L, L)
    n_a = cfg["n_a"]
    if n_a > 1:
        # DG1/DG2 ice: the random-field means plus seeded slopes and curvatures
        rng = np.random.Generator(np.random.PCG64(cfg["seeds"][0] + 100))
        Hd, Ad = np.zeros((n_a, ne)), np.zeros((n_a, ne))
        Hd[0], Ad[0] = H[0], A[0]
        Hd[1:] = rng.uniform(-0.1, 0.1, (n_a - 1, ne))
        Ad[1:] = rng.uniform(-0.02, 0.02, (n_a - 1, ne))
        H, A = Hd, Ad
    ncoord = xy.T if xy.shape[0] == nn else node_coords(nx, ny, xy)
    tau = cyclone_wind_stress(ncoord, cyclone_params(cfg["wind_seed"], L))
    vel0 = (smooth_velocity(nx, ny, cfg["vel_seed"], amp=0.3, L=L) if "vel_seed" in cfg
            else np.zeros((2, nn)))
    return dict(name=name, nx=nx, ny=ny, n_s=cfg["n_s"], n_a=n_a, n_sub=cfg["n_sub"],
                L=L, xy=xy, geometry=geometry, H=H, A=A, tau=tau,
                vel0=vel0, S0=np.zeros((3, cfg["n_s"], ne)),
                params=dict(DEFAULT_PARAMS if params is None else params))


def small_case(nx: int, ny: int, n_s: int, seed: int, L: float = DOMAIN_M, moving: bool = True,
               params: dict | None = None, geometry: str = "uniform"):
    """A small seeded case of any size (iid ice, cyclone wind, optional smooth
    initial velocity and random initial stress) for parity tests.  geometry:
    "uniform", "perturbed" (random interior vertex moves, seed + 4000) or
    "wavy" (smooth curvilinear map, bilinear elements), "wavy_iso" (the same
    map at every CG2 node: isoparametric curved elements) or "curved"
    (randomly curved isoparametric elements).  xy holds the vertices, or
    for the isoparametric geometries the CG2 node positions."""
    ne, nn, nv = sizes(nx, ny)
    H, A = ice_iid(nx, ny, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    if geometry == "uniform":
        xy = uniform_vertices(nx, ny, L, L)
    elif geometry == "perturbed":
        xy = perturbed_vertices(nx, ny, seed + 4000, L=L)
    elif geometry == "wavy":
        xy = wavy_vertices(nx, ny, L=L)
    elif geometry == "wavy_iso":
        xy = wavy_nodes(nx, ny, L=L)
    elif geometry == "curved":
        xy = curved_nodes(nx, ny, seed + 4000, L=L)
    else:
        raise ValueError(f"unknown geometry {geometry!r}")
    ncoord = xy.T if xy.shape[0] == nn else node_coords(nx, ny, xy)
    tau = cyclone_wind_stress(ncoord, cyclone_params(seed + 2000, L))
    vel0 = smooth_velocity(nx, ny, seed + 3000, L=L) if moving else np.zeros((2, nn))
    S0 = rng.uniform(-5e3, 5e3, (3, n_s, ne)) if moving else np.zeros((3, n_s, ne))
    return dict(name=f"small{nx}x{ny}_dg{n_s}", nx=nx, ny=ny, n_s=n_s, n_a=1, n_sub=10, L=L,
                xy=xy, H=H, A=A, tau=tau, vel0=vel0, S0=S0,
                params=dict(DEFAULT_PARAMS if params is None else params))


def make_ensemble(name: str, L: float = DOMAIN_M, params: dict | None = None):
    """List of member cases (dicts as make_case returns) of a named ensemble."""
    cfg = ENSEMBLES[name]
    rng = np.random.Generator(np.random.PCG64(cfg["seed"]))
    lo, hi = math.log(cfg["side_lo"]), math.log(cfg["side_hi"])
    members = []
    for m in range(cfg["n_members"]):
        side = int(round(math.exp(rng.uniform(lo, hi))))
        n_s = 6 if rng.random() < 0.5 else 3
        s1, s2, sw = (int(x) for x in rng.integers(1, 2 ** 31 - 1, 3))
        ne, nn, _ = sizes(side, side)
        H, A = ice_grf(side, side, (s1, s2), L)
        tau = cyclone_wind_stress(node_coords_uniform(side, side, L, L), cyclone_params(sw, L))
        members.append(dict(name=f"{name}[{m}]", nx=side, ny=side, n_s=n_s, n_a=1,
                            n_sub=cfg["n_sub"], L=L, xy=uniform_vertices(side, side, L, L),
                            H=H, A=A, tau=tau, vel0=np.zeros((2, nn)),
                            S0=np.zeros((3, n_s, ne)),
                            params=dict(DEFAULT_PARAMS if params is None else params)))
    return members


def perturbed_vertices(nx: int, ny: int, seed: int, amp: float = 0.2, L: float = DOMAIN_M):
    """Vertices (N_v, 2) of a non-affine quad mesh: the interior vertices of a
    uniform mesh moved by U[-amp h, amp h] in each coordinate (PCG64(seed)).
    amp < 0.25 keeps every element convex."""
    xy = uniform_vertices(nx, ny, L, L).reshape(ny + 1, nx + 1, 2)
    rng = np.random.Generator(np.random.PCG64(seed))
    hx, hy = L / nx, L / ny
    inner = xy[1:-1, 1:-1]
    inner[..., 0] += rng.uniform(-amp * hx, amp * hx, inner.shape[:2])
    inner[..., 1] += rng.uniform(-amp * hy, amp * hy, inner.shape[:2])
    return xy.reshape(-1, 2).copy()


def wavy_vertices(nx: int, ny: int, amp: float = 0.3, L: float = DOMAIN_M):
    """Vertices (N_v, 2) of a smoothly curvilinear mesh: the uniform mesh under
    x' = x + a h sin(2 pi y/L) sin(pi x/L), y' = y + a h sin(2 pi x/L) sin(pi y/L)
    (boundary fixed; a = amp, h the element size)."""
    xy = uniform_vertices(nx, ny, L, L)
    x, y = xy[:, 0] / L, xy[:, 1] / L
    h = L / max(nx, ny)
    out = xy.copy()
    out[:, 0] += amp * h * np.sin(2 * math.pi * y) * np.sin(math.pi * x)
    out[:, 1] += amp * h * np.sin(2 * math.pi * x) * np.sin(math.pi * y)
    return out


def node_coords(nx: int, ny: int, xy):
    """Coordinates (2, N_n) of the CG2 nodes of a mesh with vertices xy: images
    of the reference nodes under each element's bilinear map (vertex nodes,
    edge midpoints, element centres)."""
    v = np.asarray(xy, dtype=np.float64).reshape(ny + 1, nx + 1, 2)
    out = np.zeros((2 * ny + 1, 2 * nx + 1, 2))
    out[0::2, 0::2] = v
    out[0::2, 1::2] = 0.5 * (v[:, :-1] + v[:, 1:])
    out[1::2, 0::2] = 0.5 * (v[:-1, :] + v[1:, :])
    out[1::2, 1::2] = 0.25 * (v[:-1, :-1] + v[:-1, 1:] + v[1:, :-1] + v[1:, 1:])
    return out.reshape(-1, 2).T.copy()


def wavy_nodes(nx: int, ny: int, amp: float = 0.3, L: float = DOMAIN_M):
    """CG2 node positions (N_n, 2) of a curved mesh: the smooth map of
    wavy_vertices evaluated at every CG2 node of the uniform mesh, so that
    the isoparametric (Q2) elements follow the curved map."""
    nc = node_coords_uniform(nx, ny, L, L)
    x, y = nc[0] / L, nc[1] / L
    h = L / max(nx, ny)
    out = nc.T.copy()
    out[:, 0] += amp * h * np.sin(2 * math.pi * y) * np.sin(math.pi * x)
    out[:, 1] += amp * h * np.sin(2 * math.pi * x) * np.sin(math.pi * y)
    return out


def curved_nodes(nx: int, ny: int, seed: int, amp: float = 0.05, vamp: float = 0.1,
                 L: float = DOMAIN_M):
    """CG2 node positions (N_n, 2) of a randomly curved mesh: the nodes of a
    perturbed-vertex mesh (vertices moved by U[-vamp h, vamp h]), with every
    edge-midpoint and element-centre node moved by U[-amp h, amp h] per
    coordinate (PCG64(seed)); boundary nodes stay on the boundary.

    At a corner the Q2 map's edge derivative is the edge vector plus 4 times
    the midpoint's offset from the chord, and the centre node does not enter,
    so det J there is at least h^2 (1 - 4 vamp - 8 amp) / 4 in the unit
    square's coordinates: positive for the defaults, on any mesh size."""
    xy = perturbed_vertices(nx, ny, seed, amp=vamp, L=L)
    nodes = node_coords(nx, ny, xy).T.reshape(2 * ny + 1, 2 * nx + 1, 2).copy()
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    h = L / max(nx, ny)
    d = rng.uniform(-amp * h, amp * h, nodes.shape)
    iy, ix = np.meshgrid(np.arange(2 * ny + 1), np.arange(2 * nx + 1), indexing="ij")
    mid = (ix % 2 == 1) | (iy % 2 == 1)  # not a vertex
    d[~mid] = 0.0
    d[0, :, 1] = d[-1, :, 1] = 0.0  # south / north boundary nodes move along x only
    d[:, 0, 0] = d[:, -1, 0] = 0.0  # west / east boundary nodes move along y only
    d[0, 0] = d[0, -1] = d[-1, 0] = d[-1, -1] = 0.0
    nodes += d
    return nodes.reshape(-1, 2).copy()
