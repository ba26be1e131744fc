"""Plain FP64 CPU oracle of the mEVP momentum subcycle (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product library
never does.  The C source (``mevp_oracle.c``) restates the paper's method
(Sec. 2, Eqs. 2-3, Listing 1 / App. A, the stage split of Table 1) and shares
no code with the CUDA path.

Array layouts at this Python boundary are the library's external layouts:
  velocity / forces      (2, N_n)          node = iy*(2nx+1) + ix
  stress / strain        (3, n_s, N_e)     component order 11, 12, 22
  H, A                   (n_a, N_e)
  vertices               (N_v, 2)          vertex = jy*(nx+1) + jx
The C code stores DG fields element-major ((3, N_e, n_s), the paper's
row-major N x n_S matrices); this wrapper transposes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mevp_oracle.c")
_LIBS = {False: os.path.join(_HERE, "_build", "libmevp_oracle.so"),
         True: os.path.join(_HERE, "_build", "libmevp_oracle_omp.so")}
_lock = threading.Lock()
_handles: dict = {}


class Params(ctypes.Structure):
    """Physical and mEVP parameters (field order of the C struct)."""
    _fields_ = [(n, ctypes.c_double) for n in (
        "Pstar", "C", "e", "DeltaMin", "alpha", "beta", "dt",
        "rho_ice", "rho_water", "Cw", "coriolis_f")]

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        return cls(**{k: float(d[k]) for k, _ in cls._fields_})


def build(openmp: bool = False, force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off); returns the .so path."""
    out = _LIBS[openmp]
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-D_POSIX_C_SOURCE=199309L", "-o", tmp, _SRC, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(openmp: bool = False):
    with _lock:
        if openmp not in _handles:
            # MEVP_ORACLE_LIB: load another build of this source (the mutation
            # tests plant a mistake in a copy and check that the pins fail)
            override = os.environ.get("MEVP_ORACLE_LIB")
            lib = ctypes.CDLL(override if override else build(openmp))
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(Params)
            i = ctypes.c_int
            lib.orc_gauss.argtypes = [i, dp, dp]
            lib.orc_ngp.argtypes = [i]
            lib.orc_dg_basis.argtypes = [i, ctypes.c_double, ctypes.c_double, dp]
            lib.orc_q2_basis.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, dp]
            lib.orc_subcycles.argtypes = [i, i, dp, i, i, i, pp, dp, dp, dp, dp, dp, dp, dp, i,
                                          dp, dp, dp, dp, dp]
            lib.orc_strain.argtypes = [i, i, dp, i, i, dp, dp]
            lib.orc_stress.argtypes = [i, i, dp, i, i, i, pp, dp, dp, dp, dp, dp]
            lib.orc_divergence.argtypes = [i, i, dp, i, i, dp, dp, dp]
            lib.orc_delta.argtypes = [i, i, i, pp, dp, dp]
            lib.orc_lumped.argtypes = [i, i, dp, i, i, i, pp, dp, dp, dp]
            lib.orc_velocity.argtypes = [i, i, pp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_element_map.argtypes = [i, i, dp, i, i, i, dp, dp]
            lib.orc_max_threads.argtypes = []
            lib.orc_advect.argtypes = [i, i, dp, i, i, dp, ctypes.c_double, i, dp, dp]
            lib.orc_advect_operator.argtypes = [i, i, dp, i, i, dp, dp, dp, dp, dp]
            _handles[openmp] = lib
        return _handles[openmp]


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def sizes(nx, ny):
    return nx * ny, (2 * nx + 1) * (2 * ny + 1)


def _geo(nx, ny, xy):
    """(array, mode) of a mesh's geometry: vertices [(nx+1)(ny+1)][2] give
    bilinear element maps (mode 0), CG2 node positions [(2nx+1)(2ny+1)][2]
    give isoparametric Q2 element maps (mode 1)."""
    a = _c(xy).reshape(-1, 2)
    if a.shape[0] == (nx + 1) * (ny + 1):
        return a, 0
    if a.shape[0] == (2 * nx + 1) * (2 * ny + 1):
        return a, 1
    raise ValueError(f"geometry of {a.shape[0]} points fits neither the vertices nor the nodes")


def uniform_vertices(nx, ny, Lx, Ly):
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    X, Y = np.meshgrid(xs, ys)  # (ny+1, nx+1)
    return np.stack([X.ravel(), Y.ravel()], axis=1).copy()


def gauss(n):
    x = np.zeros(n); w = np.zeros(n)
    _check(_lib().orc_gauss(n, _p(x), _p(w)), "gauss")
    return x, w


def ngp(n_s):
    return _lib().orc_ngp(n_s)


def dg_basis(n, xi, eta):
    phi = np.zeros(n)
    _check(_lib().orc_dg_basis(n, xi, eta, _p(phi)), "dg_basis")
    return phi


def q2_basis(xi, eta):
    phi = np.zeros(9); dx = np.zeros(9); de = np.zeros(9)
    _lib().orc_q2_basis(xi, eta, _p(phi), _p(dx), _p(de))
    return phi, dx, de


def _dg_in(S, n_s, ne):
    """(3, n_s, N_e) -> C layout (3, N_e, n_s)."""
    return _c(np.asarray(S, dtype=np.float64).reshape(3, n_s, ne).transpose(0, 2, 1))


def _dg_out(Sc, n_s, ne):
    return np.ascontiguousarray(Sc.reshape(3, ne, n_s).transpose(0, 2, 1))


def _adv_in(H, n_a, ne):
    """(n_a, N_e) -> C layout (N_e, n_a)."""
    return _c(np.asarray(H, dtype=np.float64).reshape(n_a, ne).T)


def element_map(nx, ny, xy, n_s, K):
    ng = ngp(n_s) ** 2
    det = np.zeros(ng); m = np.zeros(n_s * ng)
    g, mode = _geo(nx, ny, xy)
    _check(_lib().orc_element_map(nx, ny, _p(g), mode, n_s, K, _p(det), _p(m)), "element_map")
    return det, m.reshape(n_s, ng)


def strain(nx, ny, xy, n_s, vel, openmp=False):
    ne, nn = sizes(nx, ny)
    E = np.zeros(3 * ne * n_s)
    g, mode = _geo(nx, ny, xy)
    _check(_lib(openmp).orc_strain(nx, ny, _p(g), mode, n_s, _p(_c(vel).reshape(-1)), _p(E)),
           "strain")
    return _dg_out(E, n_s, ne)


def _pstar_k(Pstar_K, ne):
    """Optional per-element P* field [N_e] (None: params['Pstar'] everywhere)."""
    if Pstar_K is None:
        return None
    a = _c(Pstar_K).reshape(-1)
    if a.shape[0] != ne:
        raise ValueError(f"Pstar_K has {a.shape[0]} entries, the mesh {ne} elements")
    return a


def stress(nx, ny, xy, n_s, n_a, params, E, H, A, S, Pstar_K=None):
    ne, nn = sizes(nx, ny)
    Sc = _dg_in(S, n_s, ne)
    prm = Params.from_dict(params)
    g, mode = _geo(nx, ny, xy)
    pk = _pstar_k(Pstar_K, ne)
    _check(_lib().orc_stress(nx, ny, _p(g), mode, n_s, n_a, ctypes.byref(prm),
                             _p(_dg_in(E, n_s, ne)), _p(_adv_in(H, n_a, ne)),
                             _p(_adv_in(A, n_a, ne)), _p(Sc), _p(pk)), "stress")
    return _dg_out(Sc, n_s, ne)


def delta(nx, ny, n_s, params, E):
    """Delta of the rheology at every Gauss point, (N_e, n_g), of the strain
    E (3, n_s, N_e)."""
    ne, nn = sizes(nx, ny)
    ng = ngp(n_s) ** 2
    out = np.zeros(ne * ng)
    prm = Params.from_dict(params)
    _check(_lib().orc_delta(nx, ny, n_s, ctypes.byref(prm), _p(_dg_in(E, n_s, ne)), _p(out)),
           "delta")
    return out.reshape(ne, ng)


def divergence(nx, ny, xy, n_s, S, return_element_forces=False, openmp=False):
    ne, nn = sizes(nx, ny)
    F = np.zeros(2 * nn)
    fel = np.zeros(18 * ne)
    g, mode = _geo(nx, ny, xy)
    _check(_lib(openmp).orc_divergence(nx, ny, _p(g), mode, n_s, _p(_dg_in(S, n_s, ne)), _p(F),
                                       _p(fel)), "divergence")
    if return_element_forces:
        return F.reshape(2, nn), fel.reshape(ne, 18)
    return F.reshape(2, nn)


def lumped(nx, ny, xy, n_s, n_a, params, H):
    ne, nn = sizes(nx, ny)
    m = np.zeros(nn); l = np.zeros(nn)
    prm = Params.from_dict(params)
    g, mode = _geo(nx, ny, xy)
    _check(_lib().orc_lumped(nx, ny, _p(g), mode, n_s, n_a, ctypes.byref(prm),
                             _p(_adv_in(H, n_a, ne)), _p(m), _p(l)), "lumped")
    return m, l


def velocity(nx, ny, params, F, vprev, vn, tau, vo, m, l):
    ne, nn = sizes(nx, ny)
    out = np.full(2 * nn, np.nan)  # every entry must be written by the stage
    prm = Params.from_dict(params)
    _check(_lib().orc_velocity(nx, ny, ctypes.byref(prm), _p(_c(F).reshape(-1)),
                               _p(_c(vprev).reshape(-1)), _p(_c(vn).reshape(-1)),
                               _p(_c(tau).reshape(-1)),
                               None if vo is None else _p(_c(vo).reshape(-1)),
                               _p(_c(m)), _p(_c(l)), _p(out)), "velocity")
    return out.reshape(2, nn)


def subcycles(nx, ny, xy, n_s, n_a, params, H, A, tau, vel0, S0, n_sub, vn=None, vo=None,
              want_last=False, openmp=False, phase_sec=None, Pstar_K=None):
    """Run n_sub mEVP subcycles; returns (vel, S) [+ (E_last, F_last, fel_last)].

    vn defaults to vel0 (start of an outer step); Pstar_K [N_e] is an optional
    per-element ice strength parameter in place of params['Pstar']."""
    ne, nn = sizes(nx, ny)
    vel = _c(vel0).reshape(-1).copy()
    vn_ = _c(vel0 if vn is None else vn).reshape(-1).copy()
    Sc = _dg_in(S0, n_s, ne)
    prm = Params.from_dict(params)
    E = np.zeros(3 * ne * n_s) if want_last else None
    F = np.zeros(2 * nn) if want_last else None
    fel = np.zeros(18 * ne) if want_last else None
    ph = np.zeros(4)
    g, mode = _geo(nx, ny, xy)
    pk = _pstar_k(Pstar_K, ne)
    rc = _lib(openmp).orc_subcycles(
        nx, ny, _p(g), mode, n_s, n_a, ctypes.byref(prm), _p(_adv_in(H, n_a, ne)),
        _p(_adv_in(A, n_a, ne)), _p(_c(tau).reshape(-1)),
        None if vo is None else _p(_c(vo).reshape(-1)), _p(vn_), _p(vel), _p(Sc), int(n_sub),
        _p(E), _p(F), _p(fel), _p(ph), _p(pk))
    _check(rc, "subcycles")
    if phase_sec is not None:
        phase_sec[:] = ph
    out = (vel.reshape(2, nn), _dg_out(Sc, n_s, ne))
    if want_last:
        out = out + (_dg_out(E, n_s, ne), F.reshape(2, nn), fel.reshape(ne, 18))
    return out


def max_threads(openmp=True):
    return _lib(openmp).orc_max_threads()


def advect(nx, ny, xy, n_a, vel, dt, n_steps, H, A, openmp=False):
    """n_steps DG upwind advection steps of H and A (n_a, N_e) with the CG2
    velocity vel (2, N_n) held fixed; returns (H, A)."""
    ne, nn = sizes(nx, ny)
    Hc, Ac = _adv_in(H, n_a, ne).copy(), _adv_in(A, n_a, ne).copy()
    g, mode = _geo(nx, ny, xy)
    _check(_lib(openmp).orc_advect(nx, ny, _p(g), mode, n_a, _p(_c(vel).reshape(-1)), float(dt),
                                   int(n_steps), _p(Hc), _p(Ac)), "advect")
    return np.ascontiguousarray(Hc.T), np.ascontiguousarray(Ac.T)


def advect_operator(nx, ny, xy, n_a, vel, H, A):
    """The semi-discrete operator L = M^-1 R applied to (H, A); (n_a, N_e) each."""
    ne, nn = sizes(nx, ny)
    LH = np.zeros(ne * n_a); LA = np.zeros(ne * n_a)
    g, mode = _geo(nx, ny, xy)
    _check(_lib().orc_advect_operator(nx, ny, _p(g), mode, n_a, _p(_c(vel).reshape(-1)),
                                      _p(_adv_in(H, n_a, ne)), _p(_adv_in(A, n_a, ne)),
                                      _p(LH), _p(LA)), "advect_operator")
    return (np.ascontiguousarray(LH.reshape(ne, n_a).T),
            np.ascontiguousarray(LA.reshape(ne, n_a).T))
