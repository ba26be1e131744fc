"""Thin Python binding of libmevp.so (the C ABI in include/mevp.h).

Argument marshalling only: every step of the mEVP subcycle runs in the CUDA
kernels behind the C ABI.  Functions carry the C names; ``State`` bundles a
mesh, a state and its device workspace (a torch uint8 tensor, so device
memory comes from torch's caching allocator) on torch's current stream.

There is no CPU fallback: if the library cannot be built or loaded, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MEVP_FP64, MEVP_MIXED = 0, 1
FIELDS = dict(U=0, V=1, S11=2, S12=3, S22=4, E11=5, E12=6, E22=7, FORCE_X=8, FORCE_Y=9, H=10,
              A=11, NODAL_MASS=12)
ERRORS = {-1: "MEVP_ERR_ARG", -2: "MEVP_ERR_CUDA", -3: "MEVP_ERR_OOM", -4: "MEVP_ERR_STATE",
          -5: "MEVP_ERR_NAN", -6: "MEVP_ERR_TIMEOUT", -7: "MEVP_ERR_UNSUPPORTED",
          -8: "MEVP_ERR_BOUNDS"}
PARAM_NAMES = ("Pstar", "C", "e", "DeltaMin", "alpha", "beta", "dt", "rho_ice", "rho_water",
               "Cw", "coriolis_f")


class MevpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class mevp_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in PARAM_NAMES]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libmevp.so (building it with nvcc first if missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # MEVP_LIBRARY: load another build of the same sources (the
        # bounds-checked build of the tests) instead of the in-tree library
        override = os.environ.get("MEVP_LIBRARY")
        path = override if override else (_build.build() if build_if_stale else _build.LIB)
        if not os.path.exists(path):
            raise ImportError(f"libmevp.so not found at {path}; run paper_2402_00466_gb300.build")
        lib = ctypes.CDLL(path)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        pvp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "mevp_mesh_create": (i, [i, i, d, d, vp, pvp]),
            "mevp_mesh_destroy": (None, [vp]),
            "mevp_mesh_create_nodes": (i, [i, i, vp, pvp]),
            "mevp_state_workspace_bytes": (i, [vp, i, i, i, ctypes.POINTER(sz)]),
            "mevp_state_create": (i, [vp, i, i, i, vp, vp, sz, pvp]),
            "mevp_state_destroy": (None, [vp]),
            "mevp_set_params": (i, [vp, ctypes.POINTER(mevp_params)]),
            "mevp_set_ice": (i, [vp, vp, vp, i]),
            "mevp_set_forcing": (i, [vp, vp, vp, i]),
            "mevp_set_velocity": (i, [vp, vp, i]),
            "mevp_set_stress": (i, [vp, vp, i]),
            "mevp_begin_step": (i, [vp]),
            "mevp_advect": (i, [vp, i]),
            "mevp_run_subcycles": (i, [vp, i]),
            "mevp_read_field": (i, [vp, i, vp, sz, i]),
            "mevp_sync": (i, [vp]),
            "mevp_run_subcycles_noalloc": (i, [i, i, i, ctypes.POINTER(mevp_params), vp, vp, vp,
                                               vp, vp, vp, vp, vp, i, vp]),
            "mevp_timing_enable": (i, [vp, i]),
            "mevp_set_option": (i, [vp, i, i]),
            "mevp_timing_read": (i, [vp, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_longlong)]),
            "mevp_set_strength_field": (i, [vp, vp, i]),
            "mevp_adjoint_kinetic_energy": (i, [vp, i, i, vp, vp, vp, i]),
            "mevp_ensemble_create": (i, [ctypes.POINTER(vp), i, pvp]),
            "mevp_ensemble_destroy": (None, [vp]),
            "mevp_ensemble_begin_step": (i, [vp]),
            "mevp_ensemble_run_subcycles": (i, [vp, i]),
            "mevp_ensemble_shapes": (i, [i, ctypes.POINTER(i), i, ctypes.POINTER(i)]),
            "mevp_ensemble_set_shape": (i, [vp, i]),
            "mevp_ensemble_autotune": (i, [vp, i, ctypes.POINTER(i)]),
            "mevp_ensemble_set_graphs": (i, [vp, i]),
            "mevp_last_error": (ctypes.c_char_p, []),
            "mevp_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _ = dp
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise MevpError(rc, mevp_last_error())


def mevp_last_error() -> str:
    return load().mevp_last_error().decode()


def mevp_version() -> str:
    return load().mevp_version().decode()


def _ptr(a):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor of float64."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != torch.float64:
            raise TypeError("expected a float64 tensor")
        a = a.contiguous()
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def mevp_mesh_create(nx: int, ny: int, Lx: float = 0.0, Ly: float = 0.0, vertex_xy=None):
    out = ctypes.c_void_p()
    xy = None if vertex_xy is None else np.ascontiguousarray(vertex_xy, dtype=np.float64)
    _check(load().mevp_mesh_create(int(nx), int(ny), float(Lx), float(Ly),
                                   None if xy is None else ctypes.c_void_p(xy.ctypes.data),
                                   ctypes.byref(out)))
    return out


def mevp_mesh_create_nodes(nx: int, ny: int, node_xy):
    """Isoparametric mesh from the CG2 node positions [(2nx+1)(2ny+1)][2]."""
    out = ctypes.c_void_p()
    xy = np.ascontiguousarray(node_xy, dtype=np.float64)
    _check(load().mevp_mesh_create_nodes(int(nx), int(ny), ctypes.c_void_p(xy.ctypes.data),
                                         ctypes.byref(out)))
    return out


def mevp_mesh_destroy(mesh):
    load().mevp_mesh_destroy(mesh)


def mevp_state_workspace_bytes(mesh, n_stress: int, n_adv: int, precision: int) -> int:
    b = ctypes.c_size_t()
    _check(load().mevp_state_workspace_bytes(mesh, n_stress, n_adv, precision, ctypes.byref(b)))
    return b.value


def mevp_state_create(mesh, n_stress, n_adv, precision, stream, workspace, workspace_bytes):
    out = ctypes.c_void_p()
    _check(load().mevp_state_create(mesh, n_stress, n_adv, precision, ctypes.c_void_p(stream),
                                    ctypes.c_void_p(workspace), workspace_bytes,
                                    ctypes.byref(out)))
    return out


def mevp_state_destroy(state):
    load().mevp_state_destroy(state)


def mevp_set_params(state, params: dict):
    p = mevp_params(**{k: float(params[k]) for k in PARAM_NAMES})
    _check(load().mevp_set_params(state, ctypes.byref(p)))


def mevp_set_ice(state, H, A):
    ph, dh, kh = _ptr(H)
    pa, da, ka = _ptr(A)
    if dh != da:
        raise ValueError("H and A must both be host or both device data")
    _check(load().mevp_set_ice(state, ph, pa, dh))


def mevp_set_forcing(state, tau, v_ocean=None):
    pt, dt, kt = _ptr(tau)
    po, do, ko = _ptr(v_ocean)
    if v_ocean is not None and do != dt:
        raise ValueError("tau and v_ocean must both be host or both device data")
    _check(load().mevp_set_forcing(state, pt, po, dt))


def mevp_set_velocity(state, uv):
    p, dev, k = _ptr(uv)
    _check(load().mevp_set_velocity(state, p, dev))


def mevp_set_stress(state, S):
    p, dev, k = _ptr(S)
    _check(load().mevp_set_stress(state, p, dev))


def mevp_set_strength_field(state, Pstar):
    """Per-element P* field [N_e] (numpy or torch float64), or None for params.Pstar."""
    p, dev, k = _ptr(Pstar)
    _check(load().mevp_set_strength_field(state, p, dev))


def mevp_adjoint_kinetic_energy(state, n, checkpoint_every, J, dJ_dPstar, dJ_dtau, on_device):
    """Thin call: pointers (or None) for J, dJ/dP* [N_e], dJ/dtau [2][N_n]."""
    vp = lambda x: None if x is None else ctypes.c_void_p(x)  # noqa: E731
    _check(load().mevp_adjoint_kinetic_energy(state, int(n), int(checkpoint_every), vp(J),
                                              vp(dJ_dPstar), vp(dJ_dtau), int(on_device)))


def mevp_begin_step(state):
    _check(load().mevp_begin_step(state))


def mevp_advect(state, n_steps: int = 1):
    _check(load().mevp_advect(state, int(n_steps)))


def mevp_run_subcycles(state, n: int):
    _check(load().mevp_run_subcycles(state, int(n)))


def mevp_read_field(state, field, out):
    """Copy field (name or enum) into ``out`` (numpy float64 or torch float64)."""
    f = FIELDS[field] if isinstance(field, str) else int(field)
    if hasattr(out, "data_ptr"):
        if not out.is_contiguous():
            raise ValueError("out must be contiguous")
        _check(load().mevp_read_field(state, f, ctypes.c_void_p(out.data_ptr()), out.numel(),
                                      int(out.is_cuda)))
    else:
        if out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array")
        _check(load().mevp_read_field(state, f, ctypes.c_void_p(out.ctypes.data), out.size, 0))
    return out


def mevp_sync(state):
    _check(load().mevp_sync(state))


def mevp_run_subcycles_noalloc(nx, ny, n_stress, params, xline, yline, H, A, tau, v_ocean,
                               vel, S, n, stream=None):
    """One outer step of n subcycles on caller-owned CUDA float64 tensors, with
    the library allocating nothing (its scratch is a fixed static device
    array; see include/mevp.h).  vel and S are updated in place."""
    import torch
    nx, ny, n_stress = int(nx), int(ny), int(n_stress)
    if nx < 1 or ny < 1:
        raise ValueError(f"nx={nx}, ny={ny} must be >= 1")
    ne, nn = nx * ny, (2 * nx + 1) * (2 * ny + 1)
    # the C entry point sees raw pointers only: every length is checked here,
    # before anything is launched
    need = dict(xline=nx + 1, yline=ny + 1, H=ne, A=ne, tau=2 * nn, vel=2 * nn,
                S=3 * n_stress * ne, v_ocean=2 * nn)
    arrs = dict(xline=xline, yline=yline, H=H, A=A, tau=tau, vel=vel, S=S)
    if v_ocean is not None:
        arrs["v_ocean"] = v_ocean
    for k, t in arrs.items():
        if t.numel() != need[k]:
            raise ValueError(f"{k} has {t.numel()} elements; a {nx}x{ny} mesh with "
                             f"{n_stress} stress dofs needs {need[k]}")
    for k, t in arrs.items():
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError(f"{k} must be a contiguous CUDA float64 tensor")
    p = mevp_params(**{k: float(params[k]) for k in PARAM_NAMES})
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    _check(load().mevp_run_subcycles_noalloc(
        nx, ny, n_stress, ctypes.byref(p), ptr(xline), ptr(yline), ptr(H), ptr(A),
        ptr(tau), ptr(v_ocean), ptr(vel), ptr(S), int(n), ctypes.c_void_p(stream)))


MEVP_OPT_FUSED = 1
MEVP_OPT_GRAPHS = 2
MEVP_OPT_NAN_CHECK = 3
MEVP_OPT_STALL_TEST = 4


def mevp_set_option(state, option: int, value: int):
    _check(load().mevp_set_option(state, int(option), int(value)))


def mevp_timing_enable(state, stride: int):
    """Event-time every `stride`-th subcycle (0 = off)."""
    _check(load().mevp_timing_enable(state, int(stride)))


def mevp_timing_read(state):
    """{'element': (ms, launches), 'node': (ms, launches)} since the last read."""
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_longlong * 2)()
    _check(load().mevp_timing_read(state, ms, n))
    return {"element": (ms[0], n[0]), "node": (ms[1], n[1])}


class State:
    """A mesh + state + torch-owned device workspace on torch's current stream.

    Host inputs are numpy arrays in the external layouts of include/mevp.h;
    device inputs are CUDA float64 tensors.

    nx, ny: elements per direction; n_stress: 3, 6 or 8 DG stress dofs;
    vertex_xy: None (uniform mesh of side L), the (nx+1)(ny+1) vertices of a
    bilinear mesh, or the (2nx+1)(2ny+1) CG2 node positions of a curved
    (isoparametric) mesh; n_adv: 1, 3 or 6 dofs of H and A; precision:
    "fp64" or "mixed".

    Methods map one to one onto the C ABI: set_params, set_ice(H, A),
    set_forcing(tau, v_ocean=None), set_velocity, set_stress,
    set_strength_field(P*), begin_step() (v^n := v, strength and node
    constants), run_subcycles(n) and advect(n) (asynchronous), sync()
    (waits; reports NaN / bounds / timeout flags), read(field) and the
    velocity() / stress() / strain() / force() shortcuts,
    adjoint_kinetic_energy(n, checkpoint_every), set_option,
    timing_enable / timing_read.
    """

    def __init__(self, nx, ny, n_stress, *, L=None, vertex_xy=None, n_adv=1,
                 precision="fp64", params=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("mevp needs a CUDA device (no CPU fallback)")
        load()
        self.nx, self.ny, self.n_stress, self.n_adv = nx, ny, n_stress, n_adv
        self.ne = nx * ny
        self.nn = (2 * nx + 1) * (2 * ny + 1)
        self.precision = {"fp64": MEVP_FP64, "mixed": MEVP_MIXED}[precision]
        Lx = Ly = float(L if L is not None else 0.0)
        if vertex_xy is not None and np.asarray(vertex_xy).reshape(-1, 2).shape[0] == self.nn:
            # the positions of every CG2 node: an isoparametric (curved) mesh
            self.mesh = mevp_mesh_create_nodes(nx, ny, vertex_xy)
        else:
            self.mesh = mevp_mesh_create(nx, ny, Lx, Ly, vertex_xy)
        self.state = None
        nbytes = mevp_state_workspace_bytes(self.mesh, n_stress, n_adv, self.precision)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.state = mevp_state_create(self.mesh, n_stress, n_adv, self.precision,
                                       self.stream.cuda_stream, aligned, nbytes)
        if params is not None:
            mevp_set_params(self.state, params)

    def close(self):
        if getattr(self, "state", None) is not None:
            mevp_state_destroy(self.state)
            self.state = None
        if getattr(self, "mesh", None) is not None:
            mevp_mesh_destroy(self.mesh)
            self.mesh = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # thin forwards
    def set_params(self, p): mevp_set_params(self.state, p)
    def set_ice(self, H, A): mevp_set_ice(self.state, H, A)
    def set_forcing(self, tau, v_ocean=None): mevp_set_forcing(self.state, tau, v_ocean)
    def set_velocity(self, uv): mevp_set_velocity(self.state, uv)
    def set_stress(self, S): mevp_set_stress(self.state, S)
    def begin_step(self): mevp_begin_step(self.state)
    def advect(self, n_steps=1): mevp_advect(self.state, n_steps)
    def run_subcycles(self, n): mevp_run_subcycles(self.state, n)
    def sync(self): mevp_sync(self.state)
    def set_strength_field(self, Pstar): mevp_set_strength_field(self.state, Pstar)

    def adjoint_kinetic_energy(self, n, checkpoint_every=10, device=False):
        """(J, dJ/dP*, dJ/dtau) of the kinetic energy after n subcycles from the
        current state (FP64 states, after begin_step); numpy, or CUDA tensors
        with device=True."""
        if device:
            import torch
            J = torch.empty((), dtype=torch.float64, device="cuda")
            gP = torch.empty(self.ne, dtype=torch.float64, device="cuda")
            gT = torch.empty((2, self.nn), dtype=torch.float64, device="cuda")
            mevp_adjoint_kinetic_energy(self.state, n, checkpoint_every, J.data_ptr(),
                                        gP.data_ptr(), gT.data_ptr(), 1)
            return J, gP, gT
        J = np.zeros(1)
        gP = np.zeros(self.ne)
        gT = np.zeros((2, self.nn))
        mevp_adjoint_kinetic_energy(self.state, n, checkpoint_every, J.ctypes.data,
                                    gP.ctypes.data, gT.ctypes.data, 0)
        return float(J[0]), gP, gT

    def timing_enable(self, stride=1): mevp_timing_enable(self.state, stride)
    def set_option(self, option, value): mevp_set_option(self.state, option, value)
    def timing_read(self): return mevp_timing_read(self.state)

    def field_shape(self, field):
        f = FIELDS[field] if isinstance(field, str) else int(field)
        if f in (0, 1, 8, 9, 12):
            return (self.nn,)
        if f in (10, 11):
            return (self.n_adv, self.ne)
        return (self.n_stress, self.ne)

    def read(self, field, device=False):
        shape = self.field_shape(field)
        if device:
            import torch
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
        else:
            out = np.empty(shape, dtype=np.float64)
        return mevp_read_field(self.state, field, out)

    def velocity(self):
        return np.stack([self.read("U"), self.read("V")])

    def stress(self):
        return np.stack([self.read("S11"), self.read("S12"), self.read("S22")])

    def strain(self):
        return np.stack([self.read("E11"), self.read("E12"), self.read("E22")])

    def force(self):
        return np.stack([self.read("FORCE_X"), self.read("FORCE_Y")])


def mevp_ensemble_create(states):
    """An ensemble over mevp State objects or raw state handles."""
    handles = [st.state if isinstance(st, State) else st for st in states]
    arr = (ctypes.c_void_p * len(handles))(*[h.value if hasattr(h, "value") else h
                                             for h in handles])
    out = ctypes.c_void_p()
    _check(load().mevp_ensemble_create(arr, len(handles), ctypes.byref(out)))
    return out


def mevp_ensemble_destroy(ens):
    load().mevp_ensemble_destroy(ens)


def mevp_ensemble_begin_step(ens):
    _check(load().mevp_ensemble_begin_step(ens))


def mevp_ensemble_run_subcycles(ens, n):
    _check(load().mevp_ensemble_run_subcycles(ens, int(n)))


def mevp_ensemble_shapes(precision):
    prec = {"fp64": MEVP_FP64, "mixed": MEVP_MIXED}.get(precision, precision)
    dims = (ctypes.c_int * 32)()
    cnt = ctypes.c_int()
    _check(load().mevp_ensemble_shapes(prec, dims, 16, ctypes.byref(cnt)))
    return [(dims[2 * i], dims[2 * i + 1]) for i in range(cnt.value)]


def mevp_ensemble_set_shape(ens, shape):
    _check(load().mevp_ensemble_set_shape(ens, int(shape)))


def mevp_ensemble_autotune(ens, trial_subcycles=20):
    best = ctypes.c_int()
    _check(load().mevp_ensemble_autotune(ens, int(trial_subcycles), ctypes.byref(best)))
    return best.value


def mevp_ensemble_set_graphs(ens, on):
    _check(load().mevp_ensemble_set_graphs(ens, int(bool(on))))


class Ensemble:
    """Several State objects advanced together (see include/mevp.h)."""

    def __init__(self, states):
        self.states = list(states)
        self.handle = mevp_ensemble_create(self.states)

    def begin_step(self): mevp_ensemble_begin_step(self.handle)
    def run_subcycles(self, n): mevp_ensemble_run_subcycles(self.handle, n)
    def set_shape(self, shape): mevp_ensemble_set_shape(self.handle, shape)
    def set_graphs(self, on): mevp_ensemble_set_graphs(self.handle, on)
    def autotune(self, trial_subcycles=20): return mevp_ensemble_autotune(self.handle, trial_subcycles)

    def close(self):
        if getattr(self, "handle", None) is not None:
            mevp_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def kinetic_energy(state, pstar, tau, n, checkpoint_every=10):
    """Differentiable J(P*, tau): the kinetic energy 1/2 sum_j m_j |v_j|^2 after
    n subcycles of an FP64 State from its current velocity and stress, as a
    function of the per-element P* field `pstar` [N_e] and the nodal wind
    stress `tau` [2, N_n] (CUDA float64 tensors).  backward() returns the
    gradients of the library's hand-written adjoint.  The call leaves the
    state after the n subcycles, like State.run_subcycles."""
    import torch

    class _KineticEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, p, t):
            state.set_strength_field(p.detach().contiguous())
            state.set_forcing(t.detach().contiguous())
            state.begin_step()
            J, gP, gT = state.adjoint_kinetic_energy(n, checkpoint_every, device=True)
            ctx.save_for_backward(gP, gT)
            return J

        @staticmethod
        def backward(ctx, gJ):
            gP, gT = ctx.saved_tensors
            return gJ * gP, gJ * gT

    return _KineticEnergy.apply(pstar, tau)
