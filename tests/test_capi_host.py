"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/mevp.h declares, and its host-only calls validate arguments."""
import os
import re

import numpy as np
import pytest

from paper_2402_00466_gb300 import mevp
from paper_2402_00466_gb300 import workloads as W
from paper_2402_00466_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "mevp.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"MEVP_API\s+[\w\s\*]*?\b(mevp_\w+)\s*\(", src)))


def test_header_declares_expected_api():
    names = declared_symbols()
    for n in ("mevp_mesh_create", "mevp_state_create", "mevp_set_params", "mevp_set_ice",
              "mevp_set_forcing", "mevp_set_velocity", "mevp_set_stress", "mevp_begin_step",
              "mevp_run_subcycles", "mevp_read_field", "mevp_sync", "mevp_last_error",
              "mevp_state_destroy", "mevp_mesh_destroy", "mevp_state_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = mevp.load()
    for n in declared_symbols():
        assert hasattr(lib, n), n
    # and the exported dynamic symbol table has no stray mevp_ entries
    out = os.popen(f"nm -D --defined-only {B.LIB}").read()
    exported = sorted(set(re.findall(r" T (mevp_\w+)", out)))
    assert exported == declared_symbols()


def test_version_string():
    assert "sm_103a" in mevp.mevp_version()


def test_mesh_create_validation():
    with pytest.raises(mevp.MevpError) as e:
        mevp.mevp_mesh_create(0, 4, 1.0, 1.0)
    assert e.value.code == -1 and "nx" in str(e.value)
    with pytest.raises(mevp.MevpError):
        mevp.mevp_mesh_create(4, 4, -1.0, 1.0)
    xy = np.zeros((9, 2))
    for j in range(3):
        for i in range(3):
            xy[j * 3 + i] = (i * 1.0, j * 1.0)
    m = mevp.mevp_mesh_create(2, 2, 0, 0, xy)  # rectilinear
    mevp.mevp_mesh_destroy(m)
    # a general (non-rectilinear) mesh of convex counter-clockwise quads
    g = xy.copy()
    g[4] += (0.2, -0.1)
    m = mevp.mevp_mesh_create(2, 2, 0, 0, g)
    mevp.mevp_mesh_destroy(m)
    # the centre vertex moved past a corner diagonal: a non-convex element
    bad = xy.copy()
    bad[4] = (1.9, 1.9)
    with pytest.raises(mevp.MevpError) as e:
        mevp.mevp_mesh_create(2, 2, 0, 0, bad)
    assert e.value.code == -1 and "convex" in str(e.value)
    # clockwise vertex order (mirrored mesh) is rejected too
    mir = xy.copy()
    mir[:, 0] *= -1.0
    with pytest.raises(mevp.MevpError) as e:
        mevp.mevp_mesh_create(2, 2, 0, 0, mir)
    assert e.value.code == -1
    nan = g.copy()
    nan[3, 1] = np.nan
    with pytest.raises(mevp.MevpError):
        mevp.mevp_mesh_create(2, 2, 0, 0, nan)
    mevp.mevp_mesh_destroy(None)  # destroying NULL is a no-op


def test_workspace_bytes_validation():
    m = mevp.mevp_mesh_create(8, 4, 1e3, 1e3)
    try:
        b3 = mevp.mevp_state_workspace_bytes(m, 3, 1, 0)
        b6 = mevp.mevp_state_workspace_bytes(m, 6, 1, 0)
        b8 = mevp.mevp_state_workspace_bytes(m, 8, 1, 0)
        assert b8 > b6 > b3 > 0 and b6 % 256 == 0
        assert mevp.mevp_state_workspace_bytes(m, 8, 1, 1) > b8  # mixed adds FP32 copies
        for bad in (1, 2, 4, 7):
            with pytest.raises(mevp.MevpError):
                mevp.mevp_state_workspace_bytes(m, bad, 1, 0)
        # DG1/DG2 ice fields: the workspace holds the per-Gauss-point
        # strength (and its FP32 copy in the mixed path) and the advection
        # stage buffers
        assert mevp.mevp_state_workspace_bytes(m, 6, 3, 0) > b6
        assert mevp.mevp_state_workspace_bytes(m, 6, 6, 0) > mevp.mevp_state_workspace_bytes(m, 6, 3, 0)
        assert (mevp.mevp_state_workspace_bytes(m, 6, 3, 1)
                > mevp.mevp_state_workspace_bytes(m, 6, 1, 1))
        for bad in (0, 2, 4):
            with pytest.raises(mevp.MevpError) as e:
                mevp.mevp_state_workspace_bytes(m, 6, bad, 0)
            assert e.value.code == -1
        with pytest.raises(mevp.MevpError):
            mevp.mevp_state_workspace_bytes(m, 6, 1, 5)
    finally:
        mevp.mevp_mesh_destroy(m)


def test_general_mesh_workspace():
    """A general mesh keeps its vertices on the device (more workspace than the
    rectilinear mesh of the same size); its mixed state adds FP32 map records."""
    xy = W.perturbed_vertices(6, 5, 3)
    g = mevp.mevp_mesh_create(6, 5, 0, 0, xy)
    r = mevp.mevp_mesh_create(6, 5, 1e3, 1e3)
    try:
        assert (mevp.mevp_state_workspace_bytes(g, 6, 1, 0)
                > mevp.mevp_state_workspace_bytes(r, 6, 1, 0))
        assert (mevp.mevp_state_workspace_bytes(g, 6, 1, 1)
                > mevp.mevp_state_workspace_bytes(r, 6, 1, 1))
    finally:
        mevp.mevp_mesh_destroy(g)
        mevp.mevp_mesh_destroy(r)


def test_geometry_record_workspace():
    """The stored geometry records: an FP64 general state holds the L D L^T
    factor of every M_K (n_s (n_s + 1) / 2 doubles per element) on top of its
    vertices, a curved one also the Jacobians at the Gauss points (4 NGP^2
    doubles); the mixed states hold the FP32 factor (n_s (n_s + 1) / 2 floats)
    beside their FP32 geometry records.  Each region is 256-byte aligned, so
    the differences are bounded from below by the record sizes."""
    nx, ny = 40, 30
    ne, nn, nv = W.sizes(nx, ny)
    g = mevp.mevp_mesh_create(nx, ny, 0, 0, W.perturbed_vertices(nx, ny, 3))
    r = mevp.mevp_mesh_create(nx, ny, 1e3, 1e3)
    c = mevp.mevp_mesh_create_nodes(nx, ny, W.curved_nodes(nx, ny, 5, L=3e3))
    try:
        for ns in (3, 6, 8):
            ngp2 = 4 if ns == 3 else 9
            w = ns * (ns + 1) // 2
            rect64 = mevp.mevp_state_workspace_bytes(r, ns, 1, 0)
            rect32 = mevp.mevp_state_workspace_bytes(r, ns, 1, 1)
            assert mevp.mevp_state_workspace_bytes(g, ns, 1, 0) >= rect64 + 8 * (2 * nv + w * ne)
            assert mevp.mevp_state_workspace_bytes(c, ns, 1, 0) >= (
                rect64 + 8 * (2 * nn + w * ne + 4 * ngp2 * ne))
            assert mevp.mevp_state_workspace_bytes(g, ns, 1, 1) >= rect32 + 4 * (6 + w) * ne
            assert mevp.mevp_state_workspace_bytes(c, ns, 1, 1) >= rect32 + 4 * (16 + w) * ne
    finally:
        for m in (g, r, c):
            mevp.mevp_mesh_destroy(m)


def test_isoparametric_mesh_validation():
    """mesh_create_nodes: the CG2 node positions of curved elements; an
    element whose map folds (det J <= 0 somewhere) is rejected; the mixed
    workspace adds the FP32 node-offset records (4 float4 per element)."""
    nx, ny = 3, 2
    nodes = W.curved_nodes(nx, ny, 5, amp=0.08, L=3e3)
    m = mevp.mevp_mesh_create_nodes(nx, ny, nodes)
    try:
        assert mevp.mevp_state_workspace_bytes(m, 6, 1, 0) > 0
        mixed = mevp.mevp_state_workspace_bytes(m, 6, 1, 1)
        r = mevp.mevp_mesh_create(nx, ny, 3e3, 3e3)
        try:
            assert mixed >= mevp.mevp_state_workspace_bytes(r, 6, 1, 1) + 64 * nx * ny
        finally:
            mevp.mevp_mesh_destroy(r)
    finally:
        mevp.mevp_mesh_destroy(m)
    bad = nodes.copy()
    nw = 2 * nx + 1
    bad[1 * nw + 1] = bad[2 * nw + 2] + (400.0, 300.0)  # centre of element 0 pulled past a corner
    with pytest.raises(mevp.MevpError) as e:
        mevp.mevp_mesh_create_nodes(nx, ny, bad)
    assert e.value.code == -1 and "det J" in str(e.value)
    nan = nodes.copy()
    nan[4, 0] = np.nan
    with pytest.raises(mevp.MevpError):
        mevp.mevp_mesh_create_nodes(nx, ny, nan)


def test_null_state_calls_fail_cleanly():
    lib = mevp.load()
    assert lib.mevp_run_subcycles(None, 1) == -1
    assert "NULL" in mevp.mevp_last_error()
    assert lib.mevp_begin_step(None) == -1
    lib.mevp_state_destroy(None)


def test_oracle_is_not_linked_into_the_library():
    out = os.popen(f"nm -D {B.LIB}").read()
    assert "orc_" not in out
    src_dir = os.path.join(os.path.dirname(B.LIB), "..", "csrc")
    for f in os.listdir(src_dir):
        assert "oracle" not in open(os.path.join(src_dir, f)).read().lower() or f.endswith(".md")


def test_noalloc_binding_checks_every_length_before_launching():
    """The no-alloc entry point takes raw device pointers, so the binding
    checks each tensor's length against the mesh first (on the CPU, before
    any device check or launch)."""
    import torch
    from paper_2402_00466_gb300 import mevp
    from paper_2402_00466_gb300 import workloads as W
    nx, ny, ns = 4, 3, 6
    ne, nn, _ = W.sizes(nx, ny)
    z = lambda *s: torch.zeros(*s, dtype=torch.float64)  # noqa: E731
    good = dict(xline=z(nx + 1), yline=z(ny + 1), H=z(ne), A=z(ne), tau=z(2, nn), v_ocean=None,
                vel=z(2, nn), S=z(3, ns, ne))
    wrong = dict(xline=z(nx), yline=z(ny + 2), H=z(ne - 1), A=z(ne + 1), tau=z(2, nn - 1),
                 v_ocean=z(nn), vel=z(2 * nn + 1), S=z(3, 3, ne))
    for k, bad in wrong.items():
        args = dict(good, **{k: bad})
        with pytest.raises(ValueError, match=k):
            mevp.mevp_run_subcycles_noalloc(nx, ny, ns, W.DEFAULT_PARAMS, n=1, **args)
