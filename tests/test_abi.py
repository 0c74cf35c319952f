"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/lq.h; the binding registers all of them.  No compute call (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ["lq_create", "lq_destroy", "lq_upload_gauge", "lq_reserve", "lq_apply_H", "lq_set_direction",
                 "lq_apply_block", "lq_sign_apply", "lq_sign_derivative_apply", "lq_newton_sign"]:
        assert need in syms


@pytest.fixture(scope="module")
def built_lib():
    from paper_1611_00195_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    return path


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_registers_every_declared_symbol(built_lib):
    from paper_1611_00195_gb300 import lq
    assert sorted(lq.EXPORTED) == declared_symbols()
    L = lq.lib()
    for name in lq.EXPORTED:
        assert getattr(L, name).argtypes is not None, name


def _header_struct(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/lq.h."""
    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*%s;" % name, src).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            parts = decl.split(None, 1)[1] if not decl.startswith("const") else decl.split(None, 2)[2]
            names += [d.strip().lstrip("*").strip() for d in parts.split(",")]
    return names


@pytest.mark.parametrize("struct,cls", [("lq_opts", "Opts"), ("lq_lattice_desc", "LatticeDesc"), ("lq_report", "Report")])
def test_binding_structs_mirror_the_header(struct, cls):
    from paper_1611_00195_gb300 import lq
    assert [f for f, _ in getattr(lq, cls)._fields_] == _header_struct(struct)


def test_default_opts_and_reserve_flags(built_lib):
    """lq_default_opts (host only) writes every field of the binding's mirror of lq_opts, and the
    binding's reserve flags are the header's."""
    from paper_1611_00195_gb300 import lq
    o = lq.Opts()
    ctypes.memset(ctypes.byref(o), 0x7f, ctypes.sizeof(o))
    lq.lib().lq_default_opts(ctypes.byref(o))
    want = dict(kmax=0, breakdown_tol=1e-14, newton_max_iter=50, newton_tol=1e-13, deflate=0, projected=0, quad_nodes=64,
                proj_tol=1e-11, hop_variant=-1, defl_kmax=0, defl_nderiv=0, two_pass=0, graph=-1, split=-1, nested_m=100,
                update_variant=-1, rebiorth=0)
    assert {f: getattr(o, f) for f, _ in o._fields_} == want
    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    for name in ("BLOCK", "ADJOINT", "TWO_PASS", "SOLVE", "REBIORTH"):
        m = re.search(r"#define LQ_RESERVE_%s\s+(\d+)" % name, src)
        assert int(m.group(1)) == getattr(lq, "LQ_RESERVE_" + name), name


def test_create_rejects_bad_descriptors_without_gpu(built_lib):
    """lq_create validates on the host and allocates nothing on the device."""
    from paper_1611_00195_gb300 import lq
    L = lq.lib()
    h = ctypes.c_void_p()
    bad = [lq.LatticeDesc(0, 4, 4, 4, -2.0, 1.0, 0.0, 1, 0),      # extent < 1
           lq.LatticeDesc(4, 4, 4, 4, -2.0, 0.5, 0.0, 1, 0),      # r != 1
           lq.LatticeDesc(4, 4, 4, 4, -2.0, 1.0, 0.0, 1, 7)]      # unknown precision
    for d in bad:
        assert L.lq_create(ctypes.byref(d), ctypes.byref(h)) == -1
    assert L.lq_create(None, ctypes.byref(h)) == -1


def test_batch_rejects_bad_arguments_without_gpu(built_lib):
    """lq_batch_apply validates the batch size and member contexts on the host first."""
    from paper_1611_00195_gb300 import lq
    L = lq.lib()
    items = (lq.BatchItem * 17)()
    assert L.lq_batch_apply(None, 1, None) == -1
    assert L.lq_batch_apply(items, 0, None) == -1
    assert L.lq_batch_apply(items, 17, None) == -1      # more than LQ_BATCH_MAX
    assert L.lq_batch_apply(items, 1, None) == -1       # null member context


@pytest.mark.parametrize("n", [1, 2, 5, 30, 64])
def test_dense_eig_host_utility(built_lib, n):
    """The host eigensolver used by the deflation-space Rayleigh-Ritz steps, against numpy."""
    import numpy as np
    from paper_1611_00195_gb300 import lq
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = np.ascontiguousarray(A)
    w = np.zeros(n, complex)
    V = np.zeros((n, n), complex)
    assert lq.lib().lq_dense_eig(n, A.ctypes.data, w.ctypes.data, V.ctypes.data) == 0
    ref = np.linalg.eigvals(A)
    for z in ref:
        assert np.min(np.abs(w - z)) < 1e-10 * max(1.0, np.abs(ref).max())
    assert np.abs(A @ V - V * w).max() < 1e-9 * max(1.0, np.abs(A).max())
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)
