"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/mf.h
(no GPU needed: nothing is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_04869_gb300 import build, native
    if not os.path.exists(native.LIB_PATH):
        build.build()
    return native.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1801_04869_gb300 import native
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(native.EXPORTS) | {"mf_default_params"}


def test_struct_layouts_match_header(lib):
    from paper_1801_04869_gb300 import native
    p = native.mf_params()
    lib.mf_default_params(ctypes.byref(p))
    assert p.n == 19.0 and p.lambda_ == 0.7 and p.iter_tol == 2e-4 and p.he_dir[2] == 1.0
    assert p.gamma == 1.0 and p.b0 == 0.0                 # the last fields: the tail's offsets


def test_law_parameters_are_checked(lib):
    import numpy as np
    from paper_1801_04869_gb300 import native
    p = native.mf_params()
    lib.mf_default_params(ctypes.byref(p))
    m = np.zeros(16 ** 3, np.uint8)
    p.nx = p.ny = 16
    p.Lx = p.Ly = 2.0
    p.mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    assert lib.mf_workspace_bytes(ctypes.byref(p)) > 0
    for g in (0.0, -1.0, float("inf"), float("nan")):
        p.gamma = g
        assert lib.mf_workspace_bytes(ctypes.byref(p)) == 0, g
    p.gamma = 2.0
    assert lib.mf_workspace_bytes(ctypes.byref(p)) > 0
    p.b0 = 0.3                                              # Kim-type jc is a bulk law
    assert lib.mf_workspace_bytes(ctypes.byref(p)) == 0
    p.dim, p.nz, p.Lz = 3, 16, 2.0
    assert lib.mf_workspace_bytes(ctypes.byref(p)) > 0
    for b in (-0.1, float("inf"), float("nan")):
        p.b0 = b
        assert lib.mf_workspace_bytes(ctypes.byref(p)) == 0, b


def test_readout_enum_matches_header():
    from paper_1801_04869_gb300 import native
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    enum = re.search(r"enum \{ (MF_READ_[^}]*)\}", src).group(1)
    vals = dict((k.strip(), int(v)) for k, v in (x.split("=") for x in enum.split(",")))
    assert vals == {"MF_READ_HZ": native.MF_READ_HZ, "MF_READ_MOMENT": native.MF_READ_MOMENT,
                    "MF_READ_J": native.MF_READ_J, "MF_READ_E": native.MF_READ_E}


def test_workspace_query_and_argument_checks(lib):
    import numpy as np
    from paper_1801_04869_gb300 import native
    p = native.mf_params()
    lib.mf_default_params(ctypes.byref(p))
    m = np.zeros(128 * 128, np.uint8)
    p.nx = p.ny = 128
    p.Lx = p.Ly = 2.0
    p.mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    p.he_sin_period = 1.0
    b = lib.mf_workspace_bytes(ctypes.byref(p))
    assert b > 128 * 128 * 8 * 6
    p.nx = 100                                    # not a power of two
    assert lib.mf_workspace_bytes(ctypes.byref(p)) == 0
    p.nx = 4096                                   # beyond the film limit
    assert lib.mf_workspace_bytes(ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    p.nx = 128
    assert lib.mf_create(ctypes.byref(p), None, 0, None, ctypes.byref(h)) == native.MF_ERR_WORKSPACE


def test_null_and_invalid_arguments_are_refused_without_a_gpu(lib):
    """The documented argument checks run before any CUDA call."""
    import ctypes
    from paper_1801_04869_gb300 import native
    assert lib.mf_autotune(None, 1, 1, None) == native.MF_ERR_ARG
    assert lib.mf_checkpoint_bytes(None) == 0
    assert lib.mf_checkpoint_save(None, None) == native.MF_ERR_ARG
    assert lib.mf_checkpoint_restore(None, None) == native.MF_ERR_ARG
    assert lib.mf_advance_batch(None, 1, None, 1, None) == native.MF_ERR_ARG
    none = (ctypes.c_void_p * 1)()
    tt = (ctypes.c_double * 1)(1.0)
    assert lib.mf_advance_batch(none, 0, tt, 1, None) == native.MF_OK      # nothing to do
    assert lib.mf_advance_batch(none, -1, tt, 1, None) == native.MF_ERR_ARG
    assert lib.mf_advance_batch(none, 1, tt, 1, None) == native.MF_ERR_ARG  # a NULL problem
    assert lib.mf_advance(None, 1.0, 1) == native.MF_ERR_ARG
    assert lib.mf_rhs(None, 0.0, None, None, None) == native.MF_ERR_ARG
    assert lib.mf_get_info(None, None) == native.MF_ERR_ARG
    assert lib.mf_film_outside_vjp(None, 1, None, None, None) == native.MF_ERR_ARG
    assert lib.mf_film_rhs_vjp(None, 1, None, None, None, None, None) == native.MF_ERR_ARG
    assert lib.mf_film_solve_gradient_work_bytes(None, 4, 2) == 0
    assert lib.mf_set_jc_map(None, None) == native.MF_ERR_ARG
    assert lib.mf_set_knot_values(None, None, 0) == native.MF_ERR_ARG
    assert lib.mf_film_rhs_vjp_warm(None, 1, None, None, None, None, None, None, None) == native.MF_ERR_ARG
    assert lib.mf_set_barrier_timeout(None, 1.0) == native.MF_ERR_ARG
    assert lib.mf_film_solve_gradient(None, 1, None, None, None, 1, None, None, None, None, 0, None,
                                      None, 0, None, None, None) == native.MF_ERR_ARG
    one = (ctypes.c_int * 1)(64)
    out = (ctypes.c_int * 1)()
    assert lib.mf_batch_plan(-1, one, one, one, None, 304, out, out, out) == -1
    assert lib.mf_batch_plan(0, None, None, None, None, 304, None, None, None) == 0
