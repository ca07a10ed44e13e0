"""The C ABI library loads, exports every symbol declared in include/*.h, and
rejects invalid arguments on the host before touching a GPU.  CPU only."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libfe():
    from paper_2208_07129_gb300 import build, fe
    build.build()
    return fe.lib()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fe_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for must in ("fe_setup", "fe_apply", "fe_destroy", "fe_set_potential", "fe_apply_host"):
        assert must in names


def test_every_declared_symbol_is_exported(libfe):
    missing = [n for n in declared_symbols() if not hasattr(libfe, n)]
    assert not missing, missing


def test_status_strings(libfe):
    from paper_2208_07129_gb300 import fe
    assert fe.status_str(fe.FE_OK) == "ok"
    assert "invalid" in fe.status_str(fe.FE_EINVAL)
    assert fe.status_str(99) == "unknown status"


def test_last_cuda_error_name(libfe):
    """The name of the CUDA error behind the last FE_ECUDA / FE_ENOMEM of this
    thread: "none" or a CUDA runtime error name, never a null pointer."""
    name = libfe.fe_last_cuda_error().decode()
    assert name == "none" or name.startswith("cuda"), name


@pytest.mark.parametrize("kw,status", [
    (dict(nx=0, ny=2, nz=2, p=2, n_q=4), 1),                       # no cells
    (dict(nx=2, ny=2, nz=2, p=9, n_q=11), 8),                      # degree outside the compiled set
    (dict(nx=2, ny=2, nz=2, p=4, n_q=4), 8),                       # n_q < p + 1
    (dict(nx=2, ny=2, nz=2, p=4, n_q=8), 8),                       # n_q > p + 3
    (dict(nx=1, ny=2, nz=2, p=2, n_q=4, periodic=True), 1),        # periodic needs >= 2 cells
    (dict(nx=2, ny=2, nz=2, p=2, n_q=4, lo=(0, 0, 0), hi=(1, 0, 1)), 1),  # empty box
])
def test_setup_rejects_before_any_launch(libfe, kw, status):
    from paper_2208_07129_gb300 import fe
    with pytest.raises(fe.FeError) as ei:
        ctx = fe.fe_setup(**kw)
        fe.fe_destroy(ctx)
    assert ei.value.status == status


def test_null_arguments(libfe):
    VP = ctypes.c_void_p
    assert libfe.fe_apply(None, None, None, 1, None) == 1
    assert libfe.fe_setup(None, 2, None, 0.5, None) == 1
    assert libfe.fe_num_dofs(None) == 0
    libfe.fe_destroy(None)


def test_eig_layer_null_arguments(libfe):
    from paper_2208_07129_gb300 import fe
    fe.lib()   # argument types
    L = fe.lib()
    assert L.fe_mass_gll(None, None) == fe.FE_EINVAL
    assert L.fe_apply_scaled(None, None, None, 1, 1.0, 0.0, 0.0, None) == fe.FE_EINVAL
    assert L.fe_chebyshev_filter(None, None, None, 1, 4, 0.0, 1.0, 2.0, None) == fe.FE_EINVAL
    assert L.fe_chfsi(None, None, 4, None, None, None, None, None) == fe.FE_EINVAL


def test_refined_mesh_calls_reject_bad_arguments(libfe):
    from paper_2208_07129_gb300 import fe
    L = fe.lib()
    assert L.fe_num_slaves(None) == 0
    assert L.fe_node_coords(None, None) == fe.FE_EINVAL
    assert L.fe_setup_refined(None, 2, None, 0.5, None) == fe.FE_EINVAL
    # a refinement box outside the coarse grid is rejected before any device work
    d = fe.fe_refined_desc()
    d.nx = d.ny = d.nz = 2
    for k in range(3):
        d.hi[k] = 1.0
        d.refine_lo[k], d.refine_hi[k] = 0, 3
    q = fe.fe_quad_desc(4, fe.FE_QUAD_GAUSS)
    out = ctypes.c_void_p()
    assert L.fe_setup_refined(ctypes.byref(d), 2, ctypes.byref(q), 0.5, ctypes.byref(out)) == fe.FE_EINVAL
    assert out.value is None
