"""C-ABI library checks that need no GPU: it loads, exports every symbol that
include/*.h declares, and its host-side mesh helper agrees with the oracle's
independent mesh (coordinates to round-off, l2g and Dirichlet flags exactly)."""
import glob
import os
import re

import numpy as np
import pytest

import paper_2004_06722_gb300 as pkg
from oracle.mesh import box_mesh, boundary_nodes, global_count

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2004_06722_gb300 import _build
        _build.build()
    return pkg.load_library()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ceedbp_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "ceedbp_setup" in names and "ceedbp_apply" in names and "ceedbp_solve" in names
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("dims,N,amp", [((2, 2, 2), 1, 0.05), ((3, 2, 1), 3, 0.05), ((2, 1, 2), 7, 0.1),
                                        ((1, 1, 1), 15, 0.05), ((2, 2, 2), 4, 0.0)])
def test_mesh_box_matches_oracle_mesh(lib, dims, N, amp):
    coords, l2g, dirichlet = pkg.mesh_box(*dims, N, amp)
    oc, ol2g = box_mesh(*dims, N, amp)
    np.testing.assert_array_equal(l2g, ol2g)
    np.testing.assert_allclose(coords, oc, rtol=0, atol=4e-16)
    np.testing.assert_array_equal(dirichlet.astype(bool), boundary_nodes(*dims, N))
    assert dirichlet.shape[0] == global_count(*dims, N)


def test_mesh_box_rejects_bad_args(lib):
    with pytest.raises(pkg.CeedbpError):
        pkg.mesh_box(0, 1, 1, 3)
    with pytest.raises(pkg.CeedbpError):
        pkg.mesh_box(1, 1, 1, 16)


def test_setup_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        pkg.Operator.box(5, 1, 1, 1, 2)


@pytest.mark.parametrize("bp,order,nelem,nglobal,arith,geom,status", [
    (7, 3, 1, 64, 0, 0, pkg.EUNSUPPORTED),           # no such bake-off problem
    (5, 0, 1, 8, 0, 0, pkg.EINVAL),                  # order below 1
    (5, 16, 1, 8, 0, 0, pkg.EINVAL),                 # order above 15
    (5, 3, 0, 64, 0, 0, pkg.EINVAL),                 # no elements
    (5, 7, 1 << 22, 64, 0, 0, pkg.EINVAL),           # E p1^3 beyond 32-bit local indices
    (5, 3, 1, 64, 5, 0, pkg.EINVAL),                 # unknown arithmetic
    (4, 3, 1, 64, pkg.ARITH_DF64, 0, pkg.EUNSUPPORTED),  # pair arithmetic: not BP2/BP4
    (2, 3, 1, 64, pkg.ARITH_DF64, 0, pkg.EUNSUPPORTED),  # pair arithmetic: not BP2/BP4
    (5, 3, 1, 64, 0, 7, pkg.EINVAL),                 # unknown geometry mode
    (3, 3, 1, 64, 0, pkg.GEOM_RECOMPUTE, pkg.EUNSUPPORTED),  # recomputed factors are BP5/BP6 only
    (6, 15, 1, 4096, 0, pkg.GEOM_RECOMPUTE, pkg.EUNSUPPORTED),  # BP6 tile too large at p1 = 16
])
def test_setup_validates_arguments_before_touching_the_device(lib, bp, order, nelem, nglobal, arith, geom, status):
    """Setup rejects invalid or unbuilt combinations from the parameters alone, before any
    data is read or any CUDA call is made (so this runs without a GPU)."""
    import ctypes
    coords = np.zeros(3 * 8, dtype=np.float64)  # never read: validation fails first
    l2g = np.zeros(8, dtype=np.int64)
    prm = pkg.Params(bp, order, 0, nelem, nglobal, arith, geom)
    ctx = ctypes.c_void_p()
    st = lib.ceedbp_setup(ctypes.byref(prm), coords.ctypes.data_as(ctypes.c_void_p),
                          l2g.ctypes.data_as(ctypes.c_void_p), None, None, None, ctypes.byref(ctx))
    assert st == status
    assert not ctx.value
    assert lib.ceedbp_last_error(None)


def test_header_is_plain_c(tmp_path):
    """include/ceedbp.h is a C ABI: it compiles as strict C99 (no C++ or CUDA types leak in)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "ceedbp.h"\nint main(void) { ceedbp_params p = {0}; (void)p; return 0; }\n')
    res = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                          os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "use_header.o")],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
