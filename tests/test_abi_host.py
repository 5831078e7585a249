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
