"""Unassembled element operators (the BK kernels of Table 1) against the oracle.

ceedbp_bk_apply computes w^e = A^e u^e (or B^e u^e) for every element without
Q, Q^T or the Dirichlet mask; the oracle builds each element matrix by full
quadrature and multiplies.  Tolerance 1e-12 relative (2-norm over all
elements), for every BP, both arithmetics of BP1/BP3/BP5/BP6 and the
recomputed factors.
"""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.element import element_matrices
from oracle.mesh import box_mesh
from oracle.quadrature import bp_rule
from synth import uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _oracle_bk(bp, dims, N, uL):
    coords, _ = box_mesh(*dims, N, 0.05)
    rule = bp_rule(bp, N)
    which = "B" if bp in (1, 2) else "A"
    out = np.zeros_like(uL)
    for e in range(coords.shape[0]):
        M = element_matrices(coords[e], N, rule, want=(which,))[which]
        out[e] = M @ uL[e]
    return out


@pytest.mark.parametrize("bp,N,dims,kw", [
    (1, 3, (2, 2, 1), {}), (2, 2, (2, 1, 2), {}), (3, 3, (2, 1, 2), {}), (4, 2, (1, 2, 2), {}),
    (5, 1, (2, 2, 2), {}), (5, 4, (2, 2, 1), {}), (5, 7, (2, 1, 2), {}), (5, 8, (1, 1, 2), {}),
    (6, 3, (2, 2, 1), {}),
    (5, 3, (2, 2, 2), {"arith": pkg.ARITH_DF64}), (5, 7, (3, 1, 1), {"arith": pkg.ARITH_DF64}),
    (6, 5, (1, 2, 1), {"arith": pkg.ARITH_DF64}),
    (1, 7, (2, 1, 2), {}), (3, 7, (2, 2, 1), {}), (3, 9, (1, 1, 2), {}), (1, 15, (1, 1, 1), {}),
    (1, 3, (2, 1, 2), {"arith": pkg.ARITH_DF64}), (1, 7, (1, 2, 1), {"arith": pkg.ARITH_DF64}),
    (3, 5, (2, 1, 1), {"arith": pkg.ARITH_DF64}), (3, 7, (2, 1, 2), {"arith": pkg.ARITH_DF64}),
    (5, 5, (2, 1, 2), {"geom": pkg.GEOM_RECOMPUTE}), (6, 3, (1, 1, 2), {"geom": pkg.GEOM_RECOMPUTE}),
])
def test_bk_apply_matches_element_matrices(bp, N, dims, kw):
    op = pkg.Operator.box(bp, *dims, N, amp=0.05, **kw)
    p3 = (N + 1) ** 3
    E = dims[0] * dims[1] * dims[2]
    shape = (E, p3) if op.ncomp == 1 else (E, p3, 3)
    uL = uniform_pm1(9, np.arange(int(np.prod(shape)))).reshape(shape)
    w = op.bk_apply(torch.from_numpy(uL).cuda()).cpu().numpy()
    ref = _oracle_bk(bp, dims, N, uL)
    err = np.linalg.norm(w - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err
    # a second call (identity map already allocated) gives the same bits
    w2 = op.bk_apply(torch.from_numpy(uL).cuda()).cpu().numpy()
    np.testing.assert_array_equal(w, w2)


def test_bk_apply_rejects_wrong_shapes():
    op = pkg.Operator.box(5, 2, 1, 1, 3)
    with pytest.raises(ValueError):
        op.bk_apply(torch.zeros(2, 63, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("bp,N,dims", [(3, 3, (2, 1, 2)), (5, 7, (2, 1, 1)), (5, 4, (1, 2, 2)), (6, 3, (1, 2, 1))])
def test_bk_apply_helmholtz(bp, N, dims):
    """With ceedbp_set_helmholtz the element operator is A^e + beta B^e (Eq. (17))."""
    beta = 3.25
    op = pkg.Operator.box(bp, *dims, N, amp=0.05)
    op.set_helmholtz(beta)
    p3 = (N + 1) ** 3
    E = dims[0] * dims[1] * dims[2]
    shape = (E, p3) if op.ncomp == 1 else (E, p3, 3)
    uL = uniform_pm1(5, np.arange(int(np.prod(shape)))).reshape(shape)
    w = op.bk_apply(torch.from_numpy(uL).cuda()).cpu().numpy()
    coords, _ = box_mesh(*dims, N, 0.05)
    rule = bp_rule(bp, N)
    ref = np.zeros_like(uL)
    for e in range(E):
        m = element_matrices(coords[e], N, rule, want=("A", "B"))
        ref[e] = (m["A"] + beta * m["B"]) @ uL[e]
    assert np.linalg.norm(w - ref) / np.linalg.norm(ref) < 1e-12
