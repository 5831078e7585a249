"""Helmholtz operator H = A + beta B (Eq. (17)) against the oracle.

ceedbp_set_helmholtz adds beta B u inside the element kernels (at the
quadrature points) and rebuilds the Jacobi diagonal of A + beta B.  One apply
must match the oracle's assembled H to 1e-12 relative, PCG the oracle's
iteration count within 1, and beta = 0 must give back A bit for bit.
"""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.problems import BakeoffProblem
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

BETA = 7.5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _vec(n, ncomp, seed):
    v = uniform_pm1(seed, np.arange(n * ncomp))
    return v if ncomp == 1 else v.reshape(n, ncomp)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("bp,N,dims", [(3, 3, (3, 2, 2)), (3, 6, (2, 1, 1)), (4, 2, (2, 2, 2)), (5, 2, (2, 3, 2)),
                                        (5, 7, (3, 2, 2)), (5, 8, (2, 1, 2)), (6, 3, (3, 2, 2)), (6, 7, (2, 1, 1))])
def test_helmholtz_apply_and_jacobi(bp, N, dims):
    op = pkg.Operator.box(bp, *dims, N, amp=0.05)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05, beta=BETA)
    u = _vec(op.nglobal, op.ncomp, 17)
    ut = torch.from_numpy(u).cuda()
    w_a = op.apply(ut).cpu().numpy()
    op.set_helmholtz(BETA)
    w = op.apply(ut).cpu().numpy()
    assert _rel(w, ref.apply(u)) < 1e-12
    assert _rel(op.jacobi().cpu().numpy(), ref.jacobi_inverse()) < 1e-12
    op.set_helmholtz(0.0)
    np.testing.assert_array_equal(op.apply(ut).cpu().numpy(), w_a)


@pytest.mark.parametrize("bp,N,dims", [(5, 7, (2, 2, 2)), (3, 3, (2, 2, 2)), (6, 3, (2, 2, 2))])
def test_helmholtz_solve(bp, N, dims):
    op = pkg.Operator.box(bp, *dims, N, amp=0.05)
    op.set_helmholtz(BETA)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05, beta=BETA)
    b = ref.rhs(_vec(op.nglobal, op.ncomp, 0))
    x, info = op.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda(), tol=1e-8)
    _, infos = ref.solve(b, tol=1e-8)
    for c in range(op.ncomp):
        assert abs(info["iters"][c] - infos[c]["iters"]) <= 1
        assert abs(info["rel_res"][c] - infos[c]["rel_res"]) <= 1e-10
    res = np.linalg.norm(ref.apply(x.cpu().numpy()) - b) / np.linalg.norm(b)
    assert res < 1e-7


def test_helmholtz_unsupported_and_invalid():
    for bp, kw in ((1, {}), (5, {"arith": pkg.ARITH_DF64}), (5, {"geom": pkg.GEOM_RECOMPUTE})):
        op = pkg.Operator.box(bp, 2, 1, 1, 3, **kw)
        with pytest.raises(pkg.CeedbpError) as ei:
            op.set_helmholtz(1.0)
        assert ei.value.status == pkg.EUNSUPPORTED
    op = pkg.Operator.box(5, 2, 1, 1, 3)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(pkg.CeedbpError) as ei:
            op.set_helmholtz(bad)
        assert ei.value.status == pkg.EINVAL
    op.set_helmholtz(2.0)
    with pytest.raises(pkg.CeedbpError) as ei:
        op.prepare_mixed(pkg.MIXED_FP32)
    assert ei.value.status == pkg.EUNSUPPORTED
