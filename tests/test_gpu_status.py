"""Failure detection through status codes, with no GPU fault: CG breakdown
(an indefinite operator, kappa = -1, makes p^T A p negative), iteration limit
(ENOCONV with the iterate and info filled), non-finite data, and host-side
argument errors that launch nothing."""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from synth import uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _rhs(op, dirichlet):
    r = torch.from_numpy(uniform_pm1(0, np.arange(op.nglobal))).cuda()
    return op.mass(r) * torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda()


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_breakdown_on_indefinite_operator(arith):
    coords, l2g, dirichlet = pkg.mesh_box(2, 2, 2, 3, 0.05)
    op = pkg.Operator(5, 3, coords, l2g, dirichlet, arith=arith)
    b = _rhs(op, dirichlet)
    op.set_kappa(torch.full((op.nelem, 4 ** 3), -1.0, dtype=torch.float64, device="cuda"))
    with pytest.raises(pkg.CeedbpError) as ei:
        op.solve(b, tol=1e-10)
    assert ei.value.status == pkg.EBREAKDOWN
    # back to a definite operator: the same context solves again
    op.set_kappa(torch.ones((op.nelem, 4 ** 3), dtype=torch.float64, device="cuda"))
    x, info = op.solve(b, tol=1e-10)
    assert info["status"] == "OK" and info["rel_res"][0] <= 1e-10


def test_noconv_fills_info():
    coords, l2g, dirichlet = pkg.mesh_box(3, 3, 3, 5, 0.05)
    op = pkg.Operator(5, 5, coords, l2g, dirichlet)
    b = _rhs(op, dirichlet)
    x, info = op.solve(b, tol=1e-14, maxit=7, raise_on_noconv=False)
    assert info["status"] == "ENOCONV" and info["iters"][0] == 7 and 0 < info["rel_res"][0] < 1
    with pytest.raises(pkg.CeedbpError) as ei:
        op.solve(b, tol=1e-14, maxit=7)
    assert ei.value.status == pkg.ENOCONV


def test_nonfinite_rhs_is_reported():
    coords, l2g, dirichlet = pkg.mesh_box(2, 2, 2, 3, 0.05)
    op = pkg.Operator(5, 3, coords, l2g, dirichlet)
    b = _rhs(op, dirichlet)
    b[int(np.flatnonzero(dirichlet == 0)[0])] = float("nan")
    with pytest.raises(pkg.CeedbpError) as ei:
        op.solve(b, tol=1e-10)
    assert ei.value.status in (pkg.EBREAKDOWN, pkg.ENOCONV)


def test_argument_errors_launch_nothing():
    coords, l2g, dirichlet = pkg.mesh_box(2, 2, 2, 3, 0.05)
    with pytest.raises(ValueError):
        pkg.Operator(5, 3, coords, np.ascontiguousarray(l2g[:, :10]), dirichlet)  # wrong l2g shape
    op = pkg.Operator(5, 3, coords, l2g, dirichlet)
    with pytest.raises(ValueError):
        op.apply(torch.zeros(op.nglobal + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(pkg.CeedbpError) as ei:
        op.solve(torch.zeros(op.nglobal, dtype=torch.float64, device="cuda"), tol=-1.0)
    assert ei.value.status == pkg.EINVAL
    p1 = pkg.Operator(1, 3, coords, l2g, dirichlet)
    with pytest.raises(pkg.CeedbpError) as ei:
        p1.set_kappa(torch.ones((p1.nelem, 5 ** 3), dtype=torch.float64, device="cuda"))
    assert ei.value.status == pkg.EUNSUPPORTED
    with pytest.raises(pkg.CeedbpError) as ei:
        p1.prepare_mixed(pkg.MIXED_FP32)
    assert ei.value.status == pkg.EUNSUPPORTED


def _staged_shape(op):
    """A launchable shape of the staged pair schedule (schedule 1) at this order."""
    for eb in (1, 2, 3, 4):
        try:
            op.set_tile(eb, 1)
            return eb
        except pkg.CeedbpError:
            continue
    pytest.skip("no staged pair shape is launchable at this order")


def test_bounded_wait_gives_up_and_is_reported():
    """The staged pair schedule waits for the bulk copy of G on an mbarrier with a bounded poll
    count.  With the limit set to 0 polls every launch gives up that wait, flags the fault, drains
    its copy (with the default limit) and returns: the apply is reported by ceedbp_check and the
    solve returns ECUDA.  No GPU fault is involved.  With the default restored the same context
    applies and solves correctly again."""
    coords, l2g, dirichlet = pkg.mesh_box(3, 3, 2, 7, 0.05)
    op = pkg.Operator(5, 7, coords, l2g, dirichlet, arith=pkg.ARITH_DF64)
    _staged_shape(op)
    b = _rhs(op, dirichlet)
    u = torch.from_numpy(uniform_pm1(4, np.arange(op.nglobal))).cuda()
    ref = op.apply(u).clone()
    op.check()
    op.set_wait_limit(0)
    op.apply(u)
    with pytest.raises(pkg.CeedbpError) as ei:
        op.check()
    assert ei.value.status == pkg.ECUDA and "bounded wait" in str(ei.value)
    op.check()  # the flag was cleared by the report
    with pytest.raises(pkg.CeedbpError) as ei:
        op.solve(b, tol=1e-10)
    assert ei.value.status == pkg.ECUDA
    op.set_wait_limit(-1)
    w = op.apply(u)
    op.check()
    assert torch.equal(w, ref)
    x, info = op.solve(b, tol=1e-10)
    assert info["status"] == "OK" and info["rel_res"][0] <= 1e-10
    op.close()


def test_wait_limit_needs_pair_path():
    op = pkg.Operator.box(5, 2, 2, 2, 3)
    with pytest.raises(pkg.CeedbpError) as ei:
        op.set_wait_limit(0)
    assert ei.value.status == pkg.EUNSUPPORTED
    op.check()  # nothing pending on an FP64 context
    op.close()
