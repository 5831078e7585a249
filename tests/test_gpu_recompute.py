"""Recomputed geometric factors (geom = RECOMPUTE) against the oracle.

The element kernel forms J, adj(J), |J| and the six factors of Eq. (23) from
the nodal coordinates every apply; the operator is the same matrix as with
stored factors, so one apply must match the oracle to 1e-12 relative, agree
with the stored-factor path to rounding, and PCG must take the same
iterations (within 1) as the oracle's.
"""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.mesh import boundary_nodes
from oracle.problems import BakeoffProblem
from synth import uniform_pm1

pytestmark = pytest.mark.gpu


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


CASES = [(5, 1, (3, 2, 2)), (5, 2, (2, 3, 2)), (5, 3, (3, 2, 3)), (5, 4, (2, 2, 2)), (5, 7, (3, 2, 2)),
         (5, 8, (2, 1, 2)), (5, 11, (2, 1, 1)), (5, 15, (1, 1, 1)),
         (6, 2, (2, 2, 2)), (6, 3, (3, 2, 2)), (6, 7, (2, 1, 1)), (6, 12, (1, 1, 1))]


@pytest.mark.parametrize("bp,N,dims", CASES)
def test_recompute_apply_matches_oracle_and_stored(bp, N, dims):
    rc = pkg.Operator.box(bp, *dims, N, amp=0.05, geom=pkg.GEOM_RECOMPUTE)
    st = pkg.Operator.box(bp, *dims, N, amp=0.05)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05)
    u = _vec(rc.nglobal, rc.ncomp, 21)
    ut = torch.from_numpy(u).cuda()
    w_rc = rc.apply(ut).cpu().numpy()
    w_st = st.apply(ut).cpu().numpy()
    assert _rel(w_rc, ref.apply(u)) < 1e-12
    assert _rel(w_rc, w_st) < 1e-13
    assert np.all(w_rc.reshape(rc.nglobal, -1)[boundary_nodes(*dims, N)] == 0)
    # the Jacobi diagonal comes from the same (temporary) stored factors
    assert _rel(rc.jacobi().cpu().numpy(), ref.jacobi_inverse()) < 1e-12


@pytest.mark.parametrize("bp,N,dims", [(5, 7, (2, 2, 2)), (5, 3, (4, 3, 3)), (6, 3, (2, 2, 2))])
def test_recompute_solve_matches_oracle(bp, N, dims):
    rc = pkg.Operator.box(bp, *dims, N, amp=0.05, geom=pkg.GEOM_RECOMPUTE)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05)
    b = ref.rhs(_vec(rc.nglobal, rc.ncomp, 0))
    x, info = rc.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda(), tol=1e-8)
    _, infos = ref.solve(b, tol=1e-8)
    for c in range(rc.ncomp):
        assert abs(info["iters"][c] - infos[c]["iters"]) <= 1
        assert abs(info["rel_res"][c] - infos[c]["rel_res"]) <= 1e-10
    res = np.linalg.norm(ref.apply(x.cpu().numpy()) - b) / np.linalg.norm(b)
    assert res < 1e-7


def test_recompute_unsupported_combinations():
    coords, l2g, dirichlet = pkg.mesh_box(2, 2, 2, 3, 0.05)
    for bp, arith in ((3, pkg.ARITH_FP64), (1, pkg.ARITH_FP64), (5, pkg.ARITH_DF64)):
        with pytest.raises(pkg.CeedbpError) as ei:
            pkg.Operator(bp, 3, coords, l2g, dirichlet, arith=arith, geom=pkg.GEOM_RECOMPUTE)
        assert ei.value.status == pkg.EUNSUPPORTED
    kappa = np.ones(8 * 4 ** 3)
    with pytest.raises(pkg.CeedbpError) as ei:
        pkg.Operator(5, 3, coords, l2g, dirichlet, kappa=kappa, geom=pkg.GEOM_RECOMPUTE)
    assert ei.value.status == pkg.EUNSUPPORTED
    op = pkg.Operator(5, 3, coords, l2g, dirichlet, geom=pkg.GEOM_RECOMPUTE)
    with pytest.raises(pkg.CeedbpError) as ei:
        op.set_kappa(torch.ones(8 * 4 ** 3, dtype=torch.float64, device="cuda"))
    assert ei.value.status == pkg.EUNSUPPORTED
    with pytest.raises(pkg.CeedbpError) as ei:
        op.prepare_mixed(pkg.MIXED_FP32)
    assert ei.value.status == pkg.EUNSUPPORTED
    with pytest.raises(pkg.CeedbpError) as ei:
        pkg.Operator(5, 3, coords, l2g, dirichlet, geom=7)
    assert ei.value.status == pkg.EINVAL
