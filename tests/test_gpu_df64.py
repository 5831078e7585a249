"""Parity of the FP64-accurate FP32-pair path (CEEDBP_ARITH_DF64) with the
CPU FP64 oracle, at the FP64 tolerances: one apply within 1e-12 relative, CG
iteration counts within 1, final relative residuals within 1e-10.  BP5/BP6
(collocated) and BP1/BP3 (Gauss quadrature)."""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.problems import BakeoffProblem
from oracle.sampled import sampled_rows
from synth import box_dims, uniform_pm1

from node_samples import probe_nodes

pytestmark = pytest.mark.gpu
APPLY_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _box(bp, dims, N, arith=pkg.ARITH_DF64, amp=0.05):
    coords, l2g, dirichlet = pkg.mesh_box(*dims, N, amp)
    return pkg.Operator(bp, N, coords, l2g, dirichlet, arith=arith)


def _vec(n, ncomp, seed):
    v = uniform_pm1(seed, np.arange(n * ncomp))
    return v if ncomp == 1 else v.reshape(n, ncomp)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("bp,N,dims", [(5, 1, (3, 2, 2)), (5, 2, (3, 3, 3)), (5, 3, (3, 2, 5)), (5, 4, (2, 3, 2)),
                                        (5, 5, (2, 2, 2)), (5, 7, (3, 2, 2)), (5, 8, (2, 1, 2)), (5, 11, (2, 1, 1)),
                                        (5, 15, (1, 1, 1)), (6, 2, (2, 2, 2)), (6, 3, (3, 2, 2)), (6, 7, (2, 1, 1)),
                                        (3, 1, (3, 2, 2)), (3, 2, (2, 3, 2)), (3, 3, (3, 2, 2)), (3, 5, (2, 2, 1)),
                                        (3, 7, (2, 1, 2)), (3, 11, (1, 1, 1)), (1, 1, (2, 2, 3)), (1, 3, (3, 2, 2)),
                                        (1, 7, (2, 1, 1)), (1, 11, (1, 1, 1)), (3, 13, (1, 1, 1)), (3, 15, (1, 1, 1)),
                                        (1, 15, (1, 1, 1))])
def test_df64_apply_parity(bp, N, dims):
    op = _box(bp, dims, N)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05)
    u = _vec(op.nglobal, op.ncomp, 11)
    w = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    err = _rel(w, ref.apply(u))
    assert err < APPLY_TOL, err


@pytest.mark.parametrize("bp,N,dims", [(5, 3, (3, 2, 2)), (5, 7, (2, 2, 2)), (6, 3, (2, 2, 2)), (5, 2, (4, 3, 3)),
                                        (3, 3, (3, 2, 2)), (3, 7, (2, 2, 1)), (1, 5, (2, 2, 2))])
def test_df64_solve_parity(bp, N, dims):
    op = _box(bp, dims, N)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05)
    b = ref.rhs(_vec(op.nglobal, op.ncomp, 0))
    x, info = op.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda(), tol=1e-8)
    x_ref, infos = ref.solve(b, tol=1e-8)
    for c in range(op.ncomp):
        assert abs(info["iters"][c] - infos[c]["iters"]) <= 1
        assert abs(info["rel_res"][c] - infos[c]["rel_res"]) <= 1e-10
    res = np.linalg.norm(ref.apply(x.cpu().numpy()) - b) / np.linalg.norm(b)
    assert res < 1e-7
    assert _rel(x.cpu().numpy(), x_ref) < 1e-6


def test_df64_manufactured_4x4x4_n7():
    op = _box(5, (4, 4, 4), 7)
    ref = BakeoffProblem(5, 4, 4, 4, 7, amp=0.05)
    b, u_exact = ref.manufactured_rhs()
    x, info = op.solve(torch.from_numpy(b).cuda(), tol=1e-8)
    x_ref, infos = ref.solve(b, tol=1e-8)
    assert abs(info["iters"][0] - infos[0]["iters"]) <= 1
    assert abs(info["rel_res"][0] - infos[0]["rel_res"]) <= 1e-10
    assert abs(np.max(np.abs(x.cpu().numpy() - u_exact)) - np.max(np.abs(x_ref - u_exact))) <= 1e-8


def test_df64_matches_fp64_path_and_is_deterministic():
    dims, N = (4, 4, 3), 7
    a = _box(5, dims, N)
    f = _box(5, dims, N, arith=pkg.ARITH_FP64)
    u = torch.from_numpy(_vec(a.nglobal, 1, 4)).cuda()
    wa, wf = a.apply(u).clone(), f.apply(u)
    assert (torch.linalg.norm(wa - wf) / torch.linalg.norm(wf)).item() < 1e-12
    assert torch.equal(wa, a.apply(u))
    b = f.mass(u)
    xa, ia = a.solve(b, fixed_iters=50)
    xa = xa.clone()
    xf, i_f = f.solve(b, fixed_iters=50)
    assert abs(ia["res_norm"][0] - i_f["res_norm"][0]) <= 1e-10 * ia["b_norm"][0]
    xa2, _ = a.solve(b, fixed_iters=50, chunk=9)
    assert torch.equal(xa, xa2)


def test_df64_x0_restart():
    op = _box(5, (3, 3, 3), 5)
    ref = BakeoffProblem(5, 3, 3, 3, 5, amp=0.05)
    b = torch.from_numpy(ref.rhs(_vec(op.nglobal, 1, 0))).cuda()
    x, i1 = op.solve(b, fixed_iters=15)
    x2, i2 = op.solve(b, x=x.clone(), tol=1e-10, x0=True)
    assert i2["rel_res"][0] <= 1e-10
    xr, _ = ref.solve(b.cpu().numpy(), tol=1e-12)
    assert _rel(x2.cpu().numpy(), xr) < 1e-8


@pytest.mark.parametrize("tile", [None, (2, 2, 16), (1, 3, 16)])
def test_df64_sampled_rows_largest_n7(tile):
    """The pair path at the bench size (E = 2^18, N = 7; the autotuned shape, the pipelined direct
    schedule and the even-odd schedule) on at least 200 rows (vertices, edges, faces and interiors
    of probe elements, the last element among them)."""
    dims, N = box_dims(18), 7
    op = _box(5, dims, N)
    if tile is not None:
        op.set_tile(*tile)
    n = op.nglobal
    u_h = uniform_pm1(9, np.arange(n))
    w = op.apply(torch.from_numpy(u_h).cuda())
    nodes = probe_nodes(dims, N, seed=18)
    assert len(nodes) >= 200
    rows = sampled_rows(5, *dims, N, 0.05, lambda ids: u_h[ids], nodes)
    got = w[torch.from_numpy(nodes).cuda()].cpu().numpy()
    err = np.linalg.norm(got - rows) / np.linalg.norm(rows)
    print(f"pair path BP5 N=7 E=2^18 (shape {op.tile_info()}): {len(nodes)} rows, relative error {err:.2e}")
    assert err <= APPLY_TOL, err
    assert np.all(got[rows == 0.0] == 0.0)
    op.close()


PIPELINED = [(1, 4), (1, 8), (1, 16), (2, 4), (2, 16)]


@pytest.mark.parametrize("bp,N,dims", [(5, 1, (3, 2, 2)), (5, 3, (3, 2, 5)), (5, 4, (2, 3, 3)), (5, 5, (3, 3, 2)),
                                        (5, 7, (5, 3, 3)), (6, 3, (2, 3, 2)), (6, 7, (3, 2, 2)), (5, 9, (3, 1, 2)),
                                        (5, 11, (2, 1, 2)), (5, 15, (1, 1, 2))])
def test_pipelined_schedule_parity_and_same_bits(bp, N, dims):
    """Every pair-kernel schedule computes the same element results: the pipelined
    sequences (ragged last block: E is not a multiple of eb * seq) match the oracle
    to 1e-12 and the per-element ring schedule bit for bit."""
    op = _box(bp, dims, N)
    ref = BakeoffProblem(bp, *dims, N, amp=0.05)
    u = _vec(op.nglobal, op.ncomp, 13)
    ut = torch.from_numpy(u).cuda()
    w_ref = ref.apply(u)
    outs = []
    for eb, seq in PIPELINED:
        try:
            op.set_tile(eb, 2, seq)
        except pkg.CeedbpError as e:
            assert e.status == pkg.EINVAL
            continue
        assert op.tile_info() == (eb, 2, seq)
        w = op.apply(ut).cpu().numpy()
        assert _rel(w, w_ref) < APPLY_TOL
        outs.append(w)
    assert len(outs) >= 3
    op.set_tile(1, 0)
    w0 = op.apply(ut).cpu().numpy()
    for w in outs:
        np.testing.assert_array_equal(w, w0)
    with pytest.raises(pkg.CeedbpError) as ei:
        op.set_tile(3, 2, 5)
    assert ei.value.status == pkg.EINVAL


EVEN_ODD = [(1, 4), (1, 8), (1, 16), (2, 8), (4, 8), (8, 8), (16, 8), (32, 4)]


@pytest.mark.parametrize("N,dims", [(3, (3, 2, 5)), (5, (3, 3, 2)), (7, (5, 3, 3)), (9, (3, 1, 2)),
                                    (11, (2, 1, 2))])
def test_even_odd_schedule_parity(N, dims):
    """The even-odd pair kernel (schedule 3): every launchable shape (ragged last sequence: E is
    not a multiple of eb * seq) matches the oracle to 1e-12; its shapes agree bit for bit among
    themselves, and with the direct schedule to the pair arithmetic's accuracy."""
    op = _box(5, dims, N)
    ref = BakeoffProblem(5, *dims, N, amp=0.05)
    u = _vec(op.nglobal, 1, 13)
    ut = torch.from_numpy(u).cuda()
    w_ref = ref.apply(u)
    outs = []
    for eb, seq in EVEN_ODD:
        try:
            op.set_tile(eb, 3, seq)
        except pkg.CeedbpError as e:
            assert e.status == pkg.EINVAL
            continue
        assert op.tile_info() == (eb, 3, seq)
        w = op.apply(ut).cpu().numpy()
        err = _rel(w, w_ref)
        assert err < APPLY_TOL, (eb, seq, err)
        outs.append(w)
    assert len(outs) >= 3
    for w in outs[1:]:
        np.testing.assert_array_equal(w, outs[0])
    op.set_tile(1, 0)
    w0 = op.apply(ut).cpu().numpy()
    assert _rel(outs[0], w0) < 1e-12


def test_even_odd_schedule_not_offered_where_not_built():
    """Schedule 3 is BP5 at odd orders 3..11: BP6 and even orders reject it."""
    for bp, N, dims in ((6, 3, (2, 2, 2)), (5, 4, (2, 2, 2)), (5, 1, (2, 2, 2))):
        op = _box(bp, dims, N)
        with pytest.raises(pkg.CeedbpError) as ei:
            op.set_tile(1, 3, 8)
        assert ei.value.status == pkg.EINVAL
        assert op.tile_info()[1] != 3
        op.close()


@pytest.mark.parametrize("bp,N,dims,tile", [(5, 7, (2, 2, 3), (1, 8)), (5, 3, (4, 3, 3), (2, 4)),
                                             (6, 3, (2, 2, 2), (1, 4))])
def test_pipelined_schedule_solve_parity(bp, N, dims, tile):
    op = _box(bp, dims, N)
    op.set_tile(tile[0], 2, tile[1])
    _solve_parity(op, bp, N, dims)


@pytest.mark.parametrize("N,dims,tile", [(7, (2, 2, 3), (1, 8)), (3, (4, 3, 3), (8, 4)), (7, (3, 3, 2), (2, 4)),
                                         (5, (3, 2, 2), (2, 16))])
def test_even_odd_schedule_solve_parity(N, dims, tile):
    """CG with the even-odd pair kernel against the oracle (orders up to 7: at higher orders on
    meshes of a few elements the pair arithmetic's 1e-12 apply error, amplified by CG, moves the
    final residual by more than the 1e-10 bar whatever the schedule)."""
    op = _box(5, dims, N)
    op.set_tile(tile[0], 3, tile[1])
    _solve_parity(op, 5, N, dims)


def _solve_parity(op, bp, N, dims):
    ref = BakeoffProblem(bp, *dims, N, amp=0.05)
    b = ref.rhs(_vec(op.nglobal, op.ncomp, 0))
    x, info = op.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda(), tol=1e-8)
    _, infos = ref.solve(b, tol=1e-8)
    for c in range(op.ncomp):
        assert abs(info["iters"][c] - infos[c]["iters"]) <= 1
        assert abs(info["rel_res"][c] - infos[c]["rel_res"]) <= 1e-10
    res = np.linalg.norm(ref.apply(x.cpu().numpy()) - b) / np.linalg.norm(b)
    assert res < 1e-7


@pytest.mark.parametrize("bp,N,k", [(3, 7, 18), (1, 7, 18)])
def test_df64_gauss_sampled_rows_at_bench_size(bp, N, k):
    """BP3 and BP1 in pair arithmetic at the bench size (E = 2^18, N = 7) on 200+ sampled rows
    (vertices, edges, faces and interiors of probe elements, the last element among them)."""
    dims = box_dims(k)
    op = _box(bp, dims, N)
    n = op.nglobal
    u_h = uniform_pm1(9, np.arange(n))
    w = op.apply(torch.from_numpy(u_h).cuda())
    nodes = probe_nodes(dims, N, seed=k + bp)
    assert len(nodes) >= 200
    rows = sampled_rows(bp, *dims, N, 0.05, lambda ids: u_h[ids], nodes)
    got = w[torch.from_numpy(nodes).cuda()].cpu().numpy()
    err = np.linalg.norm(got - rows) / np.linalg.norm(rows)
    print(f"pair path BP{bp} N={N} E=2^{k}: {len(nodes)} rows, relative error {err:.2e}")
    assert err <= APPLY_TOL, err
    op.close()


def test_df64_gauss_unsupported_cases():
    for bp, N in ((4, 3), (2, 3), (4, 7)):
        c, l, d = pkg.mesh_box(1, 1, 1, N, 0.05)
        with pytest.raises(pkg.CeedbpError) as ei:
            pkg.Operator(bp, N, c, l, d, arith=pkg.ARITH_DF64)
        assert ei.value.status == pkg.EUNSUPPORTED
