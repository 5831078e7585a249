"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (from the problem statement): one FP64 apply within 1e-12 relative
in the 2-norm; CG iteration counts within 1; final relative residuals within
1e-10.  Inputs are seeded synthetic vectors (SplitMix64 by global node id).
Sizes span several thread blocks with a ragged last block; large meshes are
checked on sampled rows the oracle evaluates one by one.
"""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.mesh import boundary_nodes
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


def _vec(n, ncomp, seed):
    v = uniform_pm1(seed, np.arange(n * ncomp))
    return v if ncomp == 1 else v.reshape(n, ncomp)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


CASES = [
    (5, 1, (3, 2, 2)), (5, 2, (3, 3, 3)), (5, 3, (3, 2, 5)), (5, 4, (2, 3, 2)), (5, 5, (2, 2, 2)),
    (5, 7, (3, 2, 2)), (5, 8, (2, 1, 2)), (5, 11, (2, 1, 1)), (5, 15, (1, 1, 1)),
    (3, 1, (3, 2, 2)), (3, 2, (2, 3, 2)), (3, 3, (3, 2, 2)), (3, 5, (2, 2, 1)), (3, 7, (2, 1, 1)), (3, 11, (1, 1, 1)),
    (1, 1, (2, 2, 3)), (1, 3, (3, 2, 2)), (1, 5, (2, 2, 1)), (1, 7, (2, 1, 1)), (1, 15, (1, 1, 1)),
    (6, 2, (2, 2, 2)), (6, 3, (3, 2, 2)), (6, 7, (2, 1, 1)),
    (2, 1, (2, 2, 2)), (2, 3, (3, 2, 2)), (2, 7, (2, 1, 1)),
    (4, 2, (2, 2, 2)), (4, 3, (3, 2, 2)), (4, 7, (2, 1, 1)),
]


@pytest.fixture(scope="module")
def problems():
    cache = {}

    def get(bp, N, dims):
        key = (bp, N, dims)
        if key not in cache:
            cache[key] = (pkg.Operator.box(bp, *dims, N, amp=0.05), BakeoffProblem(bp, *dims, N, amp=0.05))
        return cache[key]

    return get


@pytest.mark.parametrize("bp,N,dims", CASES)
def test_apply_parity(problems, bp, N, dims):
    op, ref = problems(bp, N, dims)
    u = _vec(op.nglobal, op.ncomp, 11)
    w = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    w_ref = ref.apply(u)
    assert _rel(w, w_ref) < APPLY_TOL
    if bp not in (1, 2):
        assert np.all(w.reshape(op.nglobal, -1)[boundary_nodes(*dims, N)] == 0)


@pytest.mark.parametrize("bp,N,dims", [c for c in CASES if c[0] in (1, 3, 5)])
def test_mass_and_jacobi_parity(problems, bp, N, dims):
    op, ref = problems(bp, N, dims)
    u = _vec(op.nglobal, 1, 5)
    w = op.mass(torch.from_numpy(u).cuda()).cpu().numpy()
    assert _rel(w, ref.mass(u)) < APPLY_TOL
    d = op.jacobi().cpu().numpy()
    d_ref = ref.jacobi_inverse()
    assert _rel(d, d_ref) < APPLY_TOL


@pytest.mark.parametrize("bp,N,dims", [(5, 3, (3, 2, 2)), (5, 7, (2, 2, 2)), (3, 3, (2, 2, 2)), (1, 4, (2, 2, 2)),
                                        (6, 3, (2, 2, 2)), (5, 2, (4, 3, 3)), (2, 3, (2, 2, 2)),
                                        (4, 3, (2, 2, 2))])
def test_solve_parity(problems, bp, N, dims):
    op, ref = problems(bp, N, dims)
    r = _vec(op.nglobal, op.ncomp, 0)
    b = ref.rhs(r)
    x, info = op.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda(), tol=1e-8)
    x_ref, infos = ref.solve(b, tol=1e-8)
    for c in range(op.ncomp):
        assert abs(info["iters"][c] - infos[c]["iters"]) <= 1, (info, [i["iters"] for i in infos])
        assert abs(info["rel_res"][c] - infos[c]["rel_res"]) <= 1e-10
        assert info["rel_res"][c] <= 1e-8
    # true residual of the GPU solution, measured with the oracle's operator
    res = np.linalg.norm(ref.apply(x.cpu().numpy()) - b) / np.linalg.norm(b)
    assert res < 1e-7
    assert _rel(x.cpu().numpy(), x_ref) < 1e-6


def test_manufactured_bp5_4x4x4_n7():
    """BP5, E = 4x4x4, N = 7, f = -Lap(sin sin sin), Jacobi-PCG to 1e-8."""
    op = pkg.Operator.box(5, 4, 4, 4, 7, amp=0.05)
    ref = BakeoffProblem(5, 4, 4, 4, 7, amp=0.05)
    b, u_exact = ref.manufactured_rhs()
    x, info = op.solve(torch.from_numpy(b).cuda(), tol=1e-8)
    x_ref, infos = ref.solve(b, tol=1e-8)
    assert abs(info["iters"][0] - infos[0]["iters"]) <= 1
    assert abs(info["rel_res"][0] - infos[0]["rel_res"]) <= 1e-10
    err = np.max(np.abs(x.cpu().numpy() - u_exact))
    err_ref = np.max(np.abs(x_ref - u_exact))
    assert abs(err - err_ref) <= 1e-8 and err < 1e-5


def test_fixed_iterations_match_oracle_history():
    op = pkg.Operator.box(5, 2, 2, 2, 5, amp=0.05)
    ref = BakeoffProblem(5, 2, 2, 2, 5, amp=0.05)
    b = ref.rhs(_vec(op.nglobal, 1, 0))
    for k in (1, 3, 20):
        x, info = op.solve(torch.from_numpy(b).cuda(), fixed_iters=k)
        _, infos = ref.solve(b, fixed_iters=k)
        assert info["iters"][0] == k
        assert abs(info["res_norm"][0] - infos[0]["history"][-1]) <= 1e-10 * infos[0]["b_norm"]


def test_brute_force_dense_operator():
    """Every unit vector through the GPU apply gives the oracle's dense masked matrix."""
    dims, N = (2, 2, 2), 2
    op = pkg.Operator.box(5, *dims, N, amp=0.05)
    ref = BakeoffProblem(5, *dims, N, amp=0.05)
    n = op.nglobal
    dense = np.zeros((n, n))
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    for j in range(n):
        e.zero_()
        e[j] = 1.0
        dense[:, j] = op.apply(e).cpu().numpy()
    m = ref.free.astype(float)
    A = (ref.A.toarray() * m[:, None]) * m[None, :]
    assert np.max(np.abs(dense - A)) <= 1e-13 * np.max(np.abs(A))


def test_deterministic_bits():
    op = pkg.Operator.box(5, 3, 3, 3, 7, amp=0.05)
    u = torch.from_numpy(_vec(op.nglobal, 1, 3)).cuda()
    w1 = op.apply(u).clone()
    w2 = op.apply(u)
    assert torch.equal(w1, w2)
    b = op.mass(u)
    x1, i1 = op.solve(b, fixed_iters=30)
    x1 = x1.clone()
    x2, i2 = op.solve(b, fixed_iters=30, chunk=7)
    assert torch.equal(x1, x2) and i1["res_norm"] == i2["res_norm"]
    x3, _ = op.solve(b, fixed_iters=30, use_graph=False)
    assert torch.equal(x1, x3)


def test_degenerate_single_element_all_dirichlet():
    op = pkg.Operator.box(5, 1, 1, 1, 1, amp=0.05)  # every node on the boundary
    b = torch.zeros(op.nglobal, dtype=torch.float64, device="cuda")
    x, info = op.solve(b, tol=1e-8)
    assert info["iters"][0] == 0 and torch.count_nonzero(x) == 0
    u = torch.ones(op.nglobal, dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(op.apply(u)) == 0


def test_invalid_setup_is_rejected():
    coords, l2g, dirichlet = pkg.mesh_box(1, 1, 1, 2)
    bad = l2g.copy()
    bad[0, 0] = dirichlet.shape[0] + 5
    with pytest.raises(pkg.CeedbpError) as ei:
        pkg.Operator(5, 2, coords, bad, dirichlet)
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.CeedbpError) as ei:
        pkg.Operator(7, 2, coords, l2g, dirichlet)
    assert ei.value.status == pkg.EUNSUPPORTED


# node samples per case: probe elements, interior nodes per probe element, extra random nodes
FULL_SIZE = [(5, 7, 18, dict(n_probe=5, n_interior=24, n_random=16)),
             (3, 15, 14, dict(n_probe=3, n_interior=64, n_random=8)),
             (1, 3, 21, dict(n_probe=5, n_interior=24, n_random=90))]


@pytest.mark.parametrize("bp,N,k,sample", FULL_SIZE)
def test_sampled_rows_at_largest_sweep_size(bp, N, k, sample):
    """The largest size of the 1e4..1e8 sweep (E = 2^k), in the launch configuration the bench
    times, on at least 200 rows the oracle evaluates one by one: the vertices, edges, faces and
    interior of probe elements (the first, middle and last element among them) and random
    nodes; 2-norm relative error over the sampled rows within the apply tolerance, and the
    masked Dirichlet rows exactly zero."""
    dims = box_dims(k)
    op = pkg.Operator.box(bp, *dims, N, amp=0.05)
    n = op.nglobal
    u_h = uniform_pm1(9, np.arange(n))
    w = op.apply(torch.from_numpy(u_h).cuda())
    nodes = probe_nodes(dims, N, seed=k, **sample)
    assert len(nodes) >= 200
    rows = sampled_rows(bp, *dims, N, 0.05, lambda ids: u_h[ids], nodes)
    got = w[torch.from_numpy(nodes).cuda()].cpu().numpy()
    err = _rel(got, rows)
    print(f"BP{bp} N={N} E=2^{k}: {len(nodes)} sampled rows, relative error {err:.2e}")
    assert err <= APPLY_TOL, err
    if bp != 1:
        on_boundary = rows == 0.0
        assert np.all(got[on_boundary] == 0.0)
    op.close()


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_bp6_sampled_rows_at_defect_correction_size(arith):
    """BP6 (three components sharing G) at the defect-correction configuration's size, E = 48^3,
    N = 7 (3.8e7 DOFs per component), in both arithmetics, on 200+ sampled nodes x 3 components."""
    dims, N = (48, 48, 48), 7
    op = pkg.Operator.box(6, *dims, N, amp=0.05, arith=arith)
    n = op.nglobal
    u_h = uniform_pm1(13, np.arange(n * 3)).reshape(n, 3)
    w = op.apply(torch.from_numpy(u_h).cuda())
    nodes = probe_nodes(dims, N, seed=48)
    assert len(nodes) >= 200
    rows = sampled_rows(6, *dims, N, 0.05, lambda ids: u_h[ids], nodes)
    got = w[torch.from_numpy(nodes).cuda()].cpu().numpy()
    err = _rel(got, rows)
    print(f"BP6 N=7 E=48^3 arith={arith}: {len(nodes)} nodes x 3, relative error {err:.2e}")
    assert err <= APPLY_TOL, err
    op.close()
