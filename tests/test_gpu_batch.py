"""Batched BP5 solves: every problem of a batch of uneven sizes and orders
matches its own single-problem solve (iteration counts within 1, residuals at
the tolerance) and the CPU FP64 oracle: small members by full solves, the
largest member on sampled rows of A x against b.  Both arithmetics: native
FP64 and FP64-accurate FP32 pairs."""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.problems import BakeoffProblem
from oracle.sampled import sampled_rows
from synth import batched_problems, uniform_pm1

from node_samples import probe_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _problems(n, k_max, arith=pkg.ARITH_DF64, seed=3, orders=(3, 5, 7)):
    draws = batched_problems(n_problems=n, seed=seed, k_max=k_max, orders=orders)
    probs, rhs, meshes = [], [], []
    for q in draws:
        coords, l2g, dirichlet = pkg.mesh_box(q["k"], q["k"], q["k"], q["N"], q["amp"])
        probs.append((q["N"], coords, l2g, dirichlet))
        meshes.append((q, coords, l2g, dirichlet))
        op = pkg.Operator(5, q["N"], coords, l2g, dirichlet, arith=arith)
        r = torch.from_numpy(uniform_pm1(q["rhs_seed"], np.arange(op.nglobal))).cuda()
        b = op.mass(r) * torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda()
        rhs.append((b, op))
    return draws, probs, rhs


def test_batch_matches_single_solves():
    draws, probs, rhs = _problems(24, 5)
    batch = pkg.Batch(probs, arith=pkg.ARITH_DF64)
    xs, infos = batch.solve([b for b, _ in rhs], tol=1e-8)
    for k, (b, op) in enumerate(rhs):
        x1, i1 = op.solve(b, tol=1e-8)
        assert infos[k]["status"] == "OK"
        assert abs(infos[k]["iters"][0] - i1["iters"][0]) <= 1, (k, infos[k], i1)
        assert infos[k]["rel_res"][0] <= 1e-8
        err = (torch.linalg.norm(xs[k] - x1) / torch.linalg.norm(x1)).item()
        assert err < 1e-6, (k, err)
    # two members against the oracle
    for k in range(2):
        q = draws[k]
        ref = BakeoffProblem(5, q["k"], q["k"], q["k"], q["N"], amp=q["amp"])
        bh = ref.rhs(uniform_pm1(q["rhs_seed"], np.arange(ref.n_global)))
        xr, ir = ref.solve(bh, tol=1e-8)
        assert abs(infos[k]["iters"][0] - ir[0]["iters"]) <= 1
        assert np.linalg.norm(xs[k].cpu().numpy() - xr) <= 1e-6 * np.linalg.norm(xr)
    # the same batch again (graphs reused) gives identical bits
    xs2, infos2 = batch.solve([b for b, _ in rhs], tol=1e-8)
    assert all(torch.equal(a, c) for a, c in zip(xs, xs2))
    batch.close()


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_batch_without_graphs_and_single_member(arith):
    draws, probs, rhs = _problems(3, 3, arith)
    batch = pkg.Batch(probs[:1], arith=arith)
    xs, infos = batch.solve([rhs[0][0]], tol=1e-10, use_graph=False, chunk=5)
    x1, i1 = rhs[0][1].solve(rhs[0][0], tol=1e-10)
    assert abs(infos[0]["iters"][0] - i1["iters"][0]) <= 1
    batch.close()


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_batch_every_small_member_against_oracle(arith):
    """Every member of a 16-problem batch (k <= 4, orders 3, 5, 7) solved to 1e-10 against the
    oracle's PCG (iterations within 1, both residuals at the tolerance, solution difference printed
    and bounded) and against its own single-problem solve, in both arithmetics."""
    draws, probs, rhs = _problems(16, 4, arith, seed=11)
    assert {q["N"] for q in draws} == {3, 5, 7}
    batch = pkg.Batch(probs, arith=arith)
    xs, infos = batch.solve([b for b, _ in rhs], tol=1e-10)
    worst = 0.0
    for k, q in enumerate(draws):
        assert infos[k]["status"] == "OK" and infos[k]["rel_res"][0] <= 1e-10
        ref = BakeoffProblem(5, q["k"], q["k"], q["k"], q["N"], amp=q["amp"])
        bh = ref.rhs(uniform_pm1(q["rhs_seed"], np.arange(ref.n_global)))
        xr, ir = ref.solve(bh, tol=1e-10)
        assert ir[0]["converged"]
        assert abs(infos[k]["iters"][0] - ir[0]["iters"]) <= 1, (k, q, infos[k]["iters"], ir[0]["iters"])
        err = np.linalg.norm(xs[k].cpu().numpy() - xr) / np.linalg.norm(xr)
        worst = max(worst, err)
        assert err <= 1e-8, (k, q, err)
        x1, i1 = rhs[k][1].solve(rhs[k][0], tol=1e-10)
        assert abs(infos[k]["iters"][0] - i1["iters"][0]) <= 1
    print(f"batch arith={arith}, 16 members vs oracle: worst |x - x_oracle| / |x_oracle| = {worst:.2e}")
    batch.close()


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_batch_largest_member_on_sampled_rows(arith):
    """The largest member of a batch (up to k = 12) checked by the oracle on >= 200 sampled rows:
    (b - A x) at those rows stays within the solve tolerance of |b|."""
    draws, probs, rhs = _problems(12, 12, arith, seed=5)
    batch = pkg.Batch(probs, arith=arith)
    xs, infos = batch.solve([b for b, _ in rhs], tol=1e-10)
    big = max(range(len(draws)), key=lambda i: draws[i]["k"] ** 3 * draws[i]["N"] ** 3)
    q = draws[big]
    dims = (q["k"], q["k"], q["k"])
    nodes = probe_nodes(dims, q["N"], seed=big)
    assert len(nodes) >= 200
    x_h = xs[big].cpu().numpy()
    b_h = rhs[big][0].cpu().numpy()
    ax = sampled_rows(5, *dims, q["N"], q["amp"], lambda ids: x_h[ids], nodes)
    res = np.linalg.norm(b_h[nodes] - ax) / np.linalg.norm(b_h)
    print(f"batch arith={arith}: largest member k={q['k']} N={q['N']}: sampled residual {res:.2e}")
    assert infos[big]["status"] == "OK"
    assert res <= 1e-9, res
    batch.close()


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_batch_even_orders(arith):
    """Even orders (2, 4, 6: the column kernel in FP64, the pair kernel's other shapes) batched:
    every member within one iteration of its single solve, two members against the oracle."""
    draws, probs, rhs = _problems(10, 4, arith, seed=7, orders=(2, 4, 6))
    assert {q["N"] for q in draws} == {2, 4, 6}
    batch = pkg.Batch(probs, arith=arith)
    xs, infos = batch.solve([b for b, _ in rhs], tol=1e-10)
    for k, (b, op) in enumerate(rhs):
        x1, i1 = op.solve(b, tol=1e-10)
        assert infos[k]["status"] == "OK" and infos[k]["rel_res"][0] <= 1e-10
        assert abs(infos[k]["iters"][0] - i1["iters"][0]) <= 1
    for k in range(2):
        q = draws[k]
        ref = BakeoffProblem(5, q["k"], q["k"], q["k"], q["N"], amp=q["amp"])
        bh = ref.rhs(uniform_pm1(q["rhs_seed"], np.arange(ref.n_global)))
        xr, ir = ref.solve(bh, tol=1e-10)
        assert abs(infos[k]["iters"][0] - ir[0]["iters"]) <= 1
        assert np.linalg.norm(xs[k].cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)
    batch.close()
