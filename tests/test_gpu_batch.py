"""Batched BP5 solves: every problem of a batch of uneven sizes and orders
matches its own single-problem solve (iteration counts within 1, residuals at
the tolerance) and, for small members, the CPU FP64 oracle."""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.problems import BakeoffProblem
from synth import batched_problems, uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _problems(n, k_max):
    draws = batched_problems(n_problems=n, seed=3, k_max=k_max)
    probs, rhs, meshes = [], [], []
    for q in draws:
        coords, l2g, dirichlet = pkg.mesh_box(q["k"], q["k"], q["k"], q["N"], q["amp"])
        probs.append((q["N"], coords, l2g, dirichlet))
        meshes.append((q, coords, l2g, dirichlet))
        op = pkg.Operator(5, q["N"], coords, l2g, dirichlet, arith=pkg.ARITH_DF64)
        r = torch.from_numpy(uniform_pm1(q["rhs_seed"], np.arange(op.nglobal))).cuda()
        b = op.mass(r) * torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda()
        rhs.append((b, op))
    return draws, probs, rhs


def test_batch_matches_single_solves():
    draws, probs, rhs = _problems(24, 5)
    batch = pkg.Batch(probs)
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


def test_batch_without_graphs_and_single_member():
    draws, probs, rhs = _problems(3, 3)
    batch = pkg.Batch(probs[:1])
    xs, infos = batch.solve([rhs[0][0]], tol=1e-10, use_graph=False, chunk=5)
    x1, i1 = rhs[0][1].solve(rhs[0][0], tol=1e-10)
    assert abs(infos[0]["iters"][0] - i1["iters"][0]) <= 1
    batch.close()
