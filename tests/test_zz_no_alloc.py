"""ceedbp_apply_noalloc against ceedbp_apply, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc
where they apply the operator (a global-mode stream capture held by another
thread, memory owned by another allocator, time-critical loops).  It must give
the same w as ceedbp_apply on consecutive calls (the static scratch keeps the
previous call's contents), and refuse problems larger than its scratch.  This
file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _noalloc(op, u, w):
    lib = pkg.load_library()
    torch.cuda.synchronize()
    st = lib.ceedbp_apply_noalloc(op.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                  ctypes.c_void_p(op.stream.cuda_stream))
    op.stream.synchronize()
    return st


@pytest.mark.parametrize("bp,N,dims", [(5, 7, (4, 4, 4)), (3, 3, (3, 2, 2)), (6, 2, (2, 2, 2)), (1, 5, (2, 2, 1))])
def test_noalloc_matches_apply_twice(bp, N, dims):
    op = pkg.Operator.box(bp, *dims, N, amp=0.05)
    shape = (op.nglobal,) if op.ncomp == 1 else (op.nglobal, 3)
    for seed in (1, 2):  # two calls in a row, different inputs
        u = torch.from_numpy(uniform_pm1(seed, np.arange(op.nglobal * op.ncomp)).reshape(shape)).cuda()
        ref = op.apply(u).clone()
        torch.cuda.synchronize()
        w = torch.full_like(ref, float("nan"))
        assert _noalloc(op, u, w) == pkg.OK
        err = (torch.linalg.norm(w - ref) / torch.linalg.norm(ref)).item()
        assert err <= APPLY_TOL, err
    op.close()


def _twice(op, tol=APPLY_TOL):
    shape = (op.nglobal,) if op.ncomp == 1 else (op.nglobal, 3)
    for seed in (5, 6):  # two calls in a row, different inputs
        u = torch.from_numpy(uniform_pm1(seed, np.arange(op.nglobal * op.ncomp)).reshape(shape)).cuda()
        ref = op.apply(u).clone()
        torch.cuda.synchronize()
        w = torch.full_like(ref, float("nan"))
        assert _noalloc(op, u, w) == pkg.OK
        err = (torch.linalg.norm(w - ref) / torch.linalg.norm(ref)).item()
        assert err <= tol, err


@pytest.mark.parametrize("bp,N,dims", [(5, 7, (4, 4, 2)), (6, 3, (2, 2, 3))])
def test_noalloc_pair_arithmetic(bp, N, dims):
    """Contexts in FP32-pair arithmetic: the pair kernels of ceedbp_apply, with the pair scratch
    in the same static array."""
    op = pkg.Operator.box(bp, *dims, N, amp=0.05, arith=pkg.ARITH_DF64)
    _twice(op)
    op.check()
    op.close()


def test_noalloc_recomputed_factors():
    op = pkg.Operator.box(5, 3, 3, 2, 5, amp=0.05, geom=pkg.GEOM_RECOMPUTE)
    _twice(op)
    op.close()


def test_noalloc_helmholtz_and_kappa():
    """A + beta B (Eq. (17)) and a variable coefficient set on the context are used too."""
    op = pkg.Operator.box(5, 3, 2, 2, 7, amp=0.05)
    kappa = torch.from_numpy(1.0 + 0.5 * uniform_pm1(8, np.arange(op.nelem * 8 ** 3))).cuda()
    op.set_kappa(kappa)
    _twice(op)
    op.set_helmholtz(2.5)
    _twice(op)
    op.close()


def test_noalloc_error_message_is_per_thread():
    big = pkg.Operator.box(5, 16, 16, 33, 7, amp=0.05)
    u = torch.zeros(big.nglobal, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.CeedbpError) as ei:
        big.apply_noalloc(u)
    assert ei.value.status == pkg.EINVAL and "static scratch" in str(ei.value)
    big.close()


def test_noalloc_limit_is_exact():
    """E p1^3 = 2^22 (16 x 16 x 32 elements at N = 7) is accepted and matches
    ceedbp_apply; one more layer of elements is refused before any launch."""
    op = pkg.Operator.box(5, 16, 16, 32, 7, amp=0.05)
    assert op.nelem * 8 ** 3 == 1 << 22
    u = torch.from_numpy(uniform_pm1(3, np.arange(op.nglobal))).cuda()
    ref = op.apply(u).clone()
    w = torch.empty_like(ref)
    assert _noalloc(op, u, w) == pkg.OK
    assert (torch.linalg.norm(w - ref) / torch.linalg.norm(ref)).item() <= APPLY_TOL
    op.close()
    big = pkg.Operator.box(5, 16, 16, 33, 7, amp=0.05)
    u = torch.zeros(big.nglobal, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(u)
    assert _noalloc(big, u, w) == pkg.EINVAL
    big.close()
