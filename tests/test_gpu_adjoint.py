"""Adjoint gradient dJ/dkappa for -div(kappa grad u) = f (BP5 collocated):
the fused gradient kernel against the oracle's gradient, the whole
forward/adjoint pipeline against the oracle, central finite differences
(h = 1e-6) and the torch.autograd wrapper."""
import numpy as np
import pytest
import torch

import paper_2004_06722_gb300 as pkg
from oracle.adjoint import forward_adjoint, gradient
from oracle.mesh import box_mesh
from oracle.problems import BakeoffProblem
from synth import fourier_field, fourier_modes, uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def _setup(dims, N, arith=pkg.ARITH_FP64):
    coords, l2g, dirichlet = pkg.mesh_box(*dims, N, 0.05)
    kappa = np.exp(fourier_field(fourier_modes(0), coords))        # collocated: quadrature points = nodes
    kappa_star = np.exp(fourier_field(fourier_modes(1), coords))
    op = pkg.Operator(5, N, coords, l2g, dirichlet, kappa=kappa, arith=arith)
    op.free = 1.0 - dirichlet.astype(np.float64)
    mask = torch.from_numpy(op.free).cuda()
    r = torch.from_numpy(uniform_pm1(0, np.arange(op.nglobal))).cuda()
    b = op.mass(r) * mask
    return op, kappa, kappa_star, b


def _oracle_kappas(dims, N):
    """kappa and kappa* at the oracle's own quadrature points (the mesh nodes)."""
    oc, _ = box_mesh(*dims, N, 0.05)
    return np.exp(fourier_field(fourier_modes(0), oc)), np.exp(fourier_field(fourier_modes(1), oc))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,dims", [(2, (2, 2, 2)), (3, (2, 2, 1)), (7, (2, 1, 1))])
def test_gradient_kernel_matches_oracle(N, dims):
    op, kappa, kappa_star, b = _setup(dims, N)
    ko, _ = _oracle_kappas(dims, N)
    ref = BakeoffProblem(5, *dims, N, amp=0.05, kappa=ko)
    u = uniform_pm1(3, np.arange(op.nglobal))
    lam = uniform_pm1(4, np.arange(op.nglobal))
    g = op.kappa_gradient(torch.from_numpy(u * op.free).cuda(), torch.from_numpy(lam * op.free).cuda()).cpu().numpy()
    assert _rel(g, gradient(ref, u * ref.free, lam * ref.free)) < 1e-12


@pytest.mark.parametrize("arith", [pkg.ARITH_FP64, pkg.ARITH_DF64])
def test_forward_adjoint_pipeline_matches_oracle(arith):
    dims, N = (2, 2, 2), 4
    op, kappa, kappa_star, b = _setup(dims, N, arith)
    ko, ko_star = _oracle_kappas(dims, N)
    ref = BakeoffProblem(5, *dims, N, amp=0.05, kappa=ko)
    ref_star = BakeoffProblem(5, *dims, N, amp=0.05, kappa=ko_star)
    bh = ref.rhs(uniform_pm1(0, np.arange(ref.n_global)))
    u_star_ref, _ = ref_star.solve(bh, tol=1e-14)
    u_ref, lam_ref, J_ref, _ = forward_adjoint(ref, bh, u_star_ref, tol=1e-14)
    g_ref = gradient(ref, u_ref, lam_ref)
    # GPU: u* with kappa*, then u, lambda, g with kappa
    op.set_kappa(torch.from_numpy(kappa_star).cuda())
    u_star, _ = op.solve(b, tol=1e-13)
    u_star = u_star.clone()
    op.set_kappa(torch.from_numpy(kappa).cuda())
    u, _ = op.solve(b, tol=1e-13)
    rhs, J = op.misfit(u, u_star)
    lam, _ = op.solve(rhs, tol=1e-13)
    g = op.kappa_gradient(u, lam).cpu().numpy()
    assert abs(J - J_ref) <= 1e-9 * abs(J_ref)
    assert _rel(g, g_ref) < 1e-8


def test_gradient_matches_central_differences_and_autograd():
    dims, N = (3, 3, 3), 5
    op, kappa, kappa_star, b = _setup(dims, N)
    op.set_kappa(torch.from_numpy(kappa_star).cuda())
    u_star, _ = op.solve(b, tol=1e-14)
    u_star = u_star.clone()
    k = torch.from_numpy(kappa).cuda().requires_grad_(True)
    J = pkg.kappa_misfit(k, op, b, u_star, tol=1e-14)
    (gk,) = torch.autograd.grad(J, k)
    g = gk.detach()

    def Jof(kap):
        op.set_kappa(kap)
        u, _ = op.solve(b, tol=1e-14)
        _, val = op.misfit(u, u_star)
        return val

    rng = np.random.default_rng(5)
    h = 1e-6
    k0 = torch.from_numpy(kappa).cuda()
    for _ in range(6):
        d = torch.from_numpy(rng.uniform(-1, 1, size=kappa.shape)).cuda()
        d /= d.abs().max()
        fd = (Jof(k0 + h * d) - Jof(k0 - h * d)) / (2 * h)
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_central_differences_at_16_cubed_both_measures():
    """E = 16^3, N = 7 (1.4e6 DOFs, 2.1e6 kappa values), the benchmark's adjoint workload at a
    reduced size: forcing f = 1, kappa = exp(g) from 16 Fourier modes, 20 random directions
    (entries U[-1, 1], max 1) and 5 smooth ones (log-kappa Fourier perturbations).  Central
    differences with h = 1e-6 and solves to 1e-13 against <grad J, d>: the plain relative
    error within the 1e-6 bar on every direction, and the error in the scale of the direction,
    |fd - <g,d>| / sum |g_i d_i|, within 1e-9."""
    E1, N = 16, 7
    coords, l2g, dirichlet = pkg.mesh_box(E1, E1, E1, N, 0.05)
    kappa = torch.from_numpy(np.exp(fourier_field(fourier_modes(0), coords))).cuda()
    kappa_star = torch.from_numpy(np.exp(fourier_field(fourier_modes(1), coords))).cuda()
    op = pkg.Operator(5, N, coords, l2g, dirichlet)
    mask = torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda()
    b = op.mass(torch.ones(op.nglobal, dtype=torch.float64, device="cuda")) * mask
    op.set_kappa(kappa_star)
    u_star, _ = op.solve(b, tol=1e-13, chunk=64)
    u_star = u_star.clone()
    k = kappa.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(pkg.kappa_misfit(k, op, b, u_star, tol=1e-13), k)

    def Jof(kap):
        op.set_kappa(kap)
        u, _ = op.solve(b, tol=1e-13, chunk=64)
        return op.misfit(u, u_star)[1]

    h = 1e-6
    rng = np.random.default_rng(20)
    plain, scaled, smooth = [], [], []
    for _ in range(20):
        d = torch.from_numpy(rng.uniform(-1, 1, size=tuple(kappa.shape))).cuda()
        d /= d.abs().max()
        fd = (Jof(kappa + h * d) - Jof(kappa - h * d)) / (2 * h)
        ad = float((g * d).sum())
        plain.append(abs(fd - ad) / abs(ad))
        scaled.append(abs(fd - ad) / float((g * d).abs().sum()))
    for sd in range(100, 105):
        d = torch.from_numpy(fourier_field(fourier_modes(sd), coords)).cuda()
        d /= d.abs().max()
        fd = (Jof(kappa + h * d * kappa) - Jof(kappa - h * d * kappa)) / (2 * h)
        ad = float((g * d * kappa).sum())
        smooth.append(abs(fd - ad) / abs(ad))
    print(f"E=16^3 FD: plain max {max(plain):.2e} median {np.median(plain):.2e}, scaled max {max(scaled):.2e}, "
          f"smooth max {max(smooth):.2e}")
    assert max(plain) <= 1e-6
    assert max(scaled) <= 1e-9
    assert max(smooth) <= 1e-6
    op.close()
