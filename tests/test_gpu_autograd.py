"""torch.autograd through the transport solve: forward = batched sweep, backward = adjoint sweep.
Gradients of L = sum((Gamma - T)^2) + sum(c * J) are compared with the oracle's adjoint of the same
loss, whose dL/dGamma is formed from the oracle's own Gamma."""
import numpy as np
import pytest

import oracle
from synth import configs

pytestmark = pytest.mark.gpu


def _rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _setup(ctx, seed):
    p = configs.voronoi_small(3000, n_dir=16, n_groups=2, seed=seed, n_src=6)
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    rng = np.random.default_rng(seed + 1)
    T = rng.random(p.kappa_abs.shape) * 1e-3
    c = rng.normal(size=p.kappa_abs.shape)
    return p, T, c


def _oracle_grads(p, T, c):
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, threads=8)
    rc, gk, ge = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, dl_dJ=c,
                                dl_dGamma=2.0 * (r["Gamma"] - T), threads=8)
    assert rc == 0
    return r, gk, ge


@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-4)])
def test_autograd_gradients_match_oracle_adjoint(ctx, precision, tol):
    torch = pytest.importorskip("torch")
    from paper_2207_12848_gb300 import transport_solve
    p, T, c = _setup(ctx, 71)
    ka = torch.tensor(p.kappa_abs, dtype=torch.float64, device="cuda", requires_grad=True)
    em = torch.tensor(p.emissivity, dtype=torch.float64, device="cuda", requires_grad=True)
    J, Gamma = transport_solve(ctx, ka, em, precision=precision, schedule="dataflow")
    loss = ((Gamma - torch.tensor(T, device="cuda")) ** 2).sum() + (torch.tensor(c, device="cuda") * J).sum()
    gk, ge = torch.autograd.grad(loss, (ka, em))
    r, ok_, oe = _oracle_grads(p, T, c)
    assert _rel_max(J.detach().cpu().numpy(), r["J"]) <= tol
    assert _rel_max(gk.cpu().numpy(), ok_) <= tol
    assert _rel_max(ge.cpu().numpy(), oe) <= tol


def test_autograd_only_gamma_used_and_context_reused(ctx):
    # the loss ignores J (its incoming gradient is None/zero); a second solve with other material on
    # the same context between forward and backward must not change the gradient
    torch = pytest.importorskip("torch")
    from paper_2207_12848_gb300 import transport_solve
    p, T, c = _setup(ctx, 73)
    ka = torch.tensor(p.kappa_abs, dtype=torch.float64, device="cuda", requires_grad=True)
    em = torch.tensor(p.emissivity, dtype=torch.float64, device="cuda", requires_grad=True)
    _, Gamma = transport_solve(ctx, ka, em, precision=64)
    loss = ((Gamma - torch.tensor(T, device="cuda")) ** 2).sum()
    with torch.no_grad():
        transport_solve(ctx, 2.0 * ka, em, precision=64)
    gk, ge = torch.autograd.grad(loss, (ka, em))
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, threads=8)
    rc, ok_, oe = oracle.adjoint(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity,
                                 dl_dGamma=2.0 * (r["Gamma"] - T), threads=8)
    assert rc == 0
    assert _rel_max(gk.cpu().numpy(), ok_) <= 1e-9
    assert _rel_max(ge.cpu().numpy(), oe) <= 1e-9


@pytest.mark.parametrize("kind", ["scattering", "periodic", "both"])
def test_autograd_through_the_iterations(ctx, kind):
    # forward the scattering and/or periodic iterations, backward their transpose; kappa_scat as a
    # third differentiable input where there is scattering
    torch = pytest.importorskip("torch")
    from paper_2207_12848_gb300 import transport_solve
    scat, box = kind != "periodic", kind != "scattering"
    p = configs.voronoi_small(3000, periodic_box=box, n_dir=12, n_groups=2, seed=75,
                              scatter_albedo=0.5 if scat else 0.0, n_src=6)
    ctx.set_mesh(p.mesh)
    ctx.set_directions(p.omega, p.weight)
    rng = np.random.default_rng(76)
    T = rng.random(p.kappa_abs.shape) * 1e-3
    c = rng.normal(size=p.kappa_abs.shape)
    it = dict(tol_scat=1e-12, max_it_scat=2000, tol_pbc=1e-12, max_it_pbc=2000)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
    ka, em = dev(p.kappa_abs), dev(p.emissivity)
    ks = dev(p.kappa_scat) if scat else None
    J, Gamma = transport_solve(ctx, ka, em, ks, precision=64, **it)
    loss = ((Gamma - torch.tensor(T, device="cuda")) ** 2).sum() + (torch.tensor(c, device="cuda") * J).sum()
    grads = torch.autograd.grad(loss, (ka, em, ks) if scat else (ka, em))
    k_s = p.kappa_scat if scat else None
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=k_s, threads=8, **it)
    o = oracle.adjoint_full(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, kappa_scat=k_s, dl_dJ=c,
                            dl_dGamma=2.0 * (r["Gamma"] - T), threads=8, **it)
    assert _rel_max(J.detach().cpu().numpy(), r["J"]) <= 1e-9
    names = ("grad_kappa_abs", "grad_emissivity", "grad_kappa_scat")
    for gr, name in zip(grads, names):
        assert _rel_max(gr.cpu().numpy(), o[name]) <= 1e-8, name

