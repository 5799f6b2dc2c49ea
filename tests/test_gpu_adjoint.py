"""Discrete adjoint (FP64 path): dg_rhs_vjp and dg_adjoint_step against finite differences,
the gradient of an interface functional with respect to level-set parameters against central
differences of the GPU forward map and of the oracle's forward map (relative 1e-6), and the
same gradient through torch.autograd with the DGTrajectory function.

The right-hand side has kinks (lambda = max of the one-sided wave speeds at every face), so a
finite difference is only as good as the number of kinks its step straddles.  Column by
column on a tiny mesh (few faces) a step of 1e-6 of the variable's scale straddles none and
keeps round-off at ~1e-7 (tolerance 1e-5); a directional difference on a large mesh needs
1e-9 (tolerance 2e-6).  The parameter gradients use Richardson-extrapolated central
differences (steps h and h/2, truncation O(h^4)) in the 16 level-set coefficients."""
import numpy as np
import pytest

from paper_2306_05002_gb300 import workloads as W
from tests.helpers import mass_weights, problem

pytestmark = pytest.mark.gpu


def _broken(wl, seed=3, amp=0.05):
    import oracle
    rng = np.random.default_rng(seed)
    prim = oracle.primitives(oracle.Problem(**wl.problem_kwargs()), wl.w)
    phi = np.clip(wl.w[0] + amp * rng.uniform(-1, 1, wl.N), 0.02, 0.98)
    psi = wl.w[1] + amp * rng.uniform(-1, 1, wl.N)
    P = prim[3] * (1 + 0.02 * rng.uniform(-1, 1, wl.N))
    u = prim[1] + 0.3 + 0.05 * rng.uniform(-1, 1, wl.N)
    v = prim[2] - 0.2 + 0.05 * rng.uniform(-1, 1, wl.N)
    if wl.dim == 1:
        v = 0.0 * v  # the 1D state keeps rho v = 0
    return np.array(W.conserved(wl, phi, psi, P, u, v))  # a writable copy (torch.from_numpy shares it)


@pytest.mark.parametrize("maker", [lambda: W.drop_2d(n=3, p=2, seed=2), lambda: W.drop_2d(n=2, p=3, seed=3),
                                   lambda: W.drop_2d(n=2, p=4, seed=4, water_inside=False),
                                   lambda: W.slab_1d(nx=5, p=3)])
def test_vjp_against_oracle_jacobian(orc, dg, maker):
    """mu = J^T lam with J the oracle's Jacobian by central differences, column by column."""
    import torch
    wl = maker()
    w = _broken(wl)
    pb = problem(orc, wl)
    rng = np.random.default_rng(1)
    scale = np.abs(w).max(axis=1, keepdims=True)
    Lmax = np.abs(orc.rhs(pb, w)).max(axis=1, keepdims=True)
    lam = rng.normal(size=w.shape) / np.where(Lmax > 0, Lmax, 1.0)
    if wl.dim == 1:
        lam[5] = 0.0  # rho v is not a variable of the 1D model (its state keeps rho v = 0)
    mu_fd = np.zeros_like(w)
    for v in range(7):
        for j in range(wl.N):
            h = 1e-6 * max(scale[v, 0], 1e-3)
            wp, wm = w.copy(), w.copy()
            wp[v, j] += h
            wm[v, j] -= h
            col = (orc.rhs(pb, wp) - orc.rhs(pb, wm)) / (2 * h)
            mu_fd[v, j] = np.sum(lam * col)
    s = dg.Solver(wl)
    mu = s.dg_rhs_vjp(torch.from_numpy(w.copy()).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    s.close()
    for v in range(7):
        if wl.dim == 1 and v == 5:
            continue
        ref = np.abs(mu_fd[v]).max()
        assert np.abs(mu[v] - mu_fd[v]).max() <= 1e-5 * ref, (v, np.abs(mu[v] - mu_fd[v]).max() / ref)


@pytest.mark.parametrize("maker", [lambda: W.drop_2d(n=16, p=3, seed=2), lambda: W.slab_1d(nx=40, p=4),
                                   lambda: W.drop_2d(n=8, p=5, seed=7, water_inside=False)])
def test_vjp_dot_product_with_directional_difference(dg, maker):
    """<lam, J v> (central difference of dg_rhs along v) = <J^T lam, v>."""
    import torch
    wl = maker()
    w = torch.from_numpy(_broken(wl)).cuda()
    g = torch.Generator(device="cpu").manual_seed(0)
    scale = w.abs().amax(dim=1, keepdim=True)
    vdir = (torch.randn(w.shape, generator=g, dtype=torch.float64).cuda()) * scale
    if wl.dim == 1:
        vdir[5] = 0.0  # the 1D state keeps rho v = 0
    s = dg.Solver(wl)
    L0 = s.dg_rhs(w)
    Lmax = L0.abs().amax(dim=1, keepdim=True)
    lam = torch.randn(w.shape, generator=g, dtype=torch.float64).cuda() / torch.where(Lmax > 0, Lmax, 1.0)
    h = 1e-9
    Jv = (s.dg_rhs(w + h * vdir) - s.dg_rhs(w - h * vdir)) / (2 * h)
    mu = s.dg_rhs_vjp(w, lam)
    lhs = float((lam * Jv).sum())
    rhs = float((mu * vdir).sum())
    s.close()
    assert abs(lhs - rhs) <= 2e-6 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_adjoint_step_dot_product(dg):
    """<lam_{n+1}, dPhi v> (central difference of one SSP-RK3 step) = <lam_n, v>."""
    import torch
    wl = W.drop_2d(n=16, p=3, seed=4)
    w = torch.from_numpy(_broken(wl, amp=0.01)).cuda()
    g = torch.Generator(device="cpu").manual_seed(2)
    scale = w.abs().amax(dim=1, keepdim=True)
    vdir = torch.randn(w.shape, generator=g, dtype=torch.float64).cuda() * scale
    lam1 = torch.randn(w.shape, generator=g, dtype=torch.float64).cuda() / scale
    s = dg.Solver(wl)
    h = 1e-9
    wp, wm = (w + h * vdir).contiguous(), (w - h * vdir).contiguous()
    s.dg_step(wp, wl.dt, 1)
    s.dg_step(wm, wl.dt, 1)
    lhs = float((lam1 * (wp - wm) / (2 * h)).sum())
    lam0 = s.dg_adjoint_step(w, lam1, wl.dt)
    rhs = float((lam0 * vdir).sum())
    # in place (lam_n aliasing lam_{n+1}) gives the same result
    lam_alias = lam1.clone()
    s.dg_adjoint_step(w, lam_alias, wl.dt, lam_n=lam_alias)
    # the taped step reproduces dg_step, and its reverse reproduces dg_adjoint_step
    tape = torch.empty(s.dg_tape_len(), dtype=torch.float64, device="cuda")
    wt, ws = w.clone(), w.clone()
    s.dg_step_tape(wt, wl.dt, tape)
    s.dg_step(ws, wl.dt, 1)
    lam_t = s.dg_adjoint_step_tape(w, tape, lam1, wl.dt)
    s.close()
    assert abs(lhs - rhs) <= 2e-6 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    assert torch.equal(lam_alias, lam0)
    assert torch.equal(wt, ws)
    assert torch.equal(lam_t, lam0)


def test_adjoint_step_dot_product_full_size(dg):
    """The same identity on the 128 x 128, p = 3 drop the benchmark's adjoint block differentiates
    (262,144 nodes, the level-set parametrisation with seeded coefficients): the adjoint step is
    the transpose of the step's Jacobian at full size."""
    import torch
    wl = W.adjoint_drop(n=128, p=3, theta=np.random.default_rng(50).normal(0, 0.01, 16), nsteps=1)
    w = torch.from_numpy(wl.w.copy()).cuda()
    g = torch.Generator(device="cpu").manual_seed(3)
    scale = w.abs().amax(dim=1, keepdim=True)
    vdir = torch.randn(w.shape, generator=g, dtype=torch.float64).cuda() * scale
    lam1 = torch.randn(w.shape, generator=g, dtype=torch.float64).cuda() / scale
    s = dg.Solver(wl)
    h = 1e-9
    wp, wm = (w + h * vdir).contiguous(), (w - h * vdir).contiguous()
    s.dg_step(wp, wl.dt, 1)
    s.dg_step(wm, wl.dt, 1)
    lhs = float((lam1 * (wp - wm) / (2 * h)).sum())
    rhs = float((s.dg_adjoint_step(w, lam1, wl.dt) * vdir).sum())
    s.close()
    assert abs(lhs - rhs) <= 2e-6 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _objective(orc, wl, wN, target):
    M = mass_weights(orc, wl)
    return 0.5 * np.sum(M * (wN[0] - target) ** 2), M


def _richardson(J, theta, k, h=1e-5):
    """dJ/dtheta_k by Richardson-extrapolated central differences (steps h and h/2)."""
    def d(step):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += step
        tm[k] -= step
        return (J(tp) - J(tm)) / (2 * step)
    return (4.0 * d(0.5 * h) - d(h)) / 3.0


GRAD_RTOL = 1e-6


def test_level_set_parameter_gradient(orc, dg):
    """dJ/dtheta by the adjoint (checkpointed trajectory) against central differences of J
    through the GPU forward map; J = 1/2 int (alpha_N - alpha*)^2, alpha* from other parameters."""
    import torch
    from paper_2306_05002_gb300 import adjoint as A
    n, steps, every = 16, 30, 7
    base = W.adjoint_drop(n=n, p=3, nsteps=steps)
    theta = np.array(base.meta["theta"])
    tgt_wl = W.adjoint_drop(n=n, p=3, nsteps=steps, theta=np.random.default_rng(51).normal(0, 0.01, 16))
    s = dg.Solver(base)
    dt = base.dt

    def run(wl):
        x = torch.from_numpy(wl.w.copy()).cuda()
        s.dg_step(x, dt, steps)
        return x.cpu().numpy()
    target = run(tgt_wl)[0]
    wN, ckpt = A.forward(s, torch.from_numpy(base.w.copy()).cuda(), dt, steps, every)
    J, M = _objective(orc, base, wN.cpu().numpy(), target)
    lamN = torch.zeros_like(wN)
    lamN[0] = torch.from_numpy(M * (wN[0].cpu().numpy() - target)).cuda()
    lam0 = A.backward(s, ckpt, lamN, dt, steps, every).cpu().numpy()
    lam0_recompute = A.backward(s, ckpt, lamN, dt, steps, every, tape=False).cpu().numpy()
    np.testing.assert_array_equal(lam0, lam0_recompute)
    modes = W.level_set_modes(base, base.meta["cx"], base.meta["cy"])
    grad = -(modes @ lam0[1])          # psi0 = ... - theta . modes

    def Jof(th):
        return _objective(orc, base, run(W.adjoint_drop(n=n, p=3, nsteps=steps, theta=th)), target)[0]
    fd = np.array([_richardson(Jof, theta, k) for k in range(16)])
    s.close()
    assert J > 0
    np.testing.assert_allclose(grad, fd, rtol=GRAD_RTOL, atol=GRAD_RTOL * np.abs(fd).max())


def test_level_set_parameter_gradient_against_oracle(orc, dg):
    """The same gradient on a small mesh against central differences of the oracle's own
    forward map (the oracle-derived reference gradient)."""
    import torch
    from paper_2306_05002_gb300 import adjoint as A
    n, steps = 6, 8
    base = W.adjoint_drop(n=n, p=2, nsteps=steps)
    theta = np.array(base.meta["theta"])
    pb = problem(orc, base)
    dt = base.dt
    target = orc.rk3(pb, W.adjoint_drop(n=n, p=2, nsteps=steps,
                                        theta=np.random.default_rng(51).normal(0, 0.01, 16)).w, dt, steps)[0]
    s = dg.Solver(base)
    wN, ckpt = A.forward(s, torch.from_numpy(base.w.copy()).cuda(), dt, steps, 3)
    M = mass_weights(orc, base)
    lamN = torch.zeros_like(wN)
    lamN[0] = torch.from_numpy(M * (wN[0].cpu().numpy() - target)).cuda()
    lam0 = A.backward(s, ckpt, lamN, dt, steps, 3).cpu().numpy()
    s.close()
    modes = W.level_set_modes(base, base.meta["cx"], base.meta["cy"])
    grad = -(modes @ lam0[1])

    def Jof(th):
        return _objective(orc, base, orc.rk3(pb, W.adjoint_drop(n=n, p=2, nsteps=steps, theta=th).w, dt, steps),
                          target)[0]
    fd = np.array([_richardson(Jof, theta, k) for k in range(16)])
    np.testing.assert_allclose(grad, fd, rtol=GRAD_RTOL, atol=GRAD_RTOL * np.abs(fd).max())


def test_dgtrajectory_autograd_gradient(orc, dg):
    """DGTrajectory, the torch.autograd.Function over checkpointed SSP-RK3 trajectories: the
    initial level set is built in torch from the 16 coefficients theta (psi0 = psi_circle -
    theta . modes), J = 1/2 int (alpha_N - alpha*)^2 is formed in torch, and torch.autograd.grad
    returns dJ/dtheta -- against Richardson central differences of J through the GPU forward map.
    The gradient with respect to the whole initial state equals the checkpointed adjoint sweep."""
    import torch
    from paper_2306_05002_gb300 import adjoint as A
    from paper_2306_05002_gb300.adjoint import DGTrajectory
    n, steps, every = 12, 24, 5
    base = W.adjoint_drop(n=n, p=3, nsteps=steps)
    theta_np = np.array(base.meta["theta"])
    modes_np = W.level_set_modes(base, base.meta["cx"], base.meta["cy"])
    s = dg.Solver(base)
    dt = base.dt
    tgt = W.adjoint_drop(n=n, p=3, nsteps=steps, theta=np.random.default_rng(51).normal(0, 0.01, 16))
    xt = torch.from_numpy(tgt.w.copy()).cuda()
    s.dg_step(xt, dt, steps)
    target = xt[0].clone()
    M = torch.from_numpy(mass_weights(orc, base)).cuda()
    w_base = torch.from_numpy(base.w.copy()).cuda()
    modes = torch.from_numpy(modes_np).cuda()
    psi_circle = w_base[1] + torch.from_numpy(theta_np).cuda() @ modes

    def initial_state(theta):
        return torch.cat([w_base[:1], (psi_circle - theta @ modes)[None], w_base[2:]]).contiguous()

    theta = torch.tensor(theta_np, dtype=torch.float64, device="cuda", requires_grad=True)
    w0 = initial_state(theta)
    wN = DGTrajectory.apply(w0, s, dt, steps, every)
    J = 0.5 * (M * (wN[0] - target) ** 2).sum()
    (g_theta,) = torch.autograd.grad(J, theta)
    g_theta = g_theta.cpu().numpy()

    # the state gradient through autograd equals the checkpointed adjoint sweep bit for bit
    w0_leaf = initial_state(torch.from_numpy(theta_np).cuda()).requires_grad_(True)
    wN2 = DGTrajectory.apply(w0_leaf, s, dt, steps, every)
    (g_w0,) = torch.autograd.grad(0.5 * (M * (wN2[0] - target) ** 2).sum(), w0_leaf)
    lamN = torch.zeros_like(wN2)
    lamN[0] = M * (wN2[0].detach() - target)
    _, ckpt = A.forward(s, w0_leaf.detach(), dt, steps, every)
    assert torch.equal(g_w0, A.backward(s, ckpt, lamN, dt, steps, every))

    def Jof(th):
        with torch.no_grad():
            x = initial_state(torch.from_numpy(th).cuda())
            s.dg_step(x, dt, steps)
            return float(0.5 * (M * (x[0] - target) ** 2).sum())
    fd = np.array([_richardson(Jof, theta_np, k) for k in range(16)])
    s.close()
    np.testing.assert_allclose(g_theta, fd, rtol=GRAD_RTOL, atol=GRAD_RTOL * np.abs(fd).max())


def test_dgrhs_autograd(dg):
    """DGRHS, the torch.autograd.Function of one right-hand side: its gradient is dg_rhs_vjp bit for
    bit, and <grad, v> matches a central difference of <lam, L(w)> along v (h = 1e-9, 2e-6)."""
    import torch
    from paper_2306_05002_gb300.adjoint import DGRHS
    wl = W.drop_2d(n=8, p=3, seed=2)
    s = dg.Solver(wl)
    w0 = torch.from_numpy(_broken(wl)).cuda()
    g = torch.Generator(device="cpu").manual_seed(4)
    lam = torch.randn(w0.shape, generator=g, dtype=torch.float64).cuda()
    lam /= s.dg_rhs(w0).abs().amax(dim=1, keepdim=True)
    w = w0.clone().requires_grad_(True)
    J = (lam * DGRHS.apply(w, s)).sum()
    (grad,) = torch.autograd.grad(J, w)
    assert torch.equal(grad, s.dg_rhs_vjp(w0, lam))
    vdir = torch.randn(w0.shape, generator=g, dtype=torch.float64).cuda() * w0.abs().amax(dim=1, keepdim=True)
    h = 1e-9
    with torch.no_grad():
        lhs = float(((lam * s.dg_rhs(w0 + h * vdir)).sum() - (lam * s.dg_rhs(w0 - h * vdir)).sum()) / (2 * h))
    rhs = float((grad * vdir).sum())
    s.close()
    assert abs(lhs - rhs) <= 2e-6 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_adjoint_rejects_pressure_boundary(dg):
    """The discrete adjoint covers periodic and wall boundaries; a pressure boundary is refused."""
    import torch
    wl = W.rayleigh_taylor_paper(nx=2, ny=4, p=2)
    wl.viscous = False
    s = dg.Solver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    with pytest.raises(dg.DGError):
        s.dg_rhs_vjp(w, w.clone())
    s.close()

