"""The hand-written adjoint (immobile particles) against central finite
differences in FP64, and against finite differences taken through the CPU
oracle.  Objective: J = J_drag + A (mean drag magnitude over the run plus the
interface measure at the end)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2004_04080_gb300.workloads import mixture_densities

pytestmark = pytest.mark.gpu

EPS = 1e-12
NAMES = ["tau_A", "tau_B", "G", "zeta_A", "zeta_B"]


def case(walls):
    shape = (16, 14, 12)
    base = dict(hertz_K=20.0, hertz_sigma=8.0, hertz_rcap=7.0)
    if walls:
        base.update(bc=(1, 1, 0), wall_u_lo=(-0.02, 0.0, 0.0), wall_u_hi=(0.02, 0.01, 0.0))
    theta = np.array([0.9, 1.1, 0.9, 0.2, -0.15])
    col = dict(pos=[[5.3, 6.2, 5.1], [11.6, 7.4, 6.3]], radius=[2.6, 2.4])
    a, b = mixture_densities(shape, seed=13, amp=0.05)
    return shape, base, theta, col, a, b


def params_of(base, theta):
    return dict(base, tau=(theta[0], theta[1]), G=theta[2], zeta=(theta[3], theta[4]))


def gpu_objective(shape, base, theta, col, a, b, steps, prec="fp64"):
    """(runner, [J_drag, A])"""
    from paper_2004_04080_gb300.adjoint import AdjointRunner
    from paper_2004_04080_gb300.lbgb import LBLattice

    lat = LBLattice(shape, prec, max_colloids=len(col["pos"]))
    run = AdjointRunner(lat, steps)
    J, A = run.forward(params_of(base, theta), a, b, col)
    return run, np.array([J, A])


def oracle_objective(shape, base, theta, col, a, b, steps):
    o = Oracle(*shape, len(col["pos"]))
    o.set_params(**params_of(base, theta))
    o.init_fields(a, b)
    o.add_colloids(col["pos"], col["radius"], math.inf)
    J = 0.0
    for _ in range(steps):
        o.step(1)
        F = o.term("F_liq")
        J += np.mean(np.sqrt(np.sum(F * F, axis=1) + EPS ** 2))
    J /= steps
    ra, rb, _ = o.get_fields()
    fl = o.owner() < 0
    phi = (ra[fl] - rb[fl]) / (ra[fl] + rb[fl])
    return np.array([J, np.sum(1 - phi * phi)])


def check(ad, fd, what, floor=1e-9):
    assert abs(ad - fd) <= 1e-4 * abs(fd) + floor, (what, ad, fd)


@pytest.mark.parametrize("walls", [False, True])
def test_adjoint_matches_central_differences_fp64(walls):
    """Each observable separately (J_drag, then A): adjoint gradients with
    respect to the five parameters and, along a seeded random direction, the
    initial densities agree with central differences to 1e-4 relative."""
    shape, base, theta, col, a, b = case(walls)
    steps = 20
    run, _ = gpu_objective(shape, base, theta, col, a, b, steps)
    gJ, rJ = run.backward(1.0, 0.0)
    gA, rA = run.backward(0.0, 1.0)
    for i, name in enumerate(NAMES):
        h = 1e-5
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (gpu_objective(shape, base, tp, col, a, b, steps)[1] -
              gpu_objective(shape, base, tm, col, a, b, steps)[1]) / (2 * h)
        check(gJ[i], fd[0], ("J_drag", name))
        check(gA[i], fd[1], ("A", name))
    rng = np.random.default_rng(4)
    da, db = rng.standard_normal(a.size), rng.standard_normal(b.size)
    h = 1e-6
    fd = (gpu_objective(shape, base, theta, col, a + h * da, b + h * db, steps)[1] -
          gpu_objective(shape, base, theta, col, a - h * da, b - h * db, steps)[1]) / (2 * h)
    check(float(rJ[0] @ da + rJ[1] @ db), fd[0], ("J_drag", "rho0"))
    check(float(rA[0] @ da + rA[1] @ db), fd[1], ("A", "rho0"))


def test_adjoint_matches_oracle_differences():
    """Reference gradient through the oracle: central differences of the
    oracle's observables agree with the GPU adjoint."""
    shape, base, theta, col, a, b = case(True)
    steps = 12
    run, _ = gpu_objective(shape, base, theta, col, a, b, steps)
    gJ, _ = run.backward(1.0, 0.0)
    gA, _ = run.backward(0.0, 1.0)
    for i, name in enumerate(NAMES):
        h = 1e-5
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle_objective(shape, base, tp, col, a, b, steps) -
              oracle_objective(shape, base, tm, col, a, b, steps)) / (2 * h)
        check(gJ[i], fd[0], ("J_drag", name))
        check(gA[i], fd[1], ("A", name))


def test_adjoint_fp32_agrees_with_fp64():
    shape, base, theta, col, a, b = case(False)
    steps = 20
    r64, _ = gpu_objective(shape, base, theta, col, a, b, steps, "fp64")
    g64, rho64 = r64.backward(0.0, 1.0)
    r32, _ = gpu_objective(shape, base, theta, col, a, b, steps, "fp32")
    g32, rho32 = r32.backward(0.0, 1.0)
    assert np.all(np.abs(g32 - g64) <= 1e-3 * np.abs(g64) + 1e-6)
    assert np.abs(rho32 - rho64).max() <= 1e-3 * np.abs(rho64).max()


def test_autograd_function_runs():
    import torch

    from paper_2004_04080_gb300.adjoint import AdjointRunner, LBObjective
    from paper_2004_04080_gb300.lbgb import LBLattice

    shape, base, theta, col, a, b = case(False)
    lat = LBLattice(shape, "fp32", max_colloids=2)
    run = AdjointRunner(lat, 9)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    ra = torch.tensor(a, requires_grad=True)
    rb = torch.tensor(b, requires_grad=True)
    out = LBObjective().apply(th, ra, rb, run, base, col)
    (out[0] * 2.0 + out[1]).backward()
    assert th.grad is not None and torch.all(torch.isfinite(th.grad))
    assert ra.grad.shape == ra.shape and torch.isfinite(ra.grad).all()

    # inputs on the GPU (densities in FP32): the gradients come back on each
    # input's device and in its dtype, equal to the CPU-input gradients
    th2 = th.detach().cuda().requires_grad_(True)
    ra2 = ra.detach().float().cuda().requires_grad_(True)
    rb2 = rb.detach().cuda().requires_grad_(True)
    out2 = LBObjective().apply(th2, ra2, rb2, run, base, col)
    assert out2.device == th2.device
    (out2[0] * 2.0 + out2[1]).backward()
    for x in (th2, ra2, rb2):
        assert x.grad.device == x.device and x.grad.dtype == x.dtype
    assert torch.allclose(th2.grad.cpu(), th.grad, rtol=1e-5, atol=1e-12)

    # a graph whose runner has since run another forward refuses to go back
    stale = LBObjective().apply(th, ra, rb, run, base, col)
    LBObjective().apply(th, ra, rb, run, base, col)
    with pytest.raises(RuntimeError, match="another forward"):
        stale.sum().backward()


def test_async_reverse_sweep_matches_synchronous_steps():
    """The runner's reverse sweep (states and link forces recorded on the
    device by lb_record, dJ/dF from lb_drag_gradient, gradients accumulated on
    the device) gives the gradients of a sweep of synchronous lb_adjoint_step
    calls with dJ/dF formed on the host from the read-back forces."""
    import torch

    from paper_2004_04080_gb300 import lbgb
    from paper_2004_04080_gb300.adjoint import AdjointRunner
    from paper_2004_04080_gb300.lbgb import LBLattice

    shape, base, theta, col, a, b = case(True)
    steps = 7
    lat = LBLattice(shape, "fp64", max_colloids=2)
    run = AdjointRunner(lat, steps, checkpoint_every=3)
    run.forward(params_of(base, theta), a, b, col)
    g_async, r_async = run.backward(0.7, 1.3)

    # synchronous reference: every state kept, forces read per step
    lat2 = LBLattice(shape, "fp64", max_colloids=2)
    lat2.set_params(**params_of(base, theta))
    lat2.init_fields(a, b)
    lat2.add_colloids(np.asarray(col["pos"]), col["radius"], np.full(2, np.inf))
    sb = lbgb.lb_state_bytes(lat2.h)
    states = torch.empty((steps, sb), dtype=torch.uint8, device="cuda")
    forces = []
    for t in range(steps):
        lbgb.lb_get_state(lat2.h, states[t].data_ptr())
        lat2.step(1)
        forces.append(lat2.term("F_liq"))
    fb, scb = lbgb.lb_adjoint_bytes(lat2.h)
    cur, nxt = (torch.empty(fb, dtype=torch.uint8, device="cuda") for _ in range(2))
    scratch = torch.empty(scb, dtype=torch.uint8, device="cuda")
    lbgb.lb_adjoint_seed(lat2.h, 1.3, cur.data_ptr(), scratch.data_ptr())
    grads = np.zeros(5)
    for t in reversed(range(steps)):
        # dJ/dF from the same device routine as the asynchronous sweep
        F = torch.from_numpy(forces[t]).cuda()
        dJdF_dev = torch.empty_like(F)
        lbgb.lb_drag_gradient(lat2.h, F.data_ptr(), 0.7 / (steps * 2), 1e-12, dJdF_dev.data_ptr())
        dJdF = dJdF_dev.cpu().numpy()
        lbgb.lb_adjoint_step(lat2.h, states[t].data_ptr(), cur.data_ptr(), nxt.data_ptr(), scratch.data_ptr(),
                             dJdF, grads)
        cur, nxt = nxt, cur
    g = torch.empty((2, lat2.N), dtype=torch.float64, device="cuda")
    lbgb.lb_adjoint_initial(lat2.h, cur.data_ptr(), g.data_ptr())
    # the link-force sums of the two forward runs are fixed-point sums, the
    # same bits in any order of addition, so the two sweeps agree exactly
    assert np.array_equal(g_async, grads), (g_async, grads)
    assert np.array_equal(r_async, g.cpu().numpy())


def test_adjoint_on_the_benchmarked_workload_fp64():
    """The adjoint where it is timed: the 64^3 periodic box with 8 immobile
    R = 4.5 spheres at its own parameters (G = 0.65, tau = 1, zeta = 0), 500
    steps with sqrt(500) -> 23 checkpoints, in FP64.  Each observable
    separately, the gradients with respect to tau_A, tau_B, G, zeta_A, zeta_B
    and along three seeded random directions of the initial densities agree
    with central differences to 1e-4 relative.

    The steps differ by observable and direction.  The interface measure A is
    smooth on the scale of the parameters (h = 1e-4).  The drag J_drag is the
    mean magnitude of forces that vanish by symmetry up to the 1 % noise of
    the neutral 50/50 mixture (|F| ~ 4e-7 here), so J_drag is curved on the
    scale of |F| and its differences converge only for steps well below it:
    measured on a GB300, the relative error falls like h^2 from 6.5e-2 at
    h = 1e-4 to 1.8e-5 at 1e-6 along tau, and to 6e-6 at 1e-9 along the
    densities.  Off the symmetric point (tau 0.9 / 1.1, zeta +-0.1) every
    direction agrees to 1e-6 at h = 1e-6."""
    from paper_2004_04080_gb300.workloads import workload

    w = workload("adjoint64")
    assert w.shape == (64, 64, 64) and w.n_colloids == 8 and w.steps == 500
    a, b = w.densities()
    c = w.colloids()
    col = dict(pos=c["pos"], radius=c["radius"])
    base = {k: v for k, v in w.params.items() if k not in ("tau", "G", "zeta")}
    theta = np.array([w.params["tau"][0], w.params["tau"][1], w.params["G"], w.params["zeta"][0],
                      w.params["zeta"][1]])
    steps = w.steps
    run, obj = gpu_objective(w.shape, base, theta, col, a, b, steps)
    assert run.K == 23
    assert np.all(np.isfinite(obj))
    grad = [run.backward(1.0, 0.0), run.backward(0.0, 1.0)]  # (parameters, densities) of J_drag, A
    del run

    def fd_param(i, h):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        return (gpu_objective(w.shape, base, tp, col, a, b, steps)[1] -
                gpu_objective(w.shape, base, tm, col, a, b, steps)[1]) / (2 * h)

    h_drag = {"tau_A": 2e-7, "tau_B": 2e-7, "G": 1e-4, "zeta_A": 2e-8, "zeta_B": 2e-8}
    for i, name in enumerate(NAMES):
        check(grad[0][0][i], fd_param(i, h_drag[name])[0], ("J_drag", name), floor=0.0)
        check(grad[1][0][i], fd_param(i, 1e-4)[1], ("A", name), floor=0.0)
    rng = np.random.default_rng(2024)
    for d in range(3):
        da, db = rng.standard_normal(a.size), rng.standard_normal(b.size)
        for obs, h in ((0, 1e-9), (1, 1e-4)):
            fd = (gpu_objective(w.shape, base, theta, col, a + h * da, b + h * db, steps)[1][obs] -
                  gpu_objective(w.shape, base, theta, col, a - h * da, b - h * db, steps)[1][obs]) / (2 * h)
            r = grad[obs][1]
            check(float(r[0] @ da + r[1] @ db), fd, (("J_drag", "A")[obs], "rho0 direction %d" % d), floor=0.0)
