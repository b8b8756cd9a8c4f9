"""Stochastic rounding of the FP16 deviation stores (the FP16 default;
lb_set_rounding), with the hardware's stochastic-rounding conversion."""
import numpy as np
import pytest

from paper_2004_04080_gb300.workloads import workload

pytestmark = pytest.mark.gpu


def uniform(shape, rounding, rhoA=0.7371, rhoB=1.3119):
    from paper_2004_04080_gb300.lbgb import LBLattice

    g = LBLattice(shape, "fp16", max_colloids=0)
    g.set_params(G=0.0, tau=(1.0, 1.0), rho0=(1.0, 1.0))
    N = int(np.prod(shape))
    g.init_fields(np.full(N, rhoA), np.full(N, rhoB))
    g.set_rounding(rounding, seed=5)
    return g


def test_stochastic_rounding_is_unbiased():
    """A uniform fluid at rest (no force): one step stores f*_i = w_i rho in
    FP32, and the deviation from w_i rho0 is not a half value.  Rounding to
    nearest stores the same half everywhere; stochastic rounding stores the
    two neighbouring halves, with a mean over the 262,144 sites equal to the
    FP32 value (to a few hundredths of their spacing)."""
    from paper_2004_04080_gb300.lbgb import LB_ROUND_NEAREST, LB_ROUND_STOCHASTIC

    shape = (64, 64, 64)
    rn, sr = uniform(shape, LB_ROUND_NEAREST), uniform(shape, LB_ROUND_STOCHASTIC)
    rho = [rn.populations(k).sum(axis=0) for k in range(2)]  # the stored initial state
    rn.step(1)
    sr.step(1)
    w = {0: 1 / 3, 1: 1 / 18, 7: 1 / 36}
    checked = 0
    for k in range(2):
        assert np.ptp(rho[k]) == 0.0
        fn, fs = rn.populations(k), sr.populations(k)
        for i, wi in w.items():
            exact = wi * rho[k][0]
            assert np.ptp(fn[i]) == 0.0
            vals = np.unique(fs[i])
            if len(vals) == 1:  # the value happens to be a half: nothing to round
                assert vals[0] == fn[i][0]
                continue
            lo, hi = vals
            assert lo < exact < hi
            assert fn[i][0] == (lo if exact - lo <= hi - exact else hi)
            assert abs(fs[i].mean() - exact) < 0.03 * (hi - lo), (k, i, fs[i].mean(), exact, lo, hi)
            checked += 1
    assert checked >= 4


@pytest.mark.parametrize("case", ["small_fp64", "ragged_walls"])
def test_stochastic_rounding_against_the_oracle(case):
    """FP16 with stochastic rounding stays within the 1e-3 of the FP16 form
    against the FP64 oracle (the 32^3 bijel workload after 100 steps; the
    ragged sheared-wall box with unequal tau, wetting and moving particles
    after 40 steps)."""
    from paper_2004_04080_gb300.lbgb import LB_ROUND_STOCHASTIC
    from test_gpu_parity import compare_colloids, compare_fields, run_both

    if case == "small_fp64":
        w = workload("small_fp64")
        g, o = run_both(w.shape, w.params, 0, "fp16", w.colloids(), w.densities())
        steps = w.steps
    else:
        shape = (24, 13, 11)
        params = dict(G=0.6, tau=(0.8, 1.2), zeta=(0.15, -0.15), bc=(1, 1, 0), wall_u_lo=(-0.02, 0.01, 0),
                      wall_u_hi=(0.03, 0, 0), body_force=(1e-5, 0, -2e-6), hertz_K=20, hertz_sigma=8.0,
                      hertz_rcap=7.0, side_wall_k=0.5, side_wall_d=4.0)
        col = dict(pos=[[7.2, 6.1, 5.3], [15.5, 6.5, 5.0]], radius=[3.2, 3.0], mass=[1500.0, 1200.0],
                   vel=[[0.05, 0.03, -0.01], [-0.04, 0.0, 0.02]], omega=[[0.01, 0.0, 0.02], [0, -0.02, 0]])
        g, o = run_both(shape, params, 0, "fp16", col)
        steps = 40
    g.set_rounding(LB_ROUND_STOCHASTIC, seed=3)
    g.step(steps)
    o.step(steps)
    compare_fields(g, o, 1e-3)
    compare_colloids(g, o, 1e-3)


def test_fp16_rounds_stochastically_by_default():
    """An FP16 context stores with stochastic rounding unless told otherwise
    (the adjoint, which needs reproducible recomputation, then refuses)."""
    import torch

    from paper_2004_04080_gb300 import lbgb
    from paper_2004_04080_gb300.lbgb import LB_ROUND_NEAREST, LBError, LBLattice

    g = LBLattice((16, 16, 16), "fp16", max_colloids=0)
    g.set_params(G=0.0, rho0=(1.0, 1.0))
    g.init_fields(np.full(4096, 0.7371), np.full(4096, 1.3119))
    fb, sb = lbgb.lb_adjoint_bytes(g.h)
    adj = torch.empty(fb, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    with pytest.raises(LBError):
        lbgb.lb_adjoint_seed(g.h, 1.0, adj.data_ptr(), scratch.data_ptr())
    g.set_rounding(LB_ROUND_NEAREST)
    lbgb.lb_adjoint_seed(g.h, 1.0, adj.data_ptr(), scratch.data_ptr())
    # a uniform fluid at rest stores one value per population when rounded to
    # nearest, two neighbouring halves when rounded stochastically
    g.step(1)
    assert np.ptp(g.populations(0)[1]) == 0.0
    h = LBLattice((16, 16, 16), "fp16", max_colloids=0)
    h.set_params(G=0.0, rho0=(1.0, 1.0))
    h.init_fields(np.full(4096, 0.7371), np.full(4096, 1.3119))
    h.step(1)
    assert len(np.unique(h.populations(0)[1])) == 2


def test_the_adjoint_refuses_stochastic_rounding():
    import torch

    from paper_2004_04080_gb300 import lbgb
    from paper_2004_04080_gb300.lbgb import LB_ROUND_NEAREST, LB_ROUND_STOCHASTIC, LBError

    g = uniform((16, 16, 16), LB_ROUND_STOCHASTIC)
    fb, sb = lbgb.lb_adjoint_bytes(g.h)
    adj = torch.empty(fb, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    with pytest.raises(LBError):
        lbgb.lb_adjoint_seed(g.h, 1.0, adj.data_ptr(), scratch.data_ptr())
    g.set_rounding(LB_ROUND_NEAREST)
    lbgb.lb_adjoint_seed(g.h, 1.0, adj.data_ptr(), scratch.data_ptr())
    with pytest.raises(LBError):
        g.set_rounding(7)
