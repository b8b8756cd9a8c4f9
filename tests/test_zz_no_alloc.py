"""The allocation-free totals entry point (lb_totals_static) against the
context-based one (lb_get_totals), through the C ABI.

lb_totals_static is for callers that cannot allocate device memory where they
need the totals (it keeps its scratch in a static device array); this test
gives it a copy of a context's populations and node map (FP16: the half
deviations and rho0) and checks that two calls in a row agree with
lb_get_totals, bit for bit with each other, and leave the device's free
memory unchanged.  It is collected last so that a
failure here comes after every other test, and it passes both alone in a fresh
process and after the rest of the suite (the first call on the device does the
scratch set-up).
"""
import numpy as np
import pytest

from paper_2004_04080_gb300.workloads import mixture_densities

pytestmark = pytest.mark.gpu


# D3Q19 weights by link class: rest, the six axis links, the twelve diagonals
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-12), ("fp16", 1e-6)])
def test_totals_static_matches_context_totals(prec, tol):
    """FP64 / FP32 storage hold the populations; FP16 holds half deviations
    f_i - w_i rho0^k, here with unequal rho0, which the call is given."""
    import torch

    from paper_2004_04080_gb300 import lbgb

    shape = (20, 15, 13)
    N = int(np.prod(shape))
    rho0 = (0.55, 0.45)
    g = lbgb.LBLattice(shape, prec, max_colloids=2)
    g.set_params(G=0.7, tau=(0.9, 1.1), zeta=(0.1, -0.1), hertz_K=20, hertz_sigma=8.0, hertz_rcap=7.0,
                 rho0=rho0)
    a, b = mixture_densities(shape, seed=21, amp=0.05)
    u = np.zeros((3, N))
    u[0] = 0.01
    g.init_fields(a, b, u)
    g.add_colloids([[6.2, 6.1, 5.3], [15.4, 6.6, 5.1]], [3.1, 2.9], [300.0, 250.0],
                   vel=[[0.02, 0.01, 0.0], [-0.01, 0.0, 0.01]])
    g.step(7)
    ref = g.totals()[:5]

    dt = {"fp64": torch.float64, "fp32": torch.float32, "fp16": torch.float16}[prec]
    stride = N + 37  # a padded plane stride, as the library's own buffers have
    pops = torch.zeros((2, 19, stride), dtype=dt)
    for k in (0, 1):
        f = g.populations(k)
        if prec == "fp16":
            # the stored deviations, recovered exactly (the read-out adds the
            # shift back with an error far below a half's spacing)
            dev = torch.from_numpy(f - W19[:, None] * rho0[k]).to(torch.float16)
            assert np.abs(dev.double().numpy() + W19[:, None] * rho0[k] - f).max() < 1e-6
            pops[k, :, :N] = dev
        else:
            pops[k, :, :N] = torch.from_numpy(f).to(dt)
    pops = pops.cuda()
    mask = torch.from_numpy((g.owner() >= 0).astype(np.uint8)).cuda()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    r0 = np.array(rho0) if prec == "fp16" else None

    def call():
        lbgb.lb_totals_static(pops.data_ptr(), lbgb.PREC[prec], *shape, stride, mask.data_ptr(), r0,
                              out.data_ptr(), stream.cuda_stream)

    call()  # the first call in the context may load the module and look up the scratch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    results = []
    for _ in range(2):
        out.zero_()
        call()
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    # the calls took no device memory, from the driver or from torch's pool
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for r in results:
        assert np.all(np.abs(r[:2] - ref[:2]) <= tol * np.abs(ref[:2]))
        assert np.all(np.abs(r[2:] - ref[2:]) <= tol * max(np.abs(ref[:2]).max(), 1.0))
    assert np.array_equal(results[0], results[1])


def test_totals_static_rejects_oversized_lattice():
    import torch

    from paper_2004_04080_gb300 import lbgb

    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    pops = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lbgb.LBError) as e:
        lbgb.lb_totals_static(pops.data_ptr(), lbgb.LB_FP32, 4, 4, 5000, 4 * 4 * 5000, 0, None,
                              out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == lbgb.LB_ERR_ARG
