"""sdc_step_static: the SDC step for callers that cannot allocate device
memory (an allocator or memory budget owned by another framework, or a host
that forbids device allocations after start-up).  It must give the same result
as the allocating path (sdc_init_box + sdc_step), call after call, and refuse
problems that do not fit its fixed 48 MiB scratch array.

The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from paper_1910_12578_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_12578_gb300 import build
    build.build()
    return torch


def _rel(a, b, nvar, dim):
    """Largest per-field |a - b|_inf / |b|_inf (every field against its own
    largest value, floor 1e-30)."""
    a = a.reshape(nvar, -1)
    b = b.reshape(nvar, -1)
    out = []
    for f in range(nvar):
        den = max(np.abs(b[f]).max(), 1e-30)
        out.append(np.abs(a[f] - b[f]).max() / den)
    return max(out)


def _static_call(torch, problems, U, dt, prec):
    from paper_1910_12578_gb300 import sdc
    boxes, nbox, nw, prm, keep = sdc._marshal(problems, prec)
    st = sdc.Stats()
    s = sdc.load().sdc_step_static(boxes, nbox, ctypes.byref(nw), ctypes.byref(prm),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                   ctypes.c_void_p(U.data_ptr()), float(dt), ctypes.byref(st))
    del keep
    return s, st


@pytest.mark.parametrize("case", ["1d", "box16"])
def test_static_step_matches_allocating_step_twice(torch_cuda, case):
    torch = torch_cuda
    from paper_1910_12578_gb300 import sdc
    if case == "1d":
        P, U = W.config_1d()
    else:
        P, U = W.config_box(n=16, nspec=7, seed=0, T0=0.5)
    ctx = sdc.Context(P)
    Ua = torch.from_numpy(U).cuda()
    Ub = Ua.clone()
    dt = ctx.cfl_dt(Ua, 0.5)
    for _ in range(2):  # two calls in a row through both entry points
        sa = ctx.step(Ua, dt)
        s, st = _static_call(torch, P, Ub, dt, sdc.PREC_FP64)
        assert s in (sdc.SDC_OK, sdc.SDC_ERR_NEWTON_NOCONV)
        torch.cuda.synchronize()
        assert _rel(Ub.cpu().numpy(), Ua.cpu().numpy(), P.nvar, P.dim) <= TOL64
        assert st.newton_solves == sa.newton_solves
        assert st.n_fail == sa.n_fail
    ctx.close()


def test_static_step_rejects_problems_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1910_12578_gb300 import sdc
    P, U = W.config_box(n=64, nspec=7, seed=0, T0=0.5)   # 285 MB of workspace > 48 MiB
    Ud = torch.from_numpy(U).cuda()
    before = Ud.clone()
    with pytest.raises(sdc.SdcError) as ei:
        sdc.step_static(P, Ud, 1e-3)
    assert ei.value.status == sdc.SDC_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.equal(Ud, before)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_static_step_matches_allocating_step_on_ragged_boxes(torch_cuda, prec):
    """Several uneven boxes in one call (the tile-to-box map of the static
    tables: prefix sums of tiles per box, partial tiles, box offsets), in FP64,
    with the FP32 Jacobian and with the float-pair Jacobian, against
    sdc_init_box + sdc_step on the same boxes, two calls in a row."""
    torch = torch_cuda
    from paper_1910_12578_gb300 import sdc
    net = W.alpha_chain(7, np.random.default_rng(3))
    Ps, Us = [], []
    for n, amp in (((8, 8, 8), 2.0), ((12, 16, 8), 1.6), ((16, 16, 16), 2.4), ((5, 3, 7), 1.3)):
        h = 1.0 / 64
        P = W.Problem(dim=3, n=n, dx=(h, h, h), gamma=5.0 / 3.0, net=net, n_nodes=3, n_iters=3)
        Ps.append(P)
        Us.append(W.hot_spot_state(P, amp, T0=0.5).reshape(P.nvar, -1))
    U = np.concatenate(Us, axis=1)
    ctx = sdc.Context(Ps, prec=prec)
    Ua = torch.from_numpy(U).cuda()
    Ub = Ua.clone()
    dt = ctx.cfl_dt(Ua, 0.5)
    for _ in range(2):
        sa = ctx.step(Ua, dt)
        s, st = _static_call(torch, Ps, Ub, dt, prec)
        assert s in (sdc.SDC_OK, sdc.SDC_ERR_NEWTON_NOCONV)
        torch.cuda.synchronize()
        assert _rel(Ub.cpu().numpy(), Ua.cpu().numpy(), Ps[0].nvar, 3) <= TOL64
        assert st.newton_solves == sa.newton_solves
        assert st.n_fail == sa.n_fail
        assert st.newton_iters_total == sa.newton_iters_total
    ctx.close()


def test_static_step_rejects_boxes_whose_zone_count_overflows(torch_cuda):
    """A box of 2^31 zones or more is refused before any size is formed from it."""
    torch = torch_cuda
    from paper_1910_12578_gb300 import sdc
    P, U = W.config_box(n=8, nspec=7, seed=0, T0=0.5)
    Ud = torch.from_numpy(U).cuda()
    before = Ud.clone()
    for n in ((2 ** 31 - 1,) * 3, (2 ** 16, 2 ** 15, 1), (2 ** 11, 2 ** 10, 2 ** 10)):
        Pb = W.Problem(dim=3, n=n, dx=P.dx, gamma=P.gamma, net=P.net)
        s, _ = _static_call(torch, [Pb], Ud, 1e-3, sdc.PREC_FP64)
        assert s == sdc.SDC_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.equal(Ud, before)
