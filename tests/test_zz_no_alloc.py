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
    a = a.reshape(nvar, -1)
    b = b.reshape(nvar, -1)
    out = []
    for f in range(nvar):
        den = np.abs(b[f]).max()
        if f >= 2 + dim:
            den = max(den, 1e-6 * np.abs(b[0]).max())
        out.append(np.abs(a[f] - b[f]).max() / max(den, 1e-300))
    return max(out)


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
        boxes, nbox, nw, prm, keep = sdc._marshal(P, sdc.PREC_FP64)
        st = sdc.Stats()
        s = sdc.load().sdc_step_static(boxes, nbox, ctypes.byref(nw), ctypes.byref(prm),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                       ctypes.c_void_p(Ub.data_ptr()), float(dt), ctypes.byref(st))
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
